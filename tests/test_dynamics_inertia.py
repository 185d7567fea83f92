"""The piston inertia of the multi-period march (F_I of Eq. 2.10, m_K of Table 8),
on the CPU.

The generalized mass matrix is pinned by the kinetic energy of a uniform rigid rod
over the coupling length (translation: (1/2) m v^2; tilt about mid-gap:
(1/2) (m L^2 / 12) w^2), and the march's handling of the term by running it with
the oracle's Picard step on a small grid: at every converged shaft step the oil
load of the recorded state, the side load and -M (edot - edot_l) / dt balance."""
import math

import numpy as np
import pytest

import oracle
from paper_2511_06824_gb300 import dynamics, inputs

L = inputs.GAP_L


def test_mass_matrix_is_the_uniform_rods_kinetic_energy():
    m = 0.128
    M = dynamics.inertia_matrix(m)
    assert np.array_equal(M, M.T)
    np.linalg.cholesky(M)
    v = 0.37
    # translation along x (e1 = e3) and along y (e2 = e4): (1/2) m v^2
    for ed in (np.array([v, 0, v, 0]), np.array([0, v, 0, v])):
        assert math.isclose(0.5 * ed @ M @ ed, 0.5 * m * v * v, rel_tol=1e-14)
    # tilt about mid-gap at rate w: x(z) = w (z - L/2), so e1 = -w L/2, e3 = +w L/2
    w = 2.3
    ed = np.array([-w * L / 2, 0, w * L / 2, 0])
    assert math.isclose(0.5 * ed @ M @ ed, 0.5 * (m * L * L / 12) * w * w, rel_tol=1e-14)
    # the inertia load of a uniform translation is -m a, split evenly between the ends
    F = dynamics.inertia_force(M, [2e-4, 0, 2e-4, 0], [0, 0, 0, 0], 1e-3)
    np.testing.assert_allclose(F, [-m * 0.2 / 2, 0, -m * 0.2 / 2, 0], rtol=1e-14)
    assert not np.any(dynamics.inertia_force(dynamics.inertia_matrix(0.0), [1, 2, 3, 4],
                                             [0, 0, 0, 0], 1e-3))


def oracle_stepper(scheme, nth, nz, ph, tex, state, e_prev, dt, F_ext, d_e, d_edot, opts):
    assert scheme == "general"
    r = oracle.picard_step(nth, nz, ph, tex, state, e_prev, dt, F_ext, d_e, d_edot, eps=opts.eps)
    assert r["status"] == oracle.OK
    return r


@pytest.mark.parametrize("mass", [0.0, 30.0])
def test_march_balances_oil_side_load_and_inertia(mass):
    nth, nz, steps, kappa = 24, 12, 4, 0.2
    phys = inputs.phys_vector()
    tex = inputs.smooth_texture()
    prof = inputs.trapezoid_pressure_profile(np.random.default_rng(3), 360)
    st0 = np.array([2e-6, -1e-6, 3e-6, 1e-6, 1e-5, 0, -2e-5, 0.0])
    # (30 kg, not 0.128: the lagged term converges at a rate proportional to the mass,
    # and a measurable effect on this coarse grid needs a heavy piston)
    opts = oracle_opts = type("O", (), {"eps": 1e-12, "precond": 1, "omega": 1.2, "max_iter": 10 ** 5,
                                        "precision": 0, "criterion": 0})()
    traj = dynamics.march(0, nth, nz, phys, tex, st0, prof, steps, kappa=kappa, tol_F=1e-9,
                          opts=opts, mass=mass, stepper=oracle_stepper)
    assert all(r.converged for r in traj.records)
    dt = (60.0 / 600.0) / 360.0
    M = np.diag([mass / 3] * 4)
    M[0, 2] = M[2, 0] = M[1, 3] = M[3, 1] = mass / 6
    prev = st0
    worst = 0.0
    for s, rec in enumerate(traj.records):
        ph = phys.copy()
        ph[5] = prof[s]
        ph[4] = 5.0 * math.sin(2 * math.pi * s / 360)
        side = np.array([0, 0, kappa * ph[5] * math.pi * ph[0] ** 2 * math.tan(math.radians(10)), 0])
        # oil load of the recorded state: the oracle's G with no external force
        r = oracle.picard_step(nth, nz, ph, tex, rec.state, prev[:4], dt, np.zeros(4), 2e-8, 1e-6,
                               eps=1e-12)
        inertia = -M @ ((rec.state[4:] - prev[4:]) / dt)
        worst = max(worst, np.linalg.norm(r["G"] + side + inertia) / np.linalg.norm(side))
        # the backward difference ties e to the rate
        np.testing.assert_allclose(rec.state[:4], prev[:4] + dt * rec.state[4:], rtol=1e-9,
                                   atol=1e-18)
        prev = rec.state
    assert worst <= 1e-8
    if mass:
        base = dynamics.march(0, nth, nz, phys, tex, st0, prof, steps, kappa=kappa, tol_F=1e-9,
                              opts=oracle_opts, mass=0.0, stepper=oracle_stepper)
        assert np.abs(traj.states[:, 4:] - base.states[:, 4:]).max() > 1e-3 * np.abs(base.states[:, 4:]).max()
