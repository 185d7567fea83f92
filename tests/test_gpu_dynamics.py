"""Multi-period march (shaft-angle steps of Picard iterations) on the GPU against
the same march written with the oracle's Picard step."""
import math

import numpy as np
import pytest

import oracle
from paper_2511_06824_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_06824_gb300 import build, gmaf
    build.build()
    gmaf.load()
    return gmaf


def oracle_march(nth, nz, phys, tex, st, prof, steps, kappa, eps, tol_F=1e-6, max_picard=20,
                 mass=0.128, swash=False):
    """The march with the oracle's Picard step: side load on e3, and the inertia of a
    piston of `mass` spread evenly over the gap, -M (edot - edot_l) / dt with
    M = mass / 6 [[2, 1], [1, 2]] on (e1, e3) and on (e2, e4).  swash: the gap length
    and sliding speed of the swash-plate piston of Table 8 (R_b = 40.5 mm, 10 degrees,
    L_Fmin = 30 mm, 600 rpm), L_Fmin + R_b tan(10 deg) (1 - cos phi) and its rate."""
    dt = (60.0 / 600.0) / 360.0
    M = mass / 6.0 * np.array([[2, 0, 1, 0], [0, 2, 0, 1], [1, 0, 2, 0], [0, 1, 0, 2.0]])
    out = []
    for s in range(steps):
        phi = 2 * math.pi * (s % 360) / 360
        ph = phys.copy()
        ph[5] = prof[s % 360]
        ph[4] = 5.0 * math.sin(phi)
        if swash:
            rt = 4.05e-2 * math.tan(math.radians(10.0))
            ph[1] = 3e-2 + rt * (1 - math.cos(phi))
            ph[4] = rt * (2 * math.pi * 600 / 60) * math.sin(phi)
        f = kappa * ph[5] * math.pi * ph[0] ** 2 * math.tan(math.radians(10.0))
        F = np.array([0.0, 0.0, f, 0.0])
        e_prev = st[:4].copy()
        ed_prev = st[4:].copy()
        for _ in range(max_picard):
            Fi = F - M @ ((st[4:] - ed_prev) / dt)
            r = oracle.picard_step(nth, nz, ph, tex, st, e_prev, dt, Fi, 2e-8, 1e-6, eps=eps)
            assert r["status"] == 0
            scale = max(np.linalg.norm(F), ph[5] * math.pi * ph[0] ** 2, 1.0)
            if np.linalg.norm(r["G"]) <= tol_F * scale:
                break
            st = r["state"]
        out.append(st.copy())
    return np.array(out)


@pytest.mark.parametrize("precision,tol,mass", [(0, 1e-6, 0.128), (1, 1e-4, 0.128),
                                                (0, 1e-6, 30.0), (0, 1e-6, 0.0)])
def test_march_matches_oracle(g, precision, tol, mass):
    """Mass 0.128 kg is the piston of Table 8; 30 kg makes the inertia load visible
    on this grid; 0 leaves it out."""
    from paper_2511_06824_gb300 import dynamics
    nth, nz, steps = 48, 24, 10
    phys = inputs.phys_vector()
    tex = inputs.dimple_texture(np.random.default_rng(4))
    prof = inputs.trapezoid_pressure_profile(np.random.default_rng(3), 360)
    st0 = np.array([2e-6, -1e-6, 3e-6, 1e-6, 0, 0, 0, 0.0])
    eps = 1e-12
    with g.Context() as c:
        traj = dynamics.march(c.handle, nth, nz, phys, tex, st0, prof, steps, kappa=0.2,
                              opts=g.solver_opts(eps=eps, precision=precision), mass=mass)
    ref = oracle_march(nth, nz, phys, tex, st0.copy(), prof, steps, 0.2, eps, mass=mass)
    got = traj.states
    assert all(r.converged for r in traj.records)
    scale = np.abs(ref[:, :4]).max()
    assert np.max(np.abs(got[:, :4] - ref[:, :4])) <= tol * scale
    rscale = np.abs(ref[:, 4:]).max()
    assert np.max(np.abs(got[:, 4:] - ref[:, 4:])) <= 10 * tol * rscale


@pytest.mark.parametrize("precision,tol", [(0, 1e-6), (1, 1e-4)])
def test_swash_kinematics_march_matches_oracle(g, precision, tol):
    """With the swash-plate kinematics every shaft step solves on a gap of its own
    length (30 mm at outer dead centre, growing with the stroke) at the piston's
    speed; the warm-started solves carry the previous step's fields across the change
    of gap length."""
    from paper_2511_06824_gb300 import dynamics
    nth, nz, steps = 48, 24, 10
    phys = inputs.phys_vector()
    tex = inputs.dimple_texture(np.random.default_rng(4))
    prof = inputs.trapezoid_pressure_profile(np.random.default_rng(3), 360)
    st0 = np.array([2e-6, -1e-6, 3e-6, 1e-6, 0, 0, 0, 0.0])
    eps = 1e-12
    with g.Context() as c:
        traj = dynamics.march(c.handle, nth, nz, phys, tex, st0, prof, steps, kappa=0.2,
                              opts=g.solver_opts(eps=eps, precision=precision),
                              kinematics=dynamics.SwashKinematics())
    ref = oracle_march(nth, nz, phys, tex, st0.copy(), prof, steps, 0.2, eps, swash=True)
    assert all(r.converged for r in traj.records)
    assert traj.records[0].gap_length == 3e-2 and traj.records[-1].gap_length > 3e-2
    got = traj.states
    scale = np.abs(ref[:, :4]).max()
    assert np.max(np.abs(got[:, :4] - ref[:, :4])) <= tol * scale
    rscale = np.abs(ref[:, 4:]).max()
    assert np.max(np.abs(got[:, 4:] - ref[:, 4:])) <= 10 * tol * rscale


def test_warm_start_saves_iterations_and_keeps_the_answer(g):
    """zero_init = 0 starts from the fields the previous step of this context left:
    re-solving at the same state needs almost no iterations and gives the same loads."""
    w = inputs.make("textured-128x64-k9", 2)
    dt = 2.78e-4
    F = np.array([30.0, -10.0, 5.0, 1.0])
    with g.Context() as c:
        cold = g.gmaf_picard_step(c.handle, w.n_theta, w.n_z, w.phys, w.tex, w.state, w.state[:4],
                                  dt, F, w.d_e, w.d_edot, g.solver_opts(eps=1e-12))
        warm = g.gmaf_picard_step(c.handle, w.n_theta, w.n_z, w.phys, w.tex, w.state, w.state[:4],
                                  dt, F, w.d_e, w.d_edot, g.solver_opts(eps=1e-12, zero_init=0))
        # a different shape in between invalidates the stored fields: back to a cold start
        g.gmaf_picard_step(c.handle, 64, 32, w.phys, w.tex, w.state, w.state[:4], dt, F, w.d_e,
                           w.d_edot, g.solver_opts(eps=1e-12))
        again = g.gmaf_picard_step(c.handle, w.n_theta, w.n_z, w.phys, w.tex, w.state,
                                   w.state[:4], dt, F, w.d_e, w.d_edot,
                                   g.solver_opts(eps=1e-12, zero_init=0))
    assert warm["iters"] <= 0.2 * cold["iters"]
    assert again["iters"] == cold["iters"]
    scale = np.maximum(np.abs(cold["loads"]), 1e-3 * np.linalg.norm(cold["loads"]))
    assert np.max(np.abs(warm["loads"] - cold["loads"]) / scale) < 1e-8
    np.testing.assert_allclose(warm["state"], cold["state"], rtol=1e-6, atol=1e-14)


def test_simplified_scheme_reaches_the_same_balance(g):
    """Both Picard schemes stop at force balance with e = e_l + dt edot (the general
    one by its closure, the simplified one through the predictor and Eq. 2.22), so on
    every step where both converge their states agree to the balance tolerance."""
    from paper_2511_06824_gb300 import dynamics
    nth, nz, steps = 48, 24, 6
    phys = inputs.phys_vector()
    tex = inputs.dimple_texture(np.random.default_rng(4))
    prof = inputs.trapezoid_pressure_profile(np.random.default_rng(3), 360)
    st0 = np.array([2e-6, -1e-6, 3e-6, 1e-6, 0, 0, 0, 0.0])
    opts = g.solver_opts(eps=1e-12, precision=0)
    with g.Context() as c:
        gen = dynamics.march(c.handle, nth, nz, phys, tex, st0, prof, steps, kappa=0.2,
                             opts=opts, tol_F=1e-9, scheme="general")
        sim = dynamics.march(c.handle, nth, nz, phys, tex, st0, prof, steps, kappa=0.2,
                             opts=opts, tol_F=1e-9, max_picard=40, scheme="simplified")
    assert all(r.converged for r in gen.records) and all(r.converged for r in sim.records)
    scale = np.abs(gen.states[:, :4]).max()
    assert np.abs(sim.states[:, :4] - gen.states[:, :4]).max() <= 1e-6 * scale
