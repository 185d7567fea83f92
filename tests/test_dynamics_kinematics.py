"""Swash-plate kinematics of the multi-period march (the geometry of Table 8), on
the CPU.

The coupling length is pinned by its dead-centre values (L_Fmin at outer dead
centre, L_Fmin plus the stroke 2 R_b tan(beta) at inner dead centre) and its
symmetry, the sliding speed by being the time derivative of the coupling length
(central difference over the shaft angle at 600 rpm) and by its closed-form peak,
and the march's use of both by running it with the oracle's Picard step: every
shaft step solves on the gap of its angle and balances oil and side load."""
import math

import numpy as np
import pytest

import oracle
from paper_2511_06824_gb300 import dynamics, inputs


def test_coupling_length_at_the_dead_centres():
    k = dynamics.SwashKinematics()
    tb = math.tan(math.radians(10.0))
    assert k.stroke == pytest.approx(2 * 4.05e-2 * tb, rel=1e-15)
    assert k.coupling_length(0.0) == pytest.approx(3e-2, rel=1e-15)
    assert k.coupling_length(math.pi) == pytest.approx(3e-2 + 2 * 4.05e-2 * tb, rel=1e-15)
    for phi in np.linspace(0.0, 2 * math.pi, 37):
        assert k.coupling_length(phi) == pytest.approx(k.coupling_length(2 * math.pi - phi), rel=1e-14)
        assert 3e-2 <= k.coupling_length(phi) <= 3e-2 + k.stroke + 1e-15


def test_sliding_speed_is_the_rate_of_the_coupling_length():
    k = dynamics.SwashKinematics()
    rpm = 600.0
    omega = 2 * math.pi * rpm / 60
    for phi in np.linspace(0.05, 2 * math.pi - 0.05, 23):
        h = 1e-5
        fd = (k.coupling_length(phi + h) - k.coupling_length(phi - h)) / (2 * h) * omega
        assert k.sliding_speed(phi, rpm) == pytest.approx(fd, rel=1e-8, abs=1e-12)
    # peak speed R_b omega tan(beta) at 90 degrees, zero at the dead centres
    assert k.sliding_speed(math.pi / 2, rpm) == pytest.approx(
        4.05e-2 * omega * math.tan(math.radians(10.0)), rel=1e-15)
    assert abs(k.sliding_speed(0.0, rpm)) < 1e-15 and abs(k.sliding_speed(math.pi, rpm)) < 1e-15


def oracle_stepper(scheme, nth, nz, ph, tex, state, e_prev, dt, F_ext, d_e, d_edot, opts):
    assert scheme == "general"
    r = oracle.picard_step(nth, nz, ph, tex, state, e_prev, dt, F_ext, d_e, d_edot, eps=opts.eps)
    assert r["status"] == oracle.OK
    return r


def test_march_solves_each_step_on_the_gap_of_its_angle():
    nth, nz, steps, kappa = 24, 12, 4, 0.2
    phys = inputs.phys_vector()
    tex = inputs.smooth_texture()
    prof = inputs.trapezoid_pressure_profile(np.random.default_rng(3), 360)
    st0 = np.array([2e-6, -1e-6, 3e-6, 1e-6, 1e-5, 0, -2e-5, 0.0])
    kin = dynamics.SwashKinematics()
    opts = type("O", (), {"eps": 1e-12, "precond": 1, "omega": 1.2, "max_iter": 10 ** 5,
                          "precision": 0, "criterion": 0})()
    seen = []

    def recording(scheme, n1, n2, ph, *rest):
        seen.append(ph.copy())
        return oracle_stepper(scheme, n1, n2, ph, *rest)

    traj = dynamics.march(0, nth, nz, phys, tex, st0, prof, steps, kappa=kappa, tol_F=1e-9,
                          opts=opts, mass=0.0, stepper=recording, kinematics=kin)
    assert all(r.converged for r in traj.records)
    dt = (60.0 / 600.0) / 360.0
    prev = st0
    for s, rec in enumerate(traj.records):
        phi = 2 * math.pi * s / 360
        assert rec.gap_length == kin.coupling_length(phi)
        ph = phys.copy()
        ph[1] = kin.coupling_length(phi)
        ph[4] = kin.sliding_speed(phi, 600.0)
        ph[5] = prof[s]
        side = np.array([0, 0, kappa * ph[5] * math.pi * ph[0] ** 2 * math.tan(math.radians(10)), 0])
        r = oracle.picard_step(nth, nz, ph, tex, rec.state, prev[:4], dt, np.zeros(4), 2e-8, 1e-6,
                               eps=1e-12)
        assert np.linalg.norm(r["G"] + side) <= 1e-8 * np.linalg.norm(side)
        prev = rec.state
    # every Picard step of shaft step s ran on that step's gap
    lengths = sorted({round(p[1], 15) for p in seen})
    assert len(lengths) == steps
