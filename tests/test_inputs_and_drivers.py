"""Host logic of the seeded input generators and of the dynamics driver's
synthetic load (no GPU): reproducibility, ranges and the shapes stated for them."""
import math

import numpy as np
import pytest

from paper_2511_06824_gb300 import dynamics, inputs


def test_workloads_are_seeded_and_shaped_as_named():
    a, b = inputs.make("textured-2048x1024-k9", 3), inputs.make("textured-2048x1024-k9", 3)
    assert (a.n_theta, a.n_z, a.n_cond) == (2048, 1024, 9)
    assert np.array_equal(a.state, b.state) and np.array_equal(a.tex, b.tex)
    c = inputs.make("textured-2048x1024-k9", 4)
    assert not np.array_equal(a.state, c.state)
    s = inputs.make("smooth-512x256-k9", 0)
    assert (s.n_theta, s.n_z, s.n_cond) == (512, 256, 9)
    assert np.array_equal(s.tex, inputs.smooth_texture())


def test_random_state_stays_inside_half_the_clearance():
    rng = np.random.default_rng(0)
    c = inputs.phys_vector()[2]
    for _ in range(100):
        st = inputs.random_state(rng)
        assert st.shape == (8,)
        assert np.all(st[:4] >= 0.0) and np.all(st[:4] <= 0.5 * c)
        assert np.all(np.abs(st[4:]) <= 1e-4)


def test_trapezoid_pressure_profile():
    """High plateau over about half a revolution, linear ramps of 10-40 degrees,
    values between the low and the high pressure."""
    for seed in range(5):
        p = inputs.trapezoid_pressure_profile(np.random.default_rng(seed), 360)
        assert p.shape == (360,)
        assert p.min() >= 0.1e6 - 1e-6 and p.max() <= 25e6 + 1e-6
        high = np.sum(p >= 25e6 - 1e-3)
        low = np.sum(p <= 0.1e6 + 1e-3)
        ramps = 360 - high - low
        assert 140 <= high <= 171 and 140 <= low <= 171, (high, low)
        assert 18 <= ramps <= 82
        # consecutive steps change by at most one ramp increment
        d = np.abs(np.diff(np.concatenate([p, p[:1]])))
        assert d.max() <= (25e6 - 0.1e6) / 10.0 + 1.0


def test_serving_stream_is_poisson_and_mixed():
    reqs = inputs.serving_requests(seed=7, count=400, rate_hz=20.0)
    again = inputs.serving_requests(seed=7, count=400, rate_hz=20.0)
    t = np.array([r["arrival_s"] for r in reqs])
    assert np.array_equal(t, [r["arrival_s"] for r in again])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / 20.0) < 0.15 / 20.0          # exponential, mean 1/rate
    assert abs(np.std(gaps) / gaps.mean() - 1.0) < 0.2          # coefficient of variation 1
    grids = {(r["n_theta"], r["n_z"]) for r in reqs}
    assert grids == set(inputs.SERVING_GRIDS)
    textured = np.mean([r["tex"][0] == 1 for r in reqs])
    assert 0.4 < textured < 0.6


def test_side_load_is_the_swash_plate_component_on_e3():
    p, R, kappa = 25e6, 0.01, 0.2
    f = dynamics.side_load(p, R, kappa)
    assert f.shape == (4,)
    assert f[0] == f[1] == f[3] == 0.0
    assert f[2] == pytest.approx(kappa * p * math.pi * R * R * math.tan(math.radians(10.0)))
    assert np.all(dynamics.side_load(p, R, 0.0) == 0.0)
