"""Pins of the CPU oracle against facts fixed by the paper's setup and by mathematics.

Each test names what pins it: a closed form, a brute-force restatement on tiny
inputs, a library routine (numpy's Cholesky / dense solve), or an invariant of
the method.  None of them re-types the oracle's own formula.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2511_06824_gb300 import inputs

PHYS = inputs.phys_vector()
RK, L, C, MU, V, PCH, PCASE = PHYS
SMOOTH = inputs.smooth_texture()


def tex_default(o_theta=1.234e-3, o_z=0.7e-3, depth=5e-6):
    return np.array([1.0, 0.5e-3, depth, 0.2, o_theta, o_z])


def state(e=(0, 0, 0, 0), ed=(0, 0, 0, 0)):
    return np.array(list(e) + list(ed), dtype=np.float64)


def solve_single(nth, nz, phys, tex, st, eps=1e-13, precond=1, omega=1.2):
    s, D, aE, aN, S = oracle.assemble(nth, nz, phys, tex, st)
    assert s == oracle.OK
    status, p, it, rel, trel = oracle.solve_joint(nth, nz, D, aE, aN, S, precond=precond,
                                                  omega=omega, eps=eps)
    assert status == oracle.OK, status
    return p[0], it


# ----------------------------------------------------------------------------- texture


def test_lattice_constants_give_requested_density():
    """Hexagonal lattice: whole number of columns round the piston and exact area density."""
    tex = tex_default()
    ath, az = oracle.lattice(PHYS, tex)
    ncol = 2 * math.pi * RK / ath
    assert abs(ncol - round(ncol)) < 1e-9 and round(ncol) == 30
    assert math.isclose(math.pi * 0.5e-3 ** 2 / (ath * az), 0.2, rel_tol=1e-12)
    # the ideal hexagonal pitch for 20 % would be 2.1295 mm; 30 columns is the nearest
    a0 = 0.5e-3 * math.sqrt(2 * math.pi / (math.sqrt(3) * 0.2))
    assert abs(2 * math.pi * RK / a0 - 30) < 0.5


def _brute_depth(x, z, tex, ath, az, circ):
    """Brute force: every lattice centre in a wide window, periodic distance in x."""
    _, r, depth, _, oth, oz = tex
    for k in range(math.floor(-oz / az) - 3, math.floor((L - oz) / az) + 4):
        zc = oz + k * az
        xs = oth + (0.5 * ath if k % 2 else 0.0)
        for m in range(-3, int(circ / ath) + 4):
            xc = xs + m * ath
            dx = (x - xc) % circ
            dx = min(dx, circ - dx)
            if dx * dx + (z - zc) ** 2 < r * r:
                return depth
    return 0.0


def test_texture_inside_test_matches_brute_force():
    rng = np.random.default_rng(7)
    tex = tex_default(o_theta=rng.uniform(0, 0.06), o_z=rng.uniform(0, 0.04))
    ath, az = oracle.lattice(PHYS, tex)
    circ = 2 * math.pi * RK
    pts = np.column_stack([rng.uniform(0, circ, 400), rng.uniform(0, L, 400)])
    mism = 0
    for x, z in pts:
        a = oracle.texture_depth(PHYS, tex, x, z)
        b = _brute_depth(x, z, tex, ath, az, circ)
        mism += a != b
    assert mism == 0
    # and some inside hits were actually exercised
    hits = sum(oracle.texture_depth(PHYS, tex, x, z) > 0 for x, z in pts)
    assert 40 < hits < 140


def test_texture_area_fraction_is_twenty_percent():
    """Midpoint sampling over whole lattice periods gives the lattice's area density."""
    tex = tex_default(o_theta=0.3e-3, o_z=1.0e-3)
    ath, az = oracle.lattice(PHYS, tex)
    circ = 2 * math.pi * RK
    nx, nzs = 900, 600
    z0, z1 = 1.0e-3, 1.0e-3 + 10 * 2 * az   # 20 rows = whole periods in z
    assert z1 < L
    xs = (np.arange(nx) + 0.5) * circ / nx
    zs = z0 + (np.arange(nzs) + 0.5) * (z1 - z0) / nzs
    inside = 0
    for z in zs:
        for x in xs:
            inside += oracle.texture_depth(PHYS, tex, x, z) > 0
    frac = inside / (nx * nzs)
    assert abs(frac - 0.2) < 3e-3


def test_smooth_is_depth_zero_bitwise():
    st = state((3e-6, -2e-6, 5e-6, 1e-6), (1e-5, -2e-5, 3e-5, 4e-6))
    a = oracle.assemble(32, 16, PHYS, SMOOTH, st)
    b = oracle.assemble(32, 16, PHYS, tex_default(depth=0.0), st)
    c = oracle.assemble(32, 16, PHYS, np.array([0.0, 0.5e-3, 5e-6, 0.2, 1e-3, 1e-3]), st)
    for x, y, z in zip(a[1:], b[1:], c[1:]):
        assert np.array_equal(x, y) and np.array_equal(x, z)


def test_texture_raises_conductance_only_inside_dimples():
    st = state((2e-6, 1e-6, 3e-6, -1e-6))
    tex = tex_default()
    _, D0, aE0, aN0, _ = oracle.assemble(64, 32, PHYS, SMOOTH, st)
    _, D1, aE1, aN1, _ = oracle.assemble(64, 32, PHYS, tex, st)
    assert np.all(aE1 >= aE0) and np.all(aN1 >= aN0)
    frac = np.mean(aE1 > aE0)
    assert 0.1 < frac < 0.3


# ----------------------------------------------------------------------------- film rate


def test_film_rate_is_the_derivative_of_the_film_along_the_rates():
    """Eq. 2.3 with the chain rule: dh/dt = sum_i dh/de_i edot_i.  Pinned by a central
    difference of the film itself along edot, h(e + d edot) - h(e - d edot) over 2 d,
    at seeded points with four distinct rates (a swapped axial split of the rates,
    e1 <-> e3 or e2 <-> e4, changes the result by about |edot_1 - edot_3|)."""
    rng = np.random.default_rng(11)
    worst = 0.0
    for _ in range(50):
        e = rng.uniform(-0.4 * C, 0.4 * C, 4)
        ed = rng.uniform(-1e-4, 1e-4, 4)
        theta = rng.uniform(0.0, 2 * math.pi)
        z = rng.uniform(0.0, L)
        d = 1e-5                                   # d * edot ~ 1e-9 m, well below c
        fd = (oracle.film(PHYS, SMOOTH, e + d * ed, theta, z) -
              oracle.film(PHYS, SMOOTH, e - d * ed, theta, z)) / (2 * d)
        got = oracle.film_rate(PHYS, e, ed, theta, z)
        worst = max(worst, abs(got - fd) / np.abs(ed).max())
    assert worst < 1e-6
    # the texture is static in the piston frame: it changes h, not dh/dt
    e, ed = np.array([3e-6, -2e-6, 5e-6, 1e-6]), np.array([4e-5, -7e-5, 2e-5, 9e-5])
    d = 1e-5
    tex = tex_default()
    for theta, z in [(0.3, 0.011), (2.0, 0.027), (4.4, 0.035)]:
        fd = (oracle.film(PHYS, tex, e + d * ed, theta, z) -
              oracle.film(PHYS, tex, e - d * ed, theta, z)) / (2 * d)
        assert abs(oracle.film_rate(PHYS, e, ed, theta, z) - fd) < 1e-6 * 9e-5


def test_film_rate_splits_the_rates_linearly_along_the_gap():
    """At the chamber end (z = 0) only edot_1, edot_2 move the film, at the case end
    only edot_3, edot_4, and at mid-gap each pair counts half."""
    e = np.array([3e-6, -2e-6, 5e-6, 1e-6])
    for theta in (0.0, 0.7, 1.9, 3.3):
        for k in range(4):
            ed = np.zeros(4)
            ed[k] = 1e-4
            at0 = oracle.film_rate(PHYS, e, ed, theta, 0.0)
            atL = oracle.film_rate(PHYS, e, ed, theta, L)
            if k < 2:
                assert atL == 0.0 and at0 != 0.0
            else:
                assert at0 == 0.0 and atL != 0.0
        # a pure tilt about mid-gap (edot_3 = -edot_1) leaves the mid-gap film still
        ed = np.array([1e-4, -6e-5, -1e-4, 6e-5])
        assert abs(oracle.film_rate(PHYS, e, ed, theta, 0.5 * L)) < 1e-20


# ----------------------------------------------------------------------------- assembly


def test_concentric_closed_form_coefficients():
    """e = 0, edot = 0: h = c everywhere, so a_E, a_N and the Dirichlet terms are closed forms."""
    nth, nz = 48, 20
    s, D, aE, aN, S = oracle.assemble(nth, nz, PHYS, SMOOTH, state())
    assert s == oracle.OK
    dth = 2 * math.pi / nth
    dx, dz = RK * dth, L / nz
    g = C ** 3 / (12 * MU)
    np.testing.assert_allclose(aE, g * dz / dx, rtol=1e-11)
    np.testing.assert_allclose(aN[:-1], g * dx / dz, rtol=1e-11)
    assert np.all(aN[-1] == 0.0)
    aB = g * dx / (dz / 2)
    np.testing.assert_allclose(S[0], aB * PCH, rtol=1e-11)
    np.testing.assert_allclose(S[-1], aB * PCASE, rtol=1e-11)
    assert np.all(S[1:-1] == 0.0)          # no wedge, no squeeze
    np.testing.assert_allclose(D[1:-1], 2 * g * dz / dx + 2 * g * dx / dz, rtol=1e-11)
    np.testing.assert_allclose(D[0], 2 * g * dz / dx + g * dx / dz + aB, rtol=1e-11)


def test_row_sums_are_zero_except_dirichlet_rows():
    st = state((4e-6, -3e-6, 6e-6, 2e-6), (2e-5, 1e-5, -3e-5, 0))
    nth, nz = 40, 24
    s, D, aE, aN, S = oracle.assemble(nth, nz, PHYS, tex_default(), st)
    y = oracle.apply_matrix(nth, nz, D, aE, aN, np.ones(nth * nz)).reshape(nz, nth)
    assert np.all(np.abs(y[1:-1]) <= 1e-12 * D[1:-1])
    assert np.all(y[0] > 0.1 * D[0] / 4) and np.all(y[-1] > 0.1 * D[-1] / 4)


@pytest.mark.parametrize("nth,nz", [(3, 2), (8, 4), (16, 8)])
def test_matrix_symmetric_positive_definite(nth, nz):
    st = state((5e-6, 2e-6, -4e-6, 6e-6), (1e-4, -1e-4, 5e-5, 0))
    s, D, aE, aN, S = oracle.assemble(nth, nz, PHYS, tex_default(), st)
    A = oracle.dense_matrix(nth, nz, D, aE, aN)
    assert np.array_equal(A, A.T)
    np.linalg.cholesky(A)                       # raises if not SPD
    off = np.abs(A - np.diag(np.diag(A))).sum(axis=1)
    assert np.all(np.diag(A) >= off * (1 - 1e-14))


def test_contact_is_reported():
    st = state((1.2 * C, 0, 1.2 * C, 0))
    s, *_ = oracle.assemble(16, 8, PHYS, SMOOTH, st)
    assert s == oracle.CONTACT


# ----------------------------------------------------------------------------- solver


def test_concentric_pressure_is_linear_in_z():
    """Concentric smooth piston: the exact solution is linear in z and the scheme is exact for it."""
    nth, nz = 32, 24
    p, _ = solve_single(nth, nz, PHYS, SMOOTH, state())
    zc = (np.arange(nz) + 0.5) * L / nz
    exact = PCH + (PCASE - PCH) * zc / L
    np.testing.assert_allclose(p, np.repeat(exact[:, None], nth, axis=1), rtol=1e-10)


def test_parallel_eccentric_pressure_is_linear_in_z():
    """e3 = e1, e4 = e2, no squeeze: h depends on theta only, so p is still linear in z."""
    nth, nz = 40, 20
    st = state((6e-6, -4e-6, 6e-6, -4e-6))
    p, _ = solve_single(nth, nz, PHYS, SMOOTH, st)
    zc = (np.arange(nz) + 0.5) * L / nz
    exact = PCH + (PCASE - PCH) * zc / L
    np.testing.assert_allclose(p, np.repeat(exact[:, None], nth, axis=1), rtol=1e-9)


@pytest.mark.parametrize("precond", [0, 1, 2])
def test_pcg_matches_dense_direct_solve(precond):
    nth, nz = 16, 8
    st = state((5e-6, 3e-6, 8e-6, -2e-6), (6e-5, -4e-5, 2e-5, 9e-5))
    s, D, aE, aN, S = oracle.assemble(nth, nz, PHYS, tex_default(), st)
    A = oracle.dense_matrix(nth, nz, D, aE, aN)
    exact = np.linalg.solve(A, S.ravel())
    status, p, it, rel, trel = oracle.solve_joint(nth, nz, D, aE, aN, S, precond=precond,
                                                  eps=1e-14)
    assert status == oracle.OK
    assert np.linalg.norm(p.ravel() - exact) <= 1e-10 * np.linalg.norm(exact)
    assert trel <= 1e-13


def test_joint_solve_is_block_diagonal():
    """Eq. 3.7: the joint system is the direct sum of the per-condition systems."""
    nth, nz = 16, 8
    rng = np.random.default_rng(3)
    states = [inputs.random_state(rng) for _ in range(3)]
    s, D, aE, aN, S = oracle.assemble_joint(nth, nz, PHYS, tex_default(), states)
    status, p, *_ = oracle.solve_joint(nth, nz, D, aE, aN, S, eps=1e-14)
    assert status == oracle.OK
    for k in range(3):
        A = oracle.dense_matrix(nth, nz, D[k], aE[k], aN[k])
        exact = np.linalg.solve(A, S[k].ravel())
        assert np.linalg.norm(p[k].ravel() - exact) <= 1e-10 * np.linalg.norm(exact)


def _dense_assor(A, omega):
    """M^-1 of Eq. 3.4 written with dense numpy factors (L = strict lower triangle)."""
    Dm = np.diag(np.diag(A))
    Di = np.diag(1.0 / np.diag(A))
    Lt = np.tril(A, -1)
    I = np.eye(A.shape[0])
    # (2 - w) w D^-1 (I - w L^T D^-1) D (I - w D^-1 L) D^-1
    return (2 - omega) * omega * Di @ (I - omega * Lt.T @ Di) @ Dm @ (I - omega * Di @ Lt) @ Di


@pytest.mark.parametrize("omega", [0.6, 1.0, 1.2, 1.8])
def test_assor_apply_matches_dense_definition_and_is_spd(omega):
    nth, nz = 8, 5
    rng = np.random.default_rng(11)
    states = [inputs.random_state(rng) for _ in range(2)]
    s, D, aE, aN, S = oracle.assemble_joint(nth, nz, PHYS, tex_default(), states)
    n = nth * nz
    Minv = np.zeros((2 * n, 2 * n))
    for k in range(2):
        A = oracle.dense_matrix(nth, nz, D[k], aE[k], aN[k])
        Minv[k * n:(k + 1) * n, k * n:(k + 1) * n] = _dense_assor(A, omega)
    r = rng.standard_normal(2 * n)
    z = oracle.apply_precond(nth, nz, D, aE, aN, r, precond=1, omega=omega)
    np.testing.assert_allclose(z, Minv @ r, rtol=1e-12, atol=1e-12 * np.abs(Minv @ r).max())
    # columns of the oracle's operator: symmetric positive definite
    cols = np.column_stack([oracle.apply_precond(nth, nz, D, aE, aN, np.eye(2 * n)[:, j],
                                                 precond=1, omega=omega) for j in range(2 * n)])
    assert np.allclose(cols, cols.T, rtol=1e-12, atol=1e-12 * np.abs(cols).max())
    assert np.linalg.eigvalsh(0.5 * (cols + cols.T)).min() > 0
    zj = oracle.apply_precond(nth, nz, D, aE, aN, r, precond=0)
    np.testing.assert_array_equal(zj, r / D.ravel())


@pytest.mark.parametrize("omega", [0.6, 1.2, 1.8])
def test_assor1_is_the_diagonal_of_the_dense_ssor_product(omega):
    """Eq. 3.2: {M^-1}_ii = w (2 - w) / {(D + w L) D^-1 (D + w L)^T}_ii, written with
    dense numpy factors (L = strict lower triangle in the joint index order, so the
    periodic couplings of column n_theta - 1 to column 0 are lower, those of column 0
    to column n_theta - 1 upper)."""
    nth, nz = 7, 5
    rng = np.random.default_rng(17)
    states = [inputs.random_state(rng) for _ in range(2)]
    s, D, aE, aN, S = oracle.assemble_joint(nth, nz, PHYS, tex_default(), states)
    n = nth * nz
    r = rng.standard_normal(2 * n)
    want = np.empty(2 * n)
    for k in range(2):
        A = oracle.dense_matrix(nth, nz, D[k], aE[k], aN[k])
        Dm = np.diag(np.diag(A))
        B = Dm + omega * np.tril(A, -1)
        diag = np.diag(B @ np.linalg.inv(Dm) @ B.T)
        want[k * n:(k + 1) * n] = omega * (2 - omega) * r[k * n:(k + 1) * n] / diag
    z = oracle.apply_precond(nth, nz, D, aE, aN, r, precond=2, omega=omega)
    np.testing.assert_allclose(z, want, rtol=1e-13, atol=0)
    # a wrong lower set (e.g. the west neighbour of column 0 counted as lower) would
    # change row 0 of each block: check that the first rows see only their south
    # neighbour and the last column its west and wrapped east neighbours
    assert not np.allclose(want, omega * (2 - omega) * r / D.ravel())


def test_assor_needs_fewer_iterations_than_jacobi_and_agrees():
    """Qualitative claim of Table 2 / Fig. 2a: ASSOR-II needs far fewer iterations."""
    nth, nz = 64, 32
    st = state((6e-6, 2e-6, 9e-6, -3e-6), (5e-5, -5e-5, 2e-5, 1e-5))
    pa, ia = solve_single(nth, nz, PHYS, tex_default(), st, eps=1e-12, precond=1, omega=1.6)
    pj, ij = solve_single(nth, nz, PHYS, tex_default(), st, eps=1e-12, precond=0)
    assert ia < 0.8 * ij
    assert np.linalg.norm(pa - pj) <= 1e-8 * np.linalg.norm(pj)


def test_warm_start_and_restart_semantics():
    nth, nz = 16, 8
    st = state((5e-6, 3e-6, 8e-6, -2e-6), (6e-5, -4e-5, 2e-5, 9e-5))
    s, D, aE, aN, S = oracle.assemble(nth, nz, PHYS, SMOOTH, st)
    status, p, it, rel, trel = oracle.solve_joint(nth, nz, D, aE, aN, S, eps=1e-12)
    assert status == oracle.OK and it > 0
    # already converged guess: zero iterations
    status2, p2, it2, *_ = oracle.solve_joint(nth, nz, D, aE, aN, S, p0=p, eps=1e-10)
    assert status2 == oracle.OK and it2 == 0 and np.array_equal(p2, p)
    # budget too small
    status3, *_ = oracle.solve_joint(nth, nz, D, aE, aN, S, eps=1e-12, max_iter=3)
    assert status3 == oracle.NOT_CONVERGED
    # zero right-hand side
    status4, p4, it4, *_ = oracle.solve_joint(nth, nz, D, aE, aN, np.zeros_like(S), eps=1e-12)
    assert status4 == oracle.OK and it4 == 0 and not p4.any()
    # invalid relaxation factor
    status5, *_ = oracle.solve_joint(nth, nz, D, aE, aN, S, omega=2.0)
    assert status5 == oracle.INVALID


# ----------------------------------------------------------------------------- closed forms through the whole chain


def _cosmode_integral(K_over_g):
    """Solution of P'' - P/R^2 = k with P(0) = P(L) = 0: returns (integral of P over [0, L])."""
    k = K_over_g
    # P = -k R^2 (1 - cosh((z - L/2)/R) / cosh(L/(2R)))
    return -k * RK ** 2 * (L - 2 * RK * math.tanh(L / (2 * RK)))


def _cosmode_fx(nth, nz, st, phys=PHYS):
    p, _ = solve_single(nth, nz, phys, SMOOTH, st, eps=1e-13)
    s, ld = oracle.loads(nth, nz, phys, SMOOTH, st, p)
    assert s == oracle.OK
    return ld


def test_squeeze_film_closed_form():
    """Concentric piston translating at edot_x: linearised Reynolds gives P(z) cos(theta)
    with g (P'' - P/R^2) = -a, so Fx = -pi R integral(P)."""
    a = 1e-4
    st = state((0, 0, 0, 0), (a, 0, a, 0))
    g = C ** 3 / (12 * MU)
    fx_exact = -math.pi * RK * _cosmode_integral(-a / g)
    errs = []
    for nth, nz in [(64, 32), (128, 64)]:
        ld = _cosmode_fx(nth, nz, st)
        errs.append(abs(ld[0] - fx_exact) / abs(fx_exact))
        assert abs(ld[1]) < 1e-9 * abs(ld[0])
        # pressure moment about y: symmetric P gives My = (L/2) Fx
        assert math.isclose(ld[4], 0.5 * L * ld[0], rel_tol=1e-9)
    assert fx_exact < 0                      # film squeezed at theta = 0 pushes back
    assert errs[1] < 2e-3
    assert 3.0 < errs[0] / errs[1] < 5.0      # second-order scheme


def test_wedge_film_closed_form():
    """Small axial tilt ex = delta (2z/L - 1) with sliding: first-order Reynolds gives
    g0 (P1'' - P1/R^2) = K with K = ex' (-U_b/2 + 3 g0 p0'/c)."""
    delta = 1e-4 * C
    st = state((-delta, 0, delta, 0))
    g0 = C ** 3 / (12 * MU)
    exd = 2 * delta / L
    Ub = -V
    p0d = (PCASE - PCH) / L
    K = exd * (-Ub / 2 + 3 * g0 * p0d / C)
    fx_exact = -math.pi * RK * _cosmode_integral(K / g0)
    errs = []
    for nth, nz in [(64, 32), (128, 64)]:
        ld = _cosmode_fx(nth, nz, st)
        errs.append(abs(ld[0] - fx_exact) / abs(fx_exact))
    assert errs[1] < 3e-3
    assert errs[1] < errs[0]


def test_concentric_loads():
    """Concentric: radial forces and all moments vanish; Fz_shear is a closed form."""
    nth, nz = 64, 32
    p, _ = solve_single(nth, nz, PHYS, SMOOTH, state())
    s, ld = oracle.loads(nth, nz, PHYS, SMOOTH, state(), p)
    scale = PCH * 2 * math.pi * RK * L
    for k in (0, 1, 3, 4, 5, 6, 7, 9, 10, 11):
        assert abs(ld[k]) < 1e-12 * scale
    assert ld[2] == 0.0
    Ub = -V
    fz = 2 * math.pi * RK * L * (-(C / 2) * (PCASE - PCH) / L + MU * Ub / C)
    assert math.isclose(ld[8], fz, rel_tol=1e-10)


def test_loads_converge_at_second_order():
    st = state((6e-6, -3e-6, 2e-6, 5e-6), (3e-5, 1e-5, -2e-5, 4e-5))
    res = []
    for nth, nz in [(32, 16), (64, 32), (128, 64)]:
        p, _ = solve_single(nth, nz, PHYS, SMOOTH, st, eps=1e-13)
        res.append(oracle.loads(nth, nz, PHYS, SMOOTH, st, p)[1])
    for k in (0, 1, 4, 3, 8):
        d1 = res[0][k] - res[1][k]
        d2 = res[1][k] - res[2][k]
        assert 2.8 < d1 / d2 < 5.5, (k, d1 / d2)


def test_mirror_symmetry_of_loads():
    """y -> -y: Fy, Mx, Mz change sign; Fx, Fz, My do not."""
    nth, nz = 48, 24
    st = state((6e-6, 3e-6, 2e-6, 5e-6), (3e-5, 1e-5, -2e-5, 4e-5))
    stm = st * np.array([1, -1, 1, -1, 1, -1, 1, -1])
    p, _ = solve_single(nth, nz, PHYS, SMOOTH, st)
    pm, _ = solve_single(nth, nz, PHYS, SMOOTH, stm)
    ld = oracle.loads(nth, nz, PHYS, SMOOTH, st, p)[1]
    lm = oracle.loads(nth, nz, PHYS, SMOOTH, stm, pm)[1]
    sign = np.array([1, -1, 1, -1, 1, -1] * 2)
    scale = np.abs(ld).max()
    np.testing.assert_allclose(lm, sign * ld, rtol=1e-8, atol=1e-9 * scale)
    # pressure field mirrors: theta_i -> theta_{nth-1-i}
    np.testing.assert_allclose(pm, p[:, ::-1], rtol=1e-9, atol=1e-9 * np.abs(p).max())


def test_rotation_by_whole_cells():
    nth, nz, m = 48, 24, 5
    st = state((6e-6, 3e-6, 2e-6, 5e-6), (3e-5, 1e-5, -2e-5, 4e-5))
    phi = m * 2 * math.pi / nth
    R = np.array([[math.cos(phi), -math.sin(phi)], [math.sin(phi), math.cos(phi)]])
    rot = st.copy()
    for a, b in ((0, 1), (2, 3), (4, 5), (6, 7)):
        rot[[a, b]] = R @ st[[a, b]]
    p, _ = solve_single(nth, nz, PHYS, SMOOTH, st)
    pr, _ = solve_single(nth, nz, PHYS, SMOOTH, rot)
    np.testing.assert_allclose(pr, np.roll(p, m, axis=1), rtol=1e-8, atol=1e-9 * np.abs(p).max())
    ld = oracle.loads(nth, nz, PHYS, SMOOTH, st, p)[1]
    lr = oracle.loads(nth, nz, PHYS, SMOOTH, rot, pr)[1]
    scale = np.abs(ld).max()
    for off in (0, 6):
        np.testing.assert_allclose(lr[off:off + 2], R @ ld[off:off + 2], atol=1e-8 * scale)
        np.testing.assert_allclose(lr[off + 3:off + 5], R @ ld[off + 3:off + 5], atol=1e-8 * scale)
        assert abs(lr[off + 2] - ld[off + 2]) < 1e-8 * scale


def _virtual_work_of_pressure(nth, nz, p):
    """Generalized force of the pressure on the linear tilt, computed independently
    of the oracle's loads: the virtual displacement of the surface point at axial
    position z is (1 - z/L) de_1 + (z/L) de_3 along x (likewise e_2, e_4 along y), so
    G = integral of f . dx/de over the gap with traction f = -p n, n = (cos t, sin t).
    Nodes: cell centres plus the two boundary lines; numpy's trapezoid along z on
    those nodes, the periodic trapezoid (a plain sum) around theta."""
    dth = 2 * math.pi / nth
    dz = L / nz
    th = (np.arange(nth) + 0.5) * dth
    zn = np.concatenate([[0.0], (np.arange(nz) + 0.5) * dz, [L]])
    P = np.vstack([np.full(nth, PCH), p.reshape(nz, nth), np.full(nth, PCASE)])
    fx = -P * np.cos(th)[None, :]
    fy = -P * np.sin(th)[None, :]
    lo = (1.0 - zn / L)[:, None]
    hi = (zn / L)[:, None]

    def integ(f):
        return RK * dth * np.trapezoid(f.sum(axis=1), zn)

    return np.array([integ(fx * lo), integ(fy * lo), integ(fx * hi), integ(fy * hi)])


def test_generalized_force_is_the_virtual_work_of_the_pressure():
    """S19 reading of Eq. 2.11: G = (Fx - My/L, Fy + Mx/L, My/L, -Mx/L) is exactly the
    virtual work of the linear tilt when the traction has no axial part, as for the
    pressure.  Pinned against the virtual work integrated directly from the pressure
    field (no forces or moments involved), on a tilted, eccentric, squeezing piston."""
    nth, nz = 48, 24
    st = state((6e-6, -3e-6, 2e-6, 5e-6), (3e-5, 1e-5, -2e-5, 4e-5))
    p, _ = solve_single(nth, nz, PHYS, tex_default(), st)
    s, ld = oracle.loads(nth, nz, PHYS, tex_default(), st, p)
    assert s == oracle.OK
    G = oracle.generalized_force(L, ld[:6])
    vw = _virtual_work_of_pressure(nth, nz, p)
    scale = np.abs(vw).max()
    assert scale > 1.0
    np.testing.assert_allclose(G, vw, rtol=0, atol=1e-10 * scale)
    # components of comparable size, so that a flipped sign could not hide
    assert np.all(np.abs(vw) > 1e-3 * scale)


def test_symmetric_squeeze_loads_both_ends_equally():
    """Parallel squeeze of a concentric piston (edot_1 = edot_3): the pressure mode is
    symmetric about mid-gap, so the generalized force splits Fx evenly between the two
    ends, G_1 = G_3 = Fx / 2, and nothing acts along y."""
    a = 1e-4
    st = state((0, 0, 0, 0), (a, 0, a, 0))
    nth, nz = 64, 32
    p, _ = solve_single(nth, nz, PHYS, SMOOTH, st, eps=1e-13)
    s, ld = oracle.loads(nth, nz, PHYS, SMOOTH, st, p)
    F = ld[:6] + ld[6:]
    G = oracle.generalized_force(L, F)
    assert abs(G[0] - 0.5 * F[0]) <= 1e-6 * abs(F[0])
    assert abs(G[2] - 0.5 * F[0]) <= 1e-6 * abs(F[0])
    assert abs(G[1]) <= 1e-9 * abs(F[0]) and abs(G[3]) <= 1e-9 * abs(F[0])


# ----------------------------------------------------------------------------- Jacobian and Picard


def _total(ld):
    return ld[:6] + ld[6:]


def test_edot_jacobian_is_exact_difference():
    """edot enters only the source, linearly: p and the loads are affine in edot, so the
    forward difference equals a central difference with a different step."""
    nth, nz = 32, 16
    st = state((6e-6, -3e-6, 2e-6, 5e-6), (3e-5, 1e-5, -2e-5, 4e-5))
    res = oracle.picard_step(nth, nz, PHYS, SMOOTH, st, st[:4], 1e-4, np.zeros(4), 2e-8, 1e-6,
                             eps=1e-13)
    assert res["status"] == oracle.OK
    for j in range(4):
        h = 7e-6
        lo, hi = st.copy(), st.copy()
        lo[4 + j] -= h / 2
        hi[4 + j] += h / 2
        pl, _ = solve_single(nth, nz, PHYS, SMOOTH, lo)
        ph, _ = solve_single(nth, nz, PHYS, SMOOTH, hi)
        fl = _total(oracle.loads(nth, nz, PHYS, SMOOTH, lo, pl)[1])
        fh = _total(oracle.loads(nth, nz, PHYS, SMOOTH, hi, ph)[1])
        central = (fh - fl) / h
        col = res["J"][:, 4 + j]
        np.testing.assert_allclose(col, central, rtol=1e-5, atol=1e-6 * np.abs(central).max())


def test_e_jacobian_forward_difference_is_first_order():
    nth, nz = 32, 16
    st = state((6e-6, -3e-6, 2e-6, 5e-6), (3e-5, 1e-5, -2e-5, 4e-5))
    cols = []
    for de in (4e-8, 2e-8):
        r = oracle.picard_step(nth, nz, PHYS, SMOOTH, st, st[:4], 1e-4, np.zeros(4), de, 1e-6,
                               eps=1e-13)
        cols.append(r["J"][:, :4])
    # central reference for e1
    h = 1e-8
    lo, hi = st.copy(), st.copy()
    lo[0] -= h
    hi[0] += h
    pl, _ = solve_single(nth, nz, PHYS, SMOOTH, lo)
    ph, _ = solve_single(nth, nz, PHYS, SMOOTH, hi)
    central = (_total(oracle.loads(nth, nz, PHYS, SMOOTH, hi, ph)[1]) -
               _total(oracle.loads(nth, nz, PHYS, SMOOTH, lo, pl)[1])) / (2 * h)
    e1 = np.abs(cols[0][:, 0] - central)
    e2 = np.abs(cols[1][:, 0] - central)
    big = np.abs(central) > 1e-2 * np.abs(central).max()
    ratio = e1[big] / e2[big]
    assert np.all((ratio > 1.6) & (ratio < 2.4)), ratio


def test_picard_fixed_point_concentric():
    nth, nz = 32, 16
    st = state()
    r = oracle.picard_step(nth, nz, PHYS, SMOOTH, st, st[:4], 2.78e-4, np.zeros(4), 2e-8, 1e-6,
                           eps=1e-13)
    assert r["status"] == oracle.OK
    assert np.abs(r["G"]).max() < 1e-9
    assert np.abs(r["state"]).max() < 1e-15


def test_picard_update_solves_the_linearisation():
    """The returned update equals numpy's dense solve of Eq. 2.12 with the backward-Euler
    closure, built from the returned Jacobian and generalized force."""
    nth, nz = 32, 16
    st = state((6e-6, -3e-6, 2e-6, 5e-6), (3e-5, 1e-5, -2e-5, 4e-5))
    e_prev = st[:4] - 1e-7
    dt = 2.78e-4
    Fext = np.array([30.0, -20.0, 5.0, 8.0])
    r = oracle.picard_step(nth, nz, PHYS, SMOOTH, st, e_prev, dt, Fext, 2e-8, 1e-6, eps=1e-13)
    J = r["J"]
    T = np.array([[1, 0, 0, 0, -1 / L, 0], [0, 1, 0, 1 / L, 0, 0], [0, 0, 0, 0, 1 / L, 0],
                  [0, 0, 0, -1 / L, 0, 0]])
    Je, Jd = T @ J[:, :4], T @ J[:, 4:]
    G = T @ _total(r["loads"]) + Fext
    np.testing.assert_allclose(r["G"], G, rtol=1e-12, atol=1e-9)
    gap = e_prev + dt * st[4:] - st[:4]
    delta = np.linalg.solve(Jd + dt * Je, -G - Je @ gap)
    np.testing.assert_allclose(r["state"][4:], st[4:] + delta, rtol=1e-9, atol=1e-15)
    np.testing.assert_allclose(r["state"][:4], e_prev + dt * r["state"][4:], rtol=1e-12)


def test_picard_iteration_converges_to_force_balance():
    nth, nz = 32, 16
    st = state((2e-6, 1e-6, 2e-6, 1e-6))
    e_prev = st[:4].copy()
    dt = 2.78e-4
    Fext = np.array([40.0, -25.0, 10.0, -5.0])
    norms = []
    for _ in range(5):
        r = oracle.picard_step(nth, nz, PHYS, SMOOTH, st, e_prev, dt, Fext, 2e-8, 1e-6,
                               eps=1e-13)
        assert r["status"] == oracle.OK
        norms.append(np.linalg.norm(r["G"]))
        st = r["state"]
    assert norms[-1] < 1e-6 * norms[0]


def test_simplified_picard_jacobian_matches_general_scheme_columns():
    """Eq. 2.20-2.22 solve only the base and the 4 rate perturbations: their load
    Jacobian columns equal the rate columns of the general (9-condition) step, and the
    e-columns are not formed."""
    nth, nz = 32, 16
    st = state((6e-6, -3e-6, 2e-6, 5e-6), (3e-5, 1e-5, -2e-5, 4e-5))
    dt = 2.78e-4
    Fext = np.array([30.0, -20.0, 5.0, 8.0])
    rg = oracle.picard_step(nth, nz, PHYS, SMOOTH, st, st[:4] - 1e-7, dt, Fext, 2e-8, 1e-6,
                            eps=1e-13)
    rs = oracle.picard_step_simplified(nth, nz, PHYS, SMOOTH, st, dt, Fext, 1e-6, eps=1e-13)
    assert rs["status"] == oracle.OK and rg["status"] == oracle.OK
    colscale = np.abs(rg["J"][:, 4:]).max(axis=0, keepdims=True)
    assert np.max(np.abs(rs["J"][:, 4:] - rg["J"][:, 4:]) / colscale) <= 1e-9
    assert not np.any(rs["J"][:, :4])
    np.testing.assert_allclose(rs["loads"], rg["loads"], rtol=1e-10, atol=1e-10)


def test_simplified_picard_update_follows_eqs_2_21_2_22():
    """edot_new = edot - Jd^-1 G (Eq. 2.21) and e_new = e + dt (edot_new - edot)
    (Eq. 2.22), rebuilt with numpy from the returned Jacobian and generalized force."""
    nth, nz = 32, 16
    st = state((6e-6, -3e-6, 2e-6, 5e-6), (3e-5, 1e-5, -2e-5, 4e-5))
    dt = 2.78e-4
    Fext = np.array([30.0, -20.0, 5.0, 8.0])
    r = oracle.picard_step_simplified(nth, nz, PHYS, SMOOTH, st, dt, Fext, 1e-6, eps=1e-13)
    T = np.array([[1, 0, 0, 0, -1 / L, 0], [0, 1, 0, 1 / L, 0, 0], [0, 0, 0, 0, 1 / L, 0],
                  [0, 0, 0, -1 / L, 0, 0]])
    Jd = T @ r["J"][:, 4:]
    G = T @ _total(r["loads"]) + Fext
    np.testing.assert_allclose(r["G"], G, rtol=1e-12, atol=1e-9)
    delta = np.linalg.solve(Jd, -G)
    np.testing.assert_allclose(r["state"][4:], st[4:] + delta, rtol=1e-9, atol=1e-15)
    np.testing.assert_allclose(r["state"][:4], st[:4] + dt * delta, rtol=1e-9, atol=1e-18)


def test_simplified_picard_iteration_reaches_force_balance():
    """At a fixed point of Eq. 2.21 the update is zero, so the generalized force is."""
    nth, nz = 32, 16
    st = state((2e-6, 1e-6, 2e-6, 1e-6))
    dt = 2.78e-4
    Fext = np.array([40.0, -25.0, 10.0, -5.0])
    norms = []
    for _ in range(6):
        r = oracle.picard_step_simplified(nth, nz, PHYS, SMOOTH, st, dt, Fext, 1e-6, eps=1e-13)
        assert r["status"] == oracle.OK
        norms.append(np.linalg.norm(r["G"]))
        st = r["state"]
    assert norms[-1] < 1e-9 * norms[0]
