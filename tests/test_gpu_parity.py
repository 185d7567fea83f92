"""GPU vs oracle parity through the C ABI (needs a GB300 and the built library).

Tolerances (FP64 mode): coefficients rtol 1e-11 (the film thickness is a
difference of two ~R_k numbers, so ~3e-14 relative; cubed and divided it stays
below 1e-12; cos/sin may differ by an ulp between libm and CUDA), sources rtol
1e-9 against the interior scale (h_n - h_s is a further cancellation of
~1e-3), pressure relative L2 1e-9 and loads 1e-7 normalised by
max(|F_c|, 1e-3 ||F||).  Mixed mode: pressure 1e-6, loads 1e-5.
"""
import numpy as np
import pytest

import oracle
from paper_2511_06824_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PHYS = inputs.phys_vector()


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_06824_gb300 import build, gmaf
    build.build()
    gmaf.load()
    return gmaf


@pytest.fixture(scope="module")
def ctx(g):
    c = g.Context()
    yield c.handle
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()


def zeros(n):
    return torch.zeros(n, dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def tex_dimples(seed=5):
    return inputs.dimple_texture(np.random.default_rng(seed))


def states(K, seed=1):
    rng = np.random.default_rng(seed)
    return [inputs.random_state(rng) for _ in range(K)]


def load_err(a, b):
    a, b = np.asarray(a), np.asarray(b)
    out = 0.0
    for part in (slice(0, 6), slice(6, 12)):
        x, y = a[..., part], b[..., part]
        nrm = np.linalg.norm(y, axis=-1, keepdims=True)
        scale = np.maximum(np.abs(y), 1e-3 * nrm)
        out = max(out, float(np.max(np.abs(x - y) / scale)))
    return out


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def gpu_assemble(g, ctx, nth, nz, tex, conds, allow_contact=False):
    K = len(conds)
    n = K * nth * nz
    D, aE, aN, S = zeros(n), zeros(n), zeros(n), zeros(n)
    st = g.gmaf_assemble(ctx, nth, nz, PHYS, tex, conds, D, aE, aN, S, allow_contact=allow_contact)
    sh = (K, nz, nth)
    return st, host(D).reshape(sh), host(aE).reshape(sh), host(aN).reshape(sh), host(S).reshape(sh)


# ----------------------------------------------------------------------------- assembly


@pytest.mark.parametrize("nth,nz,K,textured", [(64, 32, 1, False), (100, 37, 3, True),
                                               (3, 2, 2, True), (512, 256, 2, True),
                                               (129, 17, 9, False)])
def test_assembly_matches_oracle(g, ctx, nth, nz, K, textured):
    tex = tex_dimples() if textured else inputs.smooth_texture()
    conds = states(K, seed=nth)
    st, D, aE, aN, S = gpu_assemble(g, ctx, nth, nz, tex, conds)
    so, Do, aEo, aNo, So = oracle.assemble_joint(nth, nz, PHYS, tex, conds)
    assert st == 0 and so == 0
    np.testing.assert_allclose(aE, aEo, rtol=1e-11)
    np.testing.assert_allclose(aN, aNo, rtol=1e-11, atol=0)
    np.testing.assert_allclose(D, Do, rtol=1e-11)
    scale = np.abs(So[:, 1:-1]).max() if nz > 2 else np.abs(So).max()
    np.testing.assert_allclose(S, So, rtol=1e-9, atol=1e-9 * scale)


def test_texture_decisions_are_identical(g, ctx):
    """Dimple membership is an integer decision: the conductance jumps by (1 + depth/h)^3,
    so any disagreement would show as an O(1) relative error."""
    nth, nz = 2048, 64
    tex = tex_dimples(seed=9)
    conds = states(1, seed=2)
    _, _, aE, aN, _ = gpu_assemble(g, ctx, nth, nz, tex, conds)
    _, _, aEo, aNo, _ = oracle.assemble_joint(nth, nz, PHYS, tex, conds)
    assert np.max(np.abs(aE / aEo - 1)) < 1e-11
    assert np.max(np.abs(aN[:, :-1] / aNo[:, :-1] - 1)) < 1e-11


def test_contact_is_reported(g, ctx):
    c = inputs.CLEARANCE
    st, *_ = gpu_assemble(g, ctx, 16, 8, inputs.smooth_texture(),
                          [np.array([1.2 * c, 0, 1.2 * c, 0, 0, 0, 0, 0])], allow_contact=True)
    assert st == g.GMAF_CONTACT


# ----------------------------------------------------------------------------- solver


def solve_both(g, ctx, nth, nz, tex, conds, precond=1, omega=1.2, eps=1e-10, precision=0):
    so, D, aE, aN, S = oracle.assemble_joint(nth, nz, PHYS, tex, conds)
    K = len(conds)
    n = K * nth * nz
    p = zeros(n)
    opts = g.solver_opts(precond=precond, omega=omega, eps=eps, precision=precision)
    st, it, rel = g.gmaf_solve_joint(ctx, nth, nz, K, dev(D), dev(aE), dev(aN), dev(S), p, opts)
    sto, po, ito, relo, trelo = oracle.solve_joint(nth, nz, D, aE, aN, S, precond=precond,
                                                   omega=omega, eps=eps)
    assert sto == 0
    return host(p).reshape(K, nz, nth), it, rel, po, ito, (D, aE, aN, S)


@pytest.mark.parametrize("nth,nz,K,textured,precond", [
    (64, 32, 1, False, 1),        # single condition, smooth
    (130, 45, 9, True, 1),        # joint batch, ragged tiles, textured
    (96, 40, 4, False, 0),        # Jacobi
    (3, 2, 1, False, 1),          # smallest grid
    (257, 9, 2, True, 1),         # one tile row, ragged in theta
    (130, 45, 9, True, 2),        # ASSOR-I (Eq. 3.2)
    (3, 2, 2, False, 2),          # ASSOR-I, smallest grid (every column touches the wrap)
])
def test_fp64_solve_matches_oracle(g, ctx, nth, nz, K, textured, precond):
    tex = tex_dimples() if textured else inputs.smooth_texture()
    conds = states(K, seed=nth + nz)
    p, it, rel, po, ito, _ = solve_both(g, ctx, nth, nz, tex, conds, precond=precond)
    assert rel <= 1e-9
    assert abs(it - ito) <= 2, (it, ito)
    assert rel_l2(p, po) <= 1e-9


def test_fp64_iterates_track_the_oracle_tightly(g, ctx):
    """Same algorithm, same ordering of steps: iteration counts agree and the
    solutions agree far below the tolerance at a tight criterion."""
    conds = states(9, seed=4)
    p, it, rel, po, ito, _ = solve_both(g, ctx, 200, 60, tex_dimples(), conds, eps=1e-12)
    assert abs(it - ito) <= 1
    assert rel_l2(p, po) <= 1e-11


@pytest.mark.parametrize("nth,nz,K,precond", [(64, 32, 1, 1), (130, 45, 9, 1), (132, 40, 9, 2),
                                              (96, 40, 4, 0)])
def test_mixed_precision_solve_matches_fp64_oracle(g, ctx, nth, nz, K, precond):
    conds = states(K, seed=7)
    p, it, rel, po, ito, arrs = solve_both(g, ctx, nth, nz, tex_dimples(), conds, precision=1,
                                           precond=precond)
    assert rel <= 1e-10
    assert rel_l2(p, po) <= 1e-6
    info = g.gmaf_last_solve_info(ctx)
    assert info["outer_iterations"] >= 2


@pytest.mark.parametrize("restart,delta", [("1", "0.1"), ("0", "0.1"), ("0", "0.3"), ("0", "0.001")])
def test_mixed_refinement_modes_match_fp64_oracle(g, monkeypatch, restart, delta):
    """FP64 refinement around the FP32 PCG, both ways: restarting the inner solve
    from each FP64 residual, and continuing its recurrence with the FP64 residual
    swapped in (reliable updates every reduction by delta)."""
    monkeypatch.setenv("GMAF_MIXED_RESTART", restart)
    monkeypatch.setenv("GMAF_RELIABLE_DELTA", delta)
    nth, nz, K = 132, 45, 9
    conds = states(K, seed=19)
    c = g.Context()
    try:
        p, it, rel, po, ito, _ = solve_both(g, c.handle, nth, nz, tex_dimples(), conds, precision=1)
        info = g.gmaf_last_solve_info(c.handle)
    finally:
        c.close()
    assert rel <= 1e-10
    assert rel_l2(p, po) <= 1e-6
    assert info["outer_iterations"] >= 2
    # the continued recurrence needs about the FP64 iteration count
    if restart == "0" and delta != "0.001":
        assert it <= 1.1 * ito + 10, (it, ito)


@pytest.mark.parametrize("n_iter", [1, 2, 3, 4, 5, 8, 9])
def test_truncated_mixed_solve_matches_oracle_iterate(g, monkeypatch, n_iter):
    """Stopped after n_iter PCG iterations (budget), the mixed solve's p is the
    oracle's PCG iterate p_n to FP32 accuracy.  The staged FP32 phase A adds the p
    updates two at a time, so odd and even n end with one or two updates still
    pending for the finalize kernel; a lost or doubled update would be an O(1) error."""
    monkeypatch.setenv("GMAF_VARIANT", "604322")
    nth, nz, K = 260, 70, 3
    conds = states(K, seed=23)
    so, D, aE, aN, S = oracle.assemble_joint(nth, nz, PHYS, tex_dimples(), conds)
    p = zeros(K * nth * nz)
    c = g.Context()
    try:
        opts = g.solver_opts(eps=1e-10, precision=1, max_iter=n_iter)
        st, it, rel = g.gmaf_solve_joint(c.handle, nth, nz, K, dev(D), dev(aE), dev(aN), dev(S), p,
                                         opts, allow_not_converged=True)
        info = g.gmaf_last_solve_info(c.handle)
    finally:
        c.close()
    assert st == -3 and it == n_iter
    assert info["kernel_variant"] == 604322 and info["p_update_period"] == 2
    sto, po, ito, _, _ = oracle.solve_joint(nth, nz, D, aE, aN, S, eps=1e-10, max_iter=n_iter)
    assert ito == n_iter
    assert rel_l2(host(p).reshape(K, nz, nth), po) <= 1e-5


def test_warm_start_zero_rhs_budget_and_invalid(g, ctx):
    nth, nz = 64, 32
    conds = states(2, seed=3)
    so, D, aE, aN, S = oracle.assemble_joint(nth, nz, PHYS, inputs.smooth_texture(), conds)
    n = 2 * nth * nz
    Dd, aEd, aNd, Sd = dev(D), dev(aE), dev(aN), dev(S)
    p = zeros(n)
    opts = g.solver_opts(eps=1e-12)
    st, it, rel = g.gmaf_solve_joint(ctx, nth, nz, 2, Dd, aEd, aNd, Sd, p, opts)
    assert st == 0 and it > 10
    before = p.clone()
    st, it2, rel2 = g.gmaf_solve_joint(ctx, nth, nz, 2, Dd, aEd, aNd, Sd, p,
                                       g.solver_opts(eps=1e-10, zero_init=0))
    assert st == 0 and it2 == 0 and torch.equal(before, p)
    p.fill_(123.0)
    st, it3, rel3 = g.gmaf_solve_joint(ctx, nth, nz, 2, Dd, aEd, aNd, zeros(n), p,
                                       g.solver_opts(zero_init=0))
    assert st == 0 and it3 == 0 and not torch.any(p)
    st, it4, _ = g.gmaf_solve_joint(ctx, nth, nz, 2, Dd, aEd, aNd, Sd, p,
                                    g.solver_opts(eps=1e-12, max_iter=3), allow_not_converged=True)
    assert st == g.GMAF_NOT_CONVERGED and it4 == 3
    for bad in (g.solver_opts(omega=2.0), g.solver_opts(eps=0.0), g.solver_opts(precond=3),
                g.solver_opts(max_iter=-1)):
        with pytest.raises(g.GmafError) as ei:
            g.gmaf_solve_joint(ctx, nth, nz, 2, Dd, aEd, aNd, Sd, p, bad)
        assert ei.value.status == g.GMAF_INVALID_ARG
    with pytest.raises(g.GmafError):
        g.gmaf_solve_joint(ctx, 2, nz, 2, Dd, aEd, aNd, Sd, p)


def test_solve_is_deterministic_and_graph_matches_host_loop(g, monkeypatch):
    """Reductions are summed per task in task order, so a run does not depend on the
    scheduling of tasks to warps; with the kernel variant fixed (no tuning) two
    contexts, one driving the loop from a graph and one from the host, agree bitwise."""
    conds = states(9, seed=11)
    nth, nz = 150, 50
    so, D, aE, aN, S = oracle.assemble_joint(nth, nz, PHYS, tex_dimples(), conds)
    args = [dev(D), dev(aE), dev(aN), dev(S)]
    n = 9 * nth * nz
    monkeypatch.setenv("GMAF_NO_TUNE", "1")
    c1 = g.Context()
    outs = []
    for _ in range(2):
        p = zeros(n)
        g.gmaf_solve_joint(c1.handle, nth, nz, 9, *args, p)
        outs.append(host(p))
    c1.close()
    assert np.array_equal(outs[0], outs[1])
    monkeypatch.setenv("GMAF_NO_GRAPH", "1")
    c2 = g.Context()
    p = zeros(n)
    g.gmaf_solve_joint(c2.handle, nth, nz, 9, *args, p)
    c2.close()
    assert np.array_equal(host(p), outs[0])


# dynamic tasks (ids 1000 VEC + 10 TY + MINB), phase B staged D rows ahead
# (+ 100000 D), both phases staged (+ 300000 D), phase B filled by bulk copies
# (+ 2000000), blocks of 6 warps with a run-time task height (+ 600000000), phase A
# rebuilding the diagonal from the couplings (+ 10000000; two-row grid: every row
# carries a Dirichlet face; n_theta = 4: one strip wrapped 32 times; 388 x 97: a
# ragged last strip and a one-row last task), and the
# static schedule with phase A marching against phase B
# (ids 1000000 + 1000 VEC + MINB); float VEC > 1 kernels need n_theta % 4 == 0,
# double ones an even n_theta, the bulk-copied phase B n_theta >= 136
@pytest.mark.parametrize("precision,variant,nth,nz,K", [
    (1, 4322, 132, 45, 9), (1, 1004002, 132, 45, 9), (1, 4082, 260, 33, 4),
    (1, 204162, 132, 45, 9), (1, 204322, 260, 70, 3), (1, 604322, 132, 45, 9),
    (1, 604322, 260, 70, 3), (1, 604162, 132, 45, 9),
    (1, 2604322, 136, 45, 9), (1, 2604322, 260, 70, 3), (1, 2604322, 384, 33, 2),
    (1, 600604183, 132, 45, 9), (1, 600604183, 260, 70, 3), (1, 600604323, 132, 45, 9),
    (1, 600604163, 64, 3, 2),
    (1, 10604322, 132, 45, 9), (1, 10604322, 260, 70, 3), (1, 10604322, 64, 2, 2),
    (1, 10604322, 4, 3, 1), (1, 10604322, 388, 97, 5),
    (1, 1001004, 131, 7, 3), (0, 2322, 130, 45, 9), (0, 1002002, 130, 45, 9),
    (0, 1001003, 131, 7, 3), (0, 1001003, 3, 2, 1),
])
def test_each_schedule_matches_oracle(g, monkeypatch, precision, variant, nth, nz, K):
    monkeypatch.setenv("GMAF_VARIANT", str(variant))
    c = g.Context()
    try:
        conds = states(K, seed=nth + K)
        p, it, rel, po, ito, _ = solve_both(g, c.handle, nth, nz, tex_dimples(), conds,
                                            precision=precision)
        info = g.gmaf_last_solve_info(c.handle)
    finally:
        c.close()
    assert info["kernel_variant"] == variant
    assert rel <= 1e-9
    if precision == 0:
        assert abs(it - ito) <= 2, (it, ito)
        assert rel_l2(p, po) <= 1e-9
    else:
        assert rel_l2(p, po) <= 1e-6


@pytest.mark.parametrize("nth,nz,K,precond", [(136, 45, 9, 1), (260, 70, 3, 1), (2048, 64, 2, 1),
                                              (136, 31, 2, 1), (260, 70, 3, 0)])
def test_phase_b_forms_are_bitwise_the_staged_one(g, monkeypatch, nth, nz, K, precond):
    """The bulk-copied phase B (one lane copies whole row segments, halo and seam
    pieces included) feeds the same arithmetic in the same order as the cp.async
    staged one: bitwise the same solution and iteration count, at the narrowest
    grid the bulk copies take (136 columns), a ragged last tile (260 = 2 x 128 + 4),
    the benchmark's width and ragged row tiles (31, 45 and 70 rows), with ASSOR-II
    and with Jacobi."""
    conds = states(K, seed=nth + 3)
    so, D, aE, aN, S = oracle.assemble_joint(nth, nz, PHYS, tex_dimples(), conds)
    args = [dev(D), dev(aE), dev(aN), dev(S)]
    n = K * nth * nz
    outs = []
    for variant in ("604322", "2604322"):
        monkeypatch.setenv("GMAF_VARIANT", variant)
        c = g.Context()
        try:
            p = zeros(n)
            st, it, rel = g.gmaf_solve_joint(c.handle, nth, nz, K, *args, p,
                                             g.solver_opts(eps=1e-10, precision=1, precond=precond))
            info = g.gmaf_last_solve_info(c.handle)
        finally:
            c.close()
        assert info["kernel_variant"] == int(variant)
        outs.append((host(p), it, info["outer_iterations"]))
    for o in outs[1:]:
        assert o[1:] == outs[0][1:]
        assert np.array_equal(o[0], outs[0][0])


@pytest.mark.parametrize("variant", [1002002, 1001003])
def test_static_schedule_is_deterministic_and_graph_matches_host_loop(g, monkeypatch, variant):
    """The static schedule sums one partial per warp in warp order: for a fixed
    launch shape the graph-driven and host-driven solves agree bitwise."""
    conds = states(9, seed=12)
    nth, nz = 150, 50
    so, D, aE, aN, S = oracle.assemble_joint(nth, nz, PHYS, tex_dimples(), conds)
    args = [dev(D), dev(aE), dev(aN), dev(S)]
    n = 9 * nth * nz
    monkeypatch.setenv("GMAF_VARIANT", str(variant))
    outs = []
    for no_graph in ("0", "0", "1"):
        if no_graph == "1":
            monkeypatch.setenv("GMAF_NO_GRAPH", "1")
        c = g.Context()
        p = zeros(n)
        g.gmaf_solve_joint(c.handle, nth, nz, 9, *args, p)
        assert g.gmaf_last_solve_info(c.handle)["kernel_variant"] == variant
        c.close()
        outs.append(host(p))
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


# asynchronized criterion (Eq. 3.10): each condition is its own PCG, so the oracle is
# the oracle's solve of each condition alone
@pytest.mark.parametrize("nth,nz,K,precond", [(130, 45, 9, 1), (131, 7, 3, 1), (96, 40, 4, 0),
                                              (3, 2, 2, 1), (100, 30, 3, 2)])
def test_asynchronized_criterion_matches_per_condition_oracle(g, ctx, nth, nz, K, precond):
    conds = states(K, seed=nth + 3 * K)
    so, D, aE, aN, S = oracle.assemble_joint(nth, nz, PHYS, tex_dimples(), conds)
    n = K * nth * nz
    p = zeros(n)
    opts = g.solver_opts(precond=precond, eps=1e-10, criterion=1)
    st, it, rel = g.gmaf_solve_joint(ctx, nth, nz, K, dev(D), dev(aE), dev(aN), dev(S), p, opts)
    info = g.gmaf_last_solve_info(ctx)
    assert st == 0 and rel <= 1e-9
    pg = host(p).reshape(K, nz, nth)
    its = []
    for k in range(K):
        sl = slice(k, k + 1)
        sto, po, ito, _, _ = oracle.solve_joint(nth, nz, D[sl], aE[sl], aN[sl], S[sl],
                                                precond=precond, omega=1.2, eps=1e-10)
        assert sto == 0
        its.append(ito)
        assert rel_l2(pg[k], po) <= 1e-9, k
    assert abs(info["iterations"] - max(its)) <= 2, (info["iterations"], its)
    assert abs(info["iterations_sum"] - sum(its)) <= 2 * K, (info["iterations_sum"], its)


def test_asynchronized_picard_step_and_option_checks(g, ctx):
    rng = np.random.default_rng(21)
    st0 = inputs.random_state(rng)
    tex = tex_dimples()
    dt = 2.7777777777777778e-4
    F = np.array([30.0, -15.0, 6.0, -3.0])
    res = {}
    for crit in (0, 1):
        res[crit] = g.gmaf_picard_step(ctx, 96, 48, PHYS, tex, st0, st0[:4], dt, F, 2e-8, 1e-6,
                                       g.solver_opts(eps=1e-12, criterion=crit))
        info = g.gmaf_last_solve_info(ctx)
        if crit == 1:
            assert info["iterations_sum"] > info["iterations"]
        else:
            assert info["iterations_sum"] == 9 * info["iterations"]
    assert load_err(res[1]["loads"], res[0]["loads"]) <= 1e-7
    # the simplified scheme's 5-condition batch (one coefficient set) under both criteria
    simp = [g.gmaf_picard_step_simplified(ctx, 96, 48, PHYS, tex, st0, dt, F, 1e-6,
                                          g.solver_opts(eps=1e-12, criterion=crit))
            for crit in (0, 1)]
    assert load_err(simp[1]["loads"], simp[0]["loads"]) <= 1e-7
    assert g.gmaf_last_solve_info(ctx)["iterations_sum"] > g.gmaf_last_solve_info(ctx)["iterations"]
    p = zeros(2 * 64 * 32)
    so, D, aE, aN, S = oracle.assemble_joint(64, 32, PHYS, inputs.smooth_texture(), states(2))
    for bad in (g.solver_opts(criterion=1, precision=1), g.solver_opts(criterion=2)):
        with pytest.raises(g.GmafError) as ei:
            g.gmaf_solve_joint(ctx, 64, 32, 2, dev(D), dev(aE), dev(aN), dev(S), p, bad)
        assert ei.value.status == g.GMAF_INVALID_ARG


@pytest.mark.parametrize("precision,variant", [(0, 2322), (0, 1002002), (1, 204322), (1, 604322),
                                               (1, 4082)])
def test_two_level_reduction_matches_one_level_and_oracle(g, monkeypatch, precision, variant):
    """The chunked (two-level) reduction of the phase sums, forced on a small problem:
    same iterate as the one-level sum up to rounding, and the oracle's solution."""
    nth, nz, K = 132, 45, 9
    conds = states(K, seed=41)
    so, D, aE, aN, S = oracle.assemble_joint(nth, nz, PHYS, tex_dimples(), conds)
    args = [dev(D), dev(aE), dev(aN), dev(S)]
    n = K * nth * nz
    monkeypatch.setenv("GMAF_VARIANT", str(variant))
    out = {}
    for chunked in ("1", "1000000000"):
        monkeypatch.setenv("GMAF_CHUNKED_FROM", chunked)
        c = g.Context()
        p = zeros(n)
        st, it, rel = g.gmaf_solve_joint(c.handle, nth, nz, K, *args, p,
                                         g.solver_opts(eps=1e-10, precision=precision))
        c.close()
        assert st == 0 and rel <= 1e-9
        out[chunked] = (host(p), it)
    (p2, i2), (p1, i1) = out["1"], out["1000000000"]
    assert abs(i2 - i1) <= 1
    assert rel_l2(p2, p1) <= (1e-9 if precision == 0 else 1e-6)
    sto, po, ito, _, _ = oracle.solve_joint(nth, nz, D, aE, aN, S, precond=1, omega=1.2, eps=1e-10)
    assert rel_l2(p2.reshape(K, nz, nth), po) <= (1e-9 if precision == 0 else 1e-6)


def test_hbm_budget_is_enforced(g):
    c = g.Context(hbm_budget_bytes=1 << 20)
    n = 9 * 256 * 128
    with pytest.raises(g.GmafError) as ei:
        g.gmaf_picard_step(c.handle, 256, 128, PHYS, None, np.zeros(8), np.zeros(4), 1e-4,
                           np.zeros(4), 2e-8, 1e-6)
    assert ei.value.status == g.GMAF_OUT_OF_MEMORY
    c.close()


# ----------------------------------------------------------------------------- loads


@pytest.mark.parametrize("nth,nz,K,textured", [(64, 32, 1, False), (130, 45, 9, True),
                                               (3, 2, 2, False)])
def test_loads_match_oracle(g, ctx, nth, nz, K, textured):
    tex = tex_dimples() if textured else inputs.smooth_texture()
    conds = states(K, seed=21)
    so, D, aE, aN, S = oracle.assemble_joint(nth, nz, PHYS, tex, conds)
    sto, po, *_ = oracle.solve_joint(nth, nz, D, aE, aN, S, eps=1e-12)
    loads = zeros(12 * K)
    g.gmaf_integrate_loads(ctx, nth, nz, PHYS, tex, conds, dev(po), loads)
    got = host(loads).reshape(K, 12)
    want = np.stack([oracle.loads(nth, nz, PHYS, tex, c, po[k])[1] for k, c in enumerate(conds)])
    assert load_err(got, want) <= 1e-11


# ----------------------------------------------------------------------------- whole Picard step


@pytest.mark.parametrize("nth,nz,textured,precision", [(64, 32, False, 0), (96, 48, True, 0),
                                                       (96, 48, True, 1)])
def test_picard_step_matches_oracle(g, ctx, nth, nz, textured, precision):
    tex = tex_dimples() if textured else inputs.smooth_texture()
    st0 = states(1, seed=31)[0]
    e_prev = st0[:4] - 2e-8
    Fext = np.array([25.0, -10.0, 4.0, 3.0])
    dt = 2.78e-4
    eps = 1e-12
    r = g.gmaf_picard_step(ctx, nth, nz, PHYS, tex, st0, e_prev, dt, Fext, 2e-8, 1e-6,
                           g.solver_opts(eps=eps, precision=precision))
    o = oracle.picard_step(nth, nz, PHYS, tex, st0, e_prev, dt, Fext, 2e-8, 1e-6, eps=eps)
    assert r["status"] == 0 and o["status"] == 0
    tol_l = 1e-7 if precision == 0 else 1e-5
    assert load_err(r["loads"], o["loads"]) <= tol_l
    Jg, Jo = r["J"], o["J"]
    colscale = np.abs(Jo).max(axis=0, keepdims=True)
    assert np.max(np.abs(Jg - Jo) / colscale) <= (1e-5 if precision == 0 else 1e-3)
    np.testing.assert_allclose(r["G"], o["G"], rtol=1e-6, atol=1e-6 * np.abs(o["G"]).max())
    ds_g, ds_o = r["state"] - st0, o["state"] - st0
    assert np.linalg.norm(ds_g - ds_o) <= 1e-4 * np.linalg.norm(ds_o) + 1e-20


@pytest.mark.parametrize("nth,nz,textured,precision", [(64, 32, False, 0), (96, 48, True, 0),
                                                       (96, 48, True, 1)])
def test_simplified_picard_step_matches_oracle(g, ctx, nth, nz, textured, precision):
    """Eq. 2.20-2.22 on 5 conditions: loads, rate Jacobian, G and the update."""
    tex = tex_dimples() if textured else inputs.smooth_texture()
    st0 = states(1, seed=37)[0]
    Fext = np.array([25.0, -10.0, 4.0, 3.0])
    dt = 2.78e-4
    eps = 1e-12
    r = g.gmaf_picard_step_simplified(ctx, nth, nz, PHYS, tex, st0, dt, Fext, 1e-6,
                                      g.solver_opts(eps=eps, precision=precision))
    o = oracle.picard_step_simplified(nth, nz, PHYS, tex, st0, dt, Fext, 1e-6, eps=eps)
    assert r["status"] == 0 and o["status"] == 0
    tol_l = 1e-7 if precision == 0 else 1e-5
    assert load_err(r["loads"], o["loads"]) <= tol_l
    assert not np.any(r["J"][:, :4])
    Jg, Jo = r["J"][:, 4:], o["J"][:, 4:]
    colscale = np.abs(Jo).max(axis=0, keepdims=True)
    assert np.max(np.abs(Jg - Jo) / colscale) <= (1e-5 if precision == 0 else 1e-3)
    np.testing.assert_allclose(r["G"], o["G"], rtol=1e-6, atol=1e-6 * np.abs(o["G"]).max())
    ds_g, ds_o = r["state"] - st0, o["state"] - st0
    assert np.linalg.norm(ds_g - ds_o) <= 1e-4 * np.linalg.norm(ds_o) + 1e-20
    # the fields of the 5 conditions; the rest of the buffer is left alone
    n = nth * nz
    buf = torch.full((9 * n,), 7.0, dtype=torch.float64, device="cuda")
    g.gmaf_last_fields(ctx, nth, nz, buf)
    hb = host(buf)
    assert np.all(hb[5 * n:] == 7.0) and np.all(np.isfinite(hb[:5 * n]))


@pytest.mark.parametrize("scheme", ["general", "simplified"])
def test_rebuilt_diagonal_picard_step_matches_oracle(g, monkeypatch, scheme):
    """Phase A rebuilding the diagonal from the couplings (variant 10604322) reads the
    Dirichlet term of the first and last rows per coefficient slot: 5 slots for the
    general step's 9 conditions, 1 for the simplified step's 5.  Mixed precision
    against the oracle's step."""
    monkeypatch.setenv("GMAF_VARIANT", "10604322")
    nth, nz = 96, 48
    tex = tex_dimples()
    st0 = states(1, seed=31)[0]
    e_prev = st0[:4] - 2e-8
    Fext = np.array([25.0, -10.0, 4.0, 3.0])
    dt, eps = 2.78e-4, 1e-12
    c = g.Context()
    try:
        if scheme == "general":
            r = g.gmaf_picard_step(c.handle, nth, nz, PHYS, tex, st0, e_prev, dt, Fext, 2e-8, 1e-6,
                                   g.solver_opts(eps=eps, precision=1))
            o = oracle.picard_step(nth, nz, PHYS, tex, st0, e_prev, dt, Fext, 2e-8, 1e-6, eps=eps)
        else:
            r = g.gmaf_picard_step_simplified(c.handle, nth, nz, PHYS, tex, st0, dt, Fext, 1e-6,
                                              g.solver_opts(eps=eps, precision=1))
            o = oracle.picard_step_simplified(nth, nz, PHYS, tex, st0, dt, Fext, 1e-6, eps=eps)
        info = g.gmaf_last_solve_info(c.handle)
    finally:
        c.close()
    assert info["kernel_variant"] == 10604322
    assert r["status"] == 0 and o["status"] == 0
    assert load_err(r["loads"], o["loads"]) <= 1e-5
    np.testing.assert_allclose(r["G"], o["G"], rtol=1e-6, atol=1e-6 * np.abs(o["G"]).max())
    ds_g, ds_o = r["state"] - st0, o["state"] - st0
    assert np.linalg.norm(ds_g - ds_o) <= 1e-4 * np.linalg.norm(ds_o) + 1e-20


@pytest.mark.parametrize("precision", [0, 1])
def test_phase_timing_path_matches_graph_path(g, precision):
    """Per-phase event timing drives the loop from the host; results are bitwise the
    graph's and every phase launch is counted."""
    conds = states(9, seed=13)
    nth, nz = 140, 33
    so, D, aE, aN, S = oracle.assemble_joint(nth, nz, PHYS, tex_dimples(), conds)
    args = [dev(D), dev(aE), dev(aN), dev(S)]
    n = 9 * nth * nz
    opts = g.solver_opts(precision=precision)
    c = g.Context()
    p0 = zeros(n)
    g.gmaf_solve_joint(c.handle, nth, nz, 9, *args, p0, opts)
    g.gmaf_set_phase_timing(c.handle, True)
    p1 = zeros(n)
    st, it, rel = g.gmaf_solve_joint(c.handle, nth, nz, 9, *args, p1, opts)
    t = g.gmaf_phase_timing(c.handle)
    g.gmaf_set_phase_timing(c.handle, False)
    p2 = zeros(n)
    g.gmaf_solve_joint(c.handle, nth, nz, 9, *args, p2, opts)
    c.close()
    assert torch.equal(p0, p1) and torch.equal(p0, p2)
    assert t["phase_a"][1] >= it and t["phase_b"][1] >= it and t["phase_a"][0] > 0
    assert t["resid64"][1] >= 1
