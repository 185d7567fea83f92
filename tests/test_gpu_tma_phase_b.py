"""The block-marched TMA phase B (variants 3000000 + 10000 RPW + 1000 NS + TB: RPW
rows per consumer warp, so chunks of 8 RPW staged rows, NS chunk slots in the
ring, tasks of TB rows) against the FP64 oracle, against the cp.async staged form,
and for determinism.

It needs n_theta % 128 == 0; the shapes cover one strip (the row box holds both
seams, so both wrap boxes are loaded), several strips, ragged row tasks, tasks of
two rows and of exactly one chunk of either height, Jacobi, ASSOR-I and ASSOR-II.
Mixed precision: pressure relative L2 1e-6 against the oracle, the FP64 outer
residual 1e-9.
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()


def host(t):
    return t.detach().cpu().numpy()


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def system(nth, nz, K, seed):
    rng = np.random.default_rng(seed)
    conds = [inputs.random_state(rng) for _ in range(K)]
    tex = inputs.dimple_texture(np.random.default_rng(5))
    return oracle.assemble_joint(nth, nz, PHYS, tex, conds)


def solve(g, monkeypatch, variant, nth, nz, K, arrs, precond=1, env=None):
    so, D, aE, aN, S = arrs
    monkeypatch.setenv("GMAF_VARIANT", str(variant))
    for k, v in (env or {}).items():
        monkeypatch.setenv(k, v)
    c = g.Context()
    try:
        p = torch.zeros(K * nth * nz, dtype=torch.float64, device="cuda")
        st, it, rel = g.gmaf_solve_joint(c.handle, nth, nz, K, dev(D), dev(aE), dev(aN), dev(S), p,
                                         g.solver_opts(eps=1e-10, precision=1, precond=precond))
        info = g.gmaf_last_solve_info(c.handle)
    finally:
        c.close()
    assert st == 0
    return host(p).reshape(K, nz, nth), it, rel, info


@pytest.mark.parametrize("variant,nth,nz,K,precond", [
    (3014062, 256, 45, 9, 1),     # two strips, one task of 45 rows, 8-row chunks, ragged last chunk
    (3023030, 128, 70, 3, 1),     # one strip: both seam boxes; tasks of 30, 30, 10 rows, 16-row chunks
    (3024062, 384, 200, 2, 1),    # three strips, tasks of 62 and 14 rows
    (3023030, 128, 2, 2, 1),      # the fewest rows (both halo rows outside the grid)
    (3014062, 256, 6, 2, 1),      # a task of exactly one 8-row chunk
    (3023062, 256, 14, 2, 1),     # a task of exactly one 16-row chunk
    (3023062, 256, 45, 9, 0),     # Jacobi
    (3014062, 256, 45, 4, 2),     # ASSOR-I (its diagonal through the Jacobi path)
])
def test_tma_phase_b_matches_oracle(g, monkeypatch, variant, nth, nz, K, precond):
    arrs = system(nth, nz, K, seed=nth + nz + K)
    p, it, rel, info = solve(g, monkeypatch, variant, nth, nz, K, arrs, precond)
    assert info["kernel_variant"] == variant
    assert rel <= 1e-9
    so, D, aE, aN, S = arrs
    sto, po, ito, _, _ = oracle.solve_joint(nth, nz, D, aE, aN, S, precond=precond, omega=1.2,
                                            eps=1e-10)
    assert sto == 0
    assert rel_l2(p, po) <= 1e-6


@pytest.mark.parametrize("variant,nth,nz,K", [(3014062, 256, 45, 9), (3023062, 256, 45, 9),
                                              (3023062, 2048, 64, 2)])
def test_tma_phase_b_tracks_the_staged_one(g, monkeypatch, variant, nth, nz, K):
    """Same preconditioned recurrence as the cp.async staged phase B (604322); only
    the FP32 rounding of the dot products' grouping differs, so the two mixed solves
    take about the same iterations and agree far below the tolerance."""
    arrs = system(nth, nz, K, seed=77)
    pa, ia, _, infa = solve(g, monkeypatch, 604322, nth, nz, K, arrs)
    pb, ib, _, infb = solve(g, monkeypatch, variant, nth, nz, K, arrs)
    assert infa["kernel_variant"] == 604322 and infb["kernel_variant"] == variant
    assert abs(ia - ib) <= 0.02 * ia + 3, (ia, ib)
    assert rel_l2(pb, pa) <= 1e-8


def test_tma_phase_b_is_deterministic_and_graph_matches_host_loop(g, monkeypatch):
    """Task sums are published per task and added in task order, so neither the
    blocks that ran the tasks nor graph or host loop control change a bit."""
    nth, nz, K = 256, 45, 9
    arrs = system(nth, nz, K, seed=12)
    outs = [solve(g, monkeypatch, 3023062, nth, nz, K, arrs) for _ in range(2)]
    outs.append(solve(g, monkeypatch, 3023062, nth, nz, K, arrs, env={"GMAF_NO_GRAPH": "1"}))
    for p, it, rel, info in outs[1:]:
        assert it == outs[0][1]
        assert np.array_equal(p, outs[0][0])


def test_tma_phase_b_two_level_reduction(g, monkeypatch):
    """The two-level (chunked) reduction of the per-task sums, forced on a small
    problem, gives the one-level iterate up to rounding and the oracle's solution."""
    nth, nz, K = 256, 45, 9
    arrs = system(nth, nz, K, seed=41)
    one = solve(g, monkeypatch, 3023062, nth, nz, K, arrs, env={"GMAF_CHUNKED_FROM": "1000000000"})
    two = solve(g, monkeypatch, 3023062, nth, nz, K, arrs, env={"GMAF_CHUNKED_FROM": "1"})
    assert abs(one[1] - two[1]) <= 1
    assert rel_l2(two[0], one[0]) <= 1e-6
    so, D, aE, aN, S = arrs
    sto, po, ito, _, _ = oracle.solve_joint(nth, nz, D, aE, aN, S, precond=1, omega=1.2, eps=1e-10)
    assert rel_l2(two[0], po) <= 1e-6


def load_err(a, b):
    """Relative load error per component, forces and moments each against
    max(|F_c|, 1e-3 ||F||)."""
    a, b = np.asarray(a), np.asarray(b)
    out = 0.0
    for part in (slice(0, 6), slice(6, 12)):
        x, y = a[..., part], b[..., part]
        nrm = np.linalg.norm(y, axis=-1, keepdims=True)
        out = max(out, float(np.max(np.abs(x - y) / np.maximum(np.abs(y), 1e-3 * nrm))))
    return out


@pytest.mark.parametrize("variant,scheme", [(3014062, "general"), (3023062, "general"),
                                            (3014062, "simplified")])
def test_tma_phase_b_picard_step_matches_oracle(g, monkeypatch, variant, scheme):
    """The Picard step stores 5 coefficient slots for its 9 conditions (the simplified
    scheme one for its 5), so each task's coefficient copies come from the slot of its
    condition: loads, G, Jacobian and update against the oracle's step, mixed
    precision."""
    monkeypatch.setenv("GMAF_VARIANT", str(variant))
    nth, nz = 256, 128
    tex = inputs.dimple_texture(np.random.default_rng(5))
    st0 = inputs.random_state(np.random.default_rng(31))
    e_prev = st0[:4] - 2e-8
    F = np.array([25.0, -10.0, 4.0, 3.0])
    dt, eps = 2.78e-4, 1e-12
    c = g.Context()
    try:
        if scheme == "general":
            r = g.gmaf_picard_step(c.handle, nth, nz, PHYS, tex, st0, e_prev, dt, F, 2e-8, 1e-6,
                                   g.solver_opts(eps=eps, precision=1))
        else:
            r = g.gmaf_picard_step_simplified(c.handle, nth, nz, PHYS, tex, st0, dt, F, 1e-6,
                                              g.solver_opts(eps=eps, precision=1))
        info = g.gmaf_last_solve_info(c.handle)
    finally:
        c.close()
    if scheme == "general":
        o = oracle.picard_step(nth, nz, PHYS, tex, st0, e_prev, dt, F, 2e-8, 1e-6, eps=eps)
        Jg, Jo = r["J"], o["J"]
    else:
        o = oracle.picard_step_simplified(nth, nz, PHYS, tex, st0, dt, F, 1e-6, eps=eps)
        Jg, Jo = r["J"][:, 4:], o["J"][:, 4:]
    assert info["kernel_variant"] == variant
    assert r["status"] == 0 and o["status"] == 0
    assert load_err(r["loads"], o["loads"]) <= 1e-5
    assert np.max(np.abs(Jg - Jo) / np.abs(Jo).max(axis=0, keepdims=True)) <= 1e-3
    np.testing.assert_allclose(r["G"], o["G"], rtol=1e-6, atol=1e-6 * np.abs(o["G"]).max())
    ds_g, ds_o = r["state"] - st0, o["state"] - st0
    assert np.linalg.norm(ds_g - ds_o) <= 1e-4 * np.linalg.norm(ds_o) + 1e-20
