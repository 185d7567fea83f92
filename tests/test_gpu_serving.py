"""Continuous-batching server: results against the oracle, alone vs in a mix,
admission by device footprint, and the sequential FP64 baseline."""
import numpy as np
import pytest

import oracle
from paper_2511_06824_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PHYS = inputs.phys_vector()
F_EXT = np.array([30.0, -15.0, 6.0, -3.0])


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


def items(shapes, seed=0):
    from paper_2511_06824_gb300 import serving
    rng = np.random.default_rng(seed)
    out = []
    for k, (nth, nz, textured) in enumerate(shapes):
        tex = inputs.dimple_texture(rng) if textured else inputs.smooth_texture()
        out.append(serving.StreamItem(0.0, nth, nz, PHYS, tex, inputs.random_state(rng), F_EXT))
    return out


def run_all(g, ctx, its, budget=8 << 30, eps=1e-11, round_iters=32):
    from paper_2511_06824_gb300 import serving
    res = {}
    max_active = 0
    with g.Server(ctx, budget) as sv:
        ids = {sv.submit(serving.to_request(it, eps)): k for k, it in enumerate(its)}
        while len(res) < len(its):
            a, q = sv.run(round_iters)
            max_active = max(max_active, a)
            for r in sv.poll():
                res[ids[r["id"]]] = r
        assert sv.free_bytes() > 0
    return [res[k] for k in range(len(its))], max_active


@pytest.mark.parametrize("staged", ["1", "0"])
def test_served_step_matches_oracle(g, ctx, monkeypatch, staged):
    """Both forms of the batched phase kernels: rows staged by cp.async and
    register prefetch (the server picks its kernels when it is created)."""
    monkeypatch.setenv("GMAF_SV_STAGED", staged)
    it = items([(96, 48, True)], seed=3)[0]
    (r,), _ = run_all(g, ctx, [it], eps=1e-12)
    o = oracle.picard_step(96, 48, PHYS, it.tex, it.state, it.state[:4], 2.7777777777777778e-4,
                           F_EXT, 2e-8, 1e-6, eps=1e-12)
    assert r["status"] == 0 and o["status"] == 0
    scale = np.maximum(np.abs(o["loads"]), 1e-3 * np.linalg.norm(o["loads"]))
    assert np.max(np.abs(r["loads"] - o["loads"]) / scale) <= 1e-5
    colscale = np.abs(o["J"]).max(axis=0, keepdims=True)
    assert np.max(np.abs(r["J"] - o["J"]) / colscale) <= 1e-3
    ds_g, ds_o = r["state"] - it.state, o["state"] - it.state
    assert np.linalg.norm(ds_g - ds_o) <= 1e-3 * np.linalg.norm(ds_o)


def test_each_result_is_the_same_alone_and_in_the_mix(g, ctx):
    """Requests of uneven grids solved one per server and all in one server give
    bitwise the same loads, Jacobian, generalized force, state and iteration counts."""
    its = items([(128, 64, True), (64, 32, False), (256, 48, True), (128, 96, False),
                 (512, 32, True)], seed=11)
    mixed, max_active = run_all(g, ctx, its)
    assert max_active == len(its)
    for k, it in enumerate(its):
        (alone,), _ = run_all(g, ctx, [it])
        m = mixed[k]
        assert alone["status"] == 0 and m["status"] == 0
        assert alone["iters"] == m["iters"] and alone["outer"] == m["outer"]
        for key in ("loads", "J", "G", "state"):
            assert np.array_equal(alone[key], m[key]), (k, key)


def test_admission_is_bounded_by_the_footprint(g, ctx):
    its = items([(256, 128, True), (256, 128, False), (256, 128, True)], seed=5)
    fp = g.gmaf_request_footprint(256, 128)
    res, max_active = run_all(g, ctx, its, budget=int(fp * 1.5))
    assert max_active == 1
    assert all(r["status"] == 0 for r in res)
    res2, max_active2 = run_all(g, ctx, its, budget=int(fp * 2.5))
    assert max_active2 == 2
    for a, b in zip(res, res2):
        assert np.array_equal(a["loads"], b["loads"])
    with pytest.raises(g.GmafError) as ei:
        with g.Server(ctx, int(fp * 0.5)) as sv:
            from paper_2511_06824_gb300 import serving
            sv.submit(serving.to_request(its[0], 1e-10))
    assert ei.value.status == g.GMAF_OUT_OF_MEMORY


def test_sequential_baseline_agrees_with_served_result(g, ctx):
    from paper_2511_06824_gb300 import serving
    it = items([(128, 64, True)], seed=8)[0]
    (r,), _ = run_all(g, ctx, [it], eps=1e-12)
    s = serving.sequential_step(ctx, it, eps=1e-12)
    assert serving.load_error(s["loads"], r["loads"]) <= 1e-6
    np.testing.assert_allclose(s["G"], r["G"], rtol=1e-6, atol=1e-6 * np.abs(r["G"]).max())


def test_stream_replay_runs_and_reports_latency(g, ctx):
    from paper_2511_06824_gb300 import serving
    reqs = inputs.serving_requests(seed=2, count=6, rate_hz=50.0,
                                   grids=[(128, 64), (256, 128), (64, 32)])
    its = serving.items_from_requests(reqs)
    out = serving.serve_stream(ctx, its, 8 << 30, eps=1e-10, round_iters=32)
    assert out["completed"] == 6 and out["p99_ms"] >= out["p50_ms"] > 0
    assert all(r["status"] == 0 for r in out["results"])


def test_graph_rounds_match_host_driven_rounds(g, ctx, monkeypatch):
    """A round as a CUDA graph (default) and as host launches run the same kernels on
    the same table in the same order: bitwise the same results and counts."""
    its = items([(128, 64, True), (256, 48, True), (64, 32, False)], seed=13)
    monkeypatch.setenv("GMAF_SV_GRAPH", "0")
    host, _ = run_all(g, ctx, its, round_iters=24)
    monkeypatch.setenv("GMAF_SV_GRAPH", "1")
    graph, _ = run_all(g, ctx, its, round_iters=24)
    for a, b in zip(host, graph):
        assert a["status"] == 0 and b["status"] == 0
        assert a["iters"] == b["iters"] and a["outer"] == b["outer"]
        for key in ("loads", "J", "G", "state"):
            assert np.array_equal(a[key], b[key]), key


def test_tile_height_is_tuned_once_per_grid(g, ctx):
    """The tuner fixes each grid's task height at the first request of that grid; a
    later server, another mix or another order decomposes the grid the same way and
    gives bitwise the same results."""
    its = items([(128, 64, True), (128, 64, False), (512, 128, True), (64, 32, True)], seed=17)
    first, _ = run_all(g, ctx, its)
    again, _ = run_all(g, ctx, its[::-1])
    again = again[::-1]
    rows = {}
    for a, b, it in zip(first, again, its):
        assert a["status"] == 0 and b["status"] == 0
        assert a["tile_rows"] in (16, 32, 64)
        assert rows.setdefault((it.n_theta, it.n_z), a["tile_rows"]) == a["tile_rows"]
        assert b["tile_rows"] == a["tile_rows"]
        for key in ("loads", "J", "G", "state"):
            assert np.array_equal(a[key], b[key]), key
