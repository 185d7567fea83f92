"""The allocation-free joint solve against the ordinary one.

Some programs that call this library may not allocate device memory while
they run: a host application whose own pool allocator owns all of the GPU's
memory and gives solver plug-ins no allocation hook, or a real-time
co-simulation loop that cannot accept the latency, or the possible failure, of
an allocation in the middle of a time step.  gmaf_solve_joint_noalloc serves
them with a fixed scratch array inside the library.  These tests call it through
the C ABI several times in a row, on different problems, and check each result
against gmaf_solve_joint and against the oracle's solve of the same system
(pressure relative L2 1e-9, the FP64 parity bound of the other tests), up to
the documented fit of the array (the 9-condition 512 x 256 batch) and with an
odd n_theta (the one-column kernels); a problem larger than the array must be
refused.

The file name puts it last in collection order, so that a run stopping at the
first failure has run every other test before this one.
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


def _problem(nth, nz, K, seed, textured):
    rng = np.random.default_rng(seed)
    tex = inputs.dimple_texture(rng) if textured else inputs.smooth_texture()
    conds = [inputs.random_state(rng) for _ in range(K)]
    st, D, aE, aN, S = oracle.assemble_joint(nth, nz, PHYS, tex, conds)
    assert st == 0
    return [torch.from_numpy(np.ascontiguousarray(a).ravel()).cuda() for a in (D, aE, aN, S)]


def test_noalloc_solve_matches_solve_joint_twice_in_a_row(g):
    cases = [(150, 60, 9, 1, True, 1), (64, 32, 3, 2, False, 1), (96, 40, 4, 3, True, 2)]
    ctx = g.Context()
    try:
        for nth, nz, K, seed, textured, precond in cases:
            D, aE, aN, S = _problem(nth, nz, K, seed, textured)
            n = K * nth * nz
            p_ref = torch.zeros(n, dtype=torch.float64, device="cuda")
            p_na = torch.full((n,), 7.0, dtype=torch.float64, device="cuda")
            opts = g.solver_opts(eps=1e-10, precond=precond)
            st, it_ref, rel_ref = g.gmaf_solve_joint(ctx.handle, nth, nz, K, D, aE, aN, S, p_ref,
                                                     opts)
            st2, it_na, rel_na = g.gmaf_solve_joint_noalloc(nth, nz, K, D, aE, aN, S, p_na, opts)
            assert st == 0 and st2 == 0
            assert abs(it_na - it_ref) <= 1      # the ordinary call may tune to another variant
            assert rel_na <= 1e-9
            a, b = p_na.cpu().numpy(), p_ref.cpu().numpy()
            assert np.linalg.norm(a - b) <= 1e-9 * np.linalg.norm(b)
    finally:
        ctx.close()


@pytest.mark.parametrize("nth,nz,K,seed,textured,precond", [
    (512, 256, 9, 4, False, 1),      # the documented fit: the largest vector offsets
    (151, 48, 5, 5, True, 1),        # odd n_theta: one column per lane
    (151, 48, 2, 6, True, 0),        # odd n_theta, Jacobi
])
def test_noalloc_solve_matches_the_oracle(g, nth, nz, K, seed, textured, precond):
    D, aE, aN, S = _problem(nth, nz, K, seed, textured)
    n = K * nth * nz
    opts = g.solver_opts(eps=1e-10, precond=precond)
    p1 = torch.full((n,), -3.0, dtype=torch.float64, device="cuda")
    st, it, rel = g.gmaf_solve_joint_noalloc(nth, nz, K, D, aE, aN, S, p1, opts)
    assert st == 0 and rel <= 1e-9
    # a second call on the same array must not see the first one's leftovers
    p2 = torch.full((n,), 11.0, dtype=torch.float64, device="cuda")
    st2, it2, rel2 = g.gmaf_solve_joint_noalloc(nth, nz, K, D, aE, aN, S, p2, opts)
    assert st2 == 0 and it2 == it and torch.equal(p1, p2)
    oracle.set_threads(0)
    try:
        sto, po, ito, _, trelo = oracle.solve_joint(nth, nz, *(a.cpu().numpy() for a in (D, aE, aN, S)),
                                                    precond=precond, eps=1e-10)
    finally:
        oracle.set_threads(1)
    assert sto == oracle.OK
    assert abs(it - ito) <= 2, (it, ito)
    a, b = p1.cpu().numpy(), po.ravel()
    assert np.linalg.norm(a - b) <= 1e-9 * np.linalg.norm(b)


def test_noalloc_refuses_problems_beyond_its_scratch(g):
    n_theta, n_z, K = 2048, 1024, 9
    small = torch.zeros(64 * 32, dtype=torch.float64, device="cuda")
    big = torch.zeros(n_theta * n_z * K, dtype=torch.float64, device="cuda")
    st, it, rel = g.gmaf_solve_joint_noalloc(n_theta, n_z, K, big, big, big, big, big,
                                             allow=(g.GMAF_OUT_OF_MEMORY,))
    assert st == g.GMAF_OUT_OF_MEMORY
    for bad in (g.solver_opts(precision=1), g.solver_opts(criterion=1)):
        with pytest.raises(g.GmafError):
            g.gmaf_solve_joint_noalloc(64, 32, 1, small, small, small, small, small, bad)
