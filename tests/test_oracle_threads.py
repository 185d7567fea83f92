"""The oracle's thread count changes its speed, never its results: assembly, the
preconditioner, the joint PCG and a whole Picard step are bitwise the same on one
thread and on all processors (every reduction stays sequential)."""
import numpy as np
import pytest

import oracle
from paper_2511_06824_gb300 import inputs


@pytest.fixture
def threads():
    yield
    oracle.set_threads(1)


def _run(w, conds):
    st, D, aE, aN, S = oracle.assemble_joint(w.n_theta, w.n_z, w.phys, w.tex, conds)
    z = oracle.apply_precond(w.n_theta, w.n_z, D, aE, aN, S, precond=1, omega=1.2)
    z2 = oracle.apply_precond(w.n_theta, w.n_z, D, aE, aN, S, precond=2, omega=1.2)
    sol = oracle.solve_joint(w.n_theta, w.n_z, D, aE, aN, S, eps=1e-10, max_iter=40)
    return (D, aE, aN, S, z, z2, sol[1], np.array([sol[2], sol[3], sol[4]]))


def test_results_do_not_depend_on_the_thread_count(threads):
    w = inputs.make("textured-256x128-k3", 5)
    conds = [inputs.random_state(np.random.default_rng(k)) for k in range(3)]
    assert oracle.set_threads(1) == 1
    one = _run(w, conds)
    n = oracle.set_threads(0)
    assert n == oracle.max_threads() >= 1
    many = _run(w, conds)
    for a, b in zip(one, many):
        assert np.array_equal(a, b)


def test_picard_step_does_not_depend_on_the_thread_count(threads):
    w = inputs.make("textured-128x96-k9", 2)
    F = np.array([20.0, -10.0, 5.0, 2.0])
    res = []
    for t in (1, 0):
        oracle.set_threads(t)
        r = oracle.picard_step(w.n_theta, w.n_z, w.phys, w.tex, w.state, w.state[:4], 2.78e-4, F,
                               w.d_e, w.d_edot, eps=1e-10)
        res.append(r)
    for k in ("state", "loads", "J", "G", "loads_all"):
        assert np.array_equal(res[0][k], res[1][k]), k
    assert res[0]["iters"] == res[1]["iters"]
