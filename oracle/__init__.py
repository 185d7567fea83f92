"""GMAF oracle: plain FP64 CPU restatement of the piston-gap hot path.

TEST INFRASTRUCTURE ONLY.  The test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The CUDA library and its
Python binding never import this package, and this package imports nothing
from them.

The arithmetic lives in ``gmaf_oracle.c`` (plain C, FP64, compiled with
``-ffp-contract=off`` so that x86-64 and aarch64 produce the same bits).  This
module only compiles it and marshals numpy arrays.

Parameter vectors (plain float64 arrays):
  phys  = [R_k, L, c, mu, v_slide, p_chamber, p_case]
  tex   = [kind, radius, depth, area_density, offset_theta, offset_z]
  state = [e1, e2, e3, e4, edot1, edot2, edot3, edot4]
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gmaf_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, INVALID, CONTACT, NOT_CONVERGED, NONFINITE, NOMEM = 0, -1, -2, -3, -4, -5


def build(force: bool = False) -> str:
    """Compile gmaf_oracle.c into liboracle.so next to it (seconds).  OpenMP is used
    when the compiler has it; without it every loop runs on one thread (same results)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        r = subprocess.run(base[:5] + ["-fopenmp"] + base[5:], capture_output=True)
        if r.returncode != 0:
            subprocess.run(base, check=True)
        os.replace(tmp, _LIB)
    return _LIB


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            L.oracle_set_threads.restype = ctypes.c_int
            L.oracle_set_threads.argtypes = [ctypes.c_int]
            L.oracle_max_threads.restype = ctypes.c_int
            L.oracle_max_threads.argtypes = []
            L.oracle_film.restype = ctypes.c_double
            L.oracle_film.argtypes = [_D, _D, _D, ctypes.c_double, ctypes.c_double]
            L.oracle_film_rate.restype = ctypes.c_double
            L.oracle_film_rate.argtypes = [_D, _D, _D, ctypes.c_double, ctypes.c_double]
            L.oracle_texture_depth.restype = ctypes.c_double
            L.oracle_texture_depth.argtypes = [_D, _D, ctypes.c_double, ctypes.c_double]
            L.oracle_lattice.restype = None
            L.oracle_lattice.argtypes = [_D, _D, _D]
            L.oracle_assemble.restype = ctypes.c_int
            L.oracle_assemble.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D, _D, _D, _D, _D]
            L.oracle_dense_matrix.restype = ctypes.c_int
            L.oracle_dense_matrix.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D, _D]
            L.oracle_apply_matrix.restype = ctypes.c_int
            L.oracle_apply_matrix.argtypes = [ctypes.c_int] * 3 + [_D] * 5
            L.oracle_apply_precond.restype = ctypes.c_int
            L.oracle_apply_precond.argtypes = ([ctypes.c_int] * 3 + [_D] * 3 +
                                               [ctypes.c_int, ctypes.c_double, _D, _D])
            L.oracle_solve_joint.restype = ctypes.c_int
            L.oracle_solve_joint.argtypes = ([ctypes.c_int] * 3 + [_D] * 5 +
                                             [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_int, ctypes.c_int, _I, _D])
            L.oracle_loads.restype = ctypes.c_int
            L.oracle_loads.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D, _D, _D]
            L.oracle_generalized_force.restype = ctypes.c_int
            L.oracle_generalized_force.argtypes = [ctypes.c_double, _D, _D]
            L.oracle_picard_step.restype = ctypes.c_int
            L.oracle_picard_step.argtypes = ([ctypes.c_int, ctypes.c_int, _D, _D, _D, _D,
                                              ctypes.c_double, _D, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_int, _D, _D, _D, _I,
                                              _D, _D])
            L.oracle_picard_step_simplified.restype = ctypes.c_int
            L.oracle_picard_step_simplified.argtypes = ([ctypes.c_int, ctypes.c_int, _D, _D, _D,
                                                         ctypes.c_double, _D, ctypes.c_double,
                                                         ctypes.c_int, ctypes.c_double,
                                                         ctypes.c_double, ctypes.c_int, _D, _D, _D,
                                                         _I])
            _lib = L
    return _lib


def set_threads(n: int) -> int:
    """Threads for the oracle's independent-iteration loops (n < 1: all processors).
    Reductions stay sequential, so results do not depend on n.  Returns the count in
    effect (1 when the library was built without OpenMP)."""
    return int(lib().oracle_set_threads(int(n)))


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def no_texture():
    return np.zeros(6)


def film(phys, tex, e, theta, z):
    phys, tex, e = _f64(phys), _f64(tex), _f64(e)
    return lib().oracle_film(_p(phys), _p(tex), _p(e), float(theta), float(z))


def film_rate(phys, e, edot, theta, z):
    phys, e, edot = _f64(phys), _f64(e), _f64(edot)
    return lib().oracle_film_rate(_p(phys), _p(e), _p(edot), float(theta), float(z))


def texture_depth(phys, tex, x, z):
    phys, tex = _f64(phys), _f64(tex)
    return lib().oracle_texture_depth(_p(phys), _p(tex), float(x), float(z))


def lattice(phys, tex):
    phys, tex = _f64(phys), _f64(tex)
    out = np.zeros(2)
    lib().oracle_lattice(_p(phys), _p(tex), _p(out))
    return float(out[0]), float(out[1])


def assemble(nth, nz, phys, tex, state):
    """One condition -> (status, D, aE, aN, S), each of shape (nz, nth)."""
    phys, tex, state = _f64(phys), _f64(tex), _f64(state)
    n = nth * nz
    D, aE, aN, S = (np.zeros(n) for _ in range(4))
    st = lib().oracle_assemble(nth, nz, _p(phys), _p(tex), _p(state), _p(D), _p(aE), _p(aN), _p(S))
    sh = (nz, nth)
    return st, D.reshape(sh), aE.reshape(sh), aN.reshape(sh), S.reshape(sh)


def assemble_joint(nth, nz, phys, tex, states):
    """Stacked conditions -> (status, D, aE, aN, S) of shape (K, nz, nth)."""
    outs = [assemble(nth, nz, phys, tex, s) for s in states]
    st = min((o[0] for o in outs), default=0)
    return (st,) + tuple(np.stack([o[k] for o in outs]) for k in range(1, 5))


def dense_matrix(nth, nz, D, aE, aN):
    n = nth * nz
    out = np.zeros((n, n))
    st = lib().oracle_dense_matrix(nth, nz, _p(_f64(D).ravel()), _p(_f64(aE).ravel()),
                                   _p(_f64(aN).ravel()), _p(out))
    assert st == OK
    return out


def apply_matrix(nth, nz, D, aE, aN, x):
    D, aE, aN, x = (_f64(a).ravel() for a in (D, aE, aN, x))
    K = D.size // (nth * nz)
    y = np.zeros_like(x)
    st = lib().oracle_apply_matrix(nth, nz, K, _p(D), _p(aE), _p(aN), _p(x), _p(y))
    assert st == OK
    return y


def apply_precond(nth, nz, D, aE, aN, r, precond=1, omega=1.2):
    D, aE, aN, r = (_f64(a).ravel() for a in (D, aE, aN, r))
    K = D.size // (nth * nz)
    z = np.zeros_like(r)
    st = lib().oracle_apply_precond(nth, nz, K, _p(D), _p(aE), _p(aN), int(precond),
                                    float(omega), _p(r), _p(z))
    assert st == OK
    return z


def solve_joint(nth, nz, D, aE, aN, S, p0=None, precond=1, omega=1.2, eps=1e-10,
                max_iter=100000):
    """Joint PCG (Table 1 + Eq. 3.9).  Returns (status, p, iters, rel, true_rel)."""
    D, aE, aN, S = (_f64(a).ravel() for a in (D, aE, aN, S))
    K = D.size // (nth * nz)
    p = np.zeros_like(S) if p0 is None else _f64(p0).ravel().copy()
    it = ctypes.c_int(0)
    out = np.zeros(2)
    st = lib().oracle_solve_joint(nth, nz, K, _p(D), _p(aE), _p(aN), _p(S), _p(p),
                                  int(precond), float(omega), float(eps), int(max_iter),
                                  1 if p0 is None else 0, ctypes.byref(it), _p(out))
    return st, p.reshape(K, nz, nth), it.value, float(out[0]), float(out[1])


def loads(nth, nz, phys, tex, state, p):
    """-> (status, loads[12]) = pressure (Fx,Fy,Fz,Mx,My,Mz), shear (same)."""
    phys, tex, state, p = _f64(phys), _f64(tex), _f64(state), _f64(p).ravel()
    out = np.zeros(12)
    st = lib().oracle_loads(nth, nz, _p(phys), _p(tex), _p(state), _p(p), _p(out))
    return st, out


def generalized_force(L, F6):
    F6 = _f64(F6)
    G = np.zeros(4)
    lib().oracle_generalized_force(float(L), _p(F6), _p(G))
    return G


def picard_step_simplified(nth, nz, phys, tex, state, dt, F_ext, d_edot, precond=1, omega=1.2,
                           eps=1e-10, max_iter=100000):
    """One conventional (simplified) Picard iteration, Eq. 2.20-2.22, on the 5-condition
    joint batch (base + 4 rate perturbations).

    Returns dict(status, state, loads[12], J[6,8] (e-columns zero), G[4], iters).
    """
    phys, tex = _f64(phys), _f64(tex)
    st_vec = _f64(state).copy()
    F_ext = _f64(F_ext)
    loads_out, J, G = np.zeros(12), np.zeros(48), np.zeros(4)
    it = ctypes.c_int(0)
    st = lib().oracle_picard_step_simplified(nth, nz, _p(phys), _p(tex), _p(st_vec), float(dt),
                                             _p(F_ext), float(d_edot), int(precond), float(omega),
                                             float(eps), int(max_iter), _p(loads_out), _p(J),
                                             _p(G), ctypes.byref(it))
    return dict(status=st, state=st_vec, loads=loads_out, J=J.reshape(6, 8), G=G, iters=it.value)


def picard_step(nth, nz, phys, tex, state, e_prev, dt, F_ext, d_e, d_edot,
                precond=1, omega=1.2, eps=1e-10, max_iter=100000, want_fields=False):
    """One general Picard iteration on the 9-condition joint batch.

    Returns dict(status, state, loads[12], J[6,8], G[4], iters, loads_all[9,12], p).
    """
    phys, tex = _f64(phys), _f64(tex)
    st_vec = _f64(state).copy()
    e_prev, F_ext = _f64(e_prev), _f64(F_ext)
    loads_out, J, G = np.zeros(12), np.zeros(48), np.zeros(4)
    loads_all = np.zeros(9 * 12)
    p = np.zeros(9 * nth * nz) if want_fields else None
    it = ctypes.c_int(0)
    st = lib().oracle_picard_step(nth, nz, _p(phys), _p(tex), _p(st_vec), _p(e_prev), float(dt),
                                  _p(F_ext), float(d_e), float(d_edot), int(precond),
                                  float(omega), float(eps), int(max_iter), _p(loads_out),
                                  _p(J), _p(G), ctypes.byref(it), _p(loads_all), _p(p))
    return dict(status=st, state=st_vec, loads=loads_out, J=J.reshape(6, 8), G=G,
                iters=it.value, loads_all=loads_all.reshape(9, 12),
                p=None if p is None else p.reshape(9, nz, nth))
