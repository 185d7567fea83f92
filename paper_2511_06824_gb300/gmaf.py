"""Python binding of the C ABI in include/gmaf.h (argument marshalling only).

Every computation runs in libgmaf.so's CUDA kernels; this module converts
Python/torch arguments into the C structs and pointers and raises on a
non-zero status.  There is no CPU fallback: importing the binding without a
built library, or calling it without a CUDA device, raises.

Device arrays are torch tensors (float64, contiguous, on the context's device);
host arrays are numpy arrays or sequences.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgmaf.so")

GMAF_OK = 0
GMAF_INVALID_ARG = -1
GMAF_CONTACT = -2
GMAF_NOT_CONVERGED = -3
GMAF_NONFINITE = -4
GMAF_OUT_OF_MEMORY = -5
GMAF_CUDA_ERROR = -6
GMAF_TIMEOUT = -7
GMAF_CANCELLED = -8

EXPORTED = ("gmaf_create", "gmaf_destroy", "gmaf_set_stream", "gmaf_workspace_bytes",
            "gmaf_last_solve_info", "gmaf_assemble", "gmaf_solve_joint", "gmaf_integrate_loads",
            "gmaf_picard_step", "gmaf_status_string", "gmaf_set_phase_timing",
            "gmaf_phase_timing", "gmaf_solve_joint_noalloc", "gmaf_request_footprint",
            "gmaf_server_create", "gmaf_server_destroy", "gmaf_server_submit", "gmaf_server_run",
            "gmaf_server_poll", "gmaf_server_free_bytes", "gmaf_last_fields",
            "gmaf_picard_step_simplified", "gmaf_server_cancel")


class gmaf_grid(ctypes.Structure):
    _fields_ = [("n_theta", ctypes.c_int32), ("n_z", ctypes.c_int32)]


class gmaf_physics(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("R_k", "L", "c", "mu", "v_slide", "p_chamber",
                                               "p_case")]


class gmaf_texture(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32)] + [(k, ctypes.c_double) for k in (
        "radius", "depth", "area_density", "offset_theta", "offset_z")]


class gmaf_state(ctypes.Structure):
    _fields_ = [("e", ctypes.c_double * 4), ("edot", ctypes.c_double * 4)]


class gmaf_solver_opts(ctypes.Structure):
    _fields_ = [("precond", ctypes.c_int32), ("omega", ctypes.c_double), ("eps", ctypes.c_double),
                ("max_iter", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("zero_init", ctypes.c_int32), ("criterion", ctypes.c_int32)]


class gmaf_solve_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("outer_iterations", ctypes.c_int32),
                ("restarts", ctypes.c_int32), ("status", ctypes.c_int32),
                ("rel_residual", ctypes.c_double), ("true_rel_residual", ctypes.c_double),
                ("kernel_variant", ctypes.c_int32), ("tasks", ctypes.c_int32),
                ("iterations_sum", ctypes.c_int32), ("p_update_period", ctypes.c_int32)]


class gmaf_request(ctypes.Structure):
    _fields_ = [("grid", gmaf_grid), ("phys", gmaf_physics), ("tex", gmaf_texture),
                ("state", gmaf_state), ("e_prev", ctypes.c_double * 4), ("dt", ctypes.c_double),
                ("F_ext", ctypes.c_double * 4), ("d_e", ctypes.c_double),
                ("d_edot", ctypes.c_double), ("omega", ctypes.c_double), ("eps", ctypes.c_double),
                ("max_iter", ctypes.c_int32)]


class gmaf_result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("status", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("outer_iterations", ctypes.c_int32), ("true_rel_residual", ctypes.c_double),
                ("state", gmaf_state), ("loads", ctypes.c_double * 12), ("J", ctypes.c_double * 48),
                ("G", ctypes.c_double * 4), ("tile_rows", ctypes.c_int32)]


class GmafError(RuntimeError):
    def __init__(self, fn: str, status: int):
        self.status = status
        super().__init__(f"{fn}: {status_string(status)} ({status})")


_lib = None
_VP = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)


def load(path: str = LIB_PATH):
    """Load libgmaf.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"libgmaf.so not built at {path}; run paper_2511_06824_gb300/build.py")
    L = ctypes.CDLL(path)
    L.gmaf_create.argtypes = [ctypes.POINTER(_VP), ctypes.c_size_t, _VP]
    L.gmaf_destroy.argtypes = [_VP]
    L.gmaf_set_stream.argtypes = [_VP, _VP]
    L.gmaf_workspace_bytes.argtypes = [_VP, ctypes.POINTER(ctypes.c_size_t)]
    L.gmaf_last_solve_info.argtypes = [_VP, ctypes.POINTER(gmaf_solve_info)]
    L.gmaf_assemble.argtypes = [_VP, ctypes.POINTER(gmaf_grid), ctypes.POINTER(gmaf_physics),
                                ctypes.POINTER(gmaf_texture), ctypes.POINTER(gmaf_state),
                                ctypes.c_int32, _VP, _VP, _VP, _VP]
    L.gmaf_solve_joint.argtypes = [_VP, ctypes.POINTER(gmaf_grid), ctypes.c_int32, _VP, _VP, _VP,
                                   _VP, _VP, ctypes.POINTER(gmaf_solver_opts),
                                   ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)]
    L.gmaf_integrate_loads.argtypes = [_VP, ctypes.POINTER(gmaf_grid), ctypes.POINTER(gmaf_physics),
                                       ctypes.POINTER(gmaf_texture), ctypes.POINTER(gmaf_state),
                                       ctypes.c_int32, _VP, _VP]
    L.gmaf_picard_step.argtypes = [_VP, ctypes.POINTER(gmaf_grid), ctypes.POINTER(gmaf_physics),
                                   ctypes.POINTER(gmaf_texture), ctypes.POINTER(gmaf_state), _DP,
                                   ctypes.c_double, _DP, ctypes.c_double, ctypes.c_double,
                                   ctypes.POINTER(gmaf_solver_opts), _DP, _DP, _DP,
                                   ctypes.POINTER(ctypes.c_int32)]
    L.gmaf_picard_step_simplified.argtypes = [
        _VP, ctypes.POINTER(gmaf_grid), ctypes.POINTER(gmaf_physics), ctypes.POINTER(gmaf_texture),
        ctypes.POINTER(gmaf_state), ctypes.c_double, _DP, ctypes.c_double,
        ctypes.POINTER(gmaf_solver_opts), _DP, _DP, _DP, ctypes.POINTER(ctypes.c_int32)]
    L.gmaf_set_phase_timing.argtypes = [_VP, ctypes.c_int]
    L.gmaf_phase_timing.argtypes = [_VP, _DP, ctypes.POINTER(ctypes.c_int64)]
    L.gmaf_solve_joint_noalloc.argtypes = [ctypes.POINTER(gmaf_grid), ctypes.c_int32, _VP, _VP,
                                           _VP, _VP, _VP, ctypes.POINTER(gmaf_solver_opts), _VP,
                                           ctypes.POINTER(ctypes.c_int32),
                                           ctypes.POINTER(ctypes.c_double)]
    L.gmaf_request_footprint.argtypes = [ctypes.POINTER(gmaf_grid), ctypes.POINTER(ctypes.c_size_t)]
    L.gmaf_server_create.argtypes = [_VP, ctypes.c_size_t, ctypes.POINTER(_VP)]
    L.gmaf_server_destroy.argtypes = [_VP]
    L.gmaf_server_submit.argtypes = [_VP, ctypes.POINTER(gmaf_request), ctypes.POINTER(ctypes.c_int64)]
    L.gmaf_server_run.argtypes = [_VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                  ctypes.POINTER(ctypes.c_int32)]
    L.gmaf_server_poll.argtypes = [_VP, ctypes.POINTER(gmaf_result), ctypes.c_int32,
                                   ctypes.POINTER(ctypes.c_int32)]
    L.gmaf_server_free_bytes.argtypes = [_VP, ctypes.POINTER(ctypes.c_size_t)]
    L.gmaf_server_cancel.argtypes = [_VP, ctypes.c_int64]
    L.gmaf_last_fields.argtypes = [_VP, ctypes.POINTER(gmaf_grid), _VP]
    L.gmaf_status_string.argtypes = [ctypes.c_int]
    L.gmaf_status_string.restype = ctypes.c_char_p
    for name in EXPORTED:
        if name != "gmaf_status_string":
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def status_string(st: int) -> str:
    return load().gmaf_status_string(int(st)).decode()


# ------------------------------------------------------------------ marshalling helpers


def grid(n_theta: int, n_z: int) -> gmaf_grid:
    return gmaf_grid(int(n_theta), int(n_z))


def physics(phys: Sequence[float]) -> gmaf_physics:
    """phys = [R_k, L, c, mu, v_slide, p_chamber, p_case]"""
    return gmaf_physics(*[float(x) for x in phys])


def texture(tex: Optional[Sequence[float]]) -> gmaf_texture:
    """tex = [kind, radius, depth, area_density, offset_theta, offset_z] or None (smooth)"""
    if tex is None:
        return gmaf_texture(0, 0.0, 0.0, 0.0, 0.0, 0.0)
    return gmaf_texture(int(tex[0]), *[float(x) for x in tex[1:6]])


def state(s: Sequence[float]) -> gmaf_state:
    """s = [e1, e2, e3, e4, edot1, edot2, edot3, edot4]"""
    st = gmaf_state()
    for q in range(4):
        st.e[q] = float(s[q])
        st.edot[q] = float(s[4 + q])
    return st


def state_vector(st: gmaf_state) -> np.ndarray:
    return np.array(list(st.e) + list(st.edot), dtype=np.float64)


def solver_opts(precond=1, omega=1.2, eps=1e-10, max_iter=100000, precision=0,
                zero_init=1, criterion=0) -> gmaf_solver_opts:
    return gmaf_solver_opts(int(precond), float(omega), float(eps), int(max_iter), int(precision),
                            int(zero_init), int(criterion))


def _dev(t, n: int, name: str) -> int:
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float64 tensor")
    if t.numel() < n:
        raise ValueError(f"{name} has {t.numel()} elements, needs {n}")
    return t.data_ptr()


def _f64(a, n: int) -> np.ndarray:
    x = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if x.size != n:
        raise ValueError(f"expected {n} values")
    return x


def _check(fn: str, st: int, ok=(GMAF_OK,)) -> int:
    if st not in ok:
        raise GmafError(fn, st)
    return st


# ------------------------------------------------------------------ the ABI, one function per entry point


def gmaf_create(hbm_budget_bytes: int = 0, stream=None) -> int:
    """Returns the context handle (an integer address)."""
    L = load()
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    h = _VP()
    _check("gmaf_create", L.gmaf_create(ctypes.byref(h), int(hbm_budget_bytes), _VP(stream)))
    return h.value


def gmaf_destroy(ctx: int) -> None:
    _check("gmaf_destroy", load().gmaf_destroy(_VP(ctx)))


def gmaf_set_stream(ctx: int, stream) -> None:
    _check("gmaf_set_stream", load().gmaf_set_stream(_VP(ctx), _VP(stream)))


def gmaf_workspace_bytes(ctx: int) -> int:
    b = ctypes.c_size_t(0)
    _check("gmaf_workspace_bytes", load().gmaf_workspace_bytes(_VP(ctx), ctypes.byref(b)))
    return b.value


def gmaf_last_solve_info(ctx: int) -> dict:
    i = gmaf_solve_info()
    _check("gmaf_last_solve_info", load().gmaf_last_solve_info(_VP(ctx), ctypes.byref(i)))
    return {k: getattr(i, k) for k, _ in gmaf_solve_info._fields_}


def gmaf_assemble(ctx: int, n_theta: int, n_z: int, phys, tex, conds, D, aE, aN, S,
                  allow_contact: bool = False) -> int:
    """conds: sequence of 8-vectors.  D, aE, aN, S: float64 CUDA tensors of K*n_z*n_theta."""
    K = len(conds)
    n = K * n_theta * n_z
    arr = (gmaf_state * K)(*[state(c) for c in conds])
    g, ph, tx = grid(n_theta, n_z), physics(phys), texture(tex)
    st = load().gmaf_assemble(_VP(ctx), ctypes.byref(g), ctypes.byref(ph), ctypes.byref(tx), arr, K,
                              _dev(D, n, "D"), _dev(aE, n, "aE"), _dev(aN, n, "aN"), _dev(S, n, "S"))
    return _check("gmaf_assemble", st, (GMAF_OK, GMAF_CONTACT) if allow_contact else (GMAF_OK,))


def gmaf_solve_joint(ctx: int, n_theta: int, n_z: int, n_cond: int, D, aE, aN, S, p,
                     opts: Optional[gmaf_solver_opts] = None, allow_not_converged: bool = False,
                     allow: Sequence[int] = ()):
    """Returns (status, iterations, true relative residual).  Statuses other than
    GMAF_OK (and GMAF_NOT_CONVERGED with allow_not_converged, or any listed in
    allow) raise GmafError."""
    n = n_cond * n_theta * n_z
    g = grid(n_theta, n_z)
    o = opts or solver_opts()
    it = ctypes.c_int32(0)
    rel = ctypes.c_double(0.0)
    st = load().gmaf_solve_joint(_VP(ctx), ctypes.byref(g), int(n_cond), _dev(D, n, "D"),
                                 _dev(aE, n, "aE"), _dev(aN, n, "aN"), _dev(S, n, "S"),
                                 _dev(p, n, "p"), ctypes.byref(o), ctypes.byref(it),
                                 ctypes.byref(rel))
    ok = (GMAF_OK, GMAF_NOT_CONVERGED) if allow_not_converged else (GMAF_OK,)
    _check("gmaf_solve_joint", st, tuple(ok) + tuple(allow))
    return st, it.value, rel.value


def gmaf_integrate_loads(ctx: int, n_theta: int, n_z: int, phys, tex, conds, p, loads) -> None:
    """loads: float64 CUDA tensor of K*12 (pressure Fx..Mz, shear Fx..Mz per condition)."""
    K = len(conds)
    arr = (gmaf_state * K)(*[state(c) for c in conds])
    g, ph, tx = grid(n_theta, n_z), physics(phys), texture(tex)
    st = load().gmaf_integrate_loads(_VP(ctx), ctypes.byref(g), ctypes.byref(ph), ctypes.byref(tx),
                                     arr, K, _dev(p, K * n_theta * n_z, "p"),
                                     _dev(loads, 12 * K, "loads"))
    _check("gmaf_integrate_loads", st)


def gmaf_picard_step(ctx: int, n_theta: int, n_z: int, phys, tex, st_vec, e_prev, dt, F_ext,
                     d_e, d_edot, opts: Optional[gmaf_solver_opts] = None,
                     allow=(GMAF_OK,)) -> dict:
    """One Picard iteration; all arguments on the host.  Returns a dict with the
    status, new state (8-vector), loads[12], J[6,8], G[4] and iterations."""
    g, ph, tx = grid(n_theta, n_z), physics(phys), texture(tex)
    s = state(st_vec)
    ep = _f64(e_prev, 4)
    fe = _f64(F_ext, 4)
    loads = np.zeros(12)
    J = np.zeros(48)
    G = np.zeros(4)
    it = ctypes.c_int32(0)
    o = opts or solver_opts()
    rc = load().gmaf_picard_step(_VP(ctx), ctypes.byref(g), ctypes.byref(ph), ctypes.byref(tx),
                                 ctypes.byref(s), ep.ctypes.data_as(_DP), float(dt),
                                 fe.ctypes.data_as(_DP), float(d_e), float(d_edot), ctypes.byref(o),
                                 loads.ctypes.data_as(_DP), J.ctypes.data_as(_DP),
                                 G.ctypes.data_as(_DP), ctypes.byref(it))
    _check("gmaf_picard_step", rc, allow)
    return dict(status=rc, state=state_vector(s), loads=loads, J=J.reshape(6, 8), G=G,
                iters=it.value)


def gmaf_picard_step_simplified(ctx: int, n_theta: int, n_z: int, phys, tex, st_vec, dt, F_ext,
                                d_edot, opts: Optional[gmaf_solver_opts] = None,
                                allow=(GMAF_OK,)) -> dict:
    """One conventional (simplified) Picard iteration, Eq. 2.20-2.22; the result dict
    as gmaf_picard_step's (J's e-columns zero)."""
    g, ph, tx = grid(n_theta, n_z), physics(phys), texture(tex)
    s = state(st_vec)
    fe = _f64(F_ext, 4)
    loads = np.zeros(12)
    J = np.zeros(48)
    G = np.zeros(4)
    it = ctypes.c_int32(0)
    o = opts or solver_opts()
    rc = load().gmaf_picard_step_simplified(_VP(ctx), ctypes.byref(g), ctypes.byref(ph),
                                            ctypes.byref(tx), ctypes.byref(s), float(dt),
                                            fe.ctypes.data_as(_DP), float(d_edot), ctypes.byref(o),
                                            loads.ctypes.data_as(_DP), J.ctypes.data_as(_DP),
                                            G.ctypes.data_as(_DP), ctypes.byref(it))
    _check("gmaf_picard_step_simplified", rc, allow)
    return dict(status=rc, state=state_vector(s), loads=loads, J=J.reshape(6, 8), G=G,
                iters=it.value)


def gmaf_last_fields(ctx: int, n_theta: int, n_z: int, p_out) -> None:
    """Copy the 9 pressure fields of the last Picard step into a float64 CUDA tensor."""
    g = grid(n_theta, n_z)
    _check("gmaf_last_fields", load().gmaf_last_fields(_VP(ctx), ctypes.byref(g),
                                                        _dev(p_out, 9 * n_theta * n_z, "p_out")))


def gmaf_set_phase_timing(ctx: int, on: bool) -> None:
    _check("gmaf_set_phase_timing", load().gmaf_set_phase_timing(_VP(ctx), 1 if on else 0))


PHASES = ("phase_a", "phase_b", "init_b", "resid64")


def gmaf_phase_timing(ctx: int) -> dict:
    """{kind: (total_ms, launches)} for phase_a, phase_b, init_b, resid64."""
    ms = np.zeros(4)
    cnt = (ctypes.c_int64 * 4)()
    _check("gmaf_phase_timing", load().gmaf_phase_timing(_VP(ctx), ms.ctypes.data_as(_DP), cnt))
    return {k: (float(ms[q]), int(cnt[q])) for q, k in enumerate(PHASES)}


def gmaf_solve_joint_noalloc(n_theta: int, n_z: int, n_cond: int, D, aE, aN, S, p,
                             opts: Optional[gmaf_solver_opts] = None, stream=None,
                             allow=(GMAF_OK,)):
    """FP64 joint solve that allocates no device memory (scratch is a fixed array
    inside the library).  Returns (status, iterations, true relative residual)."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    n = n_cond * n_theta * n_z
    g = grid(n_theta, n_z)
    o = opts or solver_opts()
    it = ctypes.c_int32(0)
    rel = ctypes.c_double(0.0)
    st = load().gmaf_solve_joint_noalloc(ctypes.byref(g), int(n_cond), _dev(D, n, "D"),
                                         _dev(aE, n, "aE"), _dev(aN, n, "aN"), _dev(S, n, "S"),
                                         _dev(p, n, "p"), ctypes.byref(o), _VP(stream),
                                         ctypes.byref(it), ctypes.byref(rel))
    _check("gmaf_solve_joint_noalloc", st, allow)
    return st, it.value, rel.value


def request(n_theta, n_z, phys, tex, st_vec, e_prev, dt, F_ext, d_e, d_edot, omega=1.2,
            eps=1e-10, max_iter=100000) -> gmaf_request:
    r = gmaf_request()
    r.grid = grid(n_theta, n_z)
    r.phys = physics(phys)
    r.tex = texture(tex)
    r.state = state(st_vec)
    for q in range(4):
        r.e_prev[q] = float(e_prev[q])
        r.F_ext[q] = float(F_ext[q])
    r.dt, r.d_e, r.d_edot = float(dt), float(d_e), float(d_edot)
    r.omega, r.eps, r.max_iter = float(omega), float(eps), int(max_iter)
    return r


def gmaf_request_footprint(n_theta: int, n_z: int) -> int:
    b = ctypes.c_size_t(0)
    g = grid(n_theta, n_z)
    _check("gmaf_request_footprint", load().gmaf_request_footprint(ctypes.byref(g), ctypes.byref(b)))
    return b.value


def result_dict(r: gmaf_result) -> dict:
    return dict(id=r.id, status=r.status, iters=r.iterations, outer=r.outer_iterations,
                true_rel=r.true_rel_residual, state=state_vector(r.state),
                loads=np.array(r.loads), J=np.array(r.J).reshape(6, 8), G=np.array(r.G),
                tile_rows=r.tile_rows)


class Server:
    """Continuous-batching server of Picard-step requests (gmaf_server_*)."""

    def __init__(self, ctx: int, hbm_budget_bytes: int):
        h = _VP()
        _check("gmaf_server_create", load().gmaf_server_create(_VP(ctx), int(hbm_budget_bytes),
                                                                ctypes.byref(h)))
        self.handle = h.value

    def submit(self, req: gmaf_request) -> int:
        i = ctypes.c_int64(0)
        _check("gmaf_server_submit", load().gmaf_server_submit(_VP(self.handle), ctypes.byref(req),
                                                                ctypes.byref(i)))
        return i.value

    def run(self, iterations: int):
        a, q = ctypes.c_int32(0), ctypes.c_int32(0)
        _check("gmaf_server_run", load().gmaf_server_run(_VP(self.handle), int(iterations),
                                                          ctypes.byref(a), ctypes.byref(q)))
        return a.value, q.value

    def poll(self, max_results: int = 64) -> list:
        buf = (gmaf_result * max_results)()
        n = ctypes.c_int32(0)
        _check("gmaf_server_poll", load().gmaf_server_poll(_VP(self.handle), buf, max_results,
                                                            ctypes.byref(n)))
        return [result_dict(buf[i]) for i in range(n.value)]

    def free_bytes(self) -> int:
        b = ctypes.c_size_t(0)
        _check("gmaf_server_free_bytes", load().gmaf_server_free_bytes(_VP(self.handle),
                                                                        ctypes.byref(b)))
        return b.value

    def cancel(self, request_id: int):
        _check("gmaf_server_cancel", load().gmaf_server_cancel(_VP(self.handle),
                                                                int(request_id)))

    def close(self):
        if self.handle:
            _check("gmaf_server_destroy", load().gmaf_server_destroy(_VP(self.handle)))
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Context:
    """Owns one gmaf context on the current CUDA device and stream."""

    def __init__(self, hbm_budget_bytes: int = 0, stream=None):
        self.handle = gmaf_create(hbm_budget_bytes, stream)

    def close(self):
        if self.handle:
            gmaf_destroy(self.handle)
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
