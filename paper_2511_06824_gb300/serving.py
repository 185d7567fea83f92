"""Serving a stream of Picard-step requests, and the sequential baseline.

`serve_stream` replays a request stream against the continuous-batching server
(gmaf_server_*): a request is submitted when the wall clock passes its arrival
time, the server advances every admitted request together in rounds of
`round_iters` batched PCG iterations, requests that arrive while others run
are admitted as memory frees up, and finished results are collected after
every round.  Latency of a request = completion time - arrival time.

`sequential_stream` is the plain baseline the paper calls sequential GPU
acceleration (Sec. 3.2): one request at a time, and inside it the 9 systems
one after another in FP64 (gmaf_assemble, then gmaf_solve_joint with one
condition per call and its own criterion, then gmaf_integrate_loads), with
the 6 x 8 Jacobian and the 4 x 4 update formed on the host.

Both run the same requests and report throughput (Picard steps/s) and the
p50/p99 latency.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass
from typing import List, Optional

import numpy as np

from . import gmaf

DT = (60.0 / 600.0) / 360.0


@dataclass
class StreamItem:
    arrival_s: float
    n_theta: int
    n_z: int
    phys: np.ndarray
    tex: np.ndarray
    state: np.ndarray
    F_ext: np.ndarray


def items_from_requests(reqs, F_ext=(30.0, -15.0, 6.0, -3.0)) -> List[StreamItem]:
    return [StreamItem(r["arrival_s"], r["n_theta"], r["n_z"], r["phys"], r["tex"], r["state"],
                       np.asarray(F_ext, dtype=np.float64)) for r in reqs]


def to_request(it: StreamItem, eps: float, omega: float = 1.2, d_e: float = 2e-8,
               d_edot: float = 1e-6, max_iter: int = 100000) -> gmaf.gmaf_request:
    return gmaf.request(it.n_theta, it.n_z, it.phys, it.tex, it.state, it.state[:4], DT, it.F_ext,
                        d_e, d_edot, omega=omega, eps=eps, max_iter=max_iter)


def _summary(lat: List[float], t_first: float, t_last: float, n: int) -> dict:
    lat_ms = np.array(lat) * 1e3
    span = max(t_last - t_first, 1e-9)
    return {"completed": n, "picard_steps_per_s": n / span,
            "p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
            "mean_ms": float(lat_ms.mean()), "span_s": span}


def serve_stream(ctx: int, items: List[StreamItem], hbm_budget_bytes: int, eps: float = 1e-10,
                 round_iters: int = 64, time_scale: float = 1.0) -> dict:
    """Replay `items` (arrival times scaled by time_scale) on a server."""
    results = {}
    lat = []
    with gmaf.Server(ctx, hbm_budget_bytes) as sv:
        order = sorted(range(len(items)), key=lambda i: items[i].arrival_s)
        ids = {}
        nxt = 0
        max_active = 0
        t0 = time.perf_counter()
        while len(results) < len(items):
            now = time.perf_counter() - t0
            while nxt < len(order) and items[order[nxt]].arrival_s * time_scale <= now:
                i = order[nxt]
                ids[sv.submit(to_request(items[i], eps))] = i
                nxt += 1
            active, queued = sv.run(round_iters)
            max_active = max(max_active, active)
            t_done = time.perf_counter() - t0
            for r in sv.poll(256):
                i = ids[r["id"]]
                results[i] = r
                lat.append(t_done - items[i].arrival_s * time_scale)
            if active == 0 and queued == 0 and nxt < len(order) and len(results) < len(items):
                wait = items[order[nxt]].arrival_s * time_scale - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(wait)
        t_end = time.perf_counter() - t0
    first = min(it.arrival_s for it in items) * time_scale
    out = _summary(lat, first, t_end, len(items))
    out["max_active"] = max_active
    out["results"] = [results[i] for i in range(len(items))]
    return out


def reference_step(ctx: int, it: StreamItem, eps: float = 1e-12, omega: float = 1.2,
                   d_e: float = 2e-8, d_edot: float = 1e-6) -> dict:
    """The request's Picard step as one FP64 joint solve (gmaf_picard_step) at a tight
    eps: the accuracy reference of the equal-accuracy comparison."""
    return gmaf.gmaf_picard_step(ctx, it.n_theta, it.n_z, it.phys, it.tex, it.state, it.state[:4],
                                 DT, it.F_ext, d_e, d_edot,
                                 gmaf.solver_opts(precond=1, omega=omega, eps=eps, precision=0))


def sequential_step(ctx: int, it: StreamItem, eps: float, omega: float = 1.2, d_e: float = 2e-8,
                    d_edot: float = 1e-6) -> dict:
    """One Picard step the sequential way: 9 single-condition FP64 solves."""
    import torch
    nth, nz = it.n_theta, it.n_z
    n = nth * nz
    conds = [it.state.copy() for _ in range(9)]
    for j in range(4):
        conds[1 + j][j] += d_e
        conds[5 + j][4 + j] += d_edot
    dev = dict(dtype=torch.float64, device="cuda")
    D, aE, aN, S = (torch.empty(9 * n, **dev) for _ in range(4))
    p = torch.zeros(9 * n, **dev)
    gmaf.gmaf_assemble(ctx, nth, nz, it.phys, it.tex, conds, D, aE, aN, S)
    iters = 0
    opts = gmaf.solver_opts(precond=1, omega=omega, eps=eps, precision=0)
    for k in range(9):
        sl = slice(k * n, (k + 1) * n)
        st, i, _ = gmaf.gmaf_solve_joint(ctx, nth, nz, 1, D[sl], aE[sl], aN[sl], S[sl], p[sl], opts)
        iters += i
    loads = torch.zeros(9 * 12, **dev)
    gmaf.gmaf_integrate_loads(ctx, nth, nz, it.phys, it.tex, conds, p, loads)
    L = loads.cpu().numpy().reshape(9, 12)
    F = L[:, :6] + L[:, 6:]
    J = np.empty((6, 8))
    for c in range(8):
        J[:, c] = (F[1 + c] - F[0]) / (d_e if c < 4 else d_edot)
    Lg = it.phys[1]
    T = np.array([[1, 0, 0, 0, -1 / Lg, 0], [0, 1, 0, 1 / Lg, 0, 0], [0, 0, 0, 0, 1 / Lg, 0],
                  [0, 0, 0, -1 / Lg, 0, 0]])
    G = T @ F[0] + it.F_ext
    Je, Jd = T @ J[:, :4], T @ J[:, 4:]
    e, ed = it.state[:4], it.state[4:]
    delta = np.linalg.solve(Jd + DT * Je, -G - Je @ (it.state[:4] + DT * ed - e))
    ed_new = ed + delta
    new = np.concatenate([it.state[:4] + DT * ed_new, ed_new])
    return dict(loads=L[0], J=J, G=G, state=new, iters=iters)


def sequential_stream(ctx: int, items: List[StreamItem], eps: float = 1e-10,
                      time_scale: float = 1.0) -> dict:
    import torch
    order = sorted(range(len(items)), key=lambda i: items[i].arrival_s)
    results = {}
    lat = []
    t0 = time.perf_counter()
    for i in order:
        now = time.perf_counter() - t0
        wait = items[i].arrival_s * time_scale - now
        if wait > 0:
            time.sleep(wait)
        results[i] = sequential_step(ctx, items[i], eps)
        torch.cuda.synchronize()
        lat.append(time.perf_counter() - t0 - items[i].arrival_s * time_scale)
    t_end = time.perf_counter() - t0
    first = min(it.arrival_s for it in items) * time_scale
    out = _summary(lat, first, t_end, len(items))
    out["results"] = [results[i] for i in range(len(items))]
    return out


def load_error(a, b) -> float:
    """max_c |a_c - b_c| / max(|b_c|, 1e-3 ||b||) over the pressure and shear parts."""
    a, b = np.asarray(a), np.asarray(b)
    err = 0.0
    for part in (slice(0, 6), slice(6, 12)):
        x, y = a[part], b[part]
        scale = np.maximum(np.abs(y), 1e-3 * np.linalg.norm(y))
        err = max(err, float(np.max(np.abs(x - y) / scale)))
    return err
