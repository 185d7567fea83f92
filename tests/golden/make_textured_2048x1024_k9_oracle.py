#!/usr/bin/env python
"""Writes the oracle's Picard step of the textured 2048 x 1024 x 9 workload (seed 0,
the benchmark's configuration) as a golden fixture.

The oracle (plain C, FP64) assembles the 9 conditions (base, e_j + d_e,
edot_j + d_edot; Eq. 2.13-2.19), solves them as one joint system with ASSOR-II
PCG under the synchronized criterion (Table 1, Eq. 3.4-3.9; omega 1.2), integrates
the loads (Sec. 2.4-III) and takes the general Picard update (Eq. 2.12).  The
fixture keeps what a GPU step can be compared with: the 9 x 12 loads, the 6 x 8
Jacobian, the generalized force, the updated state, the iteration count, and per
condition the 2-norm of the pressure field and its values at 1000 seeded cells
(the full fields, 151 MB, are not stored).

Only the oracle and the seeded input generator are called.  The run takes a few
minutes with all host cores (oracle.set_threads; the results do not depend on the
thread count) and about 20 minutes on one.

    python tests/golden/make_textured_2048x1024_k9_oracle.py --eps 1e-10
    python tests/golden/make_textured_2048x1024_k9_oracle.py --eps 1e-12
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2511_06824_gb300 import inputs  # noqa: E402

WORKLOAD = "textured-2048x1024-k9"
SEED = 0
DT = (60.0 / 600.0) / 360.0
F_EXT = [40.0, -20.0, 8.0, -4.0]
SAMPLE_SEED = 2511_06824
N_SAMPLES = 1000


def path_for(eps: float) -> str:
    return os.path.join(HERE, f"{WORKLOAD}_seed{SEED}_oracle_eps{eps:.0e}.json")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--eps", type=float, default=1e-10)
    ap.add_argument("--threads", type=int, default=0, help="oracle threads (0: all)")
    a = ap.parse_args()
    w = inputs.make(WORKLOAD, SEED)
    threads = oracle.set_threads(a.threads)
    t0 = time.perf_counter()
    r = oracle.picard_step(w.n_theta, w.n_z, w.phys, w.tex, w.state, w.state[:4], DT,
                           np.array(F_EXT), w.d_e, w.d_edot, precond=1, omega=w.omega, eps=a.eps,
                           want_fields=True)
    secs = time.perf_counter() - t0
    if r["status"] != oracle.OK:
        raise SystemExit(f"oracle status {r['status']}")
    p = r["p"].reshape(9, -1)
    idx = np.sort(np.random.default_rng(SAMPLE_SEED).choice(w.n, size=N_SAMPLES, replace=False))
    out = {
        "what": "oracle Picard step (general scheme, 9 conditions) of the benchmark workload",
        "workload": WORKLOAD, "seed": SEED, "n_theta": w.n_theta, "n_z": w.n_z,
        "omega": w.omega, "eps": a.eps, "precond": "ASSOR-II", "dt": DT, "F_ext": F_EXT,
        "d_e": w.d_e, "d_edot": w.d_edot, "state_in": w.state.tolist(),
        "iterations": r["iters"], "state_out": r["state"].tolist(),
        "loads_all": r["loads_all"].tolist(), "J": r["J"].tolist(), "G": r["G"].tolist(),
        "p_norm": [float(np.linalg.norm(p[k])) for k in range(9)],
        "sample_index": idx.tolist(),
        "p_samples": [p[k][idx].tolist() for k in range(9)],
        "oracle_threads": threads, "oracle_seconds": round(secs, 1),
        "script": "tests/golden/make_textured_2048x1024_k9_oracle.py",
    }
    with open(path_for(a.eps), "w") as f:
        json.dump(out, f, indent=1)
    print(f"wrote {path_for(a.eps)}: {r['iters']} iterations, {secs:.0f} s on {threads} threads")


if __name__ == "__main__":
    main()
