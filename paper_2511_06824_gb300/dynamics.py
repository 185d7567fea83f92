"""Multi-period piston dynamics on the GPU (the time march around the Picard step).

For each shaft-angle step (Sec. 4.3: 360 steps per revolution, several Picard
iterations per step) the chamber pressure and the sliding speed are set for the
step's angle, and general Picard iterations (Eq. 2.12 with the double Jacobian,
one gmaf_picard_step each) run until the generalized force balance
||G||_2 <= tol_F * max(||F_ext||_2, 1 N) holds or the iteration budget is spent.
The eccentricity at the start of a step is the converged one of the previous
step (backward difference, Eq. 2.22).

The paper gives no formula for the external and inertia loads (Eq. 2.10 names
them only); the march uses a synthetic side load from the swash plate, the
chamber force times tan(10 deg) (swash angle of Table 8) scaled by `kappa`,
acting at the case end of the gap (generalized force on e3).  The default
kappa = 0.2 keeps the eccentricity below 0.6 c over a revolution of the oracle
on a 48 x 24 grid with the seeded trapezoid pressure (bound asked: 0.8 c).  The
load always acts along +x and nothing in the model restores the centred
position, so on finer textured grids the eccentricity keeps growing under load:
on the textured 1024 x 512 gap it reaches the wall within the first revolution
(shaft step 76 with kappa = 0.2, in FP64 as in mixed precision).

Everything per Picard iteration runs on the device through the C ABI; this
module is the host loop.  The pressure fields stay in the library's context and
each solve warm-starts from the previous iterate (opts.zero_init = 0).
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np

from . import gmaf

SWASH_ANGLE_DEG = 10.0


def side_load(p_chamber: float, radius: float, kappa: float) -> np.ndarray:
    """Generalized external force of the synthetic swash-plate side load.

    F_s = kappa * p_chamber * pi R_k^2 * tan(swash angle), a force along +x applied
    at z = L; its virtual work on the linear tilt loads e3 only."""
    f = kappa * p_chamber * math.pi * radius ** 2 * math.tan(math.radians(SWASH_ANGLE_DEG))
    return np.array([0.0, 0.0, f, 0.0])


@dataclass
class StepRecord:
    step: int
    phi_deg: float
    p_chamber: float
    v_slide: float
    picard_iterations: int
    pcg_iterations: int
    converged: bool
    state: np.ndarray
    G_norm: float
    loads: np.ndarray
    seconds: float


@dataclass
class Trajectory:
    records: List[StepRecord] = field(default_factory=list)

    @property
    def states(self) -> np.ndarray:
        return np.array([r.state for r in self.records])

    @property
    def picard_iterations(self) -> int:
        return sum(r.picard_iterations for r in self.records)

    @property
    def seconds(self) -> float:
        return sum(r.seconds for r in self.records)


def march(ctx: int, n_theta: int, n_z: int, phys, tex, state0, p_profile, steps: int,
          steps_per_rev: int = 360, rpm: float = 600.0, v_amp: float = 5.0,
          kappa: float = 0.2, tol_F: float = 1e-6, max_picard: int = 20,
          d_e: float = 2e-8, d_edot: float = 1e-6, opts: Optional[gmaf.gmaf_solver_opts] = None,
          on_step: Optional[Callable[[StepRecord], None]] = None,
          scheme: str = "general") -> Trajectory:
    """Run `steps` shaft-angle steps.  p_profile[s % steps_per_rev] is the chamber
    pressure of step s; the sliding speed is v_amp * sin(phi).

    scheme "general": the double-Jacobian Picard iteration (Eq. 2.12-2.19, 9 conditions).
    scheme "simplified": the conventional one (Eq. 2.20-2.22, 5 conditions); each time
    step starts from the predictor e = e_l + dt edot_l, so that the increments of
    Eq. 2.22 keep e = e_l + dt edot, the backward difference, at every iterate."""
    if scheme not in ("general", "simplified"):
        raise ValueError(f"unknown scheme {scheme!r}")
    phys = np.asarray(phys, dtype=np.float64).copy()
    dt = (60.0 / rpm) / steps_per_rev
    state = np.asarray(state0, dtype=np.float64).copy()
    o = opts or gmaf.solver_opts(precision=1)
    warm = gmaf.gmaf_solver_opts(o.precond, o.omega, o.eps, o.max_iter, o.precision, 0, o.criterion)
    traj = Trajectory()
    first_solve = True
    for s in range(steps):
        t0 = time.perf_counter()
        phi = 2.0 * math.pi * (s % steps_per_rev) / steps_per_rev
        ph = phys.copy()
        ph[5] = float(p_profile[s % steps_per_rev])
        ph[4] = v_amp * math.sin(phi)
        F_ext = side_load(ph[5], ph[0], kappa)
        scale = max(float(np.linalg.norm(F_ext)), 1.0)
        e_prev = state[:4].copy()
        if scheme == "simplified":
            state[:4] = e_prev + dt * state[4:]
        converged = False
        pcg = 0
        G_norm = float("inf")
        loads = np.zeros(12)
        it = 0
        for it in range(1, max_picard + 1):
            oo = o if first_solve else warm
            if scheme == "simplified":
                r = gmaf.gmaf_picard_step_simplified(ctx, n_theta, n_z, ph, tex, state, dt, F_ext,
                                                     d_edot, oo)
            else:
                r = gmaf.gmaf_picard_step(ctx, n_theta, n_z, ph, tex, state, e_prev, dt, F_ext, d_e,
                                          d_edot, oo)
            first_solve = False
            pcg += r["iters"]
            G_norm = float(np.linalg.norm(r["G"]))
            loads = r["loads"]
            if G_norm <= tol_F * scale:
                converged = True          # the state before this update balances the forces
                break
            state = r["state"]
        rec = StepRecord(step=s, phi_deg=math.degrees(phi), p_chamber=ph[5], v_slide=ph[4],
                         picard_iterations=it, pcg_iterations=pcg, converged=converged,
                         state=state.copy(), G_norm=G_norm, loads=loads.copy(),
                         seconds=time.perf_counter() - t0)
        traj.records.append(rec)
        if on_step:
            on_step(rec)
    return traj
