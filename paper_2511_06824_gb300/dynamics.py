"""Multi-period piston dynamics on the GPU (the time march around the Picard step).

For each shaft-angle step (Sec. 4.3: 360 steps per revolution, several Picard
iterations per step) the chamber pressure and the sliding speed are set for the
step's angle, and general Picard iterations (Eq. 2.12 with the double Jacobian,
one gmaf_picard_step each) run until the generalized force balance
||G||_2 <= tol_F * max(||F_ext||_2, p_chamber pi R_k^2, 1 N) holds or the
iteration budget is spent.  The scale includes the chamber force on the piston
(force_scale): the loads are resolved to about 1e-9 of the pressure force, so a
balance asked only relative to a small side load (micronewtons) could not be met.
The eccentricity at the start of a step is the converged one of the previous
step (backward difference, Eq. 2.22).

The paper gives no formula for the external and inertia loads (Eq. 2.10 names
them only).  The march uses:
- a synthetic side load from the swash plate, the chamber force times
  tan(10 deg) (swash angle of Table 8) scaled by `kappa`, acting at the case
  end of the gap (generalized force on e3).  The load always acts along +x and
  nothing in the model restores the centred position, so under a steady load
  the eccentricity keeps growing; kappa is calibrated so that the march stays
  within 0.8 c (see the benchmark's dynamics mode for the configured value);
- the piston's inertia F_I = -M e'' (Eq. 2.10) with the piston mass m_K of
  Table 8 spread evenly over the coupling length: the virtual work of -rho x''
  over the linear tilt x(z) = (1 - z/L) e1 + (z/L) e3 (likewise y with e2, e4)
  gives the generalized mass matrix M = m_K [[1/3, 1/6], [1/6, 1/3]] per
  direction.  e'' is the backward difference (edot - edot_l) / dt of the rate,
  as Eq. 2.22 uses for e.  It enters each Picard iteration through F_ext,
  evaluated at the iterate's rate (lagged by one iteration: the device update
  does not include the -M / dt term in its Jacobian, which for this piston is
  about 1e-4 of the squeeze-film damping), so a converged step balances
  oil, side load and inertia exactly.

Optionally (`kinematics=SwashKinematics()`) the piston moves as in a
swash-plate pump with the geometry of Table 8 instead of the configured fixed gap
length and sliding speed: the coupling length follows the piston stroke,
L_F(phi) = L_Fmin + R_b tan(beta) (1 - cos phi) (L_Fmin at outer dead centre,
phi = 0, growing by the stroke 2 R_b tan(beta) to inner dead centre), and the
sliding speed is its rate, dL_F/dt = R_b omega tan(beta) sin(phi), with the sign
convention of the configured v_amp sin(phi).  The paper gives Table 8's numbers
but not these relations; they are the plain kinematics of a piston whose slipper
follows a plane tilted by beta while the block turns at omega.  Each shaft step
then solves on a gap of its own length (the grid keeps its cells), and the
generalized coordinates stay the eccentricities at the two ends of the gap.

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
PISTON_MASS = 0.128          # m_K of Table 8 [kg]
PITCH_RADIUS = 4.05e-2       # R_b of Table 8 [m]: radius of the pistons' pitch circle
COUPLING_MIN = 3e-2          # L_Fmin of Table 8 [m]


@dataclass(frozen=True)
class SwashKinematics:
    """Piston motion of a swash-plate pump: coupling length and sliding speed over
    the shaft angle phi (0 at outer dead centre)."""
    pitch_radius: float = PITCH_RADIUS
    swash_deg: float = SWASH_ANGLE_DEG
    coupling_min: float = COUPLING_MIN

    @property
    def stroke(self) -> float:
        """Full piston stroke 2 R_b tan(beta)."""
        return 2.0 * self.pitch_radius * math.tan(math.radians(self.swash_deg))

    def coupling_length(self, phi: float) -> float:
        """L_F(phi) = L_Fmin + R_b tan(beta) (1 - cos phi)."""
        return self.coupling_min + 0.5 * self.stroke * (1.0 - math.cos(phi))

    def sliding_speed(self, phi: float, rpm: float) -> float:
        """dL_F/dt = R_b omega tan(beta) sin(phi), omega = 2 pi rpm / 60."""
        return 0.5 * self.stroke * (2.0 * math.pi * rpm / 60.0) * math.sin(phi)


def side_load(p_chamber: float, radius: float, kappa: float) -> np.ndarray:
    """Generalized external force of the synthetic swash-plate side load.

    F_s = kappa * p_chamber * pi R_k^2 * tan(swash angle), a force along +x applied
    at z = L; its virtual work on the linear tilt loads e3 only."""
    f = kappa * p_chamber * math.pi * radius ** 2 * math.tan(math.radians(SWASH_ANGLE_DEG))
    return np.array([0.0, 0.0, f, 0.0])


def force_scale(F_ext, p_chamber: float, radius: float) -> float:
    """Scale of the force-balance test: max(||F_ext||, p_chamber pi R_k^2, 1 N)."""
    return max(float(np.linalg.norm(F_ext)), p_chamber * math.pi * radius ** 2, 1.0)


def inertia_matrix(mass: float) -> np.ndarray:
    """Generalized mass matrix of a piston of `mass` spread evenly over the coupling
    length, on the coordinates (e1, e2, e3, e4): the kinetic energy of the linear
    tilt x(z) = (1 - t) e1 + t e3, y(z) = (1 - t) e2 + t e4 (t = z / L) is
    1/2 edot^T M edot with M = mass [[1/3, 1/6], [1/6, 1/3]] in each direction."""
    a, b = mass / 3.0, mass / 6.0
    return np.array([[a, 0.0, b, 0.0], [0.0, a, 0.0, b], [b, 0.0, a, 0.0], [0.0, b, 0.0, a]])


def inertia_force(M: np.ndarray, edot, edot_prev, dt: float) -> np.ndarray:
    """F_I = -M e'' with e'' = (edot - edot_prev) / dt (backward difference)."""
    return -M @ ((np.asarray(edot, dtype=np.float64) - np.asarray(edot_prev, dtype=np.float64)) / dt)


def gpu_stepper(ctx: int) -> Callable:
    """The Picard step of the library (general or simplified scheme) on context ctx."""
    def step(scheme, n_theta, n_z, ph, tex, state, e_prev, dt, F_ext, d_e, d_edot, opts):
        if scheme == "simplified":
            return gmaf.gmaf_picard_step_simplified(ctx, n_theta, n_z, ph, tex, state, dt, F_ext,
                                                    d_edot, opts)
        return gmaf.gmaf_picard_step(ctx, n_theta, n_z, ph, tex, state, e_prev, dt, F_ext, d_e,
                                     d_edot, opts)
    return step


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
    gap_length: float = 0.0


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
          kappa: float = 0.005, tol_F: float = 1e-6, max_picard: int = 20,
          d_e: float = 2e-8, d_edot: float = 1e-6, opts: Optional[gmaf.gmaf_solver_opts] = None,
          on_step: Optional[Callable[[StepRecord], None]] = None,
          scheme: str = "general", mass: float = PISTON_MASS,
          stepper: Optional[Callable] = None,
          kinematics: Optional[SwashKinematics] = None) -> Trajectory:
    """Run `steps` shaft-angle steps.  p_profile[s % steps_per_rev] is the chamber
    pressure of step s; the sliding speed is v_amp * sin(phi) and the gap length
    phys[1], or, with `kinematics`, the swash-plate piston's speed and coupling
    length at phi.

    scheme "general": the double-Jacobian Picard iteration (Eq. 2.12-2.19, 9 conditions).
    scheme "simplified": the conventional one (Eq. 2.20-2.22, 5 conditions); each time
    step starts from the predictor e = e_l + dt edot_l, so that the increments of
    Eq. 2.22 keep e = e_l + dt edot, the backward difference, at every iterate.
    mass: piston mass of the inertia load (0 leaves it out).
    stepper: the Picard step to call (default: the library's, on ctx); same arguments
    as the callable gpu_stepper returns."""
    if scheme not in ("general", "simplified"):
        raise ValueError(f"unknown scheme {scheme!r}")
    step_fn = stepper or gpu_stepper(ctx)
    M = inertia_matrix(mass)
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
        if kinematics is not None:
            ph[1] = kinematics.coupling_length(phi)
            ph[4] = kinematics.sliding_speed(phi, rpm)
        F_side = side_load(ph[5], ph[0], kappa)
        scale = force_scale(F_side, ph[5], ph[0])
        e_prev = state[:4].copy()
        edot_prev = state[4:].copy()
        if scheme == "simplified":
            state[:4] = e_prev + dt * state[4:]
        converged = False
        pcg = 0
        G_norm = float("inf")
        loads = np.zeros(12)
        it = 0
        for it in range(1, max_picard + 1):
            oo = o if first_solve else warm
            F_ext = F_side + inertia_force(M, state[4:], edot_prev, dt)
            r = step_fn(scheme, n_theta, n_z, ph, tex, state, e_prev, dt, F_ext, d_e, d_edot, oo)
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
                         seconds=time.perf_counter() - t0, gap_length=float(ph[1]))
        traj.records.append(rec)
        if on_step:
            on_step(rec)
    return traj
