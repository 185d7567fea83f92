"""Seeded synthetic piston-gap workloads.

This module only draws random numbers and names workload presets.  It holds no
arithmetic of the method (no film thickness, no lattice geometry, no condition
fan-out); both the CUDA path and the CPU oracle receive what it returns.

Physical set (Table 8 scale, with the clearance and gap length of the
synthetic workloads): piston radius 10 mm, gap length 40 mm, radial clearance
20 um, viscosity 0.04 Pa s, sliding speed 5 m/s, 20 MPa at the chamber end and
0.1 MPa at the case end.  Eccentricities e1..e4 ~ U[0, 0.5 c], rates
U[-1e-4, 1e-4] m/s.  Textured workloads use flat-bottom circular dimples of
radius 0.5 mm and depth 5 um on a hexagonal lattice at 20 % area density, with
a seeded lattice offset.  The paper's own pump inputs (its measured chamber
pressure and texture layout figures) are not available; these stand in for
them.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

R_K = 0.010
GAP_L = 0.040
CLEARANCE = 20e-6
MU = 0.04
V_SLIDE = 5.0
P_CHAMBER = 20e6
P_CASE = 0.1e6

DIMPLE_RADIUS = 0.5e-3
DIMPLE_DEPTH = 5e-6
DIMPLE_DENSITY = 0.2


@dataclass
class Workload:
    name: str
    n_theta: int
    n_z: int
    phys: np.ndarray          # [R_k, L, c, mu, v_slide, p_chamber, p_case]
    tex: np.ndarray           # [kind, radius, depth, area_density, offset_theta, offset_z]
    state: np.ndarray         # [e1..e4, edot1..edot4]
    n_cond: int = 9
    d_e: float = 1e-3 * CLEARANCE
    d_edot: float = 1e-6
    omega: float = 1.2
    eps: float = 1e-10
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.n_theta * self.n_z

    @property
    def dof(self) -> int:
        return self.n * self.n_cond


def phys_vector(v_slide=V_SLIDE, p_chamber=P_CHAMBER, p_case=P_CASE, clearance=CLEARANCE,
                gap_length=GAP_L, radius=R_K, mu=MU) -> np.ndarray:
    return np.array([radius, gap_length, clearance, mu, v_slide, p_chamber, p_case],
                    dtype=np.float64)


def smooth_texture() -> np.ndarray:
    return np.zeros(6, dtype=np.float64)


def dimple_texture(rng: np.random.Generator, radius=DIMPLE_RADIUS, depth=DIMPLE_DEPTH,
                   density=DIMPLE_DENSITY) -> np.ndarray:
    """Hexagonal dimple lattice with a seeded offset anywhere on the gap surface."""
    o_theta = rng.uniform(0.0, 2.0 * np.pi * R_K)
    o_z = rng.uniform(0.0, GAP_L)
    return np.array([1.0, radius, depth, density, o_theta, o_z], dtype=np.float64)


def random_state(rng: np.random.Generator, clearance=CLEARANCE, e_frac=0.5,
                 edot_max=1e-4) -> np.ndarray:
    e = rng.uniform(0.0, e_frac * clearance, size=4)
    ed = rng.uniform(-edot_max, edot_max, size=4)
    return np.concatenate([e, ed]).astype(np.float64)


def make(name: str, seed: int = 0) -> Workload:
    """Named presets.

    smooth-64x32-k1        one condition, smooth, 64 x 32, FP64
    smooth-512x256-k9      9-condition joint batch, smooth, 512 x 256
    textured-2048x1024-k9  9-condition joint batch, dimples, 2048 x 1024
    textured-1024x512-k9   9-condition joint batch, dimples, 1024 x 512 (dynamics)
    any "<smooth|textured>-<NTH>x<NZ>-k<K>" is accepted as well.
    """
    rng = np.random.default_rng(seed)
    kind, grid, k = name.split("-")
    nth, nz = (int(s) for s in grid.split("x"))
    ncond = int(k[1:])
    tex = dimple_texture(rng) if kind == "textured" else smooth_texture()
    state = random_state(rng)
    return Workload(name=name, n_theta=nth, n_z=nz, phys=phys_vector(), tex=tex, state=state,
                    n_cond=ncond)


def random_field(rng: np.random.Generator, shape, scale=1.0) -> np.ndarray:
    return (rng.standard_normal(size=shape) * scale).astype(np.float64)


def trapezoid_pressure_profile(rng: np.random.Generator, steps_per_rev=360, p_low=0.1e6,
                               p_high=25e6):
    """Seeded chamber pressure per shaft-angle step: a high plateau over about half a
    revolution, ramps of seeded width U[10, 40] degrees, seeded phase."""
    phase = rng.uniform(0.0, 360.0)
    ramp = rng.uniform(10.0, 40.0)
    plateau = 180.0 - ramp
    out = np.empty(steps_per_rev)
    for s in range(steps_per_rev):
        phi = (s * 360.0 / steps_per_rev - phase) % 360.0
        if phi < ramp:
            f = phi / ramp
        elif phi < ramp + plateau:
            f = 1.0
        elif phi < 2 * ramp + plateau:
            f = 1.0 - (phi - ramp - plateau) / ramp
        else:
            f = 0.0
        out[s] = p_low + (p_high - p_low) * f
    return out


def poisson_arrivals(rng: np.random.Generator, rate_hz: float, count: int) -> np.ndarray:
    return np.cumsum(rng.exponential(1.0 / rate_hz, size=count))


SERVING_GRIDS = [(256, 128), (512, 256), (1024, 512), (2048, 1024)]


def serving_requests(seed: int, count: int, rate_hz: float, grids=None):
    """Poisson stream of 9-condition Picard-step requests of uneven sizes, 50 % textured."""
    rng = np.random.default_rng(seed)
    grids = grids or SERVING_GRIDS
    t = poisson_arrivals(rng, rate_hz, count)
    reqs = []
    for k in range(count):
        nth, nz = grids[rng.integers(len(grids))]
        textured = bool(rng.integers(2))
        tex = dimple_texture(rng) if textured else smooth_texture()
        reqs.append(dict(arrival_s=float(t[k]), n_theta=nth, n_z=nz, tex=tex,
                         state=random_state(rng), phys=phys_vector()))
    return reqs
