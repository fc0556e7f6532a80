"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds problem descriptions and seeded random draws only: box
slabs, conductivities, stimulus boxes, fibre angles, initial fronts, batches
of instances and request arrival times.  It contains none of the numerical
method (no basis, operator, ionic model, time stepping or indicators); both
the FP64 oracle and the CUDA library read a ``Problem`` and do their own
arithmetic on it.

Units follow the monodomain problem statement of the paper (Sec. 2,
Eq. (monodomain)): cm, ms, mS/cm, uF/cm^2, and a dimensionless transmembrane
potential V for the Aliev-Panfilov cell model (rest 0, peak about 1).

The five workloads mirror the slabs the paper measures on (Niederer slab,
Sec. 3.1; spiral-wave square, Sec. 3.2), restated with the Aliev-Panfilov
model because the paper's PCG model equations are not available here.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

AP_STANDARD = (8.0, 0.15, 0.002, 0.2, 0.3, 1.0)  # k, a, eps0, mu1, mu2, time_scale [ms per model unit]

STATE_FE = 0
STATE_EXP = 1

# Geometry of the slab (Problem.geometry).  The forest always lives on the reference box
# [0, extent_0] x [0, extent_1] (x [0, extent_2]); a map x = Phi(X) takes it to the physical
# domain (the paper's curved ventricle meshes, Sec. 3.3, stand behind the shell).
GEOMETRY_BOX = 0      # Phi = identity
GEOMETRY_AFFINE = 1   # Phi(X) = A X + b, geo = (A row-major 3x3, b) (2D: the leading 2x2 block)
GEOMETRY_SHELL = 2    # ellipsoidal shell sector, geo = (a_i, b_i, c_i, a_o, b_o, c_o, phi0, dphi,
                      #   theta0, dtheta): X_0 -> azimuth, X_1 -> polar angle (2D: transmural),
                      #   X_2 -> transmural, semi-axes linear from inner to outer surface


@dataclass
class Stimulus:
    """Box-shaped stimulus: I_stim = -amplitude on nodes inside [lo, hi] for t in [t0, t1)."""
    lo: Tuple[float, float, float]
    hi: Tuple[float, float, float]
    amplitude: float = 1.0
    t0: float = 0.0
    t1: float = 1.0


@dataclass
class Problem:
    """One monodomain simulation on a box slab (fields mirror ``mdl_problem`` in include/mdl.h)."""
    dim: int = 2
    order: int = 1
    extent: Tuple[float, float, float] = (1.0, 1.0, 1.0)
    base: Tuple[int, int, int] = (32, 32, 1)
    sigma_l: float = 1.0            # mS/cm along the fibre
    sigma_t: float = 1.0            # mS/cm across the fibre
    fibre: Tuple[float, float, float] = (1.0, 0.0, 0.0)
    chi: float = 1400.0             # 1/cm
    cm: float = 1.0                 # uF/cm^2
    gamma: float = 10.0             # SIPG penalty factor
    ionic_model: int = 0            # 0 = Aliev-Panfilov, -1 = none (pure diffusion)
    ionic_params: Tuple[float, ...] = AP_STANDARD
    stimuli: List[Stimulus] = field(default_factory=list)
    dt_barrier: float = 0.01        # ms; 0 = largest 2^-k ms meeting the LTS level budget
    max_refine: int = 0
    n_lts_levels: int = 1
    tau_refine: float = math.inf
    tau_coarsen: float = -1.0
    tau_cell: float = math.inf
    dt_bar_cell: float = 0.0        # ms; substep length requested by the temporal indicator
    act_threshold: float = 0.5
    state_integrator: int = STATE_FE
    precision: int = 64             # 32 or 64
    amr_enabled: int = 0
    lts_enabled: int = 0
    geometry: int = 0               # 0 box, 1 affine map, 2 ellipsoidal shell sector (GEOMETRY_*)
    geo: Tuple[float, ...] = ()     # parameters of the map (see the GEOMETRY_* constants)
    fibre_ref: int = 0              # 1: fibre along the image of the first reference axis

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)

    @property
    def n_base(self) -> int:
        n = self.base[0] * self.base[1]
        return n * (self.base[2] if self.dim == 3 else 1)

    @property
    def n_p(self) -> int:
        return (self.order + 1) ** self.dim


def fibre_from_angle(theta: float) -> Tuple[float, float, float]:
    return (math.cos(theta), math.sin(theta), 0.0)


# --------------------------------------------------------------------------
# The five workloads.
# --------------------------------------------------------------------------

def plain_2d_q1_32x32() -> Problem:
    """Unit square, 32x32 Q1, isotropic 1.0 mS/cm, forward Euler at 0.01 ms for 20 ms, FP64."""
    return Problem(
        dim=2, order=1, extent=(1.0, 1.0, 1.0), base=(32, 32, 1),
        sigma_l=1.0, sigma_t=1.0, fibre=(1.0, 0.0, 0.0), gamma=10.0,
        stimuli=[Stimulus((0.0, 0.0, 0.0), (0.1, 0.1, 1.0), 1.0, 0.0, 1.0)],
        dt_barrier=0.01, act_threshold=0.5, state_integrator=STATE_FE,
        precision=64, amr_enabled=0, lts_enabled=0, n_lts_levels=1)


PLAIN_T_END = 20.0


def slab_2d_q1_256(seed: int = 2) -> Problem:
    """2x2 cm, 256x256 Q1 base, quadtree AMR to depth 3, 4 LTS levels, 3:1 fibres at a seeded angle."""
    rng = np.random.default_rng(seed)
    theta = float(rng.uniform(0.0, math.pi))
    return Problem(
        dim=2, order=1, extent=(2.0, 2.0, 1.0), base=(256, 256, 1),
        sigma_l=1.2, sigma_t=0.4, fibre=fibre_from_angle(theta), gamma=10.0,
        stimuli=[Stimulus((0.0, 0.0, 0.0), (0.1, 0.1, 1.0), 1.0, 0.0, 1.0)],
        dt_barrier=0.0, max_refine=3, n_lts_levels=4,
        tau_refine=SLAB2D_TAU[0], tau_coarsen=SLAB2D_TAU[1],
        tau_cell=0.5, dt_bar_cell=0.01,
        act_threshold=0.5, state_integrator=STATE_EXP,
        precision=32, amr_enabled=1, lts_enabled=1)


# Refinement thresholds for the 2D slab, calibrated once on the oracle so that
# a developed Aliev-Panfilov front (width ~0.01 cm) is refined to depth 3 and the
# rest coarsens.  tau_coarsen = tau_refine / 10 is the ratio the paper uses for its
# ventricle runs; with the indicator falling ~6x per refinement, the 1/3 ratio of
# its slab runs would coarsen freshly refined children on the next barrier.
SLAB2D_TAU = (3.0e-9, 3.0e-10)
SLAB2D_T_END = 100.0


def slab_3d_q2(seed: int = 3) -> Problem:
    """2x0.7x0.3 cm, 128x48x20 Q2 hexes, octree AMR to depth 3, 4 LTS levels, planar x=0 stimulus."""
    return Problem(
        dim=3, order=2, extent=(2.0, 0.7, 0.3), base=(128, 48, 20),
        sigma_l=1.2, sigma_t=0.3, fibre=(1.0, 0.0, 0.0), gamma=40.0,
        stimuli=[Stimulus((0.0, 0.0, 0.0), (2.0 / 128.0, 0.7, 0.3), 1.0, 0.0, 1.0)],
        dt_barrier=0.0, max_refine=3, n_lts_levels=4,
        tau_refine=SLAB3D_TAU[0], tau_coarsen=SLAB3D_TAU[1],
        tau_cell=0.5, dt_bar_cell=0.01,
        act_threshold=0.5, state_integrator=STATE_EXP,
        precision=32, amr_enabled=1, lts_enabled=1)


# 3D Q2: the indicator falls ~50-90x per refinement, so tau_coarsen = tau_refine / 1000
# keeps freshly refined children; tau_refine brings a developed planar front to depth 3.
SLAB3D_TAU = (1.0e-13, 1.0e-16)
SLAB3D_T_END = 50.0


def lv_3d_q1(base: Tuple[int, int, int] = (240, 96, 8)) -> Problem:
    """LV-like curved slab (a stand-in for the paper's idealized left ventricle, Sec. 3.3):
    an ellipsoidal shell sector with endocardial semi-axes (2.5, 2.5, 5.0) cm and epicardial
    (3.5, 3.5, 6.0) cm, azimuth 0 .. 6 rad, polar angle 0.35 .. 1.9 rad (truncated below the
    apex and past the equator), Q1 on 240 x 96 x 8 roots, fibres along the azimuth (3:1),
    4 LTS levels from the per-element CFL bounds, the apical ring stimulated.  The reference
    box has roughly the physical lengths (18 x 7.5 x 1 cm) so that reference and physical
    element sizes are alike."""
    geo = (2.5, 2.5, 5.0, 3.5, 3.5, 6.0, 0.0, 6.0, 0.35, 1.55)
    return Problem(
        dim=3, order=1, extent=(18.0, 7.5, 1.0), base=base,
        sigma_l=1.2, sigma_t=0.4, fibre=(1.0, 0.0, 0.0), gamma=10.0,
        stimuli=[Stimulus((-10.0, -10.0, 4.4), (10.0, 10.0, 10.0), 1.0, 0.0, 1.0)],
        dt_barrier=0.0, max_refine=0, n_lts_levels=4,
        tau_cell=0.5, dt_bar_cell=0.01, act_threshold=0.5, state_integrator=STATE_EXP,
        precision=32, amr_enabled=0, lts_enabled=1,
        geometry=GEOMETRY_SHELL, geo=geo, fibre_ref=1)


def lv_3d_q1_amr(base: Tuple[int, int, int] = (120, 48, 4)) -> Problem:
    """The LV-like shell sector of lv_3d_q1 on half as many roots per direction with octree
    adaptation to depth 2 (the finest elements as in lv_3d_q1 at 4x its resolution): the
    paper's idealized LV runs adapt (Sec. 3.3).  An adapting curved mesh takes its barrier step
    from the caller: 2^-6 ms, where the depth-2 elements need the 4 LTS levels (the root mesh
    alone allows 2^-2 ms).  Thresholds as the completed-request generator's 3D Q1 class
    (similar element size)."""
    return lv_3d_q1(base).replace(max_refine=2, amr_enabled=1, dt_barrier=2.0 ** -6,
                                  tau_refine=COMPLETED_TAU[(3, 1)][0], tau_coarsen=COMPLETED_TAU[(3, 1)][1])


def spiral_2d_q1(n: int = 80, h: float = 0.05) -> Problem:
    """Temporal adaptivity workload: a 2D Q1 square of n x n elements of size h (4x4 cm by
    default), isotropic 1.0 mS/cm, no AMR, 5 LTS levels, barrier step 0.1 ms and the
    temporal indicator's substep 0.01 ms as in the paper's spiral-wave run, so that the
    elements whose cell state changes fast take 16 substeps while the CFL asks for 8;
    started from a broken planar wave (spiral_state) that curls into a spiral.  tau_cell
    is calibrated on the oracle (SPIRAL_TAU_CELL)."""
    return Problem(
        dim=2, order=1, extent=(n * h, n * h, 1.0), base=(n, n, 1),
        sigma_l=1.0, sigma_t=1.0, fibre=(1.0, 0.0, 0.0), gamma=10.0,
        stimuli=[], dt_barrier=0.1, max_refine=0, n_lts_levels=5,
        tau_cell=SPIRAL_TAU_CELL, dt_bar_cell=0.01,
        act_threshold=0.5, state_integrator=STATE_EXP,
        precision=32, amr_enabled=0, lts_enabled=1)


# The paper's tau_cell (0.5) belongs to its cell model and norms; with Aliev-Panfilov the
# temporal indicator of an element on the wave's upstroke is ~0.005-0.025 on this mesh, of a
# resting one ~1e-6 (calibrated once on the oracle).
SPIRAL_TAU_CELL = 0.004


def spiral_state(points: np.ndarray, side: float, width: float = 0.02) -> Tuple[np.ndarray, np.ndarray]:
    """Broken planar wave on a square of the given side: an excited band x < side/4 in the
    lower half, the same band refractory (recovery variable raised) in the upper half, so
    the wave's free end curls.  Shapes an input state only."""
    x, y = points[:, 0], points[:, 1]
    band = 0.5 * (1.0 - np.tanh((x - 0.25 * side) / width))
    lower = 0.5 * (1.0 - np.tanh((y - 0.5 * side) / width))
    return band * lower, 1.2 * band * (1.0 - lower)


def scaled(prob: Problem, base: Tuple[int, int, int]) -> Problem:
    """Same physics on a different base grid with the extent scaled to keep h fixed."""
    ext = tuple(prob.extent[k] * base[k] / prob.base[k] if k < prob.dim else prob.extent[k]
                for k in range(3))
    stims = []
    for s in prob.stimuli:
        stims.append(dataclasses.replace(s))
    return prob.replace(base=tuple(base), extent=ext, stimuli=stims)


# --------------------------------------------------------------------------
# Seeded initial states: a developed excitation front.
# --------------------------------------------------------------------------

def front_state(points: np.ndarray, origin, radius: float, width: float,
                tail: float = 0.0) -> Tuple[np.ndarray, np.ndarray]:
    """Synthetic developed front: V = 1 inside a ball of ``radius`` around ``origin``
    with a tanh edge of ``width``, and a recovery variable that rises behind the front.

    ``points`` is (n, dim) physical coordinates; returns (V, v).  This shapes an
    input state only (it stands in for the state a corner stimulus reaches after
    several milliseconds); it is not part of the method.
    """
    o = np.asarray(origin[: points.shape[1]], dtype=np.float64)
    r = np.sqrt(((points - o) ** 2).sum(axis=1))
    V = 0.5 * (1.0 - np.tanh((r - radius) / width))
    v = np.clip((radius - r) / max(tail, 1e-30), 0.0, 1.0) * 1.5 if tail > 0 else np.zeros_like(r)
    return V, v


def planar_front_state(points: np.ndarray, x0: float, width: float, tail: float = 0.0):
    """Synthetic planar front travelling along +x: V = 1 for x < x0 with a tanh edge of
    ``width``, recovery rising behind it over ``tail``.  Input shaping only."""
    x = points[:, 0]
    V = 0.5 * (1.0 - np.tanh((x - x0) / width))
    v = np.clip((x0 - x) / max(tail, 1e-30), 0.0, 1.0) * 1.5 if tail > 0 else np.zeros_like(x)
    return V, v


# --------------------------------------------------------------------------
# Batches and request streams.
# --------------------------------------------------------------------------

def batch_instances(n: int = 64, seed: int = 4, min_e: float = 1e3, max_e: float = 1e5,
                    t_end: float = 100.0) -> List[Tuple[Problem, float]]:
    """Heterogeneous instances: half 2D Q1, half 3D (Q1/Q2); log-uniform base element count."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        ne = float(np.exp(rng.uniform(np.log(min_e), np.log(max_e))))
        if i < n // 2:
            dim, order = 2, 1
            side = max(2, int(round(math.sqrt(ne))))
            base = (side, side, 1)
            ext = (side * 0.0078125, side * 0.0078125, 1.0)
        else:
            dim = 3
            order = 1 if i < (3 * n) // 4 else 2
            # aspect 2 : 0.7 : 0.3
            s = (ne / (2.0 * 0.7 * 0.3)) ** (1.0 / 3.0)
            base = (max(2, int(round(2.0 * s))), max(2, int(round(0.7 * s))), max(2, int(round(0.3 * s))))
            hh = 0.015625 * order
            ext = (base[0] * hh, base[1] * hh, base[2] * hh)
        sl = float(rng.uniform(0.5, 2.0))
        st = float(rng.uniform(0.5, 2.0))
        sl, st = max(sl, st), min(sl, st)
        theta = float(rng.uniform(0.0, math.pi))
        n_lts = int(rng.integers(1, 5))
        corner = [float(rng.uniform(0.0, 0.8)) * ext[k] for k in range(3)]
        size = [0.1 * ext[k] for k in range(3)]
        stim = Stimulus(tuple(corner), tuple(corner[k] + size[k] for k in range(3)), 1.0, 0.0, 1.0)
        p = Problem(dim=dim, order=order, extent=ext, base=base, sigma_l=sl, sigma_t=st,
                    fibre=fibre_from_angle(theta), gamma=10.0 * order * order, stimuli=[stim],
                    dt_barrier=0.0, max_refine=0, n_lts_levels=n_lts, tau_cell=0.5,
                    state_integrator=STATE_EXP, precision=32, amr_enabled=0,
                    lts_enabled=1 if n_lts > 1 else 0)
        out.append((p, t_end))
    return out


# Refinement thresholds of the request generators per (dim, order), calibrated once on the
# oracle: tau_refine about 1/20 of the largest level-0 spatial indicator on a developed front
# (width 0.01 cm) at the generator's element size, so that a front reaches depth 2 within a
# few barrier steps; tau_coarsen at the slabs' ratios (Q1 1/10, 2D Q2 1/100, 3D Q2 1/1000:
# the indicator falls faster per refinement at Q2).
SERVE_TAU = {(2, 1): (3e-8, 3e-9), (3, 1): (1.5e-10, 1.5e-11), (3, 2): (1e-9, 1e-12), (2, 2): (5e-8, 5e-10)}
COMPLETED_TAU = {(2, 1): (2e-6, 2e-7), (3, 1): (5e-9, 5e-10), (3, 2): (4e-8, 4e-11), (2, 2): (5e-6, 5e-8)}


def poisson_requests(rate: float = 20.0, duration: float = 60.0, seed: int = 5,
                     min_e: float = 1e3, max_e: float = 2e5,
                     horizon: Tuple[float, float] = (100.0, 500.0), tau=None) -> List[Tuple[float, Problem, float]]:
    """Poisson arrivals: (arrival_s, problem, horizon_ms); horizon is the range of the uniform
    horizon draw, tau the refinement thresholds per (dim, order) (default SERVE_TAU)."""
    tau = SERVE_TAU if tau is None else tau
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= duration:
            break
        ne = float(np.exp(rng.uniform(np.log(min_e), np.log(max_e))))
        dim = 2 if rng.uniform() < 0.5 else 3
        order = 1 if rng.uniform() < 0.5 else 2
        if dim == 2:
            side = max(2, int(round(math.sqrt(ne))))
            base = (side, side, 1)
            hh = 0.0078125 * order
            ext = (side * hh, side * hh, 1.0)
        else:
            s = (ne / (2.0 * 0.7 * 0.3)) ** (1.0 / 3.0)
            base = (max(2, int(round(2.0 * s))), max(2, int(round(0.7 * s))), max(2, int(round(0.3 * s))))
            hh = 0.015625 * order
            ext = (base[0] * hh, base[1] * hh, base[2] * hh)
        theta = float(rng.uniform(0.0, math.pi))
        t_end = float(rng.uniform(horizon[0], horizon[1]))
        corner = [0.0, 0.0, 0.0]
        size = [0.1 * ext[k] for k in range(3)]
        stim = Stimulus(tuple(corner), tuple(size), 1.0, 0.0, 1.0)
        p = Problem(dim=dim, order=order, extent=ext, base=base, sigma_l=1.2, sigma_t=0.4,
                    fibre=fibre_from_angle(theta), gamma=10.0 * order * order, stimuli=[stim],
                    dt_barrier=0.0, max_refine=2, n_lts_levels=3, tau_cell=0.5,
                    tau_refine=tau[(dim, order)][0], tau_coarsen=tau[(dim, order)][1],
                    state_integrator=STATE_EXP, precision=32, amr_enabled=1, lts_enabled=1)
        out.append((t, p, t_end))
    return out


def completed_requests(rate: float = 3.0, duration: float = 20.0, seed: int = 6) -> List[Tuple[float, Problem, float]]:
    """Requests that finish inside a serving window: the Poisson generator above with 100 to
    2000 base elements, base elements 8x (2D) or 4x (3D) larger and 5-20 ms horizons (a few
    thousand barrier steps each), arriving at `rate` per second for `duration` seconds."""
    out = []
    for t, p, h in poisson_requests(rate, duration, seed, min_e=1e2, max_e=2e3, horizon=(5.0, 20.0),
                                    tau=COMPLETED_TAU):
        f = 8.0 if p.dim == 2 else 4.0
        ext = tuple(p.extent[k] * f if k < p.dim else p.extent[k] for k in range(3))
        stim = dataclasses.replace(p.stimuli[0], hi=tuple(0.1 * ext[k] for k in range(3)))
        out.append((t, p.replace(extent=ext, stimuli=[stim]), h))
    return out
