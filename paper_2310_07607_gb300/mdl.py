"""Thin ctypes binding of libmdl.so (include/mdl.h).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  There is no CPU fallback -- if the library is missing or the device
is unavailable, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmdl.so")

MDL_MAX_STIM = 4

ERRORS = {
    -1: "MDL_E_ARG", -2: "MDL_E_NOMEM", -3: "MDL_E_NOSPACE", -4: "MDL_E_CFL",
    -5: "MDL_E_NONFINITE", -6: "MDL_E_TIMEOUT", -7: "MDL_E_CUDA", -8: "MDL_E_STATE",
}


class MdlError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


class CStim(C.Structure):
    _fields_ = [("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("amplitude", C.c_double), ("t0", C.c_double), ("t1", C.c_double)]


class CProblem(C.Structure):
    _fields_ = [
        ("dim", C.c_int32), ("order", C.c_int32),
        ("extent", C.c_double * 3), ("base", C.c_int32 * 3),
        ("sigma_l", C.c_double), ("sigma_t", C.c_double), ("fibre", C.c_double * 3),
        ("chi", C.c_double), ("cm", C.c_double), ("gamma", C.c_double),
        ("ionic_model", C.c_int32), ("ionic_params", C.c_double * 8),
        ("n_stim", C.c_int32), ("stim", CStim * MDL_MAX_STIM),
        ("dt_barrier", C.c_double),
        ("max_refine", C.c_int32), ("n_lts_levels", C.c_int32),
        ("tau_refine", C.c_double), ("tau_coarsen", C.c_double),
        ("tau_cell", C.c_double), ("dt_bar_cell", C.c_double),
        ("act_threshold", C.c_double),
        ("state_integrator", C.c_int32), ("precision", C.c_int32),
        ("amr_enabled", C.c_int32), ("lts_enabled", C.c_int32),
        ("geometry", C.c_int32), ("fibre_ref", C.c_int32), ("geo", C.c_double * 12),
    ]


class CStats(C.Structure):
    _fields_ = [
        ("barriers", C.c_int64), ("dof_updates", C.c_int64), ("element_updates", C.c_int64),
        ("tick_launches", C.c_int64), ("kernel_launches", C.c_int64), ("amr_rebuilds", C.c_int64),
        ("sweep_ms", C.c_double), ("timed_barriers", C.c_int64), ("indicator_ms", C.c_double),
        ("amr_host_ms", C.c_double),
        ("transfer_ms", C.c_double), ("integral_V", C.c_double),
        ("n_elements", C.c_int64), ("level_counts", C.c_int64 * 8), ("factor_updates", C.c_int64),
    ]


EXPORTS = [
    "mdl_create", "mdl_upload_mesh", "mdl_set_initial", "mdl_set_levels", "mdl_set_indicators",
    "mdl_step_to", "mdl_step_barriers", "mdl_get_time", "mdl_get_sizes", "mdl_read_V",
    "mdl_read_state", "mdl_read_activation", "mdl_read_mesh", "mdl_read_faces",
    "mdl_read_indicators", "mdl_get_stats", "mdl_reset_stats", "mdl_set_timing",
    "mdl_device_view", "mdl_last_error", "mdl_destroy", "mdl_version", "mdl_integral_noalloc",
    "mdl_selftest_wait",
    "mdl_noalloc_last_error", "mdl_set_tick_shape", "mdl_set_sweep_variant", "mdl_set_sweep_blocks", "mdl_batch_create", "mdl_batch_footprint",
    "mdl_batch_admit", "mdl_batch_step", "mdl_batch_poll", "mdl_batch_slot", "mdl_batch_release",
    "mdl_batch_usage", "mdl_batch_shape", "mdl_batch_last_error", "mdl_batch_destroy",
    "mdl_batch_set_fused", "mdl_batch_fused_info",
    "mdl_set_initial_f32", "mdl_read_fields_f32",
]

SLOT_FREE, SLOT_RUNNING, SLOT_DONE, SLOT_FAILED = 0, 1, 2, 3
SWEEP_THREAD, SWEEP_GROUP, SWEEP_COOP, SWEEP_TENSOR = 0, 1, 2, 3

_lib = None


def load(path: Optional[str] = None):
    """Load libmdl.so (built by paper_2310_07607_gb300.build); raise if it is missing."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError("libmdl.so not built (%s): run __graft_entry__.build()" % p)
    lib = C.CDLL(p)
    vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int
    dp = C.POINTER(C.c_double)
    lib.mdl_create.argtypes = [C.POINTER(CProblem), C.POINTER(vp)]
    lib.mdl_upload_mesh.argtypes = [vp, i64, vp, vp, vp]
    lib.mdl_set_initial.argtypes = [vp, vp, vp, i64]
    lib.mdl_set_levels.argtypes = [vp, vp, i64]
    lib.mdl_set_indicators.argtypes = [vp, vp, vp, i64]
    lib.mdl_step_to.argtypes = [vp, C.c_double]
    lib.mdl_step_barriers.argtypes = [vp, i64]
    lib.mdl_get_time.argtypes = [vp, dp, C.POINTER(i64), dp]
    fp = C.POINTER(C.c_float)
    lib.mdl_set_initial_f32.argtypes = [vp, fp, fp, i64]
    lib.mdl_read_fields_f32.argtypes = [vp, fp, fp, i64, C.POINTER(i64)]
    lib.mdl_get_sizes.argtypes = [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)]
    for f in ("mdl_read_V", "mdl_read_state", "mdl_read_activation"):
        getattr(lib, f).argtypes = [vp, vp, i64, C.POINTER(i64)]
    lib.mdl_read_mesh.argtypes = [vp, vp, vp, vp, vp, i64, C.POINTER(i64)]
    lib.mdl_read_faces.argtypes = [vp, vp, vp, vp, i64, C.POINTER(i64)]
    lib.mdl_read_indicators.argtypes = [vp, vp, vp, i64, C.POINTER(i64)]
    lib.mdl_get_stats.argtypes = [vp, C.POINTER(CStats)]
    lib.mdl_reset_stats.argtypes = [vp]
    lib.mdl_set_timing.argtypes = [vp, i32]
    lib.mdl_device_view.argtypes = [vp, i32, C.POINTER(vp), C.POINTER(i64), C.POINTER(vp)]
    lib.mdl_last_error.argtypes = [vp]
    lib.mdl_last_error.restype = C.c_char_p
    lib.mdl_destroy.argtypes = [vp]
    lib.mdl_destroy.restype = None
    lib.mdl_version.restype = C.c_char_p
    lib.mdl_integral_noalloc.argtypes = [C.c_int32, C.c_int32, vp, vp, C.c_int32, vp, vp, i64, vp, vp]
    lib.mdl_selftest_wait.argtypes = [C.c_int32, C.POINTER(C.c_int32), dp]
    lib.mdl_noalloc_last_error.restype = C.c_char_p
    i32p = C.POINTER(C.c_int32)
    lib.mdl_set_tick_shape.argtypes = [vp, C.c_int32, C.c_int32]
    lib.mdl_set_sweep_variant.argtypes = [vp, C.c_int32]
    lib.mdl_set_sweep_blocks.argtypes = [vp, C.c_int32]
    lib.mdl_batch_create.argtypes = [i64, i32, C.POINTER(vp)]
    lib.mdl_batch_footprint.argtypes = [C.POINTER(CProblem), C.POINTER(i64)]
    lib.mdl_batch_admit.argtypes = [vp, C.POINTER(CProblem), vp, vp, i64, C.c_double, i32p]
    lib.mdl_batch_step.argtypes = [vp, i64, C.c_double, C.POINTER(i64)]
    lib.mdl_batch_poll.argtypes = [vp, i32p, C.c_int32, i32p]
    lib.mdl_batch_slot.argtypes = [vp, C.c_int32, C.POINTER(vp), i32p, i32p]
    lib.mdl_batch_release.argtypes = [vp, C.c_int32]
    lib.mdl_batch_usage.argtypes = [vp, C.POINTER(i64), C.POINTER(i64), i32p]
    lib.mdl_batch_set_fused.argtypes = [vp, C.c_int32]
    lib.mdl_batch_fused_info.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32, i32p, i32p, i32p, dp, dp, dp,
                                         C.POINTER(i64), C.POINTER(i64)]
    lib.mdl_batch_shape.argtypes = [vp, C.POINTER(CProblem), i32p, i32p]
    lib.mdl_batch_last_error.argtypes = [vp]
    lib.mdl_batch_last_error.restype = C.c_char_p
    lib.mdl_batch_destroy.argtypes = [vp]
    lib.mdl_batch_destroy.restype = None
    for f in EXPORTS:
        if f not in ("mdl_last_error", "mdl_destroy", "mdl_version", "mdl_noalloc_last_error",
                     "mdl_batch_last_error", "mdl_batch_destroy"):
            getattr(lib, f).restype = i32
    if path is None:
        _lib = lib
    return lib


def to_c(prob) -> CProblem:
    """Marshal a workloads.Problem into the C struct."""
    c = CProblem()
    c.dim, c.order = prob.dim, prob.order
    for k in range(3):
        c.extent[k] = float(prob.extent[k])
        c.base[k] = int(prob.base[k])
        c.fibre[k] = float(prob.fibre[k])
    c.sigma_l, c.sigma_t = prob.sigma_l, prob.sigma_t
    c.chi, c.cm, c.gamma = prob.chi, prob.cm, prob.gamma
    c.ionic_model = prob.ionic_model
    ip = list(prob.ionic_params) + [0.0] * 8
    for i in range(8):
        c.ionic_params[i] = float(ip[i])
    if len(prob.stimuli) > MDL_MAX_STIM:
        raise ValueError("at most %d stimuli" % MDL_MAX_STIM)
    c.n_stim = len(prob.stimuli)
    for i, s in enumerate(prob.stimuli):
        for k in range(3):
            c.stim[i].lo[k] = float(s.lo[k])
            c.stim[i].hi[k] = float(s.hi[k])
        c.stim[i].amplitude, c.stim[i].t0, c.stim[i].t1 = s.amplitude, s.t0, s.t1
    c.dt_barrier = prob.dt_barrier
    c.max_refine, c.n_lts_levels = prob.max_refine, prob.n_lts_levels
    c.tau_refine = prob.tau_refine if math.isfinite(prob.tau_refine) else 1e308
    c.tau_coarsen = prob.tau_coarsen
    c.tau_cell = prob.tau_cell if math.isfinite(prob.tau_cell) else 1e308
    c.dt_bar_cell = prob.dt_bar_cell
    c.act_threshold = prob.act_threshold
    c.state_integrator, c.precision = prob.state_integrator, prob.precision
    c.amr_enabled, c.lts_enabled = prob.amr_enabled, prob.lts_enabled
    c.geometry = int(getattr(prob, "geometry", 0))
    c.fibre_ref = int(getattr(prob, "fibre_ref", 0))
    geo = list(getattr(prob, "geo", ())) + [0.0] * 12
    for i in range(12):
        c.geo[i] = float(geo[i])
    return c


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class Sim:
    """One simulation context (mdl_ctx) on the current CUDA device."""

    def __init__(self, prob, lib=None, handle=None):
        self.lib = lib or load()
        self.prob = prob
        self._c = to_c(prob)
        self._owned = handle is None
        if handle is not None:      # a context owned by a batch slot
            self.h = C.c_void_p(handle)
            return
        h = C.c_void_p()
        rc = self.lib.mdl_create(C.byref(self._c), C.byref(h))
        if rc != 0:
            raise MdlError(rc, self.lib.mdl_last_error(None).decode())
        self.h = h

    # ---------------------------------------------------------------
    def _check(self, rc):
        if rc != 0:
            raise MdlError(rc, self.lib.mdl_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None) and getattr(self, "_owned", True):
            self.lib.mdl_destroy(self.h)
        self.h = None

    def set_tick_shape(self, threads: int, blocks_per_sm: int):
        self._check(self.lib.mdl_set_tick_shape(self.h, threads, blocks_per_sm))

    def set_sweep_variant(self, variant: int):
        """SWEEP_THREAD (the default), SWEEP_GROUP (Q1), SWEEP_COOP or SWEEP_TENSOR (Q2 3D FP32)."""
        self._check(self.lib.mdl_set_sweep_variant(self.h, variant))

    def set_sweep_blocks(self, max_blocks: int):
        """Upper bound on the persistent tensor-core sweep's blocks (0: two per SM)."""
        self._check(self.lib.mdl_set_sweep_blocks(self.h, max_blocks))

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------
    def upload_mesh(self, level, coords, root=None):
        level = np.ascontiguousarray(level, dtype=np.int8)
        coords = np.ascontiguousarray(coords, dtype=np.int32)
        r = None if root is None else np.ascontiguousarray(root, dtype=np.int32)
        self._check(self.lib.mdl_upload_mesh(self.h, level.size, _ptr(r), _ptr(level), _ptr(coords)))

    def set_initial(self, V, s=None):
        V = np.ascontiguousarray(V, dtype=np.float64)
        sv = None if s is None else np.ascontiguousarray(s, dtype=np.float64)
        self._check(self.lib.mdl_set_initial(self.h, _ptr(V), _ptr(sv), V.size))

    def set_initial_f32(self, V, s=None):
        """set_initial from FP32 arrays (half the transfer of the FP64 call)."""
        V = np.ascontiguousarray(V, dtype=np.float32)
        sv = None if s is None else np.ascontiguousarray(s, dtype=np.float32)
        f = C.POINTER(C.c_float)
        self._check(self.lib.mdl_set_initial_f32(self.h, V.ctypes.data_as(f),
                                                 None if sv is None else sv.ctypes.data_as(f), V.size))

    def read_fields_f32(self, V=None, s=None):
        """(V, state) in FP32 with one gather and one copy each; V, s may be caller buffers
        (e.g. pinned) of at least n_dof float32 values."""
        n = self.sizes()[1]
        V = np.empty(n, np.float32) if V is None else V
        s = np.empty(n, np.float32) if s is None else s
        for a in (V, s):
            if a.dtype != np.float32 or not a.flags.c_contiguous or a.size < n:
                raise ValueError("buffers must be contiguous float32 arrays of at least %d values" % n)
        got = C.c_int64()
        f = C.POINTER(C.c_float)
        self._check(self.lib.mdl_read_fields_f32(self.h, V.ctypes.data_as(f), s.ctypes.data_as(f),
                                                 min(V.size, s.size), C.byref(got)))
        return V[:n], s[:n]

    def set_levels(self, b):
        b = np.ascontiguousarray(b, dtype=np.int8)
        self._check(self.lib.mdl_set_levels(self.h, _ptr(b), b.size))

    def set_indicators(self, eta_s=None, eta_t=None):
        n = self.sizes()[0]
        es = None if eta_s is None else np.ascontiguousarray(eta_s, dtype=np.float64)
        et = None if eta_t is None else np.ascontiguousarray(eta_t, dtype=np.float64)
        self._check(self.lib.mdl_set_indicators(self.h, _ptr(es), _ptr(et), n))

    def step_to(self, t_end: float):
        self._check(self.lib.mdl_step_to(self.h, float(t_end)))

    def step_barriers(self, n: int):
        self._check(self.lib.mdl_step_barriers(self.h, int(n)))

    def time(self):
        t, dt = C.c_double(), C.c_double()
        k = C.c_int64()
        self._check(self.lib.mdl_get_time(self.h, C.byref(t), C.byref(k), C.byref(dt)))
        return t.value, k.value, dt.value

    @property
    def dt(self) -> float:
        return self.time()[2]

    def sizes(self):
        a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
        self._check(self.lib.mdl_get_sizes(self.h, C.byref(a), C.byref(b), C.byref(c)))
        return a.value, b.value, c.value

    def _read(self, fn, n, out=None):
        if out is None:
            out = np.empty(n, dtype=np.float64)
        elif out.dtype != np.float64 or not out.flags.c_contiguous or out.size < n:
            raise ValueError("out must be a contiguous float64 array of at least %d values" % n)
        got = C.c_int64()
        self._check(fn(self.h, _ptr(out), out.size, C.byref(got)))
        return out[:n]

    def read_V(self, out=None):
        """V in leaf order (FP64); `out` may be a caller buffer (e.g. pinned) to fill."""
        return self._read(self.lib.mdl_read_V, self.sizes()[1], out)

    def read_state(self, out=None):
        """Recovery variable in leaf order (FP64); `out` as for read_V."""
        return self._read(self.lib.mdl_read_state, self.sizes()[1], out)

    def read_activation(self):
        return self._read(self.lib.mdl_read_activation, self.sizes()[2])

    def read_mesh(self):
        n = self.sizes()[0]
        d = self.prob.dim
        root = np.empty(n, np.int32)
        level = np.empty(n, np.int8)
        coords = np.empty(n * d, np.int32)
        b = np.empty(n, np.int8)
        got = C.c_int64()
        self._check(self.lib.mdl_read_mesh(self.h, _ptr(root), _ptr(level), _ptr(coords), _ptr(b), n,
                                           C.byref(got)))
        return root, level, coords.reshape(n, d), b

    def read_faces(self):
        n = self.sizes()[0]
        d = self.prob.dim
        nf, ns = 2 * d, 1 << (d - 1)
        kind = np.empty(n * nf, np.int8)
        nbr = np.empty(n * nf * ns, np.int32)
        pos = np.empty(n * nf, np.int8)
        got = C.c_int64()
        self._check(self.lib.mdl_read_faces(self.h, _ptr(kind), _ptr(nbr), _ptr(pos), n, C.byref(got)))
        return kind.reshape(n, nf), nbr.reshape(n, nf, ns), pos.reshape(n, nf)

    def read_indicators(self):
        n = self.sizes()[0]
        es = np.empty(n)
        et = np.empty(n)
        got = C.c_int64()
        self._check(self.lib.mdl_read_indicators(self.h, _ptr(es), _ptr(et), n, C.byref(got)))
        return es, et

    def stats(self) -> dict:
        s = CStats()
        self._check(self.lib.mdl_get_stats(self.h, C.byref(s)))
        out = {f: getattr(s, f) for f, _ in CStats._fields_ if f != "level_counts"}
        out["level_counts"] = list(s.level_counts)
        return out

    def reset_stats(self):
        self._check(self.lib.mdl_reset_stats(self.h))

    def set_timing(self, on: bool):
        self._check(self.lib.mdl_set_timing(self.h, 1 if on else 0))

    def device_view(self, which: int):
        p, st = C.c_void_p(), C.c_void_p()
        n = C.c_int64()
        self._check(self.lib.mdl_device_view(self.h, which, C.byref(p), C.byref(n), C.byref(st)))
        return p.value, n.value, st.value


def integral_noalloc(prob, V_dev: int, level_dev: int, n_e: int, out_dev: int, stream: int = 0, lib=None):
    """FP64 integral of a device DOF field without device allocation (mdl_integral_noalloc).

    V_dev, level_dev and out_dev are device addresses (e.g. torch tensor data_ptr());
    the call is asynchronous on `stream`.
    """
    lib = lib or load()
    ext = (C.c_double * 3)(*[float(x) for x in prob.extent])
    base = (C.c_int32 * 3)(*[int(x) for x in prob.base])
    rc = lib.mdl_integral_noalloc(prob.dim, prob.order, C.cast(ext, C.c_void_p), C.cast(base, C.c_void_p),
                                  prob.precision, C.c_void_p(V_dev), C.c_void_p(level_dev), int(n_e),
                                  C.c_void_p(out_dev), C.c_void_p(stream))
    if rc != 0:
        raise MdlError(rc, lib.mdl_noalloc_last_error().decode())


def selftest_wait(which: int, lib=None):
    """Run one bounded device wait on a phase or count nothing completes (mdl_selftest_wait):
    which 0 the cooperative sweep's grid barrier, 1 the tensor-core sweep's mbarrier wait.
    Returns (status, elapsed_ms); status is MDL_E_TIMEOUT (-6) when the wait gave up."""
    lib = lib or load()
    st = C.c_int32(0)
    ms = C.c_double(0.0)
    rc = lib.mdl_selftest_wait(int(which), C.byref(st), C.byref(ms))
    if rc != 0:
        raise MdlError(rc, "mdl_selftest_wait failed")
    return st.value, ms.value


class Batch:
    """Resident simulations stepped together (mdl_batch_*)."""

    def __init__(self, hbm_budget_bytes: int = 0, autotune: bool = True, fused: bool = True, lib=None):
        self.lib = lib or load()
        h = C.c_void_p()
        rc = self.lib.mdl_batch_create(int(hbm_budget_bytes), 1 if autotune else 0, C.byref(h))
        if rc != 0:
            raise MdlError(rc, self.lib.mdl_batch_last_error(None).decode())
        self.h = h
        self.problems = {}
        self._check(self.lib.mdl_batch_set_fused(self.h, 1 if fused else 0))

    def fused_info(self, precision: int = 32, dim: int = 2, order: int = 1):
        """The tuner's choice for the (precision, dim, order) group -- a dict with "own" (each
        slot's own sweep) or the fused kernel's "threads" and "tile", and the measured
        "best_ms", "worst_ms" and "own_ms" per round -- or None before the tuner finished;
        and the batch's fused (rounds, launches)."""
        own, t, k = C.c_int32(), C.c_int32(), C.c_int32()
        bm, wm, om = C.c_double(), C.c_double(), C.c_double()
        r, n = C.c_int64(), C.c_int64()
        rc = self.lib.mdl_batch_fused_info(self.h, precision, dim, order, C.byref(own), C.byref(t), C.byref(k),
                                           C.byref(bm), C.byref(wm), C.byref(om), C.byref(r), C.byref(n))
        if rc not in (0, -8):
            self._check(rc)
        info = None
        if rc == 0:
            info = {"own": bool(own.value), "best_ms": bm.value, "worst_ms": wm.value, "own_ms": om.value}
            if not own.value:
                info.update(threads=t.value, tile=k.value)
        return info, (r.value, n.value)

    def _check(self, rc):
        if rc != 0:
            raise MdlError(rc, self.lib.mdl_batch_last_error(self.h).decode())

    def footprint(self, prob) -> int:
        c = to_c(prob)
        b = C.c_int64()
        self._check(self.lib.mdl_batch_footprint(C.byref(c), C.byref(b)))
        return b.value

    def admit(self, prob, t_end: float, V0=None, s0=None) -> int:
        """Admit a simulation; raises MdlError with code -3 (MDL_E_NOSPACE) when it does not fit."""
        c = to_c(prob)
        Va = None if V0 is None else np.ascontiguousarray(V0, dtype=np.float64)
        sa = None if s0 is None else np.ascontiguousarray(s0, dtype=np.float64)
        slot = C.c_int32()
        n = 0 if Va is None else Va.size
        self._check(self.lib.mdl_batch_admit(self.h, C.byref(c), _ptr(Va), _ptr(sa), n, float(t_end),
                                             C.byref(slot)))
        self.problems[slot.value] = prob
        return slot.value

    def step(self, barriers_per_slot: int = 1, wall_budget_s: float = 0.0) -> int:
        done = C.c_int64()
        self._check(self.lib.mdl_batch_step(self.h, int(barriers_per_slot), float(wall_budget_s), C.byref(done)))
        return done.value

    def poll(self, cap: int = 4096):
        out = (C.c_int32 * cap)()
        n = C.c_int32()
        self._check(self.lib.mdl_batch_poll(self.h, out, cap, C.byref(n)))
        return [out[i] for i in range(n.value)]

    def slot(self, slot: int):
        """(Sim view of the slot's context, state, error code)."""
        ctx = C.c_void_p()
        st, rc = C.c_int32(), C.c_int32()
        self._check(self.lib.mdl_batch_slot(self.h, slot, C.byref(ctx), C.byref(st), C.byref(rc)))
        return Sim(self.problems[slot], lib=self.lib, handle=ctx.value), st.value, rc.value

    def release(self, slot: int):
        self._check(self.lib.mdl_batch_release(self.h, slot))
        self.problems.pop(slot, None)

    def usage(self):
        u, b = C.c_int64(), C.c_int64()
        r = C.c_int32()
        self._check(self.lib.mdl_batch_usage(self.h, C.byref(u), C.byref(b), C.byref(r)))
        return u.value, b.value, r.value

    def shape(self, prob):
        c = to_c(prob)
        t, k = C.c_int32(), C.c_int32()
        self._check(self.lib.mdl_batch_shape(self.h, C.byref(c), C.byref(t), C.byref(k)))
        return t.value, k.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.mdl_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
