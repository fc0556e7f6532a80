"""Benchmark: explicit local space-time adaptive monodomain stepping on one GB300.

Default workload (the largest single-GPU configuration, HBM-resident): the 3D slab
2 x 0.7 x 0.3 cm, 128x48x20 Q2 DG hexes, octree AMR to depth 3 driven by the Kelly
indicator, 4 synchronous LTS levels, Aliev-Panfilov, transversely isotropic conductivity
(1.2 / 0.3 mS/cm along x), FP32 bulk arithmetic with the element residual on the tcgen05
tensor cores.  The synthetic initial state is a planar excitation front at mid-slab;
setup barriers let the AMR refine it to depth 3 (2.8M elements) before warm-up.
`--workload slab2d` runs the 2D slab (2x2 cm, 256x256 Q1, AMR 3, LTS 4), `spiral2d` the
temporal-adaptivity workload, `lv3d` the curved LV-like shell sector (mapped Q1 hexes,
per-point geometric factors, LTS 4; `lv3d_amr` with octree adaptation to depth 2), `batch64` and
`serve` the many-simulation workloads.

A step is one barrier step of Alg. 1: eta^s, refine/coarsen (device forest bookkeeping),
level assignment, all sweep ticks, eta^t, LAT, int V.  value = DOF-updates / s over the K
timed steps (device-timed with CUDA events on the library's stream, L2 flushed between
steps by writing a 512 MiB buffer).

--impl reference times the FP64 numpy oracle on the host cores instead (a bounded sample
of the same workload, see cpu_baseline).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "DOF-updates/s"
UNIT = "DOF-updates/s"
FRONT = dict(origin=(0.0, 0.0, 0.0), radius=1.0, width=0.01, tail=0.3)
PLANAR = dict(x0=1.0, width=0.012, tail=0.3)
WORKLOADS = {
    # name: (problem factory, algorithmic bytes per DOF-update, kernel name)
    "slab2d": (W.slab_2d_q1_256, 25.0, "<float,2,1>"),
    "slab3d": (W.slab_3d_q2, 17.6, "<float,3,2>"),
    "spiral2d": (W.spiral_2d_q1, 25.0, "<float,2,1>"),
    "lv3d": (W.lv_3d_q1, 110.1, "<float,3,1>"),
    "lv3d_amr": (W.lv_3d_q1_amr, 110.1, "<float,3,1>"),
}
SETUP_BARRIERS = 5
# DRAM bytes per launch of the dominant kernel (dram__bytes_read.sum + dram__bytes_write.sum)
# from one ncu capture of the same build, averaged over the launches of a barrier step in
# their proportion (tick 0 once, the finer ticks 7 times).  ncu replays each launch with
# cold caches, so this is an upper bound on the live traffic.  Set to None whenever the
# kernel changes until it is captured again.
# Keyed by (workload, kernel) at the workload's own base grid.  3D slab: captured on the same
# slab at a quarter of its x extent (base 32x48x20: the same 2,457,600 finest elements due at
# ticks 1-7, the same level-1 and level-3 elements at tick 4), tick 0 scaled to the full slab's
# 2,736,960 elements by the elements due.
TRAFFIC_PER_LAUNCH = {
    # 2D slab: the eight ticks of one barrier step
    ("slab2d", "k_tick<float,2,1>"): 6.6640e6,
    # curved LV-like slab at full size: the eight ticks of one barrier step
    ("lv3d", "k_tick_mapped<float,3,1>"): 4.4873e7,
    # 3D slab: the quarter slab's eight ticks, tick 0 and tick 4 scaled to the full slab
    ("slab3d", "k_tick_tc<3,2>"): 1.9601e9,
}
# Mapped Q1 3D (lv3d): per element step the state 128 B, metadata and the RV-T accumulator
# 49 B, and the element's geometric factors (8 nodes x 7 values + 6 faces x 4 points x 5
# values, FP32) 704 B, over 8 DOFs: 110.1 B.
# Algorithmic bytes per DOF-update of the fused sweep (Q1 2D, FP32, AP): V_old 4 + v 4 +
# V_new 4 + v 4 = 16 B, plus per element step 2d neighbour ids + 4 B level/flags + the FP64
# RV-T accumulator read-modify-write (36 B) over (p+1)^d = 4 DOFs.
ALG_BYTES_PER_DOF_UPDATE = 25.0   # Q1 2D; Q2 3D: 16 + 44/27 = 17.6 B


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    smax.append(float(p[2]))
                except ValueError:
                    continue
                for n, v in zip(names, p[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        finally:
            os.unlink(self.path)
        if sm:
            out["sm_mhz"] = statistics.median(sm)
            out["sm_max_mhz"] = max(smax)
            out["samples"] = len(sm)
        out["reasons"] = sorted(reasons)
        return out


SWEEPS = {"thread": 0, "group": 1, "coop": 2, "tensor": 3}


def prob_order(factory):
    return factory().order


def workload_name(prob):
    b = prob.base
    if getattr(prob, "geometry", 0):
        return "lv3d_q1_%dx%dx%d_shell%s_lts%d_ap_fp32" % (b[0], b[1], b[2],
                                                           "_amr%d" % prob.max_refine if prob.amr_enabled else "",
                                                           prob.n_lts_levels)
    if prob.dim == 2 and not prob.amr_enabled:
        return "spiral2d_q1_%dx%d_lts%d_taucell_ap_fp32" % (b[0], b[1], prob.n_lts_levels)
    if prob.dim == 2:
        return "slab2d_q1_%dx%d_amr3_lts4_ap_fp32" % (b[0], b[1])
    return "slab3d_q2_%dx%dx%d_amr3_lts4_ap_fp32" % (b[0], b[1], b[2])


def make_sim(prob):
    from paper_2310_07607_gb300 import mdl
    return mdl.Sim(prob)


def node_coords_of(sim, prob):
    """Physical node coordinates of the library's current mesh (leaf order)."""
    root, level, coords, _ = sim.read_mesh()
    n1 = prob.order + 1
    if prob.order == 1:
        xi = np.array([-1 / math.sqrt(3), 1 / math.sqrt(3)])
    else:
        xi = np.array([-math.sqrt(0.6), 0.0, math.sqrt(0.6)])
    d = prob.dim
    n_p = n1 ** d
    q = np.arange(n_p)
    a = [(q // n1 ** k) % n1 for k in range(d)]
    X = np.empty((len(level), n_p, d))
    for k in range(d):
        h = prob.extent[k] / (prob.base[k] * (2.0 ** level.astype(np.float64)))
        X[:, :, k] = coords[:, k:k + 1] * h[:, None] + (xi[a[k]][None, :] + 1.0) * 0.5 * h[:, None]
    return X.reshape(-1, d)


def reduce_over_ranks(total_ms, dof_updates, dist, device):
    """Whole-job figures of a multi-rank run: the slowest rank's timed milliseconds and the
    DOF-updates of all ranks (each rank runs its own replica)."""
    import torch
    t = torch.tensor([float(total_ms), float(dof_updates)], device=device, dtype=torch.float64)
    ms = t[0:1].clone()
    dof = t[1:2].clone()
    dist.all_reduce(ms, op=dist.ReduceOp.MAX)
    dist.all_reduce(dof, op=dist.ReduceOp.SUM)
    return ms.item(), dof.item()


def run_ours(args, rank, world):
    import torch
    torch.cuda.set_device(0 if world == 1 else int(os.environ.get("LOCAL_RANK", rank)))
    dist = None
    if world > 1:
        import torch.distributed as dist  # noqa: F811
        dist.init_process_group("nccl")
    from paper_2310_07607_gb300 import build
    build.build()
    factory, alg_bytes, kname = WORKLOADS[args.workload]
    if getattr(factory(), "geometry", 0):
        kname = "k_tick_mapped" + kname
    elif args.sweep == "group" and prob_order(factory) == 1:
        kname = "k_tick_group" + kname.replace(",1>", ">")
    elif args.sweep == "tensor" or (args.sweep == "default" and factory().order == 2 and factory().dim == 3):
        kname = "k_tick_tc<3,2>"
    else:
        kname = ("k_sweep" if args.sweep == "coop" else "k_tick") + kname
    prob = factory()
    if args.base:
        prob = W.scaled(prob, tuple(int(x) for x in args.base.split(",")) + ((1,) if prob.dim == 2 else ()))
    sim = make_sim(prob)
    if args.sweep != "default":
        sim.set_sweep_variant(SWEEPS[args.sweep])
    if args.tick_shape:
        t, k = (int(x) for x in args.tick_shape.split(","))
        sim.set_tick_shape(t, k)
    X = node_coords_of(sim, prob)
    if args.workload == "spiral2d":
        V0, v0 = W.spiral_state(X, prob.extent[0])
    elif prob.dim == 2:
        # a scaled base keeps the front at the same fraction of the domain
        V0, v0 = W.front_state(X, FRONT["origin"], FRONT["radius"] * prob.extent[0] / 2.0, FRONT["width"],
                               FRONT["tail"])
    else:
        V0, v0 = W.planar_front_state(X, PLANAR["x0"] * prob.extent[0] / 2.0, PLANAR["width"], PLANAR["tail"])
    sim.set_initial(V0, v0)
    sim.step_barriers(SETUP_BARRIERS)
    # clocks are sampled from the warm-up on (the sampler's start-up stays out of the timed steps)
    clk = ClockSampler(torch.cuda.current_device())
    clk.start()
    time.sleep(0.5)
    sim.step_barriers(args.warmup)
    _, _, stream_ptr = sim.device_view(1)
    stream = torch.cuda.ExternalStream(stream_ptr)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    # the first fill loads torch's fill kernel (lazy module loading, ~0.25 s): not in the timed loop
    with torch.cuda.stream(stream):
        flush.fill_(-1.0)
    torch.cuda.synchronize()
    sim.reset_stats()
    sim.set_timing(True)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(i))
        evs[i][0].record(stream)
        sim.step_barriers(1)
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    wall1 = time.perf_counter()
    if dist:
        dist.barrier()
    clocks = clk.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = sum(step_ms)
    st = sim.stats()
    n_e, n_dof, _ = sim.sizes()
    if st["timed_barriers"] != args.steps:
        raise RuntimeError("sweep timing covers %d of %d barriers" % (st["timed_barriers"], args.steps))
    if dist:
        total_ms_all, dof_all = reduce_over_ranks(total_ms, st["dof_updates"], dist, "cuda")
    else:
        total_ms_all, dof_all = total_ms, float(st["dof_updates"])
    value = dof_all / (total_ms_all / 1e3)
    # roofline of the dominant kernel (the sweep tick kernel), from its own CUDA-event timing
    peak, peak_kind = load_peaks()
    sweep_s = st["sweep_ms"] / 1e3
    alg_bytes = st["dof_updates"] * alg_bytes
    achieved = alg_bytes / sweep_s / 1e9 if sweep_s > 0 else 0.0
    traffic = (TRAFFIC_PER_LAUNCH.get((args.workload, kname))
               if args.sweep == "default" and not args.tick_shape and not args.base else None)
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": traffic, "peak_source": peak_kind,
            "alg_bytes_per_launch": round(alg_bytes / max(st["tick_launches"], 1), 1),
            "kernel": kname, "launches": st["tick_launches"],
            "avg_launch_us": round(st["sweep_ms"] * 1e3 / max(st["tick_launches"], 1), 3),
            "alg_bytes_per_dof_update": WORKLOADS[args.workload][1]}
    if traffic:
        # the same launches judged by their measured DRAM traffic (ncu, cold caches) instead of
        # the algorithmic bytes
        avg_s = st["sweep_ms"] / 1e3 / max(st["tick_launches"], 1)
        roof["traffic_frac"] = round(traffic / avg_s / 1e9 / peak, 4)
    roof["target"] = "0.6 of the HBM peak: not met"
    # end to end through the public API with host buffers: upload state, one barrier, read back
    e2e = run_e2e(sim, args, torch)
    out = None
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms_all / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(prob),
                       "sweep": args.sweep if args.sweep != "default" else ("tensor" if "k_tick_tc" in kname else "thread"),
                       "tick_shape": args.tick_shape or "128,16",
                       "domain_cm": list(prob.extent[:prob.dim]), "base": list(prob.base[:prob.dim]),
                       "max_refine": prob.max_refine, "n_lts_levels": prob.n_lts_levels,
                       "dt_barrier_ms": sim.dt, "n_elements": n_e, "n_dof": n_dof,
                       "level_counts": st["level_counts"][:prob.n_lts_levels],
                       "initial_state": ("synthetic broken planar wave (spiral onset), band x < 1/4 side"
                                         if args.workload == "spiral2d" else
                                         "synthetic developed front, r=%.2f cm, width 0.01 cm" % (prob.extent[0] / 2.0)
                                         if prob.dim == 2 else
                                         ("synthetic front at reference X_0=%.2f (a surface of constant azimuth), "
                                          "width 0.012" % (prob.extent[0] / 2.0)) if getattr(prob, "geometry", 0) else
                                         "synthetic planar front at x=%.2f cm, width 0.012 cm" % (prob.extent[0] / 2.0)),
                       "l2": "512 MiB flush buffer written between timed steps",
                       "parallelism": "replicas" if world > 1 else "single"},
            "dof_updates_per_step": st["dof_updates"] / args.steps,
            "breakdown_ms_per_step": {
                "sweep": st["sweep_ms"] / args.steps, "eta_s": st["indicator_ms"] / args.steps,
                "amr_host": st["amr_host_ms"] / args.steps, "mesh_upload_transfer": st["transfer_ms"] / args.steps},
            "amr_rebuilds": st["amr_rebuilds"],
            **({"factor_updates_per_step": st["factor_updates"] / args.steps} if prob.geometry else {}),
            "sweep_only_dof_updates_per_s": st["dof_updates"] / sweep_s if sweep_s > 0 else None,
            # host clock around the same K steps: each step also holds the L2 flush and the
            # library's end-of-call synchronisation (one read of the device bookkeeping)
            "host_wall": {"s": wall1 - wall0, "ms_per_step": (wall1 - wall0) * 1e3 / args.steps},
            "roofline": roof,
            "e2e": e2e,
            "gpu_launches": st["kernel_launches"],
            "clocks": clocks,
        }
        if world == 1 and not args.no_cpu_baseline and args.workload in CPU_SAMPLE:
            out["cpu_baseline"] = cpu_baseline(args)
    sim.close()
    if dist:
        dist.destroy_process_group()
    return out


def run_e2e(sim, args, torch):
    """Same metric through the C ABI with pinned host buffers, copies inside the timed region:
    each step uploads V and the state variable, advances one barrier step and reads both
    back (FP32 transfers, the working precision of the path)."""
    n = max(2, min(args.steps, 10))
    Vh, vh = sim.read_fields_f32()

    def pinned(m):
        return torch.empty(m, dtype=torch.float32, pin_memory=True).numpy()

    cap = Vh.size * 2
    V, v, Vo, vo = pinned(cap), pinned(cap), pinned(cap), pinned(cap)
    V[:Vh.size] = Vh
    v[:vh.size] = vh
    nd = Vh.size
    sim.reset_stats()
    h2d = d2h = 0
    t0 = time.perf_counter()
    for _ in range(n):
        sim.set_initial_f32(V[:nd], v[:nd])
        h2d += 8 * nd
        sim.step_barriers(1)
        nd = sim.sizes()[1]
        if nd > cap:
            cap = nd * 2
            Vo, vo = pinned(cap), pinned(cap)
        Vr, vr = sim.read_fields_f32(Vo, vo)
        d2h += 8 * nd
        # the results are the next step's inputs (ping-pong of the pinned buffers)
        V, Vo, v, vo = Vo, V, vo, v
    t1 = time.perf_counter()
    st = sim.stats()
    return {"value": st["dof_updates"] / (t1 - t0), "unit": UNIT, "steps": n,
            "h2d_bytes_per_step": h2d // n, "d2h_bytes_per_step": d2h // n}


# ---------------------------------------------------------------------------
# Many simulations on one GPU: a batch of 64 heterogeneous instances, and a
# continuous-batching request stream.  Both go through mdl_batch_*.
# ---------------------------------------------------------------------------

CLASS_ALG_BYTES = {(2, 1): 25.0, (3, 1): 21.5, (3, 2): 17.6, (2, 2): 16.0 + 36.0 / 9.0}


def slot_alg_bytes(prob):
    return CLASS_ALG_BYTES.get((prob.dim, prob.order), 16.0)


def run_batch(args, rank, world):
    """64 heterogeneous resident instances (32 2D Q1, 16 3D Q1, 16 3D Q2; base element counts
    log-uniform in [1e3, 1e5], seed 4) stepped in fused rounds: a step is one batch round, every
    instance advancing one barrier; per element class the sweeps of all its instances run as
    one persistent launch per global tick, replayed from a captured graph, or as the
    instances' own sweeps, whichever the batch's tuner measured faster during warm-up.  The K
    timed rounds are one batch step (issued back to back, waited for once).  One GPU: under a
    multi-rank launch it stops with an error instead of reporting one rank's rate."""
    if world > 1:
        raise SystemExit("bench.py --workload batch64 runs on one GPU (got WORLD_SIZE=%d)" % world)
    import torch
    torch.cuda.set_device(0)
    from paper_2310_07607_gb300 import build, mdl
    build.build()
    inst = W.batch_instances(64, seed=4)
    b = mdl.Batch(autotune=True, fused=not args.batch_streams)
    t_setup = time.perf_counter()
    slots = [b.admit(p, t_end) for p, t_end in inst]
    t_setup = time.perf_counter() - t_setup
    sims = {s: b.slot(s)[0] for s in slots}
    # warm-up covers the tuner (7 candidates x 2 rounds per class, one round at a time)
    classes = ((32, 2, 1, "fp32_2d_q1"), (32, 3, 1, "fp32_3d_q1"), (32, 3, 2, "fp32_3d_q2"))
    warm = 0
    while warm < args.warmup or (not args.batch_streams and warm < 40 and
                                 any(b.fused_info(pr, d, o)[0] is None for pr, d, o, _ in classes)):
        b.step(1)
        warm += 1
    base = {s: sims[s].stats() for s in slots}
    _, (r0, l0) = b.fused_info(32, 2, 1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.step(args.steps)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    now = {s: sims[s].stats() for s in slots}
    _, (r1, l1) = b.fused_info(32, 2, 1)
    du = {s: now[s]["dof_updates"] - base[s]["dof_updates"] for s in slots}
    klaunch = sum(now[s]["kernel_launches"] - base[s]["kernel_launches"] for s in slots) + (l1 - l0)
    total = float(sum(du.values()))
    alg = sum(du[s] * slot_alg_bytes(p) for s, (p, _) in zip(slots, inst))
    peak, peak_kind = load_peaks()
    n_dof = sum(sims[s].sizes()[1] for s in slots)
    # barriers each instance needs to reach its 100 ms horizon, and the projected batch time
    need = [int(math.floor(t_end / sims[s].time()[2] + 1e-9)) for s, (_, t_end) in zip(slots, inst)]
    per_round_s = secs / args.steps
    used, budget, resident = b.usage()
    shapes = {}
    for prec, dim, order, name in classes:
        info, _ = b.fused_info(prec, dim, order)
        if info:
            shapes[name] = {"choice": "own sweeps" if info["own"] else
                            "fused %d threads x %d elements per item" % (info["threads"], info["tile"]),
                            "best_round_sweep_ms": round(info["best_ms"], 3),
                            "worst_round_sweep_ms": round(info["worst_ms"], 3),
                            "own_sweeps_round_ms": round(info["own_ms"], 3)}
    out = {
        "metric": METRIC, "value": total / secs, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": warm, "ms_per_step": secs * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batch64_mixed_2dq1_3dq1_3dq2_lts1to4_ap_fp32", "instances": len(slots),
                   "mode": "streams" if args.batch_streams else "fused rounds (per element class: one sweep "
                                                             "launch per global tick from a captured graph, "
                                                             "or own sweeps, as tuned)",
                   "rounds_per_call": args.steps,
                   "n_dof_total": int(n_dof), "device_bytes": int(used), "resident": resident,
                   "timing": "host clock around one batch step of K rounds, device synchronised on both sides",
                   "l2": "working set larger than L2 (%.0f MB of state)" % (used / 1e6)},
        "roofline": {"bound": "hbm", "achieved": round(alg / secs / 1e9, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(alg / secs / 1e9 / peak, 4), "traffic": None, "peak_source": peak_kind,
                     "note": "whole batch round incl. every phase; per-class algorithmic bytes"},
        "gpu_launches": int(klaunch),
        "fused": {"rounds_timed": r1 - r0, "sweep_launches_timed": l1 - l0,
                  "sweep_launches_per_round": (l1 - l0) / max(r1 - r0, 1), "tuned_shapes": shapes},
        "horizon": {"t_end_ms": inst[0][1], "barriers_max": max(need), "barriers_min": min(need),
                    "projected_s_all_to_horizon": round(max(need) * per_round_s, 2)},
        "setup_s": round(t_setup, 2),
    }
    b.close()
    return out


def run_serve(args, rank, world):
    """Poisson request stream (rate 20/s for 60 s, seed 5; 2D/3D, Q1/Q2, AMR + LTS, horizons
    100-500 ms) through the continuous-batching loop for a bounded wall time, then the same
    stream through a plain loop (one request at a time, FP64, uniform mesh at the finest
    level, global time step) for a bounded wall time.  No request of that stream can finish
    inside the window (1e5-1e6 barrier steps each), so an added measurement follows on
    requests that do: completed_window()."""
    import torch
    torch.cuda.set_device(0)
    from paper_2310_07607_gb300 import build, mdl
    from paper_2310_07607_gb300.serve import Request, Server
    build.build()
    wall = float(os.environ.get("MDL_SERVE_WALL_S", "60"))
    reqs = [Request(rid=i, prob=p, horizon_ms=h, arrival_s=t)
            for i, (t, p, h) in enumerate(W.poisson_requests(20.0, 60.0, seed=5))]
    srv = Server(budget_bytes=0, barriers_per_round=args.serve_round, autotune=True)
    rep = srv.run(reqs, wall_limit_s=wall, drain=False)
    srv.close()
    # plain comparator: the same arrivals served one by one without adaptivity in FP64
    plain = run_plain_loop(mdl, reqs, wall)
    done = completed_window(mdl, Request, Server, args)
    return {"metric": "sims/s", "value": rep["sims_per_s"], "unit": "sims/s", "n_gpus": 1,
            "steps": None, "warmup": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "serve_poisson_rate20_60s_amr2_lts3_ap_fp32", "wall_limit_s": wall,
                       "barriers_per_round": args.serve_round},
            "adaptive": rep, "plain_fp64_uniform_loop": plain, "completed_window": done}


def probe_points(prob):
    """Coordinates of the activation-time probes: the Gauss-Legendre nodes of every root
    element (roots with axis 0 fastest, the nodes of a root with axis 0 fastest)."""
    d, n1 = prob.dim, prob.order + 1
    xi = np.polynomial.legendre.leggauss(n1)[0]
    h = [prob.extent[k] / prob.base[k] for k in range(d)]
    q = np.arange(n1 ** d)
    loc = np.stack([(xi[(q // n1 ** k) % n1] + 1.0) * 0.5 * h[k] for k in range(d)], axis=1)
    e = np.arange(int(np.prod(prob.base[:d])))
    lo = []
    for k in range(d):
        lo.append((e % prob.base[k]) * h[k])
        e = e // prob.base[k]
    lo = np.stack(lo, axis=1)
    return (lo[:, None, :] + loc[None, :, :]).reshape(-1, d)


def lat_interpolator(prob, lat):
    """The activation times of a uniform-grid run (probes on the Gauss-Legendre nodes of every
    element) as a piecewise-multilinear function on the tensor grid of those nodes; NaN where
    a neighbouring probe never activated."""
    from scipy.interpolate import RegularGridInterpolator
    d, n1 = prob.dim, prob.order + 1
    xi = np.polynomial.legendre.leggauss(n1)[0]
    axes = [((np.arange(prob.base[k])[:, None] + (xi[None, :] + 1.0) * 0.5) * (prob.extent[k] / prob.base[k])).ravel()
            for k in range(d)]
    b = [prob.base[k] for k in range(d)]
    v = np.where(np.isfinite(lat), lat, np.nan)
    if d == 2:
        grid = v.reshape(b[1], b[0], n1, n1).transpose(0, 2, 1, 3).reshape(b[1] * n1, b[0] * n1)
    else:
        grid = v.reshape(b[2], b[1], b[0], n1, n1, n1).transpose(0, 3, 1, 4, 2, 5).reshape(
            b[2] * n1, b[1] * n1, b[0] * n1)
    f = RegularGridInterpolator(tuple(axes[::-1]), grid, method="linear", bounds_error=False, fill_value=np.nan)
    return lambda pts: f(pts[:, ::-1])


def lat_difference(prob_a, lat_a, prob_p, lat_p):
    """Activation times of an adaptive run at its probes against the plain uniform-grid run
    interpolated there: probes compared (active in both), active in one only, and the mean and
    largest absolute difference (ms)."""
    ref = lat_interpolator(prob_p, lat_p)(probe_points(prob_a))
    fa, fr = np.isfinite(lat_a), np.isfinite(ref)
    both = fa & fr
    diff = np.abs(lat_a[both] - ref[both])
    return {"probes": int(both.sum()), "adaptive_only": int((fa & ~fr).sum()),
            "plain_only": int((~fa & fr).sum()),
            "mean_ms": float(diff.mean()) if diff.size else None,
            "max_ms": float(diff.max()) if diff.size else None}


def completed_window(mdl, Request, Server, args, rate=3.0, arrivals_s=20.0, cap_s=240.0):
    """Added measurement on requests that finish: the generator above with smaller, coarser
    meshes and 5-20 ms horizons (workloads.completed_requests, 3 arrivals/s for 20 s, seed 6),
    served to completion by the adaptive FP32 batch loop and by the plain FP64 loop (uniform
    mesh at the finest level, global step), each bounded by cap_s.  Accuracy: every request's
    activation times in the adaptive run against the plain run's, interpolated to the same
    probes; and, on a sample, the adaptive FP32 run against the same run in FP64."""
    gen = W.completed_requests(rate, arrivals_s, seed=6)
    mk = lambda: [Request(rid=i, prob=p, horizon_ms=h, arrival_s=t) for i, (t, p, h) in enumerate(gen)]
    lat_a = {}

    def grab(req, g):
        lat_a[req.rid] = g.read_activation()
        return None

    srv = Server(budget_bytes=0, barriers_per_round=args.serve_round, autotune=True, on_result=grab)
    reqs = mk()
    rep = srv.run(reqs, wall_limit_s=cap_s, drain=False)
    srv.close()
    # capacity: the same requests all at once (the arrival-driven run is bound by the arrival
    # rate; the plain loop, one request at a time, is saturated throughout its run)
    srv = Server(budget_bytes=0, barriers_per_round=args.serve_round, autotune=True)
    burst = srv.run([Request(rid=i, prob=p, horizon_ms=h, arrival_s=0.0) for i, (t, p, h) in enumerate(gen)],
                    wall_limit_s=cap_s, drain=False)
    srv.close()
    lat_p = {}
    plain = run_plain_loop(mdl, mk(), cap_s, keep=lat_p)
    per = []
    for i, (t, p, h) in enumerate(gen):
        if i in lat_a and i in lat_p:
            per.append(lat_difference(p, lat_a[i], plain_version(p), lat_p[i]))
    means = [x["mean_ms"] for x in per if x["mean_ms"] is not None]
    maxes = [x["max_ms"] for x in per if x["max_ms"] is not None]
    # FP32 against FP64 on a sample: the first completed request of each (dim, order)
    fp = []
    seen = set()
    for i, (t, p, h) in enumerate(gen):
        key = (p.dim, p.order)
        if i not in lat_a or key in seen:
            continue
        seen.add(key)
        g = mdl.Sim(p.replace(precision=64))
        g.step_barriers(int(math.floor(h / g.dt + 1e-9)))
        l64 = g.read_activation()
        g.close()
        f32, f64 = np.isfinite(lat_a[i]), np.isfinite(l64)
        both = f32 & f64
        fp.append({"dim": p.dim, "order": p.order, "probes": int(both.sum()),
                   "active_in_one_only": int((f32 != f64).sum()),
                   "max_ms": float(np.abs(lat_a[i][both] - l64[both]).max()) if both.any() else None})
    keep = ("completed", "failed", "wall_s", "sims_per_s", "ttr_p50_s", "ttr_p99_s", "peak_resident",
            "busy_fraction", "queue_mean")
    return {
        "label": "added measurement: requests that finish inside the window (100-2000 base elements, "
                 "base elements 8x (2D) / 4x (3D) larger than the stream above, horizons 5-20 ms); "
                 "the stream above is unchanged",
        "requests": len(gen), "arrivals_per_s": rate, "arrivals_s": arrivals_s, "cap_s": cap_s,
        "adaptive_fp32_batch": {k: rep[k] for k in keep},
        "plain_fp64_uniform_loop": {k: plain[k] for k in ("completed", "wall_s", "sims_per_s", "ttr_p50_s",
                                                          "ttr_p99_s")},
        "sims_per_s_ratio_adaptive_over_plain": (rep["sims_per_s"] / plain["sims_per_s"]
                                                 if plain["sims_per_s"] > 0 else None),
        "adaptive_fp32_batch_all_at_once": {k: burst[k] for k in ("completed", "wall_s", "sims_per_s", "ttr_p50_s",
                                                                  "ttr_p99_s", "peak_resident")},
        "capacity_ratio_adaptive_all_at_once_over_plain": (burst["sims_per_s"] / plain["sims_per_s"]
                                                           if plain["sims_per_s"] > 0 else None),
        "accuracy": {
            "lat_adaptive_vs_plain_ms": {"requests": len(per), "median_of_mean": statistics.median(means)
                                         if means else None, "max_of_max": max(maxes) if maxes else None,
                                         "probes": int(sum(x["probes"] for x in per)),
                                         "active_in_one_only": int(sum(x["adaptive_only"] + x["plain_only"]
                                                                       for x in per))},
            "lat_fp32_vs_fp64_adaptive_ms": fp,
            "parity": "the FP64 paths (adaptive and plain) equal the FP64 oracle to 1e-12 in the GPU tests",
        },
    }


def plain_version(prob):
    import dataclasses
    f = 2 ** prob.max_refine
    base = tuple(int(x * f) if k < prob.dim else x for k, x in enumerate(prob.base))
    return dataclasses.replace(prob, base=base, max_refine=0, amr_enabled=0, lts_enabled=0,
                               n_lts_levels=1, precision=64, dt_barrier=0.0)


def run_plain_loop(mdl, reqs, wall, keep=None):
    """One request at a time in arrival order, FP64, uniform mesh at the adaptive run's finest
    level, global forward Euler; bounded by `wall` seconds of serving time.  keep: a dict that
    receives the activation times of each completed request by rid."""
    t0 = time.perf_counter()
    done, ttr, proj = 0, [], []
    for r in sorted(reqs, key=lambda x: x.arrival_s):
        now = time.perf_counter() - t0
        if now >= wall:
            break
        if r.arrival_s > now:
            time.sleep(r.arrival_s - now)
        p = plain_version(r.prob)
        g = mdl.Sim(p)
        n = int(math.floor(r.horizon_ms / g.dt + 1e-9))
        start = time.perf_counter() - t0
        k = 0
        while k < n and time.perf_counter() - t0 < wall:
            m = min(64, n - k)
            g.step_barriers(m)
            k += m
        end = time.perf_counter() - t0
        if k == n:
            done += 1
            ttr.append(end - r.arrival_s)
            if keep is not None:
                keep[r.rid] = g.read_activation()
        else:
            rate = k / max(end - start, 1e-9)
            proj.append((start - r.arrival_s) + n / max(rate, 1e-9))
        g.close()
    from paper_2310_07607_gb300.serve import percentile
    el = time.perf_counter() - t0
    return {"completed": done, "sims_per_s": done / el, "wall_s": el,
            "ttr_p50_s": percentile(ttr, 0.5), "ttr_p99_s": percentile(ttr, 0.99),
            "projected_ttr_of_unfinished_s": proj[:4]}


# ---------------------------------------------------------------------------
# The FP64 oracle on the host cores (bounded sample of the same workload).
# ---------------------------------------------------------------------------

# Bounded samples of each workload for the oracle: a patch of roots with the workload's h,
# physics and thresholds, `setup` barriers (the AMR reaching depth 3 on the front) before
# `barriers` timed barrier steps.
CPU_SAMPLE = {
    "slab2d": dict(base=(64, 64, 1), setup=3, barriers=6),
    "slab3d": dict(base=(4, 2, 2), setup=3, barriers=10),
}
# peak host memory of one oracle process on the sample (its assembled sparse operator)
CPU_SAMPLE_BYTES = {"slab2d": 2.5e9, "slab3d": 4.0e9}

ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, %(root)r)
import numpy as np
import workloads as W
from oracle import lts
wl = %(workload)r
if wl == "slab2d":
    prob = W.scaled(W.slab_2d_q1_256(), %(base)r).replace(precision=64)
else:
    prob = W.scaled(W.slab_3d_q2(), %(base)r).replace(precision=64)
sim = lts.Sim(prob)
X = sim.disc.node_coords()
if wl == "slab2d":
    V0, v0 = W.front_state(X, (0.0, 0.0, 0.0), %(radius)r, %(width)r, %(tail)r)
else:
    V0, v0 = W.planar_front_state(X, %(x0)r, %(width)r, %(tail)r)
sim.V, sim.v = V0, v0
for _ in range(%(setup)d):
    sim.barrier()
res = []
for _ in range(%(steps)d):
    d0 = sim.dof_updates
    t0 = time.perf_counter()
    sim.barrier()
    res.append((sim.dof_updates - d0, time.perf_counter() - t0))
print(json.dumps(res))
"""


def _oracle_code(workload, setup, steps):
    smp = CPU_SAMPLE[workload]
    base = smp["base"]
    if workload == "slab2d":
        # same h and front width; front radius scaled with the patch so it crosses the patch
        radius = FRONT["radius"] * base[0] / 256.0
        geo = dict(radius=radius, x0=0.0, width=FRONT["width"], tail=FRONT["tail"] * radius / FRONT["radius"])
    else:
        # the planar front at the middle of the patch, as on the full slab
        x0 = PLANAR["x0"] * base[0] / 128.0
        geo = dict(radius=0.0, x0=x0, width=PLANAR["width"], tail=PLANAR["tail"])
    return ORACLE_SNIPPET % dict(root=ROOT, workload=workload, base=tuple(base), setup=setup, steps=steps, **geo)


def _oracle_env():
    return dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")


def oracle_run(workload, setup, steps):
    """One single-threaded oracle process on the workload's sample: [(DOF-updates, seconds)]."""
    r = subprocess.run([sys.executable, "-c", _oracle_code(workload, setup, steps)], capture_output=True,
                       text=True, env=_oracle_env(), timeout=1800)
    if r.returncode != 0:
        raise RuntimeError("oracle baseline failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def host_cores():
    """Cores this process may run on (the affinity mask, as nproc reports)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def mem_available():
    try:
        with open("/proc/meminfo") as f:
            for ln in f:
                if ln.startswith("MemAvailable:"):
                    return int(ln.split()[1]) * 1024
    except OSError:
        pass
    return None


def oracle_run_all_cores(workload, setup, steps, n):
    """n single-threaded oracle processes at once, one per host core, each on its own copy of
    the sample: the host's aggregate rate is their DOF-updates over the slowest one's time."""
    code = _oracle_code(workload, setup, steps)
    procs = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                              text=True, env=_oracle_env()) for _ in range(n)]
    dofs, secs, failed = 0, 0.0, None
    try:
        for p in procs:
            out, err = p.communicate(timeout=3600)
            if p.returncode != 0:
                failed = "oracle process exited %d: %s" % (p.returncode, err[-500:])
                break
            res = json.loads(out.strip().splitlines()[-1])
            dofs += sum(r[0] for r in res)
            secs = max(secs, sum(r[1] for r in res))
    finally:
        for p in procs:
            if p.poll() is None:
                p.kill()
                p.wait()
    if failed:
        raise RuntimeError(failed)
    return dofs, secs


def _sample_text(workload, n_steps):
    smp = CPU_SAMPLE[workload]
    b = smp["base"][:2] if workload == "slab2d" else smp["base"]
    return ("FP64 numpy oracle on a %s-root patch of the %s (same h, physics and thresholds), "
            "%d barrier steps after %d setup barriers that refine the front to depth 3"
            % ("x".join(str(x) for x in b), "2D slab" if workload == "slab2d" else "3D slab", n_steps,
               smp["setup"]))


def cpu_baseline(args):
    smp = CPU_SAMPLE[args.workload]
    res = oracle_run(args.workload, smp["setup"], smp["barriers"])
    d1 = sum(r[0] for r in res)
    s1 = sum(r[1] for r in res)
    nproc = host_cores()
    single = {"value": d1 / s1, "unit": UNIT, "cores": 1, "seconds": round(s1, 2)}
    # one process per core, as many as the host memory holds (each keeps its own operator)
    avail = mem_available()
    n = nproc if avail is None else max(1, min(nproc, int(0.6 * avail / CPU_SAMPLE_BYTES[args.workload])))
    try:
        dall, sall = oracle_run_all_cores(args.workload, smp["setup"], smp["barriers"], n)
    except Exception as ex:  # report the single-core figure rather than no baseline
        return {"value": single["value"], "unit": UNIT, "cores": 1, "kind": "oracle", "nproc": nproc,
                "sample": _sample_text(args.workload, len(res)), "all_cores_failed": str(ex)[:300]}
    return {"value": dall / sall, "unit": UNIT, "cores": n, "kind": "oracle",
            "sample": _sample_text(args.workload, len(res)) + "; %d processes at once, one per host core" % n,
            "nproc": nproc, "single_core": single}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    workload = args.workload if args.workload in CPU_SAMPLE else "slab3d"
    smp = CPU_SAMPLE[workload]
    res = oracle_run(workload, smp["setup"] + args.warmup, args.steps)
    dofs = sum(r[0] for r in res)
    secs = sum(r[1] for r in res)
    value = dofs / secs
    factory = WORKLOADS[workload][0]
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1e3 / len(res),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(factory()),
                   "sample": "%s-root patch, same h/physics/thresholds" % "x".join(str(x) for x in smp["base"])},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": _sample_text(workload, len(res))},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="slab3d", choices=sorted(WORKLOADS) + ["batch64", "serve"])
    ap.add_argument("--serve-round", type=int, default=16, help="barriers per slot per serving round")
    ap.add_argument("--batch-streams", action="store_true",
                    help="batch64: each instance's own sweep on its own stream instead of fused rounds")
    ap.add_argument("--tick-shape", default="", help="sweep launch shape 'threads,blocks_per_sm'")
    ap.add_argument("--base", default="", help="base grid 'nx,ny[,nz]' at the workload's element size")
    ap.add_argument("--sweep", default="default", choices=["default"] + sorted(SWEEPS),
                    help="sweep kernel variant (default: the library's choice, tensor for Q2 3D FP32 and "
                         "thread otherwise; thread per element; group: Q1 lanes per element; coop: one "
                         "cooperative launch per barrier; tensor: tcgen05 residual, Q2 3D FP32)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    elif args.workload == "batch64":
        out = run_batch(args, rank, world)
    elif args.workload == "serve":
        out = run_serve(args, rank, world) if rank == 0 else None
    else:
        out = run_ours(args, rank, world)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
