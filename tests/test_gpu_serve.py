"""Continuous-batching request loop: requests arriving while others run are admitted as
memory allows, all complete, and each result equals the same simulation run alone (with the
thread-per-element sweep every element takes in the batch's fused rounds: meshes and activated
probes identical, V within FP32 rounding of the two compilations of the element step)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def small(dim, p, seed, precision=32):
    return W.Problem(dim=dim, order=p, extent=(0.2, 0.15, 0.1), base=(4, 3, 2), sigma_l=1.2, sigma_t=0.4,
                     fibre=(0.6, 0.8, 0.0), gamma=10.0 * p * p, max_refine=1, n_lts_levels=2,
                     lts_enabled=1, amr_enabled=1, tau_refine=1e-10, tau_coarsen=1e-13, dt_barrier=0.0,
                     state_integrator=W.STATE_EXP, precision=precision,
                     stimuli=[W.Stimulus((0, 0, 0), (0.05 + 0.01 * seed, 0.05, 0.05), 1.0, 0.0, 1.0)])


def test_serving_loop_results_equal_alone():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2310_07607_gb300 import build, mdl
    from paper_2310_07607_gb300.serve import Request, Server
    build.build()
    specs = [(2, 1), (3, 1), (2, 2), (3, 2), (2, 1), (3, 1)]
    reqs = []
    for i, (d, p) in enumerate(specs):
        prob = small(d, p, i)
        dt = mdl.Sim(prob).dt
        reqs.append(Request(rid=i, prob=prob, horizon_ms=(10 + 3 * i) * dt, arrival_s=0.02 * i))

    def grab(req, g):
        return {"V": g.read_V(), "lat": g.read_activation(), "nbar": g.time()[1]}

    # a budget that holds about three of them at a time forces waiting and admission later
    fp = max(mdl.Batch(autotune=False).footprint(r.prob) for r in reqs)
    srv = Server(budget_bytes=int(3.2 * fp), barriers_per_round=4, autotune=False, on_result=grab)
    rep = srv.run(reqs, wall_limit_s=120.0, drain=True)
    srv.close()
    assert rep["completed"] == len(reqs) and rep["failed"] == 0
    assert rep["peak_resident"] <= 3
    assert np.isfinite(rep["ttr_p50_s"]) and rep["ttr_p99_s"] >= rep["ttr_p50_s"]
    for r in reqs:
        g = mdl.Sim(r.prob)
        g.set_sweep_variant(mdl.SWEEP_THREAD)
        n = int(np.floor(r.horizon_ms / g.dt + 1e-9))
        g.step_barriers(n)
        assert r.result["nbar"] == n
        Va = g.read_V()
        assert np.abs(r.result["V"] - Va).max() <= 1e-5 * max(np.abs(Va).max(), 1.0)
        la, lb = g.read_activation(), r.result["lat"]
        assert np.array_equal(np.isfinite(la), np.isfinite(lb))
        if np.isfinite(la).any():
            assert np.abs(la[np.isfinite(la)] - lb[np.isfinite(la)]).max() <= 1e-6
        g.close()


@pytest.mark.parametrize("which", [0, 1, 2, 4])
def test_completed_window_requests_fp64_match_oracle(which):
    """The physics of the serving measurement on completed requests (workloads.completed_requests:
    coarse meshes, AMR to depth 2, 3 LTS levels), on a patch of the request's roots: the FP64
    adaptive run and the plain run of the plain loop (uniform finest mesh, global step) each
    equal the FP64 oracle -- V to 1e-12 (mass-weighted), activation times to 1e-9 ms, the
    adaptive meshes identical -- so the accuracies the measurement reports for the two arms are
    those of the method, not of the kernels."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2310_07607_gb300 import build, mdl
    from oracle import lts
    from tests.helpers import forest_arrays, mass_rel_l2
    import bench
    build.build()
    t, prob, h = W.completed_requests()[which]
    patch = W.scaled(prob, (8, 8, 1) if prob.dim == 2 else (4, 2, 2)).replace(precision=64)
    # the request's corner stimulus, a quarter of the patch wide
    patch = patch.replace(stimuli=[W.Stimulus((0, 0, 0), tuple(0.25 * patch.extent[k] for k in range(3)),
                                              1.0, 0.0, 1.0)])
    for p in (patch, bench.plain_version(patch)):
        o = lts.Sim(p)
        g = mdl.Sim(p)
        assert g.dt == o.dt
        n = int(2.0 / o.dt)          # 2 ms: the stimulated front refines and spreads
        for _ in range(n):
            o.barrier()
        g.step_barriers(n)
        assert mass_rel_l2(o.disc.M, g.read_V(), o.V) <= 1e-12
        la, lo = g.read_activation(), o.lat
        assert np.array_equal(np.isfinite(la), np.isfinite(lo))
        if np.isfinite(lo).any():
            assert np.abs(la[np.isfinite(lo)] - lo[np.isfinite(lo)]).max() <= 1e-9
        if p.amr_enabled:
            lv, cc, _ = forest_arrays(o.forest)
            r2, l2, c2, _ = g.read_mesh()
            assert np.array_equal(l2, lv) and np.array_equal(c2, cc)
        g.close()
