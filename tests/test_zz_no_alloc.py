"""The allocation-free FP64 integral (mdl_integral_noalloc) on the GPU.

Callers that cannot allocate device memory (inside a stream capture, in a real-time
loop, or under a host allocator that owns all device memory) use this entry point; it
must give the same FP64 integral of V as the barrier diagnostic that a stepping call
reports in mdl_stats.integral_V.  The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

import workloads as W
from tests.helpers import forest_arrays, random_forest

pytestmark = pytest.mark.gpu


def _problem(precision):
    return W.Problem(dim=2, order=1, extent=(0.4, 0.3, 1.0), base=(4, 3, 1), sigma_l=1.2, sigma_t=0.4,
                     fibre=(0.6, 0.8, 0.0), gamma=10.0, max_refine=2, n_lts_levels=3, lts_enabled=1,
                     amr_enabled=1, tau_refine=1e30, tau_coarsen=-1.0, dt_barrier=0.0,
                     state_integrator=W.STATE_EXP, precision=precision,
                     stimuli=[W.Stimulus((0, 0, 0), (0.1, 0.1, 1.0), 1.0, 0.0, 1.0)])


@pytest.mark.parametrize("precision", [32, 64])
def test_integral_noalloc_matches_barrier_diagnostic(precision):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2310_07607_gb300 import build, mdl
    build.build()
    prob = _problem(precision)
    f = random_forest(2, prob.base, 2, prob.extent, steps=2, seed=3, tau=0.7)
    g = mdl.Sim(prob)
    lv, cc, root = forest_arrays(f)
    g.upload_mesh(lv, cc, root)
    from oracle.sipg import Disc  # node coordinates of the uploaded mesh for the initial front
    X = Disc(prob.replace(precision=64), f).node_coords()
    V0, v0 = W.front_state(X, (0, 0, 0), 0.15, 0.02, tail=0.05)
    g.set_initial(V0, v0)
    for call in range(2):
        g.step_barriers(1)
        ref = g.stats()["integral_V"]
        vptr, nd, stream = g.device_view(0)
        _, level, _, _ = g.read_mesh()
        lev = torch.tensor(level, dtype=torch.int8, device="cuda")
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        mdl.integral_noalloc(prob, vptr, lev.data_ptr(), len(level), out.data_ptr(), stream)
        torch.cuda.synchronize()
        val = out.item()
        assert np.isfinite(val)
        assert abs(val - ref) <= 1e-12 * abs(ref), (call, val, ref)
    # sizes beyond the documented maximum are rejected before any device work
    with pytest.raises(mdl.MdlError) as ei:
        mdl.integral_noalloc(prob, vptr, lev.data_ptr(), (1 << 30) + 1, out.data_ptr(), stream)
    assert ei.value.code == -1
    g.close()


@pytest.mark.parametrize("dim,order", [(2, 1), (3, 2)])
def test_integral_noalloc_levels_up_to_seven_and_out_of_range(dim, order):
    """Levels span the whole documented range 0..7 (a synthetic field, not a mesh); a level
    outside it turns the result into NaN instead of wrapping to another level's mass."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from oracle import basis
    from paper_2310_07607_gb300 import build, mdl
    build.build()
    prob = W.Problem(dim=dim, order=order, extent=(0.4, 0.3, 0.2), base=(4, 3, 2), precision=64)
    n_p = (order + 1) ** dim
    rng = np.random.default_rng(11)
    n_e = 3000
    level = rng.integers(0, 8, n_e).astype(np.int8)
    level[:8] = np.arange(8)
    V = rng.standard_normal(n_e * n_p)
    wq = basis.node_weights(dim, order)
    h = np.array([[prob.extent[k] / (prob.base[k] * 2.0 ** l) for k in range(dim)] for l in range(8)])
    m = np.prod(h / 2.0, axis=1)[level][:, None] * wq[None, :]
    ref = float(np.sum(m.reshape(-1) * V))
    Vd = torch.tensor(V, dtype=torch.float64, device="cuda")
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):
        lev = torch.tensor(level, dtype=torch.int8, device="cuda")
        torch.cuda.synchronize()
        mdl.integral_noalloc(prob, Vd.data_ptr(), lev.data_ptr(), n_e, out.data_ptr(), 0)
        torch.cuda.synchronize()
        assert abs(out.item() - ref) <= 1e-12 * np.sum(np.abs(m.reshape(-1) * V)), (out.item(), ref)
    bad = level.copy()
    bad[17] = 8
    lev = torch.tensor(bad, dtype=torch.int8, device="cuda")
    torch.cuda.synchronize()
    mdl.integral_noalloc(prob, Vd.data_ptr(), lev.data_ptr(), n_e, out.data_ptr(), 0)
    torch.cuda.synchronize()
    assert np.isnan(out.item())


def test_integral_noalloc_captured_in_a_graph():
    """After a first call outside any capture, the call is captured into a CUDA graph on a side
    stream and replayed; each replay reads the field as it is then (no allocation in between)."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from oracle import basis
    from paper_2310_07607_gb300 import build, mdl
    build.build()
    prob = W.Problem(dim=2, order=1, extent=(0.4, 0.3, 1.0), base=(4, 3, 1), precision=64)
    rng = np.random.default_rng(12)
    n_e, n_p = 2000, 4
    level = rng.integers(0, 8, n_e).astype(np.int8)
    V = rng.standard_normal(n_e * n_p)
    wq = basis.node_weights(2, 1)
    h = np.array([[prob.extent[k] / (prob.base[k] * 2.0 ** l) for k in range(2)] for l in range(8)])
    m = (np.prod(h / 2.0, axis=1)[level][:, None] * wq[None, :]).reshape(-1)
    ref, scale = float(np.sum(m * V)), float(np.sum(np.abs(m * V)))
    Vd = torch.tensor(V, dtype=torch.float64, device="cuda")
    lev = torch.tensor(level, dtype=torch.int8, device="cuda")
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    mdl.integral_noalloc(prob, Vd.data_ptr(), lev.data_ptr(), n_e, out.data_ptr(), 0)
    torch.cuda.synchronize()
    assert abs(out.item() - ref) <= 1e-12 * scale
    side = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        mdl.integral_noalloc(prob, Vd.data_ptr(), lev.data_ptr(), n_e, out.data_ptr(), side.cuda_stream)
    for factor in (1.0, -2.5):
        Vd.copy_(torch.tensor(V * factor, dtype=torch.float64, device="cuda"))
        out.fill_(float("nan"))
        torch.cuda.synchronize()
        graph.replay()
        torch.cuda.synchronize()
        assert abs(out.item() - factor * ref) <= 1e-12 * abs(factor) * scale, (factor, out.item())
