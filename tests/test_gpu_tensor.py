"""GPU parity of the tensor-core (tcgen05) Q2 3D FP32 sweep.

The tensor-core sweep computes the SIPG residual of elements whose faces all have
same-level neighbours as one tensor-core product per tile of 64 due elements: the gathered
element and face-neighbour values, shifted by the element mean and split into two FP16
terms, times the level-0 operator, also split into two FP16 terms, with FP32 accumulation
in tensor memory; other faces are added on the CUDA cores.  It is compared with the FP64
oracle (relative M-weighted L2 error of V at most 1e-3, as every FP32 result; activation
times within one finest substep) and with the CUDA-core FP32 sweep on the same inputs, on
meshes that span several tiles with a ragged last tile, with hanging faces, boundary faces,
multi-level LTS with time interpolation, an anisotropic fibre direction, and with the
persistent blocks capped so that each block walks many tiles.
"""
import numpy as np
import pytest

import workloads as W
from oracle import lts
from oracle.forest import Forest
from tests.helpers import forest_arrays, mass_rel_l2, random_forest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mdl():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2310_07607_gb300 import build, mdl as M
    build.build()
    return M


def q2_problem(base, extent, fibre, sigma=(1.2, 0.3), max_refine=2, n_lts=3, stim_hi=(0.1, 0.1, 0.1)):
    return W.Problem(dim=3, order=2, extent=extent, base=base, sigma_l=sigma[0], sigma_t=sigma[1], fibre=fibre,
                     gamma=40.0, max_refine=max_refine, n_lts_levels=n_lts, lts_enabled=1, dt_barrier=0.0,
                     state_integrator=W.STATE_EXP, precision=32,
                     stimuli=[W.Stimulus((0, 0, 0), stim_hi, 1.0, 0.0, 1.0)])


def run_pair(mdl, prob, forest, nbar, origin=(0, 0, 0), radius=0.15, width=0.02, blocks=0):
    """Oracle, CUDA-core FP32 sweep and tensor-core sweep over nbar barriers (levels from
    the oracle's own indicators each barrier, mesh fixed)."""
    o = lts.Sim(prob, forest=forest)
    X = o.disc.node_coords()
    V0, v0 = W.front_state(X, origin, radius, width, tail=0.05)
    o.V, o.v = V0.copy(), v0.copy()
    o._lat_initial()
    lv, cc, root = forest_arrays(forest)
    sims = []
    for variant in (mdl.SWEEP_THREAD, mdl.SWEEP_TENSOR):
        g = mdl.Sim(prob)
        g.upload_mesh(lv, cc, root)
        g.set_initial(V0, v0)
        g.set_sweep_variant(variant)
        if variant == mdl.SWEEP_TENSOR and blocks:
            g.set_sweep_blocks(blocks)
        sims.append(g)
    levels = []
    for _ in range(nbar):
        lev = o.assign_levels(o.eta_t)
        levels.append(lev)
        o.eta_t = o.sweep(lev)
        o.barrier_count += 1
    for g in sims:
        g.step_barriers(nbar)
    return o, sims[0], sims[1], levels


def eta_rel(a, ref, floor):
    """Largest relative difference of a and ref over entries above floor."""
    big = np.abs(ref) > floor
    return float(np.max(np.abs(a[big] - ref[big]) / np.abs(ref[big]))) if big.any() else 0.0


def check(o, gt, gx, levels, tol_pair=1e-4):
    M = o.disc.M
    Vt, Vx = gt.read_V(), gx.read_V()
    rel_o, rel_t = mass_rel_l2(M, Vx, o.V), mass_rel_l2(M, Vx, Vt)
    et_t = gt.read_indicators()[1]
    et_x = gx.read_indicators()[1]
    floor = 1e-12 * o.eta_t.max()
    err_t, err_x = eta_rel(et_t, o.eta_t, floor), eta_rel(et_x, o.eta_t, floor)
    print("V rel: tensor-oracle %.2e tensor-thread %.2e; eta_t rel: thread %.2e tensor %.2e"
          % (rel_o, rel_t, err_t, err_x))
    assert rel_o <= 1e-3
    assert rel_t <= tol_pair
    assert np.array_equal(gx.read_mesh()[3], levels[-1])
    st = gx.read_state()
    assert np.abs(st - o.v).max() <= 1e-3 * max(np.abs(o.v).max(), 1e-3)
    # the FP32 CUDA-core sweep itself reaches ~4e-3 on the refined patch
    assert err_x <= max(2e-3, 2.0 * err_t), (err_x, err_t)
    # activation times: the same activated probes, times within one finest substep
    la, lo = gx.read_activation(), o.lat
    fa, fo = np.isfinite(la), np.isfinite(lo)
    assert np.array_equal(fa, fo), (fa.sum(), fo.sum())
    if fa.any():
        assert np.abs(la[fa] - lo[fa]).max() <= o.dt / 2 ** (o.prob.n_lts_levels - 1)


def test_tensor_uniform_mesh_two_tiles(mdl):
    """240 elements (tiles of 128 and 112), fibre along x as in the 3D slab, 3 LTS levels
    from the CFL classes (boundary faces set the finer classes)."""
    base = (8, 6, 5)
    h = 2.0 / 128
    prob = q2_problem(base, (base[0] * h, base[1] * h, base[2] * h), (1.0, 0.0, 0.0), max_refine=0, n_lts=2,
                      stim_hi=(2 * h, base[1] * h, base[2] * h))
    f = Forest(3, base, 0, prob.extent)
    o, gt, gx, levels = run_pair(mdl, prob, f, 6, origin=(0, 0, 0), radius=3 * h, width=h)
    check(o, gt, gx, levels)
    gt.close(); gx.close()


@pytest.mark.parametrize("seed", [32, 7])
def test_tensor_hanging_lts_anisotropic(mdl, seed):
    """Random 2:1 forest (hanging faces on both sides), 3 LTS levels with interpolated
    coarser neighbours, fibre off every axis."""
    base = (4, 3, 2)
    prob = q2_problem(base, (0.4, 0.3, 0.2), (0.48, 0.64, 0.6), sigma=(1.2, 0.4))
    f = random_forest(3, base, 2, prob.extent, steps=2, seed=seed, tau=0.7)
    o, gt, gx, levels = run_pair(mdl, prob, f, 3)
    assert len(set(np.concatenate(levels).tolist())) >= 2
    check(o, gt, gx, levels)
    gt.close(); gx.close()


def test_tensor_many_tiles_refined_patch(mdl):
    """A refined patch inside a 10x8x4 base (several tiles, most elements regular)."""
    base = (10, 8, 4)
    h = 2.0 / 128
    prob = q2_problem(base, (base[0] * h, base[1] * h, base[2] * h), (1.0, 0.0, 0.0), max_refine=1, n_lts=3)
    f = Forest(3, base, 1, prob.extent)
    eta = np.zeros(f.n)
    X = np.array([[(lf[1][k] + 0.5) * h for k in range(3)] for lf in f.leaves])
    eta[(X[:, 0] > 3 * h) & (X[:, 0] < 7 * h)] = 1.0
    f, _ = f.adapt(eta, 0.5, -1.0)
    assert f.n > 3 * 128
    o, gt, gx, levels = run_pair(mdl, prob, f, 4, origin=(5 * h, 0, 0), radius=2 * h, width=h)
    check(o, gt, gx, levels)
    gt.close(); gx.close()


@pytest.mark.parametrize("blocks", [1, 3])
def test_tensor_few_blocks_walk_many_tiles(mdl, blocks):
    """The refined patch with the persistent sweep capped at `blocks` thread blocks, so that
    every block walks many tiles of 64 due elements back to back (metadata and operands of
    the next tile staged while the current one is computed): V, v, eta^t and activation
    times against the oracle, 6 barrier steps with levels from the oracle's indicators."""
    base = (10, 8, 4)
    h = 2.0 / 128
    prob = q2_problem(base, (base[0] * h, base[1] * h, base[2] * h), (1.0, 0.0, 0.0), max_refine=1, n_lts=3)
    f = Forest(3, base, 1, prob.extent)
    eta = np.zeros(f.n)
    X = np.array([[(lf[1][k] + 0.5) * h for k in range(3)] for lf in f.leaves])
    eta[(X[:, 0] > 3 * h) & (X[:, 0] < 7 * h)] = 1.0
    f, _ = f.adapt(eta, 0.5, -1.0)
    assert f.n >= 12 * 64
    o, gt, gx, levels = run_pair(mdl, prob, f, 6, origin=(5 * h, 0, 0), radius=2 * h, width=h, blocks=blocks)
    check(o, gt, gx, levels)
    gt.close(); gx.close()


def test_tensor_variant_rejected_elsewhere(mdl):
    for dim, p, prec in ((2, 2, 32), (3, 1, 32), (3, 2, 64)):
        prob = W.Problem(dim=dim, order=p, extent=(0.4, 0.3, 0.2), base=(4, 3, 2), precision=prec,
                         stimuli=[])
        g = mdl.Sim(prob)
        with pytest.raises(mdl.MdlError):
            g.set_sweep_variant(mdl.SWEEP_TENSOR)
        g.step_barriers(1)
        g.close()


def test_full_size_slab3d_tensor_matches_thread(mdl):
    """The 3D slab at full size (128x48x20 roots, AMR to depth 3, 4 LTS levels, 2.7M
    elements), in the benchmark's launch configuration: from one state on one refined mesh,
    one barrier step with the tensor-core sweep and one with the thread-per-element CUDA-core
    sweep (an independent evaluation of the same SIPG residual) agree to FP32 rounding in V,
    the state and eta^t, with identical meshes, levels and activation sets.  (The oracle is
    checked against both on small meshes; at this size it cannot run.)"""
    import bench as B
    prob = W.slab_3d_q2()
    a = mdl.Sim(prob)
    a.set_sweep_variant(mdl.SWEEP_THREAD)
    X = B.node_coords_of(a, prob)
    V0, v0 = W.planar_front_state(X, B.PLANAR["x0"], B.PLANAR["width"], B.PLANAR["tail"])
    a.set_initial(V0, v0)
    a.step_barriers(4)                      # AMR refines the front to depth 3
    root, level, coords, _ = a.read_mesh()
    V1, s1 = a.read_V(), a.read_state()
    assert level.max() == 3 and level.size > 2_000_000
    b = mdl.Sim(prob)
    b.set_sweep_variant(mdl.SWEEP_TENSOR)
    b.upload_mesh(level, coords.reshape(-1), root)
    b.set_initial(V1, s1)
    a.upload_mesh(level, coords.reshape(-1), root)
    a.set_initial(V1, s1)
    a.step_barriers(1)
    b.step_barriers(1)
    ma, mb = a.read_mesh(), b.read_mesh()
    for x, y in zip(ma, mb):
        assert np.array_equal(x, y)
    assert len(set(mb[3].tolist())) >= 3
    Va, Vb = a.read_V(), b.read_V()
    rel = np.linalg.norm(Vb - Va) / np.linalg.norm(Va)
    assert rel <= 1e-5, rel
    sa, sb = a.read_state(), b.read_state()
    assert np.linalg.norm(sb - sa) <= 1e-5 * np.linalg.norm(sa)
    ea, eb = a.read_indicators()[1], b.read_indicators()[1]
    big = ea > 1e-6 * ea.max()
    assert np.max(np.abs(eb[big] - ea[big]) / ea[big]) <= 1e-2
    la, lb = a.read_activation(), b.read_activation()
    assert np.array_equal(np.isfinite(la), np.isfinite(lb))
    a.close(); b.close()


def test_full_size_slab3d_tensor_conserves_integral_pure_diffusion(mdl):
    """A property that holds at any size, checked on the full 3D slab mesh (2.7M elements
    after the AMR reaches depth 3, hanging and boundary faces, the tensor-core sweep and its
    correction blocks): without ionic current and stimulus, a global forward Euler step
    changes int V = sum_q M_q V_q by -dt 1^T A u, and 1^T A = 0 for the symmetric SIPG
    operator with zero-flux boundaries.  In FP32 the residual of int V after 20 steps is set
    by the per-(level, node) rounding of M_q M_q^-1 (~1e-7) and by unbiased roundings, far
    below 1e-3 of the mass-weighted change of V; a dropped or doubled face term leaves the
    flux it carries, of the order of that change."""
    import bench as B
    prob = W.slab_3d_q2()
    a = mdl.Sim(prob)
    X = B.node_coords_of(a, prob)
    V0, v0 = W.planar_front_state(X, B.PLANAR["x0"], B.PLANAR["width"], B.PLANAR["tail"])
    a.set_initial(V0, v0)
    a.step_barriers(4)                      # AMR refines the front to depth 3
    root, level, coords, _ = a.read_mesh()
    V1, s1 = a.read_V(), a.read_state()
    a.close()
    assert level.max() == 3 and level.size > 2_000_000
    diff = prob.replace(ionic_model=-1, stimuli=[], amr_enabled=0, lts_enabled=0, n_lts_levels=1,
                        dt_barrier=0.0)
    g = mdl.Sim(diff)
    g.upload_mesh(level, coords.reshape(-1), root)
    g.set_initial(V1, s1)
    # int V of the uploaded FP32 state: M_q = prod_k (h_k / 2) w_{a_k}, h_k = extent_k / (base_k 2^l)
    w = np.array([5.0, 8.0, 5.0]) / 9.0
    wq = (w[None, None, :] * w[None, :, None] * w[:, None, None]).reshape(-1)
    h = np.array(diff.extent)[None, :] / (np.array(diff.base)[None, :] * (2.0 ** level.astype(np.float64))[:, None])
    Mq = np.prod(h / 2.0, axis=1)[:, None] * wq[None, :]
    I0 = float(np.sum(Mq * V1.reshape(level.size, 27)))
    g.step_barriers(20)
    I1 = g.stats()["integral_V"]
    Vn = g.read_V()
    g.close()
    change = float(np.sum(Mq * np.abs(Vn - V1).reshape(level.size, 27)))
    assert change > 0.0
    assert abs(I1 - I0) <= 1e-3 * change, (I0, I1, change)
