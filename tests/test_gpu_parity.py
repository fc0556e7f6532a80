"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle.

Tolerances: FP64 builds 1e-12 relative (M-weighted L2), FP32 builds 1e-3
relative; activation times within one finest substep; every integer result
(face tables, levels, meshes, clocks) bit-exact.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import lts
from oracle.forest import Forest
from tests.helpers import forest_arrays, mass_rel_l2, oracle_face_table, random_forest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mdl():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2310_07607_gb300 import build, mdl as M
    build.build()
    return M


def lat_compare(a, b, tol):
    """Same activated set; activation times within tol."""
    fa, fb = np.isfinite(a), np.isfinite(b)
    assert np.array_equal(fa, fb), (fa.sum(), fb.sum(), np.nonzero(fa != fb)[0][:10])
    if fa.any():
        assert np.abs(a[fa] - b[fa]).max() <= tol


# --------------------------------------------------------------------------
# The plain FP64 global-step workload (32x32 Q1, 20 ms) in full.
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def plain_oracle():
    prob = W.plain_2d_q1_32x32()
    sim = lts.Sim(prob)
    sim.step_to(W.PLAIN_T_END)
    return sim


def test_plain_fp64_full_run_matches_oracle(mdl, plain_oracle):
    prob = W.plain_2d_q1_32x32()
    g = mdl.Sim(prob)
    g.step_to(W.PLAIN_T_END)
    t, nb, dt = g.time()
    assert nb == 2000 and dt == 0.01
    V = g.read_V()
    assert mass_rel_l2(plain_oracle.disc.M, V, plain_oracle.V) <= 1e-12
    s = g.read_state()
    assert np.abs(s - plain_oracle.v).max() <= 1e-11
    lat_compare(g.read_activation(), plain_oracle.lat, 1e-9)
    st = g.stats()
    assert st["dof_updates"] == 2000 * 4096
    assert abs(st["integral_V"] - np.sum(plain_oracle.disc.M * plain_oracle.V)) <= 1e-12 * abs(st["integral_V"])
    g.close()


def test_plain_fp32_run_matches_oracle_within_tolerance(mdl, plain_oracle):
    prob = W.plain_2d_q1_32x32().replace(precision=32)
    g = mdl.Sim(prob)
    for T in (5.0, 10.0, 15.0, W.PLAIN_T_END):
        g.step_to(T)
    V = g.read_V()
    assert mass_rel_l2(plain_oracle.disc.M, V, plain_oracle.V) <= 1e-3
    lat_compare(g.read_activation(), plain_oracle.lat, 0.01)
    g.close()


# --------------------------------------------------------------------------
# Integer work: face tables, ordering, levels, barrier length.
# --------------------------------------------------------------------------

@pytest.mark.parametrize("dim", [2, 3])
def test_face_table_bit_exact_after_upload(mdl, dim):
    f = random_forest(dim, (5, 4, 3), 3, (1.0, 0.8, 0.6), steps=3, seed=dim)
    prob = W.Problem(dim=dim, order=1, extent=(1.0, 0.8, 0.6), base=(5, 4, 3), max_refine=3,
                     ionic_model=-1, precision=64)
    g = mdl.Sim(prob)
    lv, cc, root = forest_arrays(f)
    perm = np.random.default_rng(0).permutation(f.n)      # any order in; canonical order out
    g.upload_mesh(lv[perm], cc[perm], root[perm])
    r2, l2, c2, _ = g.read_mesh()
    assert np.array_equal(l2, lv) and np.array_equal(c2, cc) and np.array_equal(r2, root)
    k, n, p = g.read_faces()
    ko, no, po = oracle_face_table(f)
    assert np.array_equal(k, ko) and np.array_equal(n, no) and np.array_equal(p, po)
    g.close()


@pytest.mark.parametrize("which", ["slab2d", "slab3d"])
def test_auto_barrier_step_bit_exact(mdl, which):
    prob = W.slab_2d_q1_256() if which == "slab2d" else W.slab_3d_q2()
    small = W.scaled(prob, (4, 4, 2)).replace(precision=64)
    g = mdl.Sim(small)
    o = lts.Sim(small)
    assert g.dt == o.dt
    g.close()


def test_levels_from_oracle_indicators_bit_exact(mdl):
    prob = W.scaled(W.slab_2d_q1_256(), (12, 12, 1)).replace(precision=64, amr_enabled=0,
                                                           dt_bar_cell=0.0, tau_cell=0.5)
    f = random_forest(2, (12, 12, 1), 3, prob.extent, steps=3, seed=11)
    o = lts.Sim(prob, forest=f)
    g = mdl.Sim(prob)
    lv, cc, root = forest_arrays(f)
    g.upload_mesh(lv, cc, root)
    rng = np.random.default_rng(3)
    eta_t = rng.uniform(0, 1, f.n)
    prob2 = prob.replace(dt_bar_cell=o.dt / 4.0)
    o2 = lts.Sim(prob2, forest=f)
    g2 = mdl.Sim(prob2)
    g2.upload_mesh(lv, cc, root)
    g2.set_indicators(eta_t=eta_t)
    g2.step_barriers(1)
    b = g2.read_mesh()[3]
    assert np.array_equal(b, o2.assign_levels(eta_t))
    # without the temporal indicator: pure CFL levels
    g.step_barriers(1)
    assert np.array_equal(g.read_mesh()[3], o.assign_levels(np.zeros(f.n)))
    g.close(); g2.close()


# --------------------------------------------------------------------------
# Multi-level LTS sweeps with hanging faces and time interpolation.
# --------------------------------------------------------------------------

def lts_case(mdl, dim, p, seed, nbar, precision, variant=None):
    prob = W.Problem(dim=dim, order=p, extent=(0.4, 0.3, 0.2), base=(4, 3, 2), sigma_l=1.2,
                     sigma_t=0.4, fibre=(0.6, 0.8, 0.0) if dim == 2 else (0.48, 0.64, 0.6),
                     gamma=10.0 * p * p, max_refine=2, n_lts_levels=3, lts_enabled=1,
                     dt_barrier=0.0, state_integrator=W.STATE_EXP, precision=precision,
                     stimuli=[W.Stimulus((0, 0, 0), (0.1, 0.1, 0.1), 1.0, 0.0, 1.0)])
    f = random_forest(dim, prob.base, 2, prob.extent, steps=2, seed=seed, tau=0.7)
    o = lts.Sim(prob, forest=f)
    X = o.disc.node_coords()
    V0, v0 = W.front_state(X, (0, 0, 0), 0.15, 0.02, tail=0.05)
    o.V, o.v = V0.copy(), v0.copy()
    o._lat_initial()
    g = mdl.Sim(prob)
    lv, cc, root = forest_arrays(f)
    g.upload_mesh(lv, cc, root)
    g.set_initial(V0, v0)
    if variant is not None:
        g.set_sweep_variant(variant)
    levels = []
    for n in range(nbar):
        lev = o.assign_levels(o.eta_t)
        levels.append(lev)
        o.eta_t = o.sweep(lev)
        o.barrier_count += 1
    g.step_barriers(nbar)
    return prob, o, g, levels


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_lts_hanging_fp64_matches_oracle(mdl, dim, p):
    prob, o, g, levels = lts_case(mdl, dim, p, seed=dim * 10 + p, nbar=3, precision=64)
    assert len(set(np.concatenate(levels).tolist())) >= 2
    assert np.array_equal(g.read_mesh()[3], levels[-1])
    assert mass_rel_l2(o.disc.M, g.read_V(), o.V) <= 1e-12
    assert np.abs(g.read_state() - o.v).max() <= 1e-11
    es, et = g.read_indicators()
    assert np.allclose(et, o.eta_t, rtol=1e-10, atol=1e-300)
    lat_compare(g.read_activation(), o.lat, 1e-9)
    g.close()


@pytest.mark.parametrize("dim,p", [(2, 1), (3, 1), (3, 2)])
def test_lts_hanging_fp32_matches_oracle(mdl, dim, p):
    prob, o, g, levels = lts_case(mdl, dim, p, seed=dim * 10 + p, nbar=3, precision=32)
    assert mass_rel_l2(o.disc.M, g.read_V(), o.V) <= 1e-3
    es, et = g.read_indicators()
    assert np.allclose(et, o.eta_t, rtol=2e-3, atol=1e-12 * et.max())
    # activation times within one finest substep of the barrier
    lat_compare(g.read_activation(), o.lat, o.dt / 2 ** (prob.n_lts_levels - 1))
    g.close()


@pytest.mark.parametrize("variant", ["group", "coop"])
@pytest.mark.parametrize("dim,p", [(2, 1), (3, 1), (3, 2)])
def test_sweep_variants_match_oracle_fp64(mdl, dim, p, variant):
    v = {"group": mdl.SWEEP_GROUP, "coop": mdl.SWEEP_COOP}[variant]
    prob, o, g, levels = lts_case(mdl, dim, p, seed=dim * 10 + p, nbar=3, precision=64, variant=v)
    assert mass_rel_l2(o.disc.M, g.read_V(), o.V) <= 1e-12
    assert np.abs(g.read_state() - o.v).max() <= 1e-11
    lat_compare(g.read_activation(), o.lat, 1e-9)
    g.close()


@pytest.mark.parametrize("dim", [2, 3])
def test_thread_and_coop_sweeps_identical(mdl, dim):
    out = []
    for v in (mdl.SWEEP_THREAD, mdl.SWEEP_COOP):
        prob, o, g, levels = lts_case(mdl, dim, 1, seed=dim, nbar=3, precision=32, variant=v)
        out.append((g.read_V(), g.read_state(), g.read_indicators()[1], g.read_activation()))
        g.close()
    # the same per-element arithmetic in two kernels: equal up to the multiply-add contraction
    # the compiler chooses in each (FP32 rounding), activation sets identical
    for a, b in zip(*out):
        fa, fb = np.isfinite(a), np.isfinite(b)
        assert np.array_equal(fa, fb)
        assert np.allclose(a[fa], b[fa], rtol=1e-5, atol=1e-12 * max(np.abs(a[fa]).max(), 1e-300))


# --------------------------------------------------------------------------
# Indicators and adaptation (replay protocol).
# --------------------------------------------------------------------------

@pytest.mark.parametrize("dim,p,precision", [(2, 1, 64), (2, 1, 32), (3, 1, 64), (3, 2, 64)])
def test_eta_s_matches_oracle(mdl, dim, p, precision):
    prob = W.Problem(dim=dim, order=p, extent=(0.4, 0.3, 0.2), base=(4, 3, 2), sigma_l=1.2,
                     sigma_t=0.4, fibre=(0.6, 0.8, 0.0) if dim == 2 else (0.48, 0.64, 0.6),
                     gamma=10.0 * p * p, max_refine=2, n_lts_levels=3, lts_enabled=1,
                     amr_enabled=1, tau_refine=1e30, tau_coarsen=-1.0, dt_barrier=0.0,
                     precision=precision)
    f = random_forest(dim, prob.base, 2, prob.extent, steps=2, seed=5, tau=0.7)
    o = lts.Sim(prob, forest=f)
    X = o.disc.node_coords()
    V0, v0 = W.front_state(X, (0, 0, 0), 0.15, 0.02, tail=0.05)
    g = mdl.Sim(prob)
    lv, cc, root = forest_arrays(f)
    g.upload_mesh(lv, cc, root)
    g.set_initial(V0, v0)
    g.step_barriers(1)                 # eta^s is computed on the barrier-start values
    es, _ = g.read_indicators()
    ref = o.disc.eta_s(V0)
    tol = 1e-10 if precision == 64 else 2e-3
    assert np.abs(es - ref).max() <= tol * ref.max()
    g.close()


@pytest.mark.parametrize("dim", [2, 3])
def test_adapt_replay_bit_exact_mesh_and_transfer(mdl, dim):
    prob = W.Problem(dim=dim, order=1, extent=(0.4, 0.3, 0.2), base=(4, 3, 2), max_refine=3,
                     n_lts_levels=4, lts_enabled=1, amr_enabled=1, tau_refine=0.8, tau_coarsen=0.2,
                     dt_barrier=0.0, precision=64, state_integrator=W.STATE_EXP)
    f = random_forest(dim, prob.base, 3, prob.extent, steps=2, seed=9, tau=0.7)
    o = lts.Sim(prob, forest=f)
    X = o.disc.node_coords()
    V0, v0 = W.front_state(X, (0, 0, 0), 0.15, 0.03, tail=0.05)
    o.V, o.v = V0.copy(), v0.copy()
    g = mdl.Sim(prob)
    lv, cc, root = forest_arrays(f)
    g.upload_mesh(lv, cc, root)
    g.set_initial(V0, v0)
    rng = np.random.default_rng(21)
    for step in range(3):
        eta = rng.uniform(0, 1, o.disc.ne)
        g.set_indicators(eta_s=eta)
        newf, plan = o.forest.adapt(eta, prob.tau_refine, prob.tau_coarsen)
        o.transfer(newf, plan)
        lev = o.assign_levels(o.eta_t)
        o.eta_t = o.sweep(lev)
        o.barrier_count += 1
        g.step_barriers(1)
        r2, l2, c2, b2 = g.read_mesh()
        lvo, cco, rto = forest_arrays(o.forest)
        assert np.array_equal(l2, lvo) and np.array_equal(c2, cco)
        assert np.array_equal(b2, lev)
        assert mass_rel_l2(o.disc.M, g.read_V(), o.V) <= 1e-12
    g.close()


# --------------------------------------------------------------------------
# Edge cases.
# --------------------------------------------------------------------------

def test_single_element_and_no_stimulus(mdl):
    prob = W.plain_2d_q1_32x32().replace(base=(1, 1, 1), extent=(0.05, 0.05, 1.0), stimuli=[])
    o = lts.Sim(prob)
    V0 = np.array([0.3, 0.31, 0.29, 0.3])
    o.V = V0.copy()
    o.step_to(1.0)
    g = mdl.Sim(prob)
    g.set_initial(V0)
    g.step_to(1.0)
    assert mass_rel_l2(o.disc.M, g.read_V(), o.V) <= 1e-12
    g.close()


def test_bad_calls_raise_and_leave_context_usable(mdl):
    prob = W.plain_2d_q1_32x32().replace(base=(4, 4, 1), extent=(0.125, 0.125, 1.0))
    g = mdl.Sim(prob)
    with pytest.raises(mdl.MdlError):
        g.set_initial(np.zeros(7))
    with pytest.raises(mdl.MdlError):
        g.set_levels(np.full(16, 3, np.int8))       # no LTS levels in a plain run
    with pytest.raises(mdl.MdlError):
        g.upload_mesh(np.zeros(3, np.int8), np.zeros((3, 2), np.int32))  # does not tile
    g.step_to(0.05)
    assert g.time()[1] == 5
    g.close()


def test_nonfinite_state_is_reported(mdl):
    prob = W.plain_2d_q1_32x32().replace(base=(4, 4, 1), extent=(0.125, 0.125, 1.0))
    g = mdl.Sim(prob)
    V = np.zeros(64)
    V[5] = np.nan
    g.set_initial(V)
    with pytest.raises(mdl.MdlError) as ei:
        g.step_barriers(2)
    assert ei.value.code == -5
    g.close()


@pytest.mark.parametrize("dim", [2, 3])
def test_coarsen_only_replay_bit_exact(mdl, dim):
    """No refine mark: the device's exact coarsenable-family count decides alone whether the
    host adapts; the resulting meshes must equal the oracle's."""
    prob = W.Problem(dim=dim, order=1, extent=(0.4, 0.3, 0.2), base=(4, 3, 2), max_refine=3,
                     n_lts_levels=4, lts_enabled=1, amr_enabled=1, tau_refine=0.8, tau_coarsen=0.2,
                     dt_barrier=0.0, precision=64, state_integrator=W.STATE_EXP)
    f = random_forest(dim, prob.base, 3, prob.extent, steps=3, seed=13, tau=0.6)
    o = lts.Sim(prob, forest=f)
    g = mdl.Sim(prob)
    lv, cc, root = forest_arrays(f)
    g.upload_mesh(lv, cc, root)
    rng = np.random.default_rng(4)
    for step in range(3):
        # below tau_refine everywhere; about half the leaves below tau_coarsen
        eta = rng.uniform(0.0, 0.4, o.disc.ne)
        if step == 2:
            eta[:] = 0.5            # nothing may change
        g.set_indicators(eta_s=eta)
        newf, plan = o.forest.adapt(eta, prob.tau_refine, prob.tau_coarsen)
        o.transfer(newf, plan)
        lev = o.assign_levels(o.eta_t)
        o.eta_t = o.sweep(lev)
        o.barrier_count += 1
        before = g.stats()["amr_rebuilds"]
        g.step_barriers(1)
        r2, l2, c2, b2 = g.read_mesh()
        lvo, cco, rto = forest_arrays(o.forest)
        assert np.array_equal(l2, lvo) and np.array_equal(c2, cco)
        changed = any(pl[0] != 'keep' for pl in plan)
        assert (g.stats()["amr_rebuilds"] - before) == (1 if changed else 0)
    g.close()


@pytest.mark.parametrize("dim,base,seed,tau", [(2, (3, 2, 1), 5, 0.75), (3, (2, 2, 1), 1, 0.7)])
def test_depth_seven_forest_faces_and_adapt_bit_exact(mdl, dim, base, seed, tau):
    """Leaves down to the deepest level (7): face tables after an upload and the meshes of two
    adaptations equal the oracle's (the device finds neighbours by a search over the leaves'
    sort keys, so a forest this deep must resolve neighbours across many levels of keys)."""
    prob = W.Problem(dim=dim, order=1, extent=(0.3, 0.2, 0.1), base=base, max_refine=7,
                     n_lts_levels=1, lts_enabled=0, amr_enabled=1, tau_refine=0.8, tau_coarsen=0.2,
                     dt_barrier=1e-4, precision=32, ionic_model=-1)
    f = random_forest(dim, base, 7, prob.extent, steps=7, seed=seed, tau=tau)
    assert max(lf[0] for lf in f.leaves) == 7
    g = mdl.Sim(prob)
    lv, cc, root = forest_arrays(f)
    g.upload_mesh(lv, cc, root)
    k, n, p = g.read_faces()
    ko, no, po = oracle_face_table(f)
    assert np.array_equal(k, ko) and np.array_equal(n, no) and np.array_equal(p, po)
    rng = np.random.default_rng(seed)
    for step in range(2):
        eta = rng.uniform(0, 1, f.n)
        g.set_indicators(eta_s=eta)
        f, _ = f.adapt(eta, prob.tau_refine, prob.tau_coarsen)
        g.step_barriers(1)
        r2, l2, c2, _ = g.read_mesh()
        lvo, cco, rto = forest_arrays(f)
        assert np.array_equal(l2, lvo) and np.array_equal(c2, cco) and np.array_equal(r2, rto)
    k, n, p = g.read_faces()
    ko, no, po = oracle_face_table(f)
    assert np.array_equal(k, ko) and np.array_equal(n, no) and np.array_equal(p, po)
    g.close()


def test_finest_grid_larger_than_a_dense_cell_map(mdl):
    """512 x 512 roots with 7 refinement levels: 4.3e9 finest cells, far more than a map of
    4 bytes per finest cell could hold; the context needs memory per leaf only.  The uniform
    root mesh has the closed-form face table of a Cartesian grid."""
    prob = W.Problem(dim=2, order=1, extent=(1.0, 1.0, 1.0), base=(512, 512, 1), max_refine=7,
                     n_lts_levels=1, lts_enabled=0, amr_enabled=1, tau_refine=0.8, tau_coarsen=0.2,
                     dt_barrier=1e-3, precision=32, ionic_model=-1)
    g = mdl.Sim(prob)
    k, n, _ = g.read_faces()
    nx = ny = 512
    e = np.arange(nx * ny)
    x, y = e % nx, e // nx
    want_k = np.ones((nx * ny, 4), np.int8)
    want_n = np.stack([e - 1, e + 1, e - nx, e + nx], axis=1).astype(np.int32)
    for f, edge in enumerate([x == 0, x == nx - 1, y == 0, y == ny - 1]):
        want_k[edge, f] = 0
        want_n[edge, f] = -1
    assert np.array_equal(k, want_k) and np.array_equal(n[:, :, 0], want_n)
    # refine the corner leaf at the origin down to the deepest level
    for step in range(7):
        g.set_indicators(eta_s=np.where(np.arange(g.sizes()[0]) == 0, 1.0, 0.5))
        g.step_barriers(1)
    r2, l2, c2, _ = g.read_mesh()
    assert l2.max() == 7 and l2[0] == 7 and np.array_equal(c2[0], [0, 0])
    g.close()


def test_full_size_slab2d_replay_matches_oracle(mdl):
    """The benchmark workload at full size (256x256 roots, AMR to depth 3, 4 LTS levels, FP32)
    from the synthetic developed front, in the benchmark's launch configuration, with the
    oracle's eta^s replayed: meshes and levels bit-exact, V within 1e-3, activation times
    within one finest substep; and the device's own eta^s within FP32 error of the oracle's."""
    prob = W.slab_2d_q1_256()
    o = lts.Sim(prob.replace(precision=64))
    X = o.disc.node_coords()
    V0, v0 = W.front_state(X, (0.0, 0.0, 0.0), 1.0, 0.01, 0.3)
    o.V, o.v = V0.copy(), v0.copy()
    o._lat_initial()
    g = mdl.Sim(prob)
    g.set_initial(V0, v0)
    assert g.dt == o.dt
    for n in range(4):
        es = o.disc.eta_s(o.V)
        g.set_indicators(eta_s=es)
        newf, plan = o.forest.adapt(es, prob.tau_refine, prob.tau_coarsen)
        o.transfer(newf, plan)
        lev = o.assign_levels(o.eta_t)
        o.eta_t = o.sweep(lev)
        o.barrier_count += 1
        g.step_barriers(1)
        r2, l2, c2, b2 = g.read_mesh()
        lvo, cco, rto = forest_arrays(o.forest)
        assert np.array_equal(l2, lvo) and np.array_equal(c2, cco)
        assert np.array_equal(b2, lev)
        assert mass_rel_l2(o.disc.M, g.read_V(), o.V) <= 1e-3
    assert o.disc.ne > 100000 and len(set(lev.tolist())) >= 3
    lat_compare(g.read_activation(), o.lat, o.dt / 8)
    # free-running indicator: the device's own eta^s on the current state
    es_o = o.disc.eta_s(o.V)
    g.step_barriers(1)
    es_g, _ = g.read_indicators()
    es_g = es_g[:es_o.size]       # eta^s lives on the mesh before this barrier's adaptation
    big = es_o > 1e-3 * es_o.max()
    assert np.abs(es_g[big] - es_o[big]).max() <= 5e-3 * es_o.max()
    g.close()


def test_long_horizon_fp32_amr_lts_replay_matches_oracle(mdl):
    """FP32 AMR + 4 LTS levels on an 8x8-root patch of the 2D slab (the slab's h, physics and
    thresholds; the developed front scaled to the patch) over 4096 barrier steps (0.25 ms),
    with the oracle's eta^s replayed every barrier: meshes and levels bit-exact, V within
    1e-3 (M-weighted) at every checkpoint, the same probes activated, and activation times
    within the FP32 crossing-time tolerance, including the probes the front reaches after
    t = 0.  That tolerance is max(one finest substep, 4e-5 ms): the finest substep here is
    7.6e-6 ms, below what FP32 resolves -- V drifts from the FP64 oracle by ~1e-5..4e-5 at
    the front over 10^3..10^4 steps, and divided by the upstroke slope (dV/dt ~ 1..3 per ms)
    that moves a threshold crossing by ~1e-5 ms."""
    prob = W.scaled(W.slab_2d_q1_256(), (8, 8, 1))
    o = lts.Sim(prob.replace(precision=64))
    X = o.disc.node_coords()
    r = 1.0 * 8 / 256
    V0, v0 = W.front_state(X, (0.0, 0.0, 0.0), r, 0.01, 0.3 * r)
    o.V, o.v = V0.copy(), v0.copy()
    o._lat_initial()
    initially = np.isfinite(o.lat).copy()
    g = mdl.Sim(prob)
    g.set_initial(V0, v0)
    assert g.dt == o.dt
    fine = max(o.dt / 8, 4e-5)
    n_bar, checks, rebuilds = 4096, 0, 0
    for n in range(n_bar):
        es = o.disc.eta_s(o.V)
        g.set_indicators(eta_s=es)
        newf, plan = o.forest.adapt(es, prob.tau_refine, prob.tau_coarsen)
        if any(pl[0] != 'keep' for pl in plan) or newf.n != o.forest.n:
            o.transfer(newf, plan)
            rebuilds += 1
        lev = o.assign_levels(o.eta_t)
        o.eta_t = o.sweep(lev)
        o.barrier_count += 1
        g.step_barriers(1)
        if (n + 1) % 512 == 0:
            r2, l2, c2, b2 = g.read_mesh()
            lvo, cco, rto = forest_arrays(o.forest)
            assert np.array_equal(l2, lvo) and np.array_equal(c2, cco), n
            assert np.array_equal(b2, lev), n
            rel = mass_rel_l2(o.disc.M, g.read_V(), o.V)
            la = g.read_activation()
            both = np.isfinite(la) & np.isfinite(o.lat)
            print("barrier %d: V rel %.2e, LAT max diff %.2e ms over %d probes"
                  % (n + 1, rel, np.abs(la[both] - o.lat[both]).max() if both.any() else 0.0, both.sum()))
            assert rel <= 1e-3, (n, rel)
            lat_compare(la, o.lat, fine)
            checks += 1
    assert checks == 8 and rebuilds >= 10 and len(set(lev.tolist())) >= 3
    crossed = np.isfinite(o.lat) & ~initially
    assert crossed.sum() >= 8, crossed.sum()
    assert np.all(o.lat[crossed] > 0.0)
    g.close()


# --------------------------------------------------------------------------
# Temporal adaptivity: the cell-model substep b^cell (Eq. num-substeps) set free-running
# from the element's own temporal indicator, on the spiral-wave workload (broken wave).
# --------------------------------------------------------------------------

def spiral_case(mdl, precision):
    prob = W.spiral_2d_q1(12).replace(precision=precision)
    o = lts.Sim(prob)
    X = o.disc.node_coords()
    V0, v0 = W.spiral_state(X, prob.extent[0])
    o.V, o.v = V0.copy(), v0.copy()
    o._lat_initial()
    g = mdl.Sim(prob)
    g.set_initial(V0, v0)
    bcfl = np.array([lts.b_from_bound(o.dt, c) for c in o.cfl()])
    return prob, o, g, bcfl


def test_spiral_cell_substeps_fp64_free_running(mdl):
    """FP64: levels (b^CFL and b^cell from the GPU's own eta^t) bit-exact every barrier,
    b^cell raising some elements above their CFL level, V and eta^t at 1e-12 / 1e-10."""
    prob, o, g, bcfl = spiral_case(mdl, 64)
    raised = 0
    for n in range(6):
        lev = o.assign_levels(o.eta_t)
        raised += int(np.sum(lev > bcfl))
        o.eta_t = o.sweep(lev)
        o.barrier_count += 1
        g.step_barriers(1)
        assert np.array_equal(g.read_mesh()[3], lev), n
    assert raised > 0
    assert mass_rel_l2(o.disc.M, g.read_V(), o.V) <= 1e-12
    assert np.allclose(g.read_indicators()[1], o.eta_t, rtol=1e-10, atol=1e-300)
    lat_compare(g.read_activation(), o.lat, 1e-9)
    g.close()


def test_spiral_cell_substeps_fp32_replay(mdl):
    """FP32 with the oracle's levels replayed each barrier: V within 1e-3."""
    prob, o, g, bcfl = spiral_case(mdl, 32)
    for n in range(6):
        lev = o.assign_levels(o.eta_t)
        o.eta_t = o.sweep(lev)
        o.barrier_count += 1
        g.set_levels(lev.astype(np.int8))
        g.step_barriers(1)
    assert mass_rel_l2(o.disc.M, g.read_V(), o.V) <= 1e-3
    g.close()


def test_fp32_field_transfers_match_fp64_calls(mdl):
    """set_initial_f32 / read_fields_f32 against the FP64 calls on an FP32 context: the same
    stored values (FP32 either way), bit for bit, also after a step."""
    prob = W.slab_2d_q1_256().replace(base=(24, 20, 1), extent=(24 * 2.0 / 256, 20 * 2.0 / 256, 1.0))
    a, b = mdl.Sim(prob), mdl.Sim(prob)
    X = lts.Sim(prob.replace(amr_enabled=0)).disc.node_coords()   # base grid, leaf order
    V, s = W.front_state(X, (0, 0, 0), 0.1, 0.01, tail=0.3)
    assert V.size == a.sizes()[1]
    a.set_initial(V, s)
    b.set_initial_f32(V.astype(np.float32), s.astype(np.float32))
    for sim_steps in (0, 2):
        a.step_barriers(sim_steps)
        b.step_barriers(sim_steps)
        Vb, sb = b.read_fields_f32()
        assert np.array_equal(a.read_V(), Vb.astype(np.float64))
        assert np.array_equal(a.read_state(), sb.astype(np.float64))
    a.close(); b.close()


def test_fp32_field_transfers_through_pinned_buffers(mdl):
    """Page-locked host buffers are read and written by the layout kernels directly (no staging
    copy): the same stored and returned values as with ordinary host arrays, bit for bit, on
    the padded Q2 3D rows and on Q1 2D; 81 values (a partial group of four at the end) too."""
    import torch
    for prob in (W.scaled(W.slab_3d_q2(), (3, 2, 2)).replace(amr_enabled=0, max_refine=0),
                 W.scaled(W.slab_3d_q2(), (3, 1, 1)).replace(amr_enabled=0, max_refine=0),
                 W.slab_2d_q1_256().replace(base=(12, 10, 1), extent=(12 * 2.0 / 256, 10 * 2.0 / 256, 1.0),
                                            amr_enabled=0, max_refine=0)):
        a, b = mdl.Sim(prob), mdl.Sim(prob)
        n = a.sizes()[1]
        rng = np.random.default_rng(8)
        V = rng.uniform(0, 1, n).astype(np.float32)
        s = rng.uniform(0, 0.5, n).astype(np.float32)
        pin = [torch.empty(n, dtype=torch.float32, pin_memory=True).numpy() for _ in range(4)]
        pin[0][:] = V
        pin[1][:] = s
        a.set_initial_f32(V, s)
        b.set_initial_f32(pin[0], pin[1])
        for steps in (0, 2):
            a.step_barriers(steps)
            b.step_barriers(steps)
            Va, sa = a.read_fields_f32()
            b.read_fields_f32(pin[2], pin[3])
            assert np.array_equal(Va, pin[2]) and np.array_equal(sa, pin[3])
        assert np.array_equal(a.read_V(), b.read_V())
        a.close(); b.close()
