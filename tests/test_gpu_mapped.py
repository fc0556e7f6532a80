"""GPU parity on curved (mapped) meshes: the thread-per-element sweep with per-point geometric
factors against the FP64 oracle's mapped operator (oracle/mapped.py), on ellipsoidal shell
sectors whose elements differ in size (so the per-element CFL bounds give several LTS levels)
with circumferential fibres, and on a sheared affine mesh.  FP64 to 1e-12 (M-weighted V),
LTS levels and activated probes identical; FP32 within the 1e-3 tolerance, activation times
within one finest substep."""
import numpy as np
import pytest

import workloads as W
from oracle import lts
from tests.helpers import mass_rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mdl():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2310_07607_gb300 import build, mdl as M
    build.build()
    return M


def shell_problem(dim, p, precision, base=None):
    """A thin ellipsoidal shell sector: azimuth 0.2 .. 0.3 rad, polar angle 1.52 .. 1.62 rad
    (3D), inner semi-axes (0.5, 0.45, 0.8) cm, outer (0.8, 0.75, 1.1) cm, so that elements at
    the outer surface are 1.6x wider than at the inner one and their CFL bounds differ by more
    than 2 (several LTS levels); fibres along the azimuth; a stimulus on the low-azimuth end."""
    if base is None:
        base = (6, 4, 1) if dim == 2 else (6, 4, 2)
    geo = (0.5, 0.45, 0.8, 0.8, 0.75, 1.1, 0.2, 0.1, 1.52, 0.1)
    stim = W.Stimulus((-3.0, -3.0, -3.0), (3.0, 0.115, 3.0), 1.0, 0.0, 1.0)
    return W.Problem(dim=dim, order=p, extent=(1.0, 1.0, 1.0), base=base, sigma_l=1.2, sigma_t=0.4,
                     fibre=(1.0, 0.0, 0.0), gamma=10.0 * p * p, geometry=W.GEOMETRY_SHELL, geo=geo,
                     fibre_ref=1, n_lts_levels=4, lts_enabled=1, dt_barrier=0.0,
                     state_integrator=W.STATE_EXP, precision=precision, stimuli=[stim])


def run_pair(mdl, prob, nbar, V0=None, v0=None):
    o = lts.Sim(prob)
    if V0 is not None:
        o.V, o.v = V0.copy(), v0.copy()
        o._lat_initial()
    g = mdl.Sim(prob)
    if V0 is not None:
        g.set_initial(V0, v0)
    assert g.dt == o.dt
    levels = []
    for _ in range(nbar):
        o.barrier()
        levels.append(o.levels.copy())
    g.step_barriers(nbar)
    return o, g, levels


def front(o, prob):
    X = o.disc.node_coords()
    return W.front_state(X, (0.5, 0.1, 0.0), 0.12, 0.01, tail=0.05)


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_shell_fp64_matches_oracle(mdl, dim, p):
    prob = shell_problem(dim, p, 64)
    o0 = lts.Sim(prob)
    V0, v0 = front(o0, prob)
    o, g, levels = run_pair(mdl, prob, int(2.0 / lts.Sim(prob).dt), V0, v0)   # 2 ms
    if (dim, p) != (3, 2):
        assert len(set(np.concatenate(levels).tolist())) >= 2      # several LTS levels
    assert (np.isfinite(o.lat) & (o.lat > 0)).any()                # probes crossed during the run
    assert np.array_equal(g.read_mesh()[3], levels[-1])
    assert mass_rel_l2(o.disc.M, g.read_V(), o.V) <= 1e-12
    assert np.abs(g.read_state() - o.v).max() <= 1e-11
    es, et = g.read_indicators()
    assert np.allclose(et, o.eta_t, rtol=1e-10, atol=1e-300)
    la, lo = g.read_activation(), o.lat
    assert np.array_equal(np.isfinite(la), np.isfinite(lo))
    if np.isfinite(lo).any():
        assert np.abs(la[np.isfinite(lo)] - lo[np.isfinite(lo)]).max() <= 1e-9
    st = g.stats()
    assert abs(st["integral_V"] - o.disc.M @ o.V) <= 1e-12 * abs(o.disc.M @ o.V)
    g.close()


@pytest.mark.parametrize("dim,p", [(2, 1), (3, 1), (3, 2)])
def test_shell_fp32_matches_oracle_within_tolerance(mdl, dim, p):
    prob = shell_problem(dim, p, 32)
    o = lts.Sim(prob.replace(precision=64))
    V0, v0 = front(o, prob)
    o.V, o.v = V0.copy(), v0.copy()
    o._lat_initial()
    g = mdl.Sim(prob)
    g.set_initial(V0, v0)
    nbar = int(2.0 / o.dt)        # 2 ms
    for _ in range(nbar):
        o.barrier()
    g.step_barriers(nbar)
    assert mass_rel_l2(o.disc.M, g.read_V(), o.V) <= 1e-3
    la, lo = g.read_activation(), o.lat
    assert np.array_equal(np.isfinite(la), np.isfinite(lo))
    if np.isfinite(lo).any():
        assert np.abs(la[np.isfinite(lo)] - lo[np.isfinite(lo)]).max() <= o.dt / 2 ** (prob.n_lts_levels - 1)
    g.close()


@pytest.mark.parametrize("dim,p", [(2, 2), (3, 1)])
def test_sheared_affine_mesh_fp64_matches_oracle(mdl, dim, p):
    A = (1.3, 0.4, -0.2, 0.1, 0.9, 0.3, 0.25, -0.15, 1.1)
    prob = W.Problem(dim=dim, order=p, extent=(0.4, 0.3, 0.2), base=(5, 4, 3), sigma_l=1.2, sigma_t=0.4,
                     fibre=(0.6, 0.8, 0.0) if dim == 2 else (0.48, 0.64, 0.6), gamma=10.0 * p * p,
                     geometry=W.GEOMETRY_AFFINE, geo=A + (0.05, 0.1, -0.2), n_lts_levels=2, lts_enabled=1,
                     dt_barrier=0.0, state_integrator=W.STATE_FE, precision=64,
                     stimuli=[W.Stimulus((-1.0, -1.0, -1.0), (0.15, 0.1, 1.0), 1.0, 0.0, 1.0)])
    o, g, _ = run_pair(mdl, prob, 30)
    assert mass_rel_l2(o.disc.M, g.read_V(), o.V) <= 1e-12
    assert np.abs(g.read_state() - o.v).max() <= 1e-11
    g.close()


def test_mapped_geometry_rejects_what_it_does_not_support(mdl):
    prob = shell_problem(2, 1, 32)
    with pytest.raises(mdl.MdlError):
        mdl.Sim(prob.replace(amr_enabled=1, max_refine=1))
    with pytest.raises(mdl.MdlError):
        mdl.Sim(prob.replace(geo=(0.5, 0.45, 0.8, 0.4, 0.75, 1.1, 0.2, 0.1, 1.52, 0.1)))   # a shrinks, b grows
    with pytest.raises(mdl.MdlError):
        mdl.Sim(prob.replace(dim=3, base=(3, 2, 2), geo=(0.5, 0.45, 0.8, 0.8, 0.75, 1.1, 0.2, 0.1, 3.0, 0.5)))
    g = mdl.Sim(prob)
    with pytest.raises(mdl.MdlError):
        g.set_sweep_variant(mdl.SWEEP_GROUP)
    with pytest.raises(mdl.MdlError):
        g.upload_mesh(np.zeros(24, np.int8), np.zeros((24, 2), np.int32))
    g.step_barriers(2)                                   # still usable
    assert g.time()[1] == 2
    g.close()


def test_mapped_slots_in_a_fused_batch_give_their_alone_values(mdl):
    """A mapped slot in a fused batch sweeps on its own (the fused kernel has box elements
    only), so it gives the bits it gives alone; the box slots beside it are unaffected."""
    shell = shell_problem(3, 1, 32)
    box = W.Problem(dim=2, order=1, extent=(0.4, 0.3, 1.0), base=(8, 6, 1), sigma_l=1.2, sigma_t=0.4,
                    fibre=(0.6, 0.8, 0.0), gamma=10.0, n_lts_levels=2, lts_enabled=1, dt_barrier=0.0,
                    state_integrator=W.STATE_EXP, precision=32,
                    stimuli=[W.Stimulus((0, 0, 0), (0.1, 0.1, 1.0), 1.0, 0.0, 1.0)])
    nbar = 6
    alone = mdl.Sim(shell)
    alone.step_barriers(nbar)
    Va = alone.read_V()
    alone.close()
    b = mdl.Batch(autotune=False, fused=True)
    s1 = b.admit(shell, nbar * mdl.Sim(shell).dt)
    s2 = b.admit(box, nbar * mdl.Sim(box).dt)
    while b.step(barriers_per_slot=3) > 0:
        pass
    g, state, rc = b.slot(s1)
    assert state == mdl.SLOT_DONE and rc == 0
    assert np.array_equal(g.read_V(), Va)
    assert b.slot(s2)[1] == mdl.SLOT_DONE
    b.close()


@pytest.mark.parametrize("dim,p,precision", [(2, 1, 64), (2, 2, 64), (3, 1, 64), (3, 2, 64), (3, 1, 32), (3, 2, 32)])
def test_shell_kelly_indicator_matches_oracle(mdl, dim, p, precision):
    """The spatial indicator on the mapped mesh, computed at the start of every barrier step:
    after n steps it holds the indicator of the state n - 1 steps in (FP64 to 1e-10, FP32 with
    FP64 face accumulation to 2e-3 of the largest value)."""
    prob = shell_problem(dim, p, precision)
    o = lts.Sim(prob.replace(precision=64))
    V0, v0 = front(o, prob)
    o.V, o.v = V0.copy(), v0.copy()
    o._lat_initial()
    g = mdl.Sim(prob)
    g.set_initial(V0, v0)
    nbar = 5
    for _ in range(nbar - 1):
        o.barrier()
    want = o.disc.eta_s(o.V)
    o.barrier()
    g.step_barriers(nbar)
    es, _ = g.read_indicators()
    assert want.max() > 0
    if precision == 64:
        assert np.allclose(es, want, rtol=1e-10, atol=1e-14 * want.max())
    else:
        assert np.abs(es - want).max() <= 2e-3 * want.max()
    g.close()


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_shell_adaptation_replay_matches_oracle(mdl, dim, p):
    """Adaptation on the curved shell (2:1 meshes with hanging faces): with the oracle's random
    indicators replayed, four barrier steps of refinement and coarsening give the same meshes
    and LTS levels (the device recomputes the factors and each element's bound where the face
    kinds change), V to 1e-12 (the hanging-face terms and the mass-weighted restriction); then
    the device's own indicator on the adapted mesh equals the oracle's (to 1e-9 of the largest)."""
    from tests.helpers import forest_arrays
    base = shell_problem(dim, p, 64, base=(6, 4, 1) if dim == 2 else (4, 3, 2))
    dt0 = lts.Sim(base).dt
    prob = base.replace(max_refine=2, amr_enabled=1, tau_refine=0.7, tau_coarsen=0.3, dt_barrier=dt0 / 32)
    o = lts.Sim(prob)
    V0, v0 = front(o, prob)
    o.V, o.v = V0.copy(), v0.copy()
    o._lat_initial()
    g = mdl.Sim(prob)
    g.set_initial(V0, v0)
    rng = np.random.default_rng(dim * 10 + p)
    hanging = False
    for step in range(4):
        eta = rng.uniform(0, 1, o.disc.ne)
        g.set_indicators(eta_s=eta)
        newf, plan = o.forest.adapt(eta, prob.tau_refine, prob.tau_coarsen)
        o.transfer(newf, plan)
        lev = o.assign_levels(o.eta_t)
        o.eta_t = o.sweep(lev)
        o.barrier_count += 1
        g.step_barriers(1)
        r2, l2, c2, b2 = g.read_mesh()
        lvo, cco, _ = forest_arrays(o.forest)
        assert np.array_equal(l2, lvo) and np.array_equal(c2, cco)
        assert np.array_equal(b2, lev)
        assert mass_rel_l2(o.disc.M, g.read_V(), o.V) <= 1e-12, step
        hanging = hanging or (l2.max() > l2.min())
    assert hanging
    want = o.disc.eta_s(o.V)
    g.step_barriers(1)
    # the indicator array holds the values of the barrier-start mesh, element by element; that
    # step then adapts with them (every indicator is far below tau_coarsen, so the mesh only
    # coarsens and the first entries read back are the start mesh's first elements)
    es, _ = g.read_indicators()
    assert len(es) <= len(want)
    # flux jumps across faces are differences of nearly equal fluxes, and on a hanging face the
    # coarse side is evaluated through other tables than the oracle's basis: held to 1e-9 of the
    # largest indicator, and the larger ones to 1e-8 relative
    w = want[:len(es)]
    err = np.abs(es - w)
    i = int(np.argmax(err / want.max()))
    assert err.max() <= 1e-9 * want.max(), (i, es[i], w[i], err.max() / want.max())
    big = w > 1e-3 * want.max()
    assert np.allclose(es[big], w[big], rtol=1e-8, atol=0), np.max(np.abs(es[big] / w[big] - 1))
    g.close()
