"""Batches of resident simulations (mdl_batch_*): same results alone and in a mix (streams mode:
bit for bit; fused rounds: the thread-per-element sweep's values up to FP32 rounding), the fused
sweep's tuned launch shape and launch count, admission by device-memory footprint, completion
polling and slot release."""
import numpy as np
import pytest

import workloads as W
from tests.helpers import forest_arrays, random_forest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mdl():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2310_07607_gb300 import build, mdl as M
    build.build()
    return M


def instance(dim, p, seed, precision=32, amr=1):
    ext = (0.4, 0.3, 0.2)
    return W.Problem(dim=dim, order=p, extent=ext, base=(4, 3, 2), sigma_l=1.2, sigma_t=0.4,
                     fibre=(0.6, 0.8, 0.0) if dim == 2 else (0.48, 0.64, 0.6), gamma=10.0 * p * p,
                     max_refine=2, n_lts_levels=3, lts_enabled=1, amr_enabled=amr,
                     tau_refine=2e-9 if dim == 2 else 1e-11, tau_coarsen=2e-10 if dim == 2 else 1e-14,
                     dt_barrier=0.0, state_integrator=W.STATE_EXP, precision=precision,
                     stimuli=[W.Stimulus((0, 0, 0), (0.05 + 0.02 * seed, 0.1, 0.1), 1.0, 0.0, 1.0)])


def initial(mdl, prob):
    g = mdl.Sim(prob)
    root, level, coords, _ = g.read_mesh()
    g.close()
    n1 = prob.order + 1
    xi = np.polynomial.legendre.leggauss(n1)[0]
    d = prob.dim
    q = np.arange(n1 ** d)
    X = np.empty((len(level), n1 ** d, d))
    for k in range(d):
        h = prob.extent[k] / (prob.base[k] * 2.0 ** level)
        X[:, :, k] = coords[:, k:k + 1] * h[:, None] + (xi[(q // n1 ** k) % n1][None, :] + 1) * 0.5 * h[:, None]
    return W.front_state(X.reshape(-1, d), (0, 0, 0), 0.12, 0.02, tail=0.05)


def test_alone_equals_in_mix_bitwise(mdl):
    """Streams mode: every slot runs its own barriers (its own sweep variant) on its stream."""
    probs = [instance(2, 1, 0), instance(3, 1, 1), instance(3, 2, 2), instance(2, 1, 3, precision=64),
             instance(2, 2, 4, amr=0)]
    nbar = 6
    alone = []
    for p in probs:
        V0, v0 = initial(mdl, p)
        g = mdl.Sim(p)
        g.set_initial(V0, v0)
        g.step_barriers(nbar)
        alone.append((g.read_V(), g.read_state(), g.read_activation(), g.read_mesh()[1]))
        g.close()
    b = mdl.Batch(autotune=True, fused=False)
    slots = []
    for p in probs:
        V0, v0 = initial(mdl, p)
        dt = mdl.Sim(p).dt
        slots.append(b.admit(p, nbar * dt, V0, v0))
    # uneven stepping: rounds of 2 barriers until every slot has reached its end time
    while True:
        done = b.step(barriers_per_slot=2)
        if done == 0:
            break
    finished = sorted(b.poll())
    assert finished == sorted(slots)
    for s, (Va, va, la, lva) in zip(slots, alone):
        g, state, rc = b.slot(s)
        assert state == mdl.SLOT_DONE and rc == 0
        assert g.time()[1] == nbar
        assert np.array_equal(g.read_mesh()[1], lva)
        assert np.array_equal(g.read_V(), Va)
        assert np.array_equal(g.read_state(), va)
        assert np.array_equal(g.read_activation(), la)
    # every class got a tuned launch shape
    for p in probs:
        t, k = b.shape(p)
        assert t in (64, 128, 256) and 1 <= k <= 32
    for s in slots:
        b.release(s)
    assert b.usage()[2] == 0
    b.close()


def test_admission_by_footprint_and_release(mdl):
    p = instance(2, 1, 0)
    fp = mdl.Batch(autotune=False).footprint(p)
    assert fp > 0
    b = mdl.Batch(hbm_budget_bytes=int(fp * 1.5), autotune=False)
    s0 = b.admit(p, 0.001)
    with pytest.raises(mdl.MdlError) as ei:
        b.admit(p, 0.001)
    assert ei.value.code == -3
    b.release(s0)
    s1 = b.admit(p, 0.001)
    assert s1 == s0
    b.close()


def test_slot_finishes_at_its_own_end_time(mdl):
    b = mdl.Batch(autotune=False)
    p = instance(2, 1, 0)
    dt = mdl.Sim(p).dt
    a = b.admit(p, 3 * dt)
    c = b.admit(p, 7 * dt)
    b.step(barriers_per_slot=4)
    assert b.poll() == [a]
    b.step(barriers_per_slot=4)
    assert b.poll() == [c]
    assert b.slot(a)[0].time()[1] == 3 and b.slot(c)[0].time()[1] == 7
    b.close()


def fused_probs():
    return [instance(2, 1, 0), instance(3, 1, 1), instance(3, 2, 2), instance(2, 1, 3, precision=64),
            instance(2, 2, 4, amr=0), instance(2, 1, 5).replace(n_lts_levels=2),
            instance(3, 1, 6).replace(n_lts_levels=4)]


def run_alone(mdl, probs, nbar, variant=None):
    out = []
    for p in probs:
        V0, v0 = initial(mdl, p)
        g = mdl.Sim(p)
        if variant is not None:
            g.set_sweep_variant(variant)
        g.set_initial(V0, v0)
        g.step_barriers(nbar)
        out.append((g.read_V(), g.read_state(), g.read_activation(), g.read_mesh()))
        g.close()
    return out


def test_fused_rounds_match_alone_thread_sweep(mdl):
    """Fused rounds: one sweep launch per global tick, element class and precision over all
    slots of the class (uneven LTS levels: 2, 3 and 4 levels in one batch), replayed from a
    captured graph, several rounds per step issued back to back.  Each slot must give the
    values it gives alone with the thread-per-element sweep: meshes, levels and activated
    probes identical, V and the state within FP32 rounding of two compilations of the same
    element step (FP64 slots within 1e-12).  The launch count must be one per global tick of
    each group."""
    probs = fused_probs()
    nbar = 14
    alone = run_alone(mdl, probs, nbar, mdl.SWEEP_THREAD)
    b = mdl.Batch(autotune=False, fused=True)
    slots = []
    for p in probs:
        V0, v0 = initial(mdl, p)
        slots.append(b.admit(p, nbar * mdl.Sim(p).dt, V0, v0))
    while b.step(barriers_per_slot=4) > 0:
        pass
    assert sorted(b.poll()) == sorted(slots)
    for s, p, (Va, va, la, ma) in zip(slots, probs, alone):
        g, state, rc = b.slot(s)
        assert state == mdl.SLOT_DONE and rc == 0
        assert g.time()[1] == nbar
        mb = g.read_mesh()
        for x, y in zip(ma, mb):
            assert np.array_equal(x, y)
        tol = 1e-12 if p.precision == 64 else 1e-5
        Vb, vb, lb = g.read_V(), g.read_state(), g.read_activation()
        assert np.abs(Vb - Va).max() <= tol * max(np.abs(Va).max(), 1.0), (p.dim, p.order, np.abs(Vb - Va).max())
        assert np.abs(vb - va).max() <= tol * max(np.abs(va).max(), 1.0)
        fa, fb = np.isfinite(la), np.isfinite(lb)
        assert np.array_equal(fa, fb)
        if fa.any():
            assert np.abs(la[fa] - lb[fa]).max() <= 1e-6
    info, (rounds, launches) = b.fused_info(32, 2, 1)
    assert rounds == nbar
    # per round, 2^Bmax launches for each (precision, class) group: FP32 2D Q1 (levels 3 and
    # 2: Bmax 2), FP32 3D Q1 (3 and 4: 3), FP32 3D Q2 (2), FP64 2D Q1 (2), FP32 2D Q2 (2)
    assert launches == nbar * (4 + 8 + 4 + 4 + 4)
    for s in slots:
        b.release(s)
    b.close()


def test_fused_tuner_picks_per_class_and_slots_finish(mdl):
    """With autotune, the first rounds time every fused launch shape and the slots' own sweeps
    per (precision, class) group, one round at a time, and keep the fastest; the later rounds
    run back to back.  A slot's rounds may then mix the fused (thread-per-element) step and its
    own sweep variant (the tensor-core sweep for Q2 3D FP32), so each slot is held to the
    FP32 tolerance against its run alone (FP64 slots: 1e-12), and every group present must
    report its choice with the fastest candidate no slower than the slowest."""
    probs = fused_probs()
    # the Q2 3D slot without adaptation: an indicator within rounding of its threshold could
    # otherwise adapt differently under the two sweep variants
    probs[2] = probs[2].replace(amr_enabled=0)
    nbar = 20                     # 7 candidates x 2 rounds of tuning, then 6 back to back
    alone = run_alone(mdl, probs, nbar)
    b = mdl.Batch(autotune=True, fused=True)
    slots = []
    for p in probs:
        V0, v0 = initial(mdl, p)
        slots.append(b.admit(p, nbar * mdl.Sim(p).dt, V0, v0))
    while b.step(barriers_per_slot=3) > 0:
        pass
    assert sorted(b.poll()) == sorted(slots)
    for s, p, (Va, va, la, ma) in zip(slots, probs, alone):
        g, state, rc = b.slot(s)
        assert state == mdl.SLOT_DONE and rc == 0
        assert g.time()[1] == nbar
        Vb = g.read_V()
        tol = 1e-12 if p.precision == 64 else 1e-3
        assert np.linalg.norm(Vb - Va) <= tol * np.linalg.norm(Va), (p.dim, p.order)
    for prec, dim, order in [(32, 2, 1), (32, 3, 1), (32, 3, 2), (64, 2, 1), (32, 2, 2)]:
        info, (rounds, _) = b.fused_info(prec, dim, order)
        assert info is not None, (prec, dim, order)
        assert info["best_ms"] <= info["worst_ms"] and info["own_ms"] > 0
        if not info["own"]:
            assert info["threads"] in (64, 128, 256) and info["tile"] >= 128
    assert rounds == nbar
    # a class never admitted has no choice
    assert b.fused_info(64, 3, 2)[0] is None
    for s in slots:
        b.release(s)
    b.close()


def test_fused_group_larger_than_one_launch(mdl):
    """More slots of one class than one fused launch takes (256): the group sweeps in chunks,
    each slot still gives the values it gives alone with the thread-per-element sweep."""
    probs = [instance(2, 1, i % 5, amr=0).replace(base=(2, 2, 1), extent=(0.2, 0.15, 1.0)) for i in range(300)]
    nbar = 4
    b = mdl.Batch(autotune=False, fused=True)
    slots = [b.admit(p, nbar * mdl.Sim(p).dt) for p in probs]
    while b.step(barriers_per_slot=nbar) > 0:
        pass
    for i in (0, 255, 256, 299):
        g = mdl.Sim(probs[i])
        g.set_sweep_variant(mdl.SWEEP_THREAD)
        g.step_barriers(nbar)
        gb, state, rc = b.slot(slots[i])
        assert state == mdl.SLOT_DONE and rc == 0 and gb.time()[1] == nbar
        Va, Vb = g.read_V(), gb.read_V()
        assert np.abs(Vb - Va).max() <= 1e-5 * max(np.abs(Va).max(), 1.0)
        g.close()
    _, (rounds, launches) = b.fused_info(32, 2, 1)
    assert rounds == nbar and launches == nbar * 2 * 4      # two chunks, 2^2 ticks each
    for s in slots:
        b.release(s)
    b.close()
