"""Pins for the oracle's time marching (Alg. 1), indicators, AMR and activation times."""
import math

import numpy as np
import pytest
import scipy.integrate

import workloads as W
from oracle import basis, ionic, lts
from oracle.forest import Forest
from oracle.sipg import Disc


def diffusion_prob(dim=2, p=1, base=(6, 6, 1), extent=(1.0, 1.0, 1.0), n_lts=3):
    return W.Problem(dim=dim, order=p, extent=extent, base=base, sigma_l=1.2, sigma_t=0.4,
                     fibre=(0.6, 0.8, 0.0), chi=1400.0, cm=1.0, gamma=10.0 * p * p,
                     ionic_model=-1, max_refine=2, n_lts_levels=n_lts, lts_enabled=1,
                     dt_barrier=0.0)


def refined_forest(prob, frac=0.5):
    f = Forest(prob.dim, prob.base, prob.max_refine, prob.extent)
    eta = np.array([1.0 if lf[1][0] < prob.base[0] * frac else 0.0 for lf in f.leaves])
    f, _ = f.adapt(eta, 0.5, -1.0)
    eta = np.array([1.0 if (lf[0] == 1 and lf[1][0] < 2) else 0.0 for lf in f.leaves])
    f, _ = f.adapt(eta, 0.5, -1.0)
    return f


def smooth_state(sim):
    X = sim.disc.node_coords()
    return np.cos(math.pi * X[:, 0]) * np.cos(math.pi * X[:, 1]) + 0.5


# --------------------------------------------------------------------------
# Conservation and equivalences.
# --------------------------------------------------------------------------

def test_global_fe_conserves_integral_pure_diffusion():
    prob = diffusion_prob(n_lts=1).replace(lts_enabled=0, dt_barrier=1e-4)
    sim = lts.Sim(prob, forest=refined_forest(prob))
    rng = np.random.default_rng(0)
    V = rng.standard_normal(sim.disc.ne * sim.disc.n_p)
    I0 = np.sum(sim.disc.M * V)
    V, _ = lts.global_fe(prob, sim.A, sim.disc.M, V, np.zeros_like(V), prob.dt_barrier, 100,
                         lambda t: 0.0)
    assert abs(np.sum(sim.disc.M * V) - I0) <= 1e-12 * np.sum(sim.disc.M * np.abs(V))


def test_single_level_lts_is_global_forward_euler_bitwise():
    """With equal S_e the sweep is exactly global forward Euler at dt / S (AP, no stimulus)."""
    prob = W.plain_2d_q1_32x32().replace(base=(8, 8, 1), extent=(0.25, 0.25, 1.0), stimuli=[],
                                         lts_enabled=1, n_lts_levels=3, dt_barrier=0.02,
                                         state_integrator=W.STATE_EXP)
    rng = np.random.default_rng(1)
    sim = lts.Sim(prob)
    V0 = rng.uniform(0, 1, sim.disc.ne * sim.disc.n_p)
    v0 = rng.uniform(0, 0.5, V0.size)
    sim.V, sim.v = V0.copy(), v0.copy()
    lev = np.full(sim.disc.ne, 2)
    for _ in range(3):
        sim.sweep(lev)
        sim.barrier_count += 1
    Vg, vg = lts.global_fe(prob, sim.A, sim.disc.M, V0, v0, 0.02 / 4, 12, lambda t: 0.0)
    assert np.array_equal(sim.V, Vg)
    assert np.array_equal(sim.v, vg)


def test_lts_converges_first_order_to_fine_global_step():
    prob = diffusion_prob()
    f = refined_forest(prob)
    errs = []
    for scale in (1, 2, 4):
        sim = lts.Sim(prob, forest=f)
        dt0 = sim.dt
        sim.dt = dt0 / scale
        V0 = smooth_state(sim)
        sim.V = V0.copy()
        # substep levels follow the refinement levels (dt_e <= CFL_e holds for each)
        lev = sim.disc.levels.copy()
        assert len(set(lev.tolist())) == 3
        assert np.all(np.ldexp(sim.dt, -lev) <= sim.cfl())
        T = 8 * dt0
        for _ in range(8 * scale):
            sim.sweep(lev)
            sim.barrier_count += 1
        nfine = 8 * scale * (1 << sim.B)
        Vg, _ = lts.global_fe(prob, sim.A, sim.disc.M, V0, np.zeros_like(V0), T / nfine, nfine,
                              lambda t: 0.0)
        errs.append(math.sqrt(np.sum(sim.disc.M * (sim.V - Vg) ** 2)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 1.6 < r1 < 2.5 and 1.6 < r2 < 2.5, errs


def test_lts_integral_drift_vanishes_with_dt():
    """Multi-level LTS is not conservative, but the drift of int V is O(dt)."""
    prob = diffusion_prob()
    f = refined_forest(prob)
    drifts = []
    for scale in (1, 4):
        sim = lts.Sim(prob, forest=f)
        T = 8 * sim.dt
        sim.dt /= scale
        sim.V = smooth_state(sim)
        I0 = np.sum(sim.disc.M * sim.V)
        lev = sim.disc.levels.copy()
        for _ in range(8 * scale):
            sim.sweep(lev)
            sim.barrier_count += 1
        drifts.append(abs(np.sum(sim.disc.M * sim.V) - I0))
    assert drifts[1] < drifts[0] / 2.5


def test_levels_from_cfl_and_auto_barrier():
    prob = diffusion_prob()
    sim = lts.Sim(prob, forest=refined_forest(prob))
    cfl = sim.cfl()
    lev = sim.assign_levels(np.zeros(sim.disc.ne))
    for e in range(sim.disc.ne):
        b = lev[e]
        assert math.ldexp(sim.dt, -int(b)) <= cfl[e]
        if b > 0:
            assert math.ldexp(sim.dt, -int(b) + 1) > cfl[e]
    # auto barrier is the largest power of two meeting the budget for every class
    assert math.log2(sim.dt) == round(math.log2(sim.dt))
    assert lev.max() <= prob.n_lts_levels - 1
    sim2 = lts.Sim(prob.replace(dt_barrier=2 * sim.dt), forest=refined_forest(prob))
    worst = lts.auto_dt_barrier(prob, sim.disc)
    assert worst == sim.dt


def test_cell_indicator_raises_level():
    prob = diffusion_prob().replace(tau_cell=0.1, dt_bar_cell=1e-9)
    sim = lts.Sim(prob, forest=refined_forest(prob))
    eta = np.zeros(sim.disc.ne)
    eta[0] = 1.0
    with pytest.raises(lts.CFLViolation):
        sim.assign_levels(eta)
    prob = prob.replace(dt_bar_cell=0.0)
    sim = lts.Sim(prob, forest=refined_forest(prob))
    base = sim.assign_levels(np.zeros(sim.disc.ne))
    prob2 = prob.replace(dt_bar_cell=sim.dt / 4.0 * 1.0000001)
    sim2 = lts.Sim(prob2, forest=refined_forest(prob))
    lev = sim2.assign_levels(eta)
    assert lev[0] == max(base[0], 2) and np.array_equal(lev[1:], base[1:])


# --------------------------------------------------------------------------
# RV-T temporal indicator against the exact Bochner norm of the cell ODE.
# --------------------------------------------------------------------------

def test_rvt_indicator_converges_to_bochner_norm():
    prob = W.Problem(dim=2, order=1, extent=(0.1, 0.1, 1.0), base=(1, 1, 1), stimuli=[],
                     lts_enabled=1, n_lts_levels=9, dt_barrier=2.0, state_integrator=W.STATE_EXP)
    V0, v0 = 0.35, 0.05

    def rhs(t, y):
        V, v = np.array([y[0]]), np.array([y[1]])
        return [-ionic.i_ion(prob, V, v)[0], ionic.g(prob, V, v)[0]]
    sol = scipy.integrate.solve_ivp(rhs, (0.0, 2.0), [V0, v0], rtol=1e-11, atol=1e-13,
                                    dense_output=True, method='DOP853')
    Ia = ionic.i_ion(prob, np.array([V0]), np.array([v0]))[0]
    ga = ionic.g(prob, np.array([V0]), np.array([v0]))[0]

    def integrand(t):
        V, v = sol.sol(t)
        return ((ionic.i_ion(prob, np.array([V]), np.array([v]))[0] - Ia) ** 2
                + (ionic.g(prob, np.array([V]), np.array([v]))[0] - ga) ** 2)
    area = 0.1 * 0.1
    ex = math.sqrt(scipy.integrate.quad(integrand, 0.0, 2.0, limit=400, epsabs=1e-14)[0] * area) / 2.0
    errs = []
    for b in (5, 6, 7, 8):
        sim = lts.Sim(prob)
        sim.V[:] = V0
        sim.v[:] = v0
        eta = sim.sweep(np.array([b]))
        errs.append(abs(eta[0] - ex))
    rates = [errs[i] / errs[i + 1] for i in range(3)]
    assert errs[-1] < 0.02 * ex
    assert all(1.6 < r < 2.6 for r in rates), (errs, ex)


# --------------------------------------------------------------------------
# AMR: balance, plan, transfer.
# --------------------------------------------------------------------------

@pytest.mark.parametrize("dim", [2, 3])
def test_adapt_random_marks_keeps_balance_and_plan(dim):
    f = Forest(dim, (4, 3, 2), 3, (1.0, 0.75, 0.5))
    rng = np.random.default_rng(7)
    for step in range(5):
        eta = rng.uniform(0, 1, f.n)
        nf, plan = f.adapt(eta, 0.8, 0.3)
        assert nf.is_balanced()
        assert len(plan) == nf.n
        # every old leaf is accounted for exactly once
        used = []
        for pl in plan:
            if pl[0] == 'keep':
                used.append(pl[1])
            elif pl[0] == 'child':
                used.append(pl[1])
            else:
                used.extend(pl[1])
        assert set(used) == set(range(f.n))
        # refined leaves had eta >= tau or were forced by balance; coarsened had all eta <= tau_c
        for pl in plan:
            if pl[0] == 'parent':
                assert all(eta[c] <= 0.3 for c in pl[1])
        for i, lf in enumerate(f.leaves):
            if eta[i] >= 0.8 and lf[0] < 3:
                assert lf not in nf.index
        f = nf
    assert max(lf[0] for lf in f.leaves) >= 2


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (3, 1)])
def test_transfer_exact_for_polynomials_and_projection_identity(dim, p):
    prob = W.Problem(dim=dim, order=p, extent=(1.0, 1.0, 1.0), base=(2, 2, 2), ionic_model=-1,
                     max_refine=2)
    sim = lts.Sim(prob)
    X = sim.disc.node_coords()
    poly = lambda X: 0.3 + X[:, 0] ** p - 0.7 * X[:, 1] * X[:, 0] ** (p - 1) + 0.2 * X[:, dim - 1]
    sim.V = poly(X)
    sim.v = 2.0 * poly(X)
    eta = np.zeros(sim.disc.ne); eta[0] = 1.0
    nf, plan = sim.forest.adapt(eta, 0.5, -1.0)
    old_int = np.sum(sim.disc.M * sim.V)
    sim.transfer(nf, plan)
    assert np.abs(sim.V - poly(sim.disc.node_coords())).max() < 1e-13
    assert abs(np.sum(sim.disc.M * sim.V) - old_int) < 1e-13
    # coarsen back: projection of a prolonged polynomial is the identity
    eta = np.zeros(sim.disc.ne)
    nf2, plan2 = sim.forest.adapt(eta, 0.5, 0.1)
    assert nf2.n == 2 ** dim
    sim.transfer(nf2, plan2)
    assert np.abs(sim.V - poly(sim.disc.node_coords())).max() < 1e-13


def test_coarsening_preserves_integral_of_rough_field():
    prob = W.Problem(dim=2, order=1, extent=(1.0, 1.0, 1.0), base=(2, 2, 1), ionic_model=-1, max_refine=2)
    sim = lts.Sim(prob)
    eta = np.ones(sim.disc.ne)
    nf, plan = sim.forest.adapt(eta, 0.5, -1.0)
    sim.transfer(nf, plan)
    rng = np.random.default_rng(2)
    sim.V = rng.standard_normal(sim.V.size)
    I0 = np.sum(sim.disc.M * sim.V)
    nf, plan = sim.forest.adapt(np.zeros(sim.disc.ne), 0.5, 0.1)
    sim.transfer(nf, plan)
    assert sim.disc.ne == 4
    assert abs(np.sum(sim.disc.M * sim.V) - I0) < 1e-13


# --------------------------------------------------------------------------
# Local activation times.
# --------------------------------------------------------------------------

def test_lat_planar_front_is_linear_in_x():
    prob = W.plain_2d_q1_32x32().replace(base=(64, 2, 1), extent=(2.0, 2.0 / 32, 1.0),
                                         stimuli=[W.Stimulus((0, 0, 0), (0.05, 1.0, 1.0), 1.0, 0.0, 1.0)])
    sim = lts.Sim(prob)
    sim.step_to(40.0)
    xs = sim.probe_x[:, 0]
    sel = (xs > 0.5) & (xs < 1.5)
    lat = sim.lat[sel]
    assert np.isfinite(lat).all()
    A = np.stack([xs[sel], np.ones(sel.sum())], axis=1)
    coef, res, *_ = np.linalg.lstsq(A, lat, rcond=None)
    fit = A @ coef
    cv = 1.0 / coef[0]          # cm/ms
    assert 0.02 < cv < 0.08
    assert np.abs(fit - lat).max() < 0.02 * (lat.max() - lat.min())
    # nodes that share x share the activation time (planar front)
    order = np.argsort(xs[sel])
    assert np.all(np.diff(lat[order]) >= -1e-9)


def test_lat_initially_active_points_read_start_time():
    prob = W.plain_2d_q1_32x32().replace(base=(4, 4, 1), extent=(0.125, 0.125, 1.0), stimuli=[])
    sim0 = lts.Sim(prob)
    V0 = np.where(sim0.disc.node_coords()[:, 0] < 0.05, 1.0, 0.0)
    sim = lts.Sim(prob, V0=V0)
    assert np.all(sim.lat[sim.probe_x[:, 0] < 0.05] == 0.0)
    assert np.all(np.isinf(sim.lat[sim.probe_x[:, 0] > 0.06]))
