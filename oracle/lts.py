"""Explicit local space-time adaptive time marching (Sec. 2.3, Alg. 1).

Per barrier step [t_n, t_n + dt]:
  1. eta^s on the current mesh (Eq. dg-error-estimate), refine then coarsen with
     solution transfer (Alg. 1, adapt steps);
  2. substeps S_e = 2^max(b^CFL_e, b^cell_e) (Eq. num-substeps), with
     b^CFL_e the smallest integer b >= 0 with dt 2^-b <= CFL_e (Sec. 2.3,
     Eq. cfl-monodomain), b^cell_e the smallest b >= 0 with dt 2^-b <= dt_bar if
     eta^t_e > tau_cell, else 0;
  3. sweeps over the dyadic tick clock i = 0 .. 2^B - 1 (B = n_lts_levels - 1):
     element e is due at tick i iff (2^B / S_e) divides i.  Due elements buffer
     their value and take one forward-Euler step on phi and one exponential step
     on the state, all from the values at the tick start (Jacobi reading of the
     queue loop; with equal S_e it is exactly global forward Euler).  A coarser
     neighbour that is mid-interval is seen through the linear time interpolant
     between its buffered value and its new value (Alg. 1, interpolation step).
     Ticks where nothing is due are empty, so the update sequence is the one of
     Alg. 1 with S_max = max_e S_e.
  4. RV-T temporal indicator accumulated over the element's own substeps by the
     midpoint rule (Eq. ratti-veroni-temporal):
       acc_e += dt_e sum_q M_q [ (I(u_mid, t_mid) - I(u_a, t_a))^2 + (g(u_mid) - g(u_a))^2 ]
       eta^t_e = sqrt(acc_e) / dt
  5. local activation times (Sec. 3.3 LAT definition) on a fixed probe lattice
     (the GL nodes of the root mesh), phi piecewise linear in time between each
     owning element's steps, first strict crossing of the threshold.

The dyadic barrier length for the 'n LTS levels' workloads (dt_barrier = 0) is
the largest 2^-k ms such that every admissible element class (any level up to
max_refine, any face configuration) has b^CFL <= n_lts_levels - 1.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
from __future__ import annotations

import itertools
import math
from typing import Optional

import numpy as np

from . import basis, ionic
from .forest import Forest
from .mapped import MappedDisc
from .sipg import Disc, eval_element


class CFLViolation(RuntimeError):
    pass


def b_from_bound(dt: float, bound: float) -> int:
    """Smallest integer b >= 0 with dt * 2^-b <= bound (exact ldexp loop)."""
    b = 0
    while math.ldexp(dt, -b) > bound:
        b += 1
        if b > 60:
            raise CFLViolation("bound %g unreachable from dt %g" % (bound, dt))
    return b


def own_block(disc: Disc, level: int, configs) -> np.ndarray:
    """Own-DOF block of A for an element of `level` with face configuration `configs`.

    configs[f] for f = 2 axis + (side > 0): 0 boundary, 1 same level, 2 neighbour
    one level coarser, 3 neighbours one level finer.  Assembled from the volume
    block and the element's own quadrant of each face block.
    """
    n_p = disc.n_p
    B = disc.volume_block(level).copy()
    d = disc.dim
    for f, c in enumerate(configs):
        k, s = f // 2, (1 if f % 2 else -1)
        if c == 0:
            continue
        if c == 1:
            sigs = [(level, level, ())]
        elif c == 2:
            sigs = [(level, level - 1, (0,) * (d - 1))]
        else:
            sigs = [(level, level + 1, tuple((b >> t) & 1 for t in range(d - 1)))
                    for b in range(1 << (d - 1))]
        for (l_me, l_nb, pos) in sigs:
            if s > 0:   # this element is the minus side
                Bf = disc.face_block(k, (l_me, l_nb, pos))
                B += Bf[:n_p, :n_p]
            else:       # this element is the plus side
                Bf = disc.face_block(k, (l_nb, l_me, pos))
                B += Bf[n_p:, n_p:]
    return B


def gershgorin_cfl(Bown: np.ndarray, Mq: np.ndarray) -> float:
    L = -Bown / Mq[:, None]
    return 1.0 / np.max(np.abs(L).sum(axis=1))


def auto_dt_barrier(prob, disc: Disc, cfl=None) -> float:
    """Largest 2^-k ms with b^CFL <= n_lts_levels - 1 for every admissible element class
    (on a mapped mesh, which does not adapt: for every element of the mesh, cfl)."""
    d = disc.dim
    wq = basis.node_weights(d, disc.p)
    cmin = math.inf
    if cfl is not None:
        cmin = float(np.min(cfl))
    for level in range(prob.max_refine + 1 if cfl is None else 0):
        choices = [0, 1] + ([2] if level > 0 else []) + ([3] if level < prob.max_refine else [])
        Mq = wq * np.prod(disc.forest.h(level) / 2.0)
        for cfg in itertools.product(choices, repeat=2 * d):
            cmin = min(cmin, gershgorin_cfl(own_block(disc, level, cfg), Mq))
    B = prob.n_lts_levels - 1
    k = -20
    while math.ldexp(1.0, -k - B) > cmin:
        k += 1
    return math.ldexp(1.0, -k)


class Sim:
    """FP64 reference simulation of one problem."""

    def __init__(self, prob, V0: Optional[np.ndarray] = None, v0: Optional[np.ndarray] = None,
                 forest: Optional[Forest] = None):
        self.prob = prob
        self.forest = forest if forest is not None else Forest(prob.dim, prob.base, prob.max_refine,
                                                               prob.extent)
        self.B = prob.n_lts_levels - 1 if prob.lts_enabled else 0
        self.mapped = getattr(prob, "geometry", 0) != 0
        if self.mapped and prob.amr_enabled and not prob.dt_barrier > 0:
            # the admissible elements of an adapting curved mesh are not a finite set of
            # classes: the barrier step is the caller's
            raise ValueError("mapped geometry with adaptation: dt_barrier must be given")
        self._rebuild()
        n = self.disc.ne * self.disc.n_p
        self.V = np.zeros(n) if V0 is None else np.array(V0, dtype=np.float64)
        self.v = np.zeros(n) if v0 is None else np.array(v0, dtype=np.float64)
        self.barrier_count = 0
        self.eta_t = np.zeros(self.disc.ne)
        self.eta_s = np.zeros(self.disc.ne)
        if prob.dt_barrier > 0:
            self.dt = float(prob.dt_barrier)
        else:
            self.dt = auto_dt_barrier(prob, self.disc, self.cfl() if self.mapped else None)
        self._probes()
        self.lat = np.full(self.n_probe, np.inf)
        self._lat_initial()
        self.levels = np.zeros(self.disc.ne, dtype=np.int64)
        self.dof_updates = 0

    @property
    def t(self) -> float:
        return self.barrier_count * self.dt

    def tick_time(self, i: int) -> float:
        """Start time of tick i of the current barrier: (n 2^B + i) dt / 2^B, never accumulated."""
        nt = 1 << self.B
        return (self.barrier_count * nt + i) * self.dt / nt

    # ------------------------------------------------------------------
    def _rebuild(self):
        self.disc = (MappedDisc if self.mapped else Disc)(self.prob, self.forest)
        self.A = self.disc.assemble()
        self._cfl = None
        self._stim_masks()

    def cfl(self) -> np.ndarray:
        if self._cfl is None:
            self._cfl = self.disc.cfl(self.A)
        return self._cfl

    def _stim_masks(self):
        X = self.disc.node_coords()
        self.stim_masks = []
        for s in self.prob.stimuli:
            m = np.ones(X.shape[0], dtype=bool)
            for k in range(self.prob.dim):
                m &= (X[:, k] >= s.lo[k] - 1e-12) & (X[:, k] <= s.hi[k] + 1e-12)
            self.stim_masks.append(m)

    def i_stim(self, t: float, sel=slice(None)) -> np.ndarray:
        """I_stim per DOF at time t: -amplitude inside the box while t0 <= t < t1."""
        n = self.V[sel].shape[0]
        out = np.zeros(n)
        for s, m in zip(self.prob.stimuli, self.stim_masks):
            if s.t0 <= t < s.t1:
                out -= s.amplitude * m[sel]
        return out

    def current_I(self, V, v, t, sel=slice(None)):
        """I = I_ion / C_m + I_stim (Eq. contGal with the AP current already per unit capacitance)."""
        return ionic.i_ion(self.prob, V, v) + self.i_stim(t, sel)

    # ------------------------------------------------------------------
    def _probes(self):
        """Probe lattice: the GL nodes of every root element, owned by the leaf containing them."""
        prob = self.prob
        d = prob.dim
        xi = basis.node_points(d, prob.order)
        f = self.forest
        h0 = f.h(0)
        pts = []
        for rz in range(f.base[2]):
            for ry in range(f.base[1]):
                for rx in range(f.base[0]):
                    lo = np.array([rx, ry, rz][:d], dtype=np.float64) * h0
                    pts.append(lo[None, :] + (xi + 1.0) * 0.5 * h0[None, :])
        self.probe_x = np.concatenate(pts, axis=0)
        self.n_probe = self.probe_x.shape[0]
        self._probe_owner()

    def _probe_owner(self):
        """Owner leaf of every probe and the sparse map P (probe values = P @ V).

        Probe q of root r lies in the leaf of level l whose local cell index is
        floor((xi_q + 1)/2 * 2^l) per direction (half-open cells).
        """
        import scipy.sparse as sp
        prob = self.prob
        d = prob.dim
        f = self.forest
        xi = basis.node_points(d, prob.order)
        n_p = xi.shape[0]
        lv, c = self.disc.leaf_arrays()
        root = c >> lv[:, None]
        loc = c - (root << lv[:, None])
        rid = root[:, 0] + f.base[0] * (root[:, 1] + (f.base[1] * root[:, 2] if d == 3 else 0))
        # cell of root node q at level l, per direction
        cell = np.floor((xi[None, :, :] + 1.0) * 0.5 * (2.0 ** lv)[:, None, None]).astype(np.int64)
        inside = np.all(cell == loc[:, None, :], axis=2)                      # (ne, n_p)
        e_idx, q_idx = np.nonzero(inside)
        ids = rid[e_idx] * n_p + q_idx
        owner = np.full(self.n_probe, -1, dtype=np.int64)
        owner[ids] = e_idx
        assert (owner >= 0).all()
        hs = np.array([f.h(l) for l in range(f.L + 1)])
        h = hs[lv[e_idx]]
        lower = c[e_idx] * h
        xl = 2.0 * (self.probe_x[ids] - lower) / h - 1.0
        phi, _ = basis.eval_basis(d, prob.order, xl)                          # (npr, n_p)
        rows = np.repeat(ids, n_p)
        cols = (e_idx[:, None] * n_p + np.arange(n_p)[None, :]).ravel()
        self.probe_owner = owner
        self.P = sp.csr_matrix((phi.ravel(), (rows, cols)), shape=(self.n_probe, f.n * n_p))

    def _lat_initial(self):
        th = self.prob.act_threshold
        val = self.P @ self.V
        hit = (val > th) & np.isinf(self.lat)
        self.lat[hit] = self.t

    # ------------------------------------------------------------------
    def assign_levels(self, eta_t: np.ndarray) -> np.ndarray:
        """b_e = max(b^CFL_e, b^cell_e) (Eq. num-substeps)."""
        prob = self.prob
        ne = self.disc.ne
        if not prob.lts_enabled:
            return np.zeros(ne, dtype=np.int64)
        cfl = self.cfl()
        b_cell_on = b_from_bound(self.dt, prob.dt_bar_cell) if prob.dt_bar_cell > 0 else 0
        out = np.empty(ne, dtype=np.int64)
        memo = {}
        for e in range(ne):
            c = cfl[e]
            if c not in memo:
                memo[c] = b_from_bound(self.dt, c)
            bt = b_cell_on if eta_t[e] > prob.tau_cell else 0
            out[e] = max(memo[c], bt)
        if out.max(initial=0) > self.B:
            raise CFLViolation("element needs %d levels, budget %d" % (out.max(), self.B))
        return out

    # ------------------------------------------------------------------
    def sweep(self, levels: np.ndarray):
        """One barrier step of Alg. 1 on a fixed mesh with fixed levels; returns eta^t."""
        prob = self.prob
        disc = self.disc
        n_p = disc.n_p
        ne = disc.ne
        B = self.B
        nt = 1 << B
        stride = (1 << (B - levels)).astype(np.int64)           # ticks per element step
        dte = self.dt / (1 << levels).astype(np.float64)          # element step length
        t_a = self.t
        V_a = self.V.copy()
        v_a = self.v.copy()
        I_a = self.current_I(V_a, v_a, t_a)
        g_a = ionic.g(prob, V_a, v_a)
        Vcur = self.V.copy()
        Vbuf = self.V.copy()
        vcur = self.v.copy()
        acc = np.zeros(ne)
        M = disc.M
        th = prob.act_threshold
        dof_e = np.repeat(np.arange(ne), n_p)
        for i in range(nt):
            due = (i % stride) == 0
            if not due.any():
                continue
            t_i = self.tick_time(i)
            # values seen at tick start: own/finer = current, coarser mid-interval = interpolant
            start = (i // stride) * stride
            theta = (i - start) / stride
            th_dof = theta[dof_e]
            U = np.where(th_dof == 0.0, Vcur, Vbuf + th_dof * (Vcur - Vbuf))
            r = self.A @ U
            due_dof = due[dof_e]
            idx = np.nonzero(due_dof)[0]
            Vo = Vcur[idx]
            vo = vcur[idx]
            dt_d = dte[dof_e[idx]]
            I_o = self.current_I(Vo, vo, t_i, idx)
            Vn = Vo + dt_d * (-r[idx] / M[idx] - I_o)
            vn = ionic.step_state(prob, Vo, vo, dt_d, prob.state_integrator)
            # RV-T accumulation by the midpoint rule
            Vm = 0.5 * (Vo + Vn)
            vm = 0.5 * (vo + vn)
            t_m = t_i + 0.5 * dt_d
            Im = ionic.i_ion(prob, Vm, vm) + self._stim_at(idx, t_m)
            gm = ionic.g(prob, Vm, vm)
            term = M[idx] * ((Im - I_a[idx]) ** 2 + (gm - g_a[idx]) ** 2)
            els = np.nonzero(due)[0]
            acc[els] += dte[els] * term.reshape(-1, n_p).sum(axis=1)
            # LAT on probes owned by due elements: first strict crossing, linear in time
            Vnew_full = Vcur.copy()
            Vnew_full[idx] = Vn
            po = self.P @ Vcur
            pn = self.P @ Vnew_full
            hit = due[self.probe_owner] & np.isinf(self.lat) & (po <= th) & (pn > th)
            if hit.any():
                frac = (th - po[hit]) / (pn[hit] - po[hit])
                self.lat[hit] = t_i + dte[self.probe_owner[hit]] * frac
            Vbuf[idx] = Vo
            Vcur[idx] = Vn
            vcur[idx] = vn
            self.dof_updates += idx.size
        self.V = Vcur
        self.v = vcur
        return np.sqrt(acc) / self.dt

    def _stim_at(self, idx, t):
        """I_stim at DOFs idx and per-DOF times t."""
        out = np.zeros(idx.size)
        t = np.broadcast_to(np.asarray(t, dtype=np.float64), idx.shape)
        for s, m in zip(self.prob.stimuli, self.stim_masks):
            on = (s.t0 <= t) & (t < s.t1)
            out -= s.amplitude * (m[idx] & on)
        return out

    # ------------------------------------------------------------------
    def transfer(self, new_forest: Forest, plan):
        """Solution transfer (Alg. 1, adapt steps): prolong by evaluating the parent
        polynomial at the child nodes; restrict by the L2 projection onto the parent
        computed with the children's GL rule (exact for the diagonal GL mass)."""
        d, p = self.prob.dim, self.prob.order
        n_p = (p + 1) ** d
        xi = basis.node_points(d, p)
        wq = basis.node_weights(d, p)
        oldV = self.V.reshape(-1, n_p)
        oldv = self.v.reshape(-1, n_p)
        nn = new_forest.n
        newV = np.empty((nn, n_p))
        newv = np.empty((nn, n_p))
        eta_t = np.empty(nn)
        # parent basis at the nodes of child b: child b occupies [-1,0] or [0,1] per direction
        phis = []
        for b in range(1 << d):
            off = np.array([((b >> k) & 1) for k in range(d)], dtype=np.float64)
            phi, _ = basis.eval_basis(d, p, (xi + 2.0 * off[None, :] - 1.0) / 2.0)
            phis.append(phi)
        kind = np.array([0 if pl[0] == 'keep' else (1 if pl[0] == 'child' else 2) for pl in plan])
        keep = np.nonzero(kind == 0)[0]
        src = np.array([pl[1] for pl in plan if pl[0] == 'keep'], dtype=np.int64)
        newV[keep] = oldV[src]; newv[keep] = oldv[src]; eta_t[keep] = self.eta_t[src]
        ch = np.nonzero(kind == 1)[0]
        if ch.size:
            par = np.array([plan[i][1] for i in ch], dtype=np.int64)
            bits = np.array([plan[i][2] for i in ch], dtype=np.int64)
            for b in range(1 << d):
                m = bits == b
                newV[ch[m]] = oldV[par[m]] @ phis[b].T
                newv[ch[m]] = oldv[par[m]] @ phis[b].T
            eta_t[ch] = self.eta_t[par]
        pa = np.nonzero(kind == 2)[0]
        new_disc = MappedDisc(self.prob, new_forest) if self.mapped else None
        if pa.size:
            kids = np.array([plan[i][1] for i in pa], dtype=np.int64)         # (npar, 2^d)
            if self.mapped:
                # the children's GL masses against the parent's: M_p u_p = sum_c sum_qc M_c psi_p u_c
                Mo = self.disc.M.reshape(-1, n_p)
                Mn = new_disc.M.reshape(-1, n_p)
                accV = np.zeros((pa.size, n_p)); accv = np.zeros((pa.size, n_p))
                for b in range(1 << d):
                    accV += (Mo[kids[:, b]] * oldV[kids[:, b]]) @ phis[b]
                    accv += (Mo[kids[:, b]] * oldv[kids[:, b]]) @ phis[b]
                newV[pa] = accV / Mn[pa]
                newv[pa] = accv / Mn[pa]
            else:
                wc = wq / (2.0 ** d)                                          # child weights in parent measure
                accV = np.zeros((pa.size, n_p)); accv = np.zeros((pa.size, n_p))
                for b in range(1 << d):
                    accV += (wc[None, :] * oldV[kids[:, b]]) @ phis[b]
                    accv += (wc[None, :] * oldv[kids[:, b]]) @ phis[b]
                newV[pa] = accV / wq[None, :]
                newv[pa] = accv / wq[None, :]
            eta_t[pa] = self.eta_t[kids].mean(axis=1)
        self.forest = new_forest
        self._rebuild()
        self.V = newV.reshape(-1)
        self.v = newv.reshape(-1)
        self.eta_t = eta_t
        self._probe_owner()

    # ------------------------------------------------------------------
    def barrier(self):
        prob = self.prob
        if prob.amr_enabled:
            self.eta_s = self.disc.eta_s(self.V)
            newf, plan = self.forest.adapt(self.eta_s, prob.tau_refine, prob.tau_coarsen)
            if any(pl[0] != 'keep' for pl in plan) or newf.n != self.forest.n:
                self.transfer(newf, plan)
        self.levels = self.assign_levels(self.eta_t)
        self.eta_t = self.sweep(self.levels)
        self.barrier_count += 1

    def step_to(self, t_end: float):
        n = int(math.floor((t_end - self.t) / self.dt + 1e-9))
        for _ in range(n):
            self.barrier()


def global_fe(prob, A, M, V, v, dt, nsteps, i_stim_fn, t0=0.0):
    """Plain global forward Euler on phi and the chosen state integrator (no AMR, no LTS)."""
    V = V.copy(); v = v.copy()
    for n in range(nsteps):
        t = t0 + n * dt
        I = ionic.i_ion(prob, V, v) + i_stim_fn(t)
        Vn = V + dt * (-(A @ V) / M - I)
        v = ionic.step_state(prob, V, v, dt, prob.state_integrator)
        V = Vn
    return V, v
