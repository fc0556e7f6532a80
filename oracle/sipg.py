"""SIPG monodomain operator on a forest of boxes (Sec. 2.1).

The primal DG form (Eq. monodomain-primal-formulation) with the anisotropic
SIPG flux (Eq. monodomain-numerical-flux) is read as the standard symmetric
interior penalty bilinear form

  a(u, v) = sum_e int_e D grad u . grad v
          - sum_F int_F ( {D grad u} . [v] + {D grad v} . [u] )
          + sum_F int_F kappa_F [u] . [v],

  [w] = w+ n+ + w- n-,  {w} = (w+ + w-)/2,
  kappa_F = gamma * ( n.D+ n / h+ + n.D- n / h- ) / 2,

with h the element extent normal to F, F running over interior faces only
(zero flux on the outer boundary, Eq. monodomain C), and K = -A, A_ij = a(psi_j, psi_i)
(Eq. monodomain-ode-massmatrix-form).  The paper writes the face terms with a
'+' sign and the penalty inside the flux; read literally that is destabilising,
so the standard SIPG signs are used -- they are fixed by the symmetry, the
semi-definiteness with A 1 = 0, and the convergence order checked in the tests.

D = (sigma_t I + (sigma_l - sigma_t) f f^T) / (chi C_m)   (Eq. contGal, D = kappa / (chi C_m)).

Hanging faces (2:1): every fine subface is integrated with the fine face GL rule,
the coarse side's trace being evaluated at the mapped points.

Two independent routes compute A u: ``assemble`` builds the global sparse matrix
from element and face blocks evaluated by quadrature with the general basis
evaluation (the paper's own pre-assembled design, Sec. 2.3), and
``apply_matrix_free`` applies the operator by 1D sum factorisation of traces and
derivatives.  The tests require them to agree.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
from __future__ import annotations

import math
from typing import Dict, List, Tuple

import numpy as np
import scipy.sparse as sp

from . import basis
from .forest import Forest


def diffusion_tensor(prob) -> np.ndarray:
    """D = kappa / (chi C_m) with kappa = sigma_t I + (sigma_l - sigma_t) f f^T."""
    d = prob.dim
    f = np.array(prob.fibre[:d], dtype=np.float64)
    nf = np.linalg.norm(f)
    f = f / nf if nf > 0 else np.eye(d)[0]
    kappa = prob.sigma_t * np.eye(d) + (prob.sigma_l - prob.sigma_t) * np.outer(f, f)
    return kappa / (prob.chi * prob.cm)


class Disc:
    """Discretisation of one problem on one forest."""

    def __init__(self, prob, forest: Forest):
        self.prob = prob
        self.forest = forest
        self.dim = prob.dim
        self.p = prob.order
        self.n1 = self.p + 1
        self.n_p = self.n1 ** self.dim
        self.D = diffusion_tensor(prob)
        self.gamma = float(prob.gamma)
        self.nodes, self.weights = basis.gauss_legendre(self.p)
        self.ne = forest.n
        self.levels = np.array([lf[0] for lf in forest.leaves], dtype=np.int64)
        self._blocks = {}
        self._faces()
        self.M = self.mass()

    # ------------------------------------------------------------------
    def _faces(self):
        """Interior (sub)faces as records (minus, plus, axis, (lm, lp, pos))."""
        f = self.forest
        recs = []
        for i, lf in enumerate(f.leaves):
            lvl = lf[0]
            for k in range(self.dim):
                nb = f.neighbour(lf, k, +1)
                if nb[0] == 'same':
                    recs.append((i, nb[1], k, (lvl, lvl, ())))
                elif nb[0] == 'finer':
                    for b, j in enumerate(nb[1]):
                        pos = tuple((b >> t) & 1 for t in range(self.dim - 1))
                        recs.append((i, j, k, (lvl, lvl + 1, pos)))
                elif nb[0] == 'coarser':
                    recs.append((i, nb[1], k, (lvl, lvl - 1, tuple(nb[2]))))
        self.faces = recs

    def mass(self) -> np.ndarray:
        """Diagonal GL mass M_q = w_q det J per DOF (Sec. 2.1: collocation makes M diagonal)."""
        wq = basis.node_weights(self.dim, self.p)
        detj = np.array([np.prod(self.forest.h(l) / 2.0) for l in range(self.forest.L + 1)])
        return (detj[self.levels][:, None] * wq[None, :]).reshape(-1)

    def leaf_arrays(self):
        """(level (ne,), integer coordinates (ne, dim)) of the leaves."""
        c = np.array([lf[1][:self.dim] for lf in self.forest.leaves], dtype=np.int64).reshape(-1, self.dim)
        return self.levels, c

    def node_coords(self) -> np.ndarray:
        """Physical coordinates of every DOF node, (ne * n_p, dim): lower + (xi + 1)/2 h."""
        xi = basis.node_points(self.dim, self.p)
        lv, c = self.leaf_arrays()
        hs = np.array([self.forest.h(l) for l in range(self.forest.L + 1)])   # (L+1, dim)
        h = hs[lv]                                                            # (ne, dim)
        lower = c * h
        out = lower[:, None, :] + (xi[None, :, :] + 1.0) * 0.5 * h[:, None, :]
        return out.reshape(-1, self.dim)

    # ------------------------------------------------------------------
    # Local blocks by quadrature with general basis evaluation.
    # ------------------------------------------------------------------
    def volume_block(self, level: int) -> np.ndarray:
        """A_e[i, j] = sum_q W_q grad psi_i(x_q) . D grad psi_j(x_q)."""
        key = ('vol', int(level))
        if key not in self._blocks:
            self._blocks[key] = self._volume_block(level)
        return self._blocks[key]

    def _volume_block(self, level: int) -> np.ndarray:
        h = self.forest.h(level)
        xi = basis.node_points(self.dim, self.p)
        W = basis.node_weights(self.dim, self.p) * np.prod(h / 2.0)
        _, dphi = basis.eval_basis(self.dim, self.p, xi)
        g = dphi * (2.0 / h)[None, None, :]           # physical gradients (q, j, l)
        Dg = np.einsum('kl,qjl->qjk', self.D, g)        # D grad psi_j
        return np.einsum('q,qik,qjk->ij', W, g, Dg)

    def _face_geometry(self, k: int, sig):
        """Canonical placement of the two sides of a face of signature sig = (lm, lp, pos).

        Returns (xm, hm, xp, hp, xf_lower, hf): lower corners and extents of the
        minus/plus elements and the lower corner / extents of the (finer) face.
        """
        lm, lp, pos = sig
        hm = self.forest.h(lm)
        hp = self.forest.h(lp)
        d = self.dim
        tang = [l for l in range(d) if l != k]
        xm = np.zeros(d)
        xp = np.zeros(d)
        xp[k] = hm[k]
        if lp == lm + 1:            # plus side finer
            for t, l in enumerate(tang):
                xp[l] = pos[t] * hp[l]
            xf, hf = xp.copy(), hp.copy()
        elif lp == lm - 1:          # minus side finer
            for t, l in enumerate(tang):
                xm[l] = pos[t] * hm[l]
            xf, hf = xm.copy(), hm.copy()
        else:
            xf, hf = xm.copy(), hm.copy()
        xf[k] = hm[k]
        return xm, hm, xp, hp, xf, hf

    def _face_points(self, k: int, sig):
        """Face quadrature points (physical), weights, and both sides' basis values/gradients."""
        d = self.dim
        xm, hm, xp, hp, xf, hf = self._face_geometry(k, sig)
        tang = [l for l in range(d) if l != k]
        n1 = self.n1
        npts = n1 ** (d - 1)
        X = np.zeros((npts, d))
        W = np.ones(npts)
        for t_idx in range(npts):
            r = t_idx
            for l in tang:
                a = r % n1
                r //= n1
                X[t_idx, l] = xf[l] + (self.nodes[a] + 1.0) * 0.5 * hf[l]
                W[t_idx] *= self.weights[a] * hf[l] / 2.0
            X[t_idx, k] = xf[k]
        xim = 2.0 * (X - xm[None, :]) / hm[None, :] - 1.0
        xip = 2.0 * (X - xp[None, :]) / hp[None, :] - 1.0
        xim[:, k] = 1.0
        xip[:, k] = -1.0
        phim, dphim = basis.eval_basis(d, self.p, xim)
        phip, dphip = basis.eval_basis(d, self.p, xip)
        gm = dphim * (2.0 / hm)[None, None, :]
        gp = dphip * (2.0 / hp)[None, None, :]
        return X, W, (phim, gm, hm), (phip, gp, hp), hf

    def kappa(self, k: int, hm, hp) -> float:
        """kappa_F = gamma * (n.D n / h- + n.D n / h+) / 2 with h the extents normal to F."""
        Dnn = self.D[k, k]
        return self.gamma * 0.5 * (Dnn / hm[k] + Dnn / hp[k])

    def face_block(self, k: int, sig) -> np.ndarray:
        """Cached face block (the block only depends on the axis and the signature)."""
        key = ('face', k, sig)
        if key not in self._blocks:
            self._blocks[key] = self._face_block(k, sig)
        return self._blocks[key]

    def _face_block(self, k: int, sig) -> np.ndarray:
        """2 n_p x 2 n_p block of one interior (sub)face; rows/cols [minus DOFs, plus DOFs].

        For test psi_i on side s and trial psi_j on side t (sign + on the minus
        side, - on the plus side, n the minus side's outward normal e_k):
          B = sum_pts W [ -1/2 (D grad psi_j^t . n) sgn_s psi_i^s
                          -1/2 (D grad psi_i^s . n) sgn_t psi_j^t
                          + kappa sgn_s sgn_t psi_i^s psi_j^t ].
        """
        X, W, (phim, gm, hm), (phip, gp, hp), _ = self._face_points(k, sig)
        kap = self.kappa(k, hm, hp)
        phi = np.concatenate([phim, phip], axis=1)                 # (pts, 2np)
        flux = np.concatenate([np.einsum('l,qjl->qj', self.D[k], gm),
                               np.einsum('l,qjl->qj', self.D[k], gp)], axis=1)  # D grad psi . e_k
        sgn = np.concatenate([np.ones(self.n_p), -np.ones(self.n_p)])
        B = (-0.5 * np.einsum('q,qj,i,qi->ij', W, flux, sgn, phi)
             - 0.5 * np.einsum('q,qi,j,qj->ij', W, flux, sgn, phi)
             + kap * np.einsum('q,i,j,qi,qj->ij', W, sgn, sgn, phi, phi))
        return B

    # ------------------------------------------------------------------
    def assemble(self) -> sp.csr_matrix:
        """Global SIPG matrix A (so that M dphi/dt = -A phi - M I), by element and face blocks."""
        n_p = self.n_p
        rows, cols, vals = [], [], []
        li = np.arange(n_p)
        for lvl in np.unique(self.levels):
            B = self.volume_block(int(lvl))
            els = np.nonzero(self.levels == lvl)[0]
            r = (els[:, None, None] * n_p + li[None, :, None]) + 0 * li[None, None, :]
            c = (els[:, None, None] * n_p + li[None, None, :]) + 0 * li[None, :, None]
            rows.append(r.ravel()); cols.append(c.ravel())
            vals.append(np.broadcast_to(B[None], (len(els), n_p, n_p)).ravel())
        groups: Dict[Tuple, List[Tuple[int, int]]] = {}
        for (m, p, k, sig) in self.faces:
            groups.setdefault((k, sig), []).append((m, p))
        for (k, sig), pairs in groups.items():
            B = self.face_block(k, sig)
            pairs = np.array(pairs, dtype=np.int64)
            dof = np.concatenate([pairs[:, 0:1] * n_p + li[None, :],
                                  pairs[:, 1:2] * n_p + li[None, :]], axis=1)  # (nf, 2np)
            r = np.broadcast_to(dof[:, :, None], (len(pairs), 2 * n_p, 2 * n_p))
            c = np.broadcast_to(dof[:, None, :], (len(pairs), 2 * n_p, 2 * n_p))
            rows.append(r.ravel()); cols.append(c.ravel())
            vals.append(np.broadcast_to(B[None], (len(pairs), 2 * n_p, 2 * n_p)).ravel())
        N = self.ne * n_p
        A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(N, N)).tocsr()
        A.sum_duplicates()
        return A

    # ------------------------------------------------------------------
    # Matrix-free apply by 1D sum factorisation (independent second route).
    # ------------------------------------------------------------------
    def _ax(self, k: int) -> int:
        """Array axis of reference direction k in the (e, a_{d-1}, ..., a_0) DOF layout."""
        return self.dim - k

    def _apply1d(self, U: np.ndarray, Mat: np.ndarray, k: int) -> np.ndarray:
        ax = self._ax(k)
        Ut = np.moveaxis(U, ax, -1)
        R = Ut @ Mat.T
        return np.moveaxis(R, -1, ax)

    def apply_matrix_free(self, u: np.ndarray) -> np.ndarray:
        d, n1 = self.dim, self.n1
        shape = (self.ne,) + (n1,) * d
        U = np.asarray(u, dtype=np.float64).reshape(shape)
        R = np.zeros(shape)
        nodes = self.nodes
        _, D1 = basis.basis_1d(nodes, nodes)           # D1[i, j] = l_j'(x_i)
        # node_weights is ordered with a_0 fastest; reshape to (a_{d-1}, ..., a_0)
        wq = basis.node_weights(d, self.p).reshape((n1,) * d)
        # volume: sum_k (2/h_k) D1_k^T [ W (sum_l D_kl (2/h_l) D1_l u) ]
        for lvl in np.unique(self.levels):
            els = np.nonzero(self.levels == lvl)[0]
            h = self.forest.h(int(lvl))
            Ue = U[els]
            W = wq[None] * np.prod(h / 2.0)
            G = [self._apply1d(Ue, D1, l) * (2.0 / h[l]) for l in range(d)]
            for k in range(d):
                Fk = sum(self.D[k, l] * G[l] for l in range(d))
                R[els] += self._apply1d(W * Fk, D1.T, k) * (2.0 / h[k])
        # faces
        bL = np.array([basis.lagrange(nodes, j, -1.0) for j in range(n1)])
        bR = np.array([basis.lagrange(nodes, j, 1.0) for j in range(n1)])
        dL = np.array([basis.lagrange_deriv(nodes, j, -1.0) for j in range(n1)])
        dR = np.array([basis.lagrange_deriv(nodes, j, 1.0) for j in range(n1)])
        # interpolation from a coarse face onto half c of it: P_c[i, m] = l_m((x_i + 2c - 1)/2)
        P = [basis.basis_1d(nodes, (nodes - 1.0) / 2.0), basis.basis_1d(nodes, (nodes + 1.0) / 2.0)]
        groups: Dict[Tuple, List[Tuple[int, int]]] = {}
        for (m, p, k, sig) in self.faces:
            groups.setdefault((k, sig), []).append((m, p))
        for (k, sig), pairs in groups.items():
            pairs = np.array(pairs, dtype=np.int64)
            lm, lp, pos = sig
            hm, hp = self.forest.h(lm), self.forest.h(lp)
            tang = [l for l in range(d) if l != k]
            # fine side decides the face points; coarse side interpolated with P_pos
            coarse_m = (lp == lm + 1)
            coarse_p = (lp == lm - 1)
            hf = hp if coarse_m else hm
            Wf = np.ones((n1,) * d)
            for t, l in enumerate(tang):
                w1 = self.weights * hf[l] / 2.0
                shp = [1] * d
                shp[self._ax(l) - 1] = n1
                Wf = Wf * w1.reshape(shp)
            # collapse the normal axis to size 1
            Wf = np.take(Wf, [0], axis=self._ax(k) - 1)

            def side(Uside, h, bnd, dnd, coarse):
                tr = self._apply1d(Uside, bnd[None, :], k)             # trace at face nodes
                dn = self._apply1d(Uside, dnd[None, :], k) * (2.0 / h[k])
                grads = {k: dn}
                for l in tang:
                    grads[l] = self._apply1d(tr, D1, l) * (2.0 / h[l])
                if coarse:
                    def interp(X, lderiv=None):
                        for t, l in enumerate(tang):
                            Bm, Gm = P[pos[t]]
                            X = self._apply1d(X, Gm if l == lderiv else Bm, l)
                        return X
                    tr_i = interp(tr)
                    grads_i = {k: interp(dn)}
                    for l in tang:
                        grads_i[l] = interp(tr, lderiv=l) * (2.0 / h[l])
                    return tr_i, grads_i
                return tr, grads

            def side_T(C_val, C_grad, h, bnd, dnd, coarse):
                """Adjoint of side(): maps coefficient fields at face points back to DOFs."""
                out = 0.0
                if coarse:
                    def interpT(X, lderiv=None):
                        for t, l in enumerate(tang):
                            Bm, Gm = P[pos[t]]
                            X = self._apply1d(X, (Gm if l == lderiv else Bm).T, l)
                        return X
                    tr_c = interpT(C_val)
                    dn_c = interpT(C_grad[k]) * (2.0 / h[k])
                    for l in tang:
                        tr_c = tr_c + interpT(C_grad[l], lderiv=l) * (2.0 / h[l])
                else:
                    tr_c = C_val
                    dn_c = C_grad[k] * (2.0 / h[k])
                    for l in tang:
                        tr_c = tr_c + self._apply1d(C_grad[l], D1.T, l) * (2.0 / h[l])
                out = self._apply1d(tr_c, bnd[:, None], k) + self._apply1d(dn_c, dnd[:, None], k)
                return out

            Um = U[pairs[:, 0]]
            Up = U[pairs[:, 1]]
            trm, gm = side(Um, hm, bR, dR, coarse_m)
            trp, gp = side(Up, hp, bL, dL, coarse_p)
            kap = self.kappa(k, hm, hp)
            jump = trm - trp
            fm = sum(self.D[k, l] * gm[l] for l in range(d))
            fp = sum(self.D[k, l] * gp[l] for l in range(d))
            favg = 0.5 * (fm + fp)
            Wb = Wf[None]
            # minus side tests: value part  W(-favg + kap jump);  gradient part  -1/2 W jump D_k.
            cval_m = Wb * (-favg + kap * jump)
            cval_p = Wb * (favg - kap * jump)
            cg = {l: -0.5 * Wb * jump * self.D[k, l] for l in range(d)}
            rm = side_T(cval_m, cg, hm, bR, dR, coarse_m)
            rp = side_T(cval_p, cg, hp, bL, dL, coarse_p)
            np.add.at(R, pairs[:, 0], rm)
            np.add.at(R, pairs[:, 1], rp)
        return R.reshape(-1)

    # ------------------------------------------------------------------
    def cfl(self, A: sp.csr_matrix = None) -> np.ndarray:
        """Gershgorin bound (Eq. cfl-monodomain) per element.

        L_e = M_e^{-1} K_e with K_e the element's own diagonal block of K = -A;
        CFL_e = min_i 1 / (|L_ii| + sum_{j != i} |L_ij|)  (absolute value on the
        diagonal: K is negative semi-definite, the bound is on |lambda|).
        """
        if A is None:
            A = self.assemble()
        n_p = self.n_p
        C = A.tocoo()
        own = (C.row // n_p) == (C.col // n_p)
        rows, cols, vals = C.row[own], C.col[own], C.data[own]
        Ke = np.zeros((self.ne, n_p, n_p))
        np.add.at(Ke, (rows // n_p, rows % n_p, cols % n_p), -vals)
        L = Ke / self.M.reshape(self.ne, n_p)[:, :, None]
        return 1.0 / np.max(np.abs(L).sum(axis=2), axis=1)

    # ------------------------------------------------------------------
    def _eta_s_groups(self):
        """The faces grouped by (axis, signature) with each group's face data: the flux rows
        D grad psi . e_k of both sides at the face points, the weights, h_F and W_F (fixed
        for a mesh: built once per Disc)."""
        if getattr(self, "_eta_groups", None) is None:
            groups: Dict[Tuple, List[Tuple[int, int]]] = {}
            for (m, p, k, sig) in self.faces:
                groups.setdefault((k, sig), []).append((m, p))
            out = []
            for (k, sig), pairs in groups.items():
                X, W, (phim, gm, hm), (phip, gp, hp), hf = self._face_points(k, sig)
                fm = np.einsum('l,qjl->qj', self.D[k], gm)
                fp = np.einsum('l,qjl->qj', self.D[k], gp)
                area = np.prod([hf[l] for l in range(self.dim) if l != k])
                hF = area ** (1.0 / (self.dim - 1))
                WF = area / 2.0 ** (self.dim - 1)
                out.append((np.array(pairs, dtype=np.int64), fm, fp, W, hF, WF))
            self._eta_groups = out
        return self._eta_groups

    def eta_s(self, u: np.ndarray) -> np.ndarray:
        """Kelly-type spatial indicator (Eq. dg-error-estimate).

        eta_e = sqrt( sum_{F in faces of e} h_F / (2p) || W_F [D grad phi . n] ||^2_{L2(F)} )
        reading: h_F = |F|^(1/(d-1)), W_F = |F| / 2^(d-1) (the face map's Jacobian
        determinant), the norm over the physical (sub)face by its GL rule, boundary
        faces contributing nothing, hanging faces summed over their subfaces.
        """
        n_p = self.n_p
        U = np.asarray(u, dtype=np.float64).reshape(self.ne, n_p)
        acc = np.zeros(self.ne)
        for pairs, fm, fp, W, hF, WF in self._eta_s_groups():
            J = U[pairs[:, 0]] @ fm.T - U[pairs[:, 1]] @ fp.T      # (nf, pts)
            c = hF / (2.0 * self.p) * ((WF * J) ** 2 * W[None, :]).sum(axis=1)
            np.add.at(acc, pairs[:, 0], c)
            np.add.at(acc, pairs[:, 1], c)
        return np.sqrt(acc)


def eval_element(disc: Disc, e: int, u_e: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Value of element e's polynomial (DOFs u_e) at physical points x (m, dim)."""
    lf = disc.forest.leaves[e]
    h = disc.forest.h(lf[0])
    xi = 2.0 * (np.atleast_2d(x) - disc.forest.lower(lf)[None, :]) / h[None, :] - 1.0
    phi, _ = basis.eval_basis(disc.dim, disc.p, xi)
    return phi @ u_e
