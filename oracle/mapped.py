"""SIPG operator on a forest mapped to a curved domain (Sec. 2.1 on curved elements, Sec. 3.3).

The bilinear form is the one of ``sipg`` (Eq. monodomain-primal-formulation with the flux
of Eq. monodomain-numerical-flux), now on the images of the reference elements under the
map x = Phi(X) of ``geometry``.  Everything is evaluated at the same GL points as on the
box, with the element Jacobian J = DPhi(X) diag(h / 2):

  mass          M_q = w_q det(h/2) |det DPhi(X_q)|                 (diagonal GL mass)
  gradients     grad psi = DPhi^-T g, g the box gradient diag(2/h) grad_xi psi
  volume        A_e[i, j] = sum_q M_q grad psi_i . D(x_q) grad psi_j
  face point    normal n = DPhi^-T e_k / |DPhi^-T e_k| (e_k the reference normal),
                area weight dS = W_box |det DPhi| |DPhi^-T e_k| (Nanson's formula),
                element extent normal to the face h_n = h_k / |DPhi^-T e_k|,
                kappa = gamma n.D n (1/h_n- + 1/h_n+) / 2,
and the face block has the terms of ``sipg.Disc._face_block`` with these values at each
point.  Both sides of a face see the same physical point and the same DPhi there (the map
is global), so the two traces meet exactly on conforming and on hanging faces.

The diffusion tensor is constant (the problem's fibre) or, with ``prob.fibre_ref``, has
its fibre along the image of the first reference axis, f = DPhi e_0 / |DPhi e_0|, at
every point.

With an affine map the element maps are affine and every integrand is a polynomial the GL
rule integrates exactly, as on the box.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import basis, geometry
from .sipg import Disc


def tensor_at(prob, J: np.ndarray) -> np.ndarray:
    """D = (sigma_t I + (sigma_l - sigma_t) f f^T) / (chi C_m) at points with DPhi = J (N, d, d)."""
    d = prob.dim
    n = J.shape[0]
    if prob.fibre_ref:
        f = J[:, :, 0] / np.linalg.norm(J[:, :, 0], axis=1)[:, None]
    else:
        f0 = np.array(prob.fibre[:d], dtype=np.float64)
        nf = np.linalg.norm(f0)
        f0 = f0 / nf if nf > 0 else np.eye(d)[0]
        f = np.broadcast_to(f0, (n, d))
    kappa = prob.sigma_t * np.eye(d)[None] + (prob.sigma_l - prob.sigma_t) * np.einsum('ni,nj->nij', f, f)
    return kappa / (prob.chi * prob.cm)


class MappedDisc(Disc):
    """Discretisation of one problem on one forest under the problem's map."""

    def __init__(self, prob, forest):
        super().__init__(prob, forest)

    def ref_coords(self) -> np.ndarray:
        """Reference (box) coordinates of every DOF node."""
        return Disc.node_coords(self)

    def node_coords(self) -> np.ndarray:
        """Physical coordinates of every DOF node: Phi of the reference node."""
        return geometry.phi(self.prob, self.ref_coords())

    def mass(self) -> np.ndarray:
        box = Disc.mass(self)
        J = geometry.dphi(self.prob, self.ref_coords())
        return box * np.abs(np.linalg.det(J))

    def _lower(self, e: int) -> np.ndarray:
        lvl, c = self.forest.leaves[e][0], self.forest.leaves[e][1]
        return np.array(c[:self.dim], dtype=np.float64) * self.forest.h(lvl)

    def element_volume_block(self, e: int) -> np.ndarray:
        lvl = self.forest.leaves[e][0]
        h = self.forest.h(lvl)
        xi = basis.node_points(self.dim, self.p)
        X = self._lower(e)[None, :] + (xi + 1.0) * 0.5 * h[None, :]
        J = geometry.dphi(self.prob, X)
        W = basis.node_weights(self.dim, self.p) * np.prod(h / 2.0) * np.abs(np.linalg.det(J))
        _, dphi_ref = basis.eval_basis(self.dim, self.p, xi)
        g = dphi_ref * (2.0 / h)[None, None, :]                       # box gradients (q, j, l)
        Jit = np.linalg.inv(J).transpose(0, 2, 1)                      # DPhi^-T
        gm = np.einsum('qkl,qjl->qjk', Jit, g)                         # physical gradients
        D = tensor_at(self.prob, J)
        Dg = np.einsum('qkl,qjl->qjk', D, gm)
        return np.einsum('q,qik,qjk->ij', W, gm, Dg)

    def element_face_block(self, m: int, k: int, sig) -> np.ndarray:
        """2 n_p x 2 n_p block of the interior (sub)face of minus element m, normal axis k."""
        Xr, Wb, (phim, gmb, hm), (phip, gpb, hp), _ = self._face_points(k, sig)
        xm, _, _, _, _, _ = self._face_geometry(k, sig)
        X = Xr + (self._lower(m) - xm)[None, :]                         # reference points
        J = geometry.dphi(self.prob, X)
        Jit = np.linalg.inv(J).transpose(0, 2, 1)
        nk = Jit[:, :, k]                                               # DPhi^-T e_k
        ln = np.linalg.norm(nk, axis=1)
        n = nk / ln[:, None]
        dS = Wb * np.abs(np.linalg.det(J)) * ln
        D = tensor_at(self.prob, J)
        Dn = np.einsum('qkl,ql->qk', D, n)
        gm = np.einsum('qkl,qjl->qjk', Jit, gmb)
        gp = np.einsum('qkl,qjl->qjk', Jit, gpb)
        flux = np.concatenate([np.einsum('qk,qjk->qj', Dn, gm), np.einsum('qk,qjk->qj', Dn, gp)], axis=1)
        nDn = np.einsum('qk,qk->q', Dn, n)
        kap = self.gamma * nDn * 0.5 * (ln / hm[k] + ln / hp[k])        # 1/h_n = |DPhi^-T e_k| / h_k
        phi = np.concatenate([phim, phip], axis=1)
        sgn = np.concatenate([np.ones(self.n_p), -np.ones(self.n_p)])
        return (-0.5 * np.einsum('q,qj,i,qi->ij', dS, flux, sgn, phi)
                - 0.5 * np.einsum('q,qi,j,qj->ij', dS, flux, sgn, phi)
                + np.einsum('q,q,i,j,qi,qj->ij', dS, kap, sgn, sgn, phi, phi))

    def assemble(self) -> sp.csr_matrix:
        """Global SIPG matrix, element by element and face by face (no two blocks alike)."""
        n_p = self.n_p
        li = np.arange(n_p)
        rows, cols, vals = [], [], []
        for e in range(self.ne):
            B = self.element_volume_block(e)
            dof = e * n_p + li
            rows.append(np.repeat(dof, n_p)); cols.append(np.tile(dof, n_p)); vals.append(B.ravel())
        for (m, p, k, sig) in self.faces:
            B = self.element_face_block(m, k, sig)
            dof = np.concatenate([m * n_p + li, p * n_p + li])
            rows.append(np.repeat(dof, 2 * n_p)); cols.append(np.tile(dof, 2 * n_p)); vals.append(B.ravel())
        N = self.ne * n_p
        A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(N, N)).tocsr()
        A.sum_duplicates()
        return A

    def apply_matrix_free(self, u):
        raise NotImplementedError("mapped geometry: the oracle assembles the operator only")

    def eta_s(self, u: np.ndarray) -> np.ndarray:
        """Kelly-type spatial indicator (Eq. dg-error-estimate) on the mapped mesh:

        eta_e = sqrt( sum_{F of e} h_F / (2p) sum_t dS_t (W_F(t) [D grad phi . n](t))^2 ),
        with the physical face area |F| = sum_t dS_t, h_F = |F|^(1/(d-1)) and W_F(t) the
        face map's Jacobian at the point (dS_t over the reference GL weight), the jump taken
        with each side's own gradient at the shared physical point.  On a box this is the
        indicator of ``sipg.Disc.eta_s`` (W_F = |F| / 2^(d-1))."""
        n_p = self.n_p
        U = np.asarray(u, dtype=np.float64).reshape(self.ne, n_p)
        acc = np.zeros(self.ne)
        for (m, p, k, sig) in self.faces:
            Xr, Wb, (phim, gmb, hm), (phip, gpb, hp), hf = self._face_points(k, sig)
            xm, _, _, _, _, _ = self._face_geometry(k, sig)
            X = Xr + (self._lower(m) - xm)[None, :]
            J = geometry.dphi(self.prob, X)
            Jit = np.linalg.inv(J).transpose(0, 2, 1)
            nk = Jit[:, :, k]
            ln = np.linalg.norm(nk, axis=1)
            n = nk / ln[:, None]
            dS = Wb * np.abs(np.linalg.det(J)) * ln
            D = tensor_at(self.prob, J)
            Dn = np.einsum('qkl,ql->qk', D, n)
            gm = np.einsum('qkl,qjl->qjk', Jit, gmb)
            gp = np.einsum('qkl,qjl->qjk', Jit, gpb)
            jump = (np.einsum('qk,qjk,j->q', Dn, gm, U[m]) - np.einsum('qk,qjk,j->q', Dn, gp, U[p]))
            tang = [l for l in range(self.dim) if l != k]
            wref = Wb / np.prod([hf[l] / 2.0 for l in tang])             # reference GL weights
            WF = dS / wref
            area = dS.sum()
            hF = area ** (1.0 / (self.dim - 1))
            c = hF / (2.0 * self.p) * np.sum(dS * (WF * jump) ** 2)
            acc[m] += c
            acc[p] += c
        return np.sqrt(acc)
