"""Nodal basis of the GL-collocated DG space (Sec. 2.1, paragraph after Eq. monodomain-ode-form).

The ansatz and test spaces are tensor-product Lagrange polynomials whose nodes
are the roots of the Legendre polynomial (the Gauss-Legendre points), and all
integrals use the same Gauss-Legendre rule, so the mass matrix is diagonal and
the ionic term is pointwise.  Reference element [-1, 1]^d.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
from __future__ import annotations

import numpy as np


def gauss_legendre(p: int):
    """(p+1)-point Gauss-Legendre nodes and weights on [-1, 1]."""
    x, w = np.polynomial.legendre.leggauss(p + 1)
    return np.asarray(x, dtype=np.float64), np.asarray(w, dtype=np.float64)


def lagrange(nodes: np.ndarray, j: int, x) -> np.ndarray:
    """l_j(x) = prod_{m != j} (x - x_m) / (x_j - x_m)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.ones_like(x)
    for m in range(len(nodes)):
        if m != j:
            out = out * (x - nodes[m]) / (nodes[j] - nodes[m])
    return out


def lagrange_deriv(nodes: np.ndarray, j: int, x) -> np.ndarray:
    """l_j'(x) by the product rule: sum_k 1/(x_j - x_k) prod_{m != j,k} (x - x_m)/(x_j - x_m)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    for k in range(len(nodes)):
        if k == j:
            continue
        term = np.full_like(x, 1.0 / (nodes[j] - nodes[k]))
        for m in range(len(nodes)):
            if m != j and m != k:
                term = term * (x - nodes[m]) / (nodes[j] - nodes[m])
        out = out + term
    return out


def basis_1d(nodes: np.ndarray, x):
    """Matrices B[i, j] = l_j(x_i) and G[i, j] = l_j'(x_i) for points x."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    B = np.stack([lagrange(nodes, j, x) for j in range(n)], axis=1)
    G = np.stack([lagrange_deriv(nodes, j, x) for j in range(n)], axis=1)
    return B, G


def local_index(dim: int, p: int):
    """Tensor index (a_0, a_1[, a_2]) of each local DOF; x index fastest."""
    n1 = p + 1
    idx = []
    for q in range(n1 ** dim):
        a = []
        r = q
        for _ in range(dim):
            a.append(r % n1)
            r //= n1
        idx.append(tuple(a))
    return np.array(idx, dtype=np.int64)


def eval_basis(dim: int, p: int, xi: np.ndarray):
    """Values and reference gradients of all (p+1)^dim basis functions at points xi (m, dim).

    Returns (phi (m, n_p), dphi (m, n_p, dim)).
    """
    nodes, _ = gauss_legendre(p)
    xi = np.atleast_2d(np.asarray(xi, dtype=np.float64))
    A = local_index(dim, p)
    B = []
    G = []
    for k in range(dim):
        b, g = basis_1d(nodes, xi[:, k])
        B.append(b)
        G.append(g)
    m = xi.shape[0]
    n_p = A.shape[0]
    phi = np.ones((m, n_p))
    dphi = np.ones((m, n_p, dim))
    for q in range(n_p):
        for k in range(dim):
            phi[:, q] *= B[k][:, A[q, k]]
            for l in range(dim):
                dphi[:, q, l] *= (G[k][:, A[q, k]] if k == l else B[k][:, A[q, k]])
    return phi, dphi


def node_points(dim: int, p: int) -> np.ndarray:
    """Reference coordinates of the local nodes (= volume quadrature points), (n_p, dim)."""
    nodes, _ = gauss_legendre(p)
    A = local_index(dim, p)
    return nodes[A]


def node_weights(dim: int, p: int) -> np.ndarray:
    """Tensor GL weights of the local nodes, (n_p,)."""
    _, w = gauss_legendre(p)
    A = local_index(dim, p)
    return np.prod(w[A], axis=1)
