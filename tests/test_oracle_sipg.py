"""Pins for the oracle's SIPG operator, CFL bound and spatial indicator.

Each check is independent of the oracle's own arithmetic: exact
integration of the bilinear form, invariants (symmetry, semi-definiteness,
constants in the kernel), the closed-form heat solution's convergence order,
and closed-form indicator values for piecewise-linear fields.
"""
import itertools
import math

import numpy as np
import pytest
import scipy.linalg

import workloads as W
from oracle import basis, lts
from oracle.forest import Forest
from oracle.sipg import Disc


def make_prob(dim, p, base, extent, D_iso=None, aniso=True, gamma=None):
    if D_iso is not None:
        return W.Problem(dim=dim, order=p, extent=extent, base=base, sigma_l=D_iso, sigma_t=D_iso,
                         chi=1.0, cm=1.0, gamma=gamma or 10.0 * p * p, ionic_model=-1, max_refine=3)
    fib = (0.6, 0.8, 0.0) if dim == 2 else (0.48, 0.64, 0.6)
    return W.Problem(dim=dim, order=p, extent=extent, base=base, sigma_l=1.2, sigma_t=0.4, fibre=fib,
                     chi=1.0, cm=1.0, gamma=gamma or 10.0 * p * p, ionic_model=-1, max_refine=3)


def hanging_forest(dim, base, extent, marks=((1,), (2,))):
    f = Forest(dim, base, 3, extent)
    for m in marks:
        eta = np.zeros(f.n)
        for i in m:
            eta[i % f.n] = 1.0
        f, _ = f.adapt(eta, 0.5, -1.0)
    return f


# --------------------------------------------------------------------------
# Exact integration of the SIPG bilinear form (brute force, no quadrature).
# --------------------------------------------------------------------------

def exact_A(prob, forest):
    """Exact A of a 2D mesh by exact integration of the bilinear form.

    Basis functions are products X_a(x) Y_b(y) of 1D Lagrange polynomials built
    from the closed-form nodes (+-1/sqrt(3), or 0, +-sqrt(3/5)) as explicit
    coefficient polynomials; every volume and (sub)face integral factorises
    into 1D polynomial integrals taken by exact antiderivatives (no quadrature
    rule involved).
    """
    from numpy.polynomial import Polynomial as Poly
    p = prob.order
    if p == 1:
        nodes = [-1 / math.sqrt(3), 1 / math.sqrt(3)]
    else:
        nodes = [-math.sqrt(0.6), 0.0, math.sqrt(0.6)]
    from oracle.sipg import diffusion_tensor
    D = diffusion_tensor(prob)
    gamma = float(prob.gamma)

    def lag_poly(j, x0, h):
        """l_j(2 (s - x0)/h - 1) as a polynomial in the physical coordinate s."""
        ref = Poly([-2.0 * x0 / h - 1.0, 2.0 / h])
        e = Poly([1.0])
        for m in range(p + 1):
            if m != j:
                e = e * (ref - nodes[m]) / (nodes[j] - nodes[m])
        return e

    def integ(P, lo, hi):
        I = P.integ()
        return I(hi) - I(lo)

    elems = []
    for lf in forest.leaves:
        lvl, c = lf
        h = [prob.extent[k] / (prob.base[k] * 2 ** lvl) for k in range(2)]
        x0 = [c[k] * h[k] for k in range(2)]
        F = []   # F[k][a] = (poly, derivative poly) of l_a along axis k in physical coordinate s
        for k in range(2):
            row = []
            for a in range(p + 1):
                P = lag_poly(a, x0[k], h[k])
                row.append((P, P.deriv()))
            F.append(row)
        elems.append(dict(x0=x0, h=h, F=F))
    n1 = p + 1
    n_p = n1 * n1
    N = len(elems) * n_p
    A = np.zeros((N, N))
    idx = [(q % n1, q // n1) for q in range(n_p)]      # (a along x, b along y)

    for e, E in enumerate(elems):
        lo = E['x0']; hi = [E['x0'][k] + E['h'][k] for k in range(2)]
        F = E['F']
        for i, (ai, bi) in enumerate(idx):
            for j, (aj, bj) in enumerate(idx):
                # d/dx psi = X' Y, d/dy psi = X Y'
                val = 0
                for k in range(2):
                    for l in range(2):
                        xi_ = F[0][ai][1 if k == 0 else 0]
                        yi_ = F[1][bi][1 if k == 1 else 0]
                        xj_ = F[0][aj][1 if l == 0 else 0]
                        yj_ = F[1][bj][1 if l == 1 else 0]
                        val += D[k][l] * integ(xi_ * xj_, lo[0], hi[0]) * integ(yi_ * yj_, lo[1], hi[1])
                A[e * n_p + i, e * n_p + j] += float(val)

    def face_fns(E, k, xF):
        """For each local DOF: (value, d/dx, d/dy) on the face x_k = xF as polys in the tangential coordinate."""
        t = 1 - k
        out = []
        for (a, b) in idx:
            an, at = (a, b) if k == 0 else (b, a)        # index along normal / tangential axis
            Pn, dPn = E['F'][k][an]
            Pt, dPt = E['F'][t][at]
            vn, dvn = Pn(xF), dPn(xF)
            val = Pt * vn
            dn = Pt * dvn
            dt = dPt * vn
            grads = [dn, dt] if k == 0 else [dt, dn]
            out.append((val, grads))
        return out

    for a, b in itertools.combinations(range(len(elems)), 2):
        for (mi, pi) in ((a, b), (b, a)):
            m, pl = elems[mi], elems[pi]
            for k in range(2):
                t = 1 - k
                if abs(m['x0'][k] + m['h'][k] - pl['x0'][k]) > 1e-12:
                    continue
                lo = max(m['x0'][t], pl['x0'][t])
                hi = min(m['x0'][t] + m['h'][t], pl['x0'][t] + pl['h'][t])
                if hi <= lo + 1e-12:
                    continue
                xF = m['x0'][k] + m['h'][k]
                kap = gamma * (D[k][k] / m['h'][k] + D[k][k] / pl['h'][k]) / 2
                sides = [(face_fns(m, k, xF), mi, 1), (face_fns(pl, k, xF), pi, -1)]
                for (Sf, si, ss) in sides:
                    for (Tf, ti, ts) in sides:
                        for i in range(n_p):
                            vi, gi = Sf[i]
                            fi = D[k][0] * gi[0] + D[k][1] * gi[1]
                            for j in range(n_p):
                                uj, gj = Tf[j]
                                fj = D[k][0] * gj[0] + D[k][1] * gj[1]
                                P = (-0.5 * ss) * (fj * vi) + (-0.5 * ts) * (fi * uj) \
                                    + (kap * ss * ts) * (vi * uj)
                                A[si * n_p + i, ti * n_p + j] += float(integ(P, lo, hi))
    return A


def test_exact_integration_two_elements_q1_anisotropic():
    prob = make_prob(2, 1, (2, 1, 1), (1.0, 0.5, 1.0))
    f = Forest(2, prob.base, 3, prob.extent)
    A = Disc(prob, f).assemble().toarray()
    S = exact_A(prob, f)
    assert np.abs(A - S).max() <= 1e-12 * np.abs(S).max()


def test_exact_integration_hanging_face_q1():
    prob = make_prob(2, 1, (2, 1, 1), (1.0, 0.5, 1.0))
    f = Forest(2, prob.base, 3, prob.extent)
    eta = np.array([0.0, 1.0])
    f, _ = f.adapt(eta, 0.5, -1.0)          # right root refined: 1 coarse + 4 fine, 2 hanging subfaces
    assert f.n == 5
    A = Disc(prob, f).assemble().toarray()
    S = exact_A(prob, f)
    assert np.abs(A - S).max() <= 1e-12 * np.abs(S).max()


def test_exact_integration_two_elements_q2():
    prob = make_prob(2, 2, (2, 1, 1), (1.0, 0.5, 1.0))
    f = Forest(2, prob.base, 3, prob.extent)
    A = Disc(prob, f).assemble().toarray()
    S = exact_A(prob, f)
    assert np.abs(A - S).max() <= 1e-12 * np.abs(S).max()


# --------------------------------------------------------------------------
# Invariants: symmetry, PSD, constants in the kernel, matrix-free == assembled.
# --------------------------------------------------------------------------

@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_operator_invariants_with_hanging_faces(dim, p):
    prob = make_prob(dim, p, (3, 2, 2), (1.0, 0.8, 0.6))
    f = hanging_forest(dim, prob.base, prob.extent)
    assert f.is_balanced()
    d = Disc(prob, f)
    assert any(s[0] != s[1] for (_, _, _, s) in d.faces)     # has hanging subfaces
    A = d.assemble().toarray()
    nrm = np.abs(A).max()
    assert np.abs(A - A.T).max() <= 1e-13 * nrm
    assert np.abs(A @ np.ones(A.shape[0])).max() <= 1e-13 * nrm
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert ev.min() >= -1e-12 * ev.max()
    # exactly one zero mode (connected mesh, zero-flux boundary)
    assert (ev < 1e-10 * ev.max()).sum() == 1
    rng = np.random.default_rng(3)
    for _ in range(3):
        u = rng.standard_normal(A.shape[0])
        mf = d.apply_matrix_free(u)
        assert np.abs(mf - A @ u).max() <= 1e-13 * np.abs(A @ u).max()
    # columns through the matrix-free route on unit vectors
    for j in rng.choice(A.shape[0], 5, replace=False):
        e = np.zeros(A.shape[0]); e[j] = 1.0
        assert np.abs(d.apply_matrix_free(e) - A[:, j]).max() <= 1e-13 * nrm


# --------------------------------------------------------------------------
# Closed-form heat solution: spatial convergence order p+1.
# --------------------------------------------------------------------------

def heat_error(dim, p, n, T=0.02, refine_patch=False):
    prob = make_prob(dim, p, (n, n, n), (1.0, 1.0, 1.0), D_iso=1.0)
    f = Forest(dim, prob.base, 3, prob.extent)
    if refine_patch:
        eta = np.zeros(f.n)
        for i, lf in enumerate(f.leaves):
            c = lf[1]
            if c[0] < n // 2 and c[1] < n // 2:
                eta[i] = 1.0
        f, _ = f.adapt(eta, 0.5, -1.0)
    d = Disc(prob, f)
    A = d.assemble().toarray()
    X = d.node_coords()
    lam = math.pi ** 2 * dim
    u0 = np.prod(np.cos(math.pi * X), axis=1) + 0.3
    ue = np.exp(-lam * T) * np.prod(np.cos(math.pi * X), axis=1) + 0.3
    Ms = np.sqrt(d.M)
    S = A / Ms[:, None] / Ms[None, :]
    w, Q = scipy.linalg.eigh(0.5 * (S + S.T))
    uT = (Q @ (np.exp(-T * w) * (Q.T @ (Ms * u0)))) / Ms
    return math.sqrt(np.sum(d.M * (uT - ue) ** 2))


@pytest.mark.parametrize("dim,p,ns", [(2, 1, (4, 8, 16)), (2, 2, (2, 4, 8)), (3, 1, (2, 4, 6))])
def test_heat_convergence_order(dim, p, ns):
    errs = [heat_error(dim, p, n) for n in ns]
    rates = [math.log(errs[i] / errs[i + 1]) / math.log(ns[i + 1] / ns[i]) for i in range(len(ns) - 1)]
    assert rates[-1] > p + 1 - 0.3, (errs, rates)


@pytest.mark.parametrize("p,ns", [(1, (4, 8, 16)), (2, (2, 4, 8))])
def test_heat_convergence_order_with_hanging_patch(p, ns):
    errs = [heat_error(2, p, n, refine_patch=True) for n in ns]
    rates = [math.log(errs[i] / errs[i + 1]) / math.log(ns[i + 1] / ns[i]) for i in range(len(ns) - 1)]
    assert rates[-1] > p + 1 - 0.35, (errs, rates)


# --------------------------------------------------------------------------
# CFL (Gershgorin) and element classes.
# --------------------------------------------------------------------------

@pytest.mark.parametrize("dim,p", [(2, 1), (3, 1), (2, 2)])
def test_own_block_classes_match_assembled_diagonal_blocks(dim, p):
    prob = make_prob(dim, p, (3, 2, 2), (1.0, 0.8, 0.6))
    f = hanging_forest(dim, prob.base, prob.extent)
    d = Disc(prob, f)
    A = d.assemble().toarray()
    code = {'boundary': 0, 'same': 1, 'coarser': 2, 'finer': 3}
    for e, lf in enumerate(f.leaves):
        cfg = [code[f.neighbour(lf, ax, s)[0]] for ax in range(dim) for s in (-1, 1)]
        Bo = lts.own_block(d, lf[0], cfg)
        s = slice(e * d.n_p, (e + 1) * d.n_p)
        assert np.abs(Bo - A[s, s]).max() <= 1e-13 * np.abs(A).max()


def test_gershgorin_against_exact_matrix():
    prob = make_prob(2, 1, (2, 1, 1), (1.0, 0.5, 1.0))
    f = Forest(2, prob.base, 3, prob.extent)
    d = Disc(prob, f)
    S = exact_A(prob, f)
    cfl = d.cfl()
    for e in range(2):
        s = slice(e * 4, (e + 1) * 4)
        L = -S[s, s] / d.M[s][:, None]
        ref = min(1.0 / (abs(L[i, i]) + sum(abs(L[i, j]) for j in range(4) if j != i)) for i in range(4))
        assert abs(cfl[e] - ref) <= 1e-12 * ref


def test_cfl_bound_gives_stable_forward_euler():
    """At dt = min CFL_e the pure-diffusion energy ||phi||_M never grows."""
    prob = make_prob(2, 1, (6, 6, 1), (1.0, 1.0, 1.0), D_iso=1.0)
    f = hanging_forest(2, prob.base, prob.extent, marks=((7, 14, 21),))
    d = Disc(prob, f)
    A = d.assemble()
    dt = d.cfl(A).min()
    rng = np.random.default_rng(5)
    V = rng.standard_normal(d.ne * d.n_p)
    E = np.sum(d.M * V * V)
    for _ in range(200):
        V = V - dt * (A @ V) / d.M
        En = np.sum(d.M * V * V)
        assert En <= E * (1 + 1e-12)
        E = En


# --------------------------------------------------------------------------
# Kelly-type indicator: closed forms.
# --------------------------------------------------------------------------

@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (3, 1)])
def test_eta_s_vanishes_for_linear_fields(dim, p):
    prob = make_prob(dim, p, (3, 2, 2), (1.0, 0.8, 0.6))
    f = hanging_forest(dim, prob.base, prob.extent)
    d = Disc(prob, f)
    X = d.node_coords()
    u = 0.3 + X @ np.arange(1, dim + 1)
    assert np.abs(d.eta_s(u)).max() < 1e-12


@pytest.mark.parametrize("dim", [2, 3])
def test_eta_s_kink_closed_form(dim):
    """phi = max(0, x - x_F), x_F on an element face: only the two neighbours of that
    face see a flux jump D_xx, so eta_e = sqrt(h_F/(2p) |F| (W_F D_xx)^2)."""
    n = 4
    prob = make_prob(dim, 1, (n, n, n), (1.0, 1.0, 1.0))
    f = Forest(dim, prob.base, 3, prob.extent)
    d = Disc(prob, f)
    X = d.node_coords()
    xF = 0.5
    u = np.maximum(0.0, X[:, 0] - xF)
    es = d.eta_s(u)
    h = 1.0 / n
    area = h ** (dim - 1)
    hF = area ** (1.0 / (dim - 1))
    WF = area / 2 ** (dim - 1)
    ref = math.sqrt(hF / 2.0 * area * (WF * d.D[0, 0]) ** 2)
    for e, lf in enumerate(f.leaves):
        cx = lf[1][0]
        expect = ref if cx in (n // 2 - 1, n // 2) else 0.0
        assert abs(es[e] - expect) <= 1e-12 * ref + 1e-18


# --------------------------------------------------------------------------
# Statements of the paper (tests/golden/paper_statements.json).
# --------------------------------------------------------------------------

def paper_statements():
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_statements.json")) as fh:
        return json.load(fh)


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (3, 1)])
def test_refinement_divides_cfl_by_four(dim, p):
    """Sec. 2.3: one refinement divides the stable step by about 4 (CFL_e ~ h^2 on box meshes)."""
    g = paper_statements()["cfl_refinement_ratio"]
    prob = make_prob(dim, p, (3, 3, 3), (1.0, 1.0, 1.0), D_iso=1.0)
    f = Forest(dim, prob.base, 3, prob.extent)
    # the interior element of the base grid, and of the uniformly refined grid
    c0 = Disc(prob, f).cfl()
    f1, _ = f.adapt(np.ones(f.n), 0.5, -1.0)
    c1 = Disc(prob, f1).cfl()
    ratio = c0.min() / c1.min()
    assert abs(ratio - g["value"]) <= g["rel_tol"] * g["value"]


def test_larger_penalty_lowers_cfl_bound():
    """Sec. 3.3: gamma = 8 decreases the CFL bound relative to gamma = 4."""
    g = paper_statements()["penalty_reference"]["value"]
    cfls = []
    for gamma in (g, 2 * g):
        prob = make_prob(2, 1, (4, 4, 1), (1.0, 1.0, 1.0), gamma=gamma)
        cfls.append(Disc(prob, Forest(2, prob.base, 3, prob.extent)).cfl().min())
    assert cfls[1] < cfls[0]


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2)])
def test_small_penalty_loses_semidefiniteness(dim, p):
    """Sec. 3.3: penalties << 4 are unstable; the SIPG operator then has a negative eigenvalue,
    while at gamma = 4 it is positive semi-definite."""
    st = paper_statements()["penalty_unstable_below"]
    lam = {}
    for gamma in (st["value"], st["factor"] * st["value"]):
        prob = make_prob(dim, p, (3, 3, 1), (1.0, 1.0, 1.0), gamma=gamma)
        A = Disc(prob, Forest(dim, prob.base, 3, prob.extent)).assemble().toarray()
        lam[gamma] = np.linalg.eigvalsh(0.5 * (A + A.T)).min() / np.abs(A).max()
    assert lam[st["value"]] >= -1e-12
    assert lam[st["factor"] * st["value"]] < -1e-6
