"""Shared test helpers: moving meshes and states between the oracle and the library."""
import math

import numpy as np

import workloads as W


def mass_rel_l2(M, a, b):
    """||a - b||_M / ||b||_M (M = diagonal GL mass per DOF)."""
    return math.sqrt(np.sum(M * (a - b) ** 2) / max(np.sum(M * b * b), 1e-300))


def forest_arrays(forest):
    """(level int8, coords int32 (n, dim), root int32) of an oracle forest, in its leaf order."""
    d = forest.dim
    lv = np.array([lf[0] for lf in forest.leaves], dtype=np.int8)
    cc = np.array([lf[1][:d] for lf in forest.leaves], dtype=np.int32).reshape(-1, d)
    b = forest.base
    root = np.array([(lf[1][0] >> lf[0]) + b[0] * ((lf[1][1] >> lf[0]) + b[1] * ((lf[1][2] >> lf[0]) if d == 3 else 0))
                     for lf in forest.leaves], dtype=np.int32)
    return lv, cc, root


def oracle_face_table(forest):
    """Face table of an oracle forest in the library's read_faces layout."""
    d = forest.dim
    nf, ns = 2 * d, 1 << (d - 1)
    n = forest.n
    kind = np.zeros((n, nf), np.int8)
    nbr = -np.ones((n, nf, ns), np.int32)
    pos = np.zeros((n, nf), np.int8)
    code = {'boundary': 0, 'same': 1, 'coarser': 2, 'finer': 3}
    for i, lf in enumerate(forest.leaves):
        for ax in range(d):
            for s in (-1, 1):
                f = 2 * ax + (1 if s > 0 else 0)
                nb = forest.neighbour(lf, ax, s)
                kind[i, f] = code[nb[0]]
                if nb[0] in ('same',):
                    nbr[i, f, 0] = nb[1]
                elif nb[0] == 'coarser':
                    nbr[i, f, 0] = nb[1]
                    pos[i, f] = sum(bit << t for t, bit in enumerate(nb[2]))
                elif nb[0] == 'finer':
                    nbr[i, f, :] = nb[1]
    return kind, nbr, pos


def random_forest(dim, base, L, extent, steps=3, seed=0, tau=0.8):
    from oracle.forest import Forest
    f = Forest(dim, base, L, extent)
    rng = np.random.default_rng(seed)
    for _ in range(steps):
        eta = rng.uniform(0, 1, f.n)
        f, _ = f.adapt(eta, tau, 0.15)
    return f
