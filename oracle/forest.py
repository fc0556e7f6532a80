"""Forest-of-trees h-refinement on a box slab (Sec. 2.2; Alg. 1, refine and coarsen steps).

Root elements form a regular base grid; refinement replaces a leaf by 2^d equal
children, coarsening reverts it.  Leaves are stored as (level, c) with c the
integer cell coordinate on the level-`level` grid, and ordered by
(root id, Morton key of the lower corner on the finest grid), so that the
children of one parent are contiguous in child order cx + 2 cy + 4 cz.

Readings taken where the paper delegates to MFEM:
  * 2:1 face balance is enforced (face neighbours differ by at most one level);
  * refine if eta >= tau_refine and level < max_refine (Alg. 1; Sec. 2.2 words the
    inequalities the other way round, Alg. 1 is followed);
  * then coarsen a complete family of leaves if every child has eta <= tau_coarsen,
    none was refined this step, and every face neighbour outside the family is no
    finer than the children (so the parent keeps 2:1);
  * refinement needed by the balance is closed over (refine coarser neighbours).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
from __future__ import annotations

from typing import Dict, List, Tuple

import numpy as np

Leaf = Tuple[int, Tuple[int, int, int]]  # (level, (cx, cy, cz))


class Forest:
    def __init__(self, dim: int, base, max_refine: int, extent):
        self.dim = dim
        self.base = tuple(int(b) for b in base[:3]) + (1,) * (3 - len(base))
        if dim == 2:
            self.base = (self.base[0], self.base[1], 1)
        self.L = int(max_refine)
        self.extent = tuple(float(e) for e in extent[:3])
        leaves = []
        for cz in range(self.base[2]):
            for cy in range(self.base[1]):
                for cx in range(self.base[0]):
                    leaves.append((0, (cx, cy, cz)))
        self.set_leaves(leaves)

    # ---------------- ordering ----------------
    def key(self, leaf: Leaf) -> int:
        lvl, c = leaf
        L = self.L
        root = [c[k] >> lvl for k in range(3)]
        rid = root[0] + self.base[0] * (root[1] + self.base[1] * root[2])
        loc = [(c[k] - (root[k] << lvl)) << (L - lvl) for k in range(3)]
        m = 0
        for bit in range(L):
            for k in range(self.dim):
                m |= ((loc[k] >> bit) & 1) << (bit * self.dim + k)
        return rid * (1 << (self.dim * L)) + m

    def set_leaves(self, leaves: List[Leaf]):
        self.leaves = sorted(leaves, key=self.key)
        self.index: Dict[Leaf, int] = {lf: i for i, lf in enumerate(self.leaves)}

    @property
    def n(self) -> int:
        return len(self.leaves)

    # ---------------- geometry ----------------
    def h(self, level: int) -> np.ndarray:
        return np.array([self.extent[k] / (self.base[k] * (1 << level)) for k in range(self.dim)])

    def lower(self, leaf: Leaf) -> np.ndarray:
        lvl, c = leaf
        h = self.h(lvl)
        return np.array([c[k] * h[k] for k in range(self.dim)])

    def ncells(self, level: int, k: int) -> int:
        return self.base[k] << level if (k < self.dim) else 1

    # ---------------- neighbours ----------------
    def neighbour(self, leaf: Leaf, axis: int, side: int):
        """Face neighbour across face (axis, side), side in {-1, +1}.

        Returns ('boundary',), ('same', j), ('coarser', j, pos) with pos the
        tangential position bits of this leaf on the coarse face, or
        ('finer', [j0, j1, ...]) ordered by tangential child bits.
        """
        lvl, c = leaf
        cn = list(c)
        cn[axis] += side
        if cn[axis] < 0 or cn[axis] >= self.ncells(lvl, axis):
            return ('boundary',)
        same = (lvl, tuple(cn))
        if same in self.index:
            return ('same', self.index[same])
        if lvl > 0:
            par = (lvl - 1, tuple(x >> 1 for x in cn) if self.dim == 3
                   else (cn[0] >> 1, cn[1] >> 1, 0))
            if par in self.index:
                tang = [k for k in range(self.dim) if k != axis]
                pos = tuple(c[k] & 1 for k in tang)
                return ('coarser', self.index[par], pos)
        tang = [k for k in range(self.dim) if k != axis]
        out = []
        nsub = 1 << (self.dim - 1)
        for b in range(nsub):
            ch = [0, 0, 0]
            ch[axis] = 2 * cn[axis] + (0 if side > 0 else 1)
            for t, k in enumerate(tang):
                ch[k] = 2 * cn[k] + ((b >> t) & 1)
            if self.dim == 2:
                ch[2] = 0
            lf = (lvl + 1, tuple(ch))
            if lf not in self.index:
                raise ValueError("forest not 2:1 balanced at %r" % (leaf,))
            out.append(self.index[lf])
        return ('finer', out)

    def is_balanced(self) -> bool:
        for lf in self.leaves:
            for ax in range(self.dim):
                for s in (-1, 1):
                    try:
                        self.neighbour(lf, ax, s)
                    except ValueError:
                        return False
        return True

    def face_table(self):
        """Per leaf and face f = 2*axis + (side > 0): (kind, data) as returned by neighbour()."""
        out = []
        for lf in self.leaves:
            row = []
            for ax in range(self.dim):
                for s in (-1, 1):
                    row.append(self.neighbour(lf, ax, s))
            out.append(row)
        return out

    # ---------------- adaptation ----------------
    @staticmethod
    def children(leaf: Leaf, dim: int) -> List[Leaf]:
        lvl, c = leaf
        out = []
        for b in range(1 << dim):
            ch = (2 * c[0] + (b & 1), 2 * c[1] + ((b >> 1) & 1),
                  (2 * c[2] + ((b >> 2) & 1)) if dim == 3 else 0)
            out.append((lvl + 1, ch))
        return out

    @staticmethod
    def parent(leaf: Leaf, dim: int) -> Leaf:
        lvl, c = leaf
        return (lvl - 1, (c[0] >> 1, c[1] >> 1, (c[2] >> 1) if dim == 3 else 0))

    def adapt(self, eta_s: np.ndarray, tau_refine: float, tau_coarsen: float):
        """One refine-then-coarsen step (Alg. 1).  Returns (new_forest, plan).

        plan[i] for new leaf i is ('keep', old) | ('child', old_parent, child_bits)
        | ('parent', [old children in child order]).
        """
        dim = self.dim
        old = self.leaves
        eta = np.asarray(eta_s, dtype=np.float64)
        refine = set()
        for i, lf in enumerate(old):
            if eta[i] >= tau_refine and lf[0] < self.L:
                refine.add(lf)
        # balance closure: refine coarser neighbours of any too-fine child
        leafset = set(old)
        queue = list(refine)          # the closure does not depend on the processing order
        refined = set()
        while queue:
            lf = queue.pop()
            if lf in refined or lf not in leafset:
                continue
            refined.add(lf)
            leafset.discard(lf)
            for ch in self.children(lf, dim):
                leafset.add(ch)
            # new children at level lvl+1: any neighbour leaf at level lvl-1 violates 2:1
            lvl, c = lf
            for ax in range(dim):
                for s in (-1, 1):
                    cn = list(c)
                    cn[ax] += s
                    if cn[ax] < 0 or cn[ax] >= self.ncells(lvl, ax):
                        continue
                    if lvl >= 1:
                        par = (lvl - 1, (cn[0] >> 1, cn[1] >> 1, (cn[2] >> 1) if dim == 3 else 0))
                        if par in leafset and par not in refined:
                            queue.append(par)
        # coarsening of complete, untouched families
        fams: Dict[Leaf, List[Leaf]] = {}
        for lf in old:
            if lf[0] == 0 or lf in refined:
                continue
            fams.setdefault(self.parent(lf, dim), []).append(lf)
        coarsen = []
        for par, members in fams.items():
            if len(members) != (1 << dim):
                continue
            if any(eta[self.index[m]] > tau_coarsen for m in members):
                continue
            if any(m in refine for m in members):
                continue
            ok = True
            lvl_c = par[0] + 1
            for m in members:
                lvl, c = m
                for ax in range(dim):
                    for s in (-1, 1):
                        cn = list(c)
                        cn[ax] += s
                        if cn[ax] < 0 or cn[ax] >= self.ncells(lvl, ax):
                            continue
                        if self.parent((lvl, tuple(cn)), dim) == par:
                            continue  # inside the family
                        # a finer neighbour in the post-refine mesh blocks coarsening
                        for ch in self.children((lvl, tuple(cn)), dim):
                            if ch in leafset:
                                ok = False
                        if not ok:
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if ok:
                coarsen.append((par, members))
        if not refined and not coarsen:
            # nothing changes: the same leaves in the same order, every one kept
            return self, [('keep', i) for i in range(self.n)]
        for par, members in coarsen:
            for m in members:
                leafset.discard(m)
            leafset.add(par)
        new = Forest.__new__(Forest)
        new.dim, new.base, new.L, new.extent = self.dim, self.base, self.L, self.extent
        new.set_leaves(list(leafset))
        plan = []
        coarsened = {par: members for par, members in coarsen}
        for lf in new.leaves:
            if lf in self.index:
                plan.append(('keep', self.index[lf]))
            elif lf in coarsened:
                plan.append(('parent', [self.index[m] for m in
                                        sorted(coarsened[lf], key=self.key)]))
            else:
                par = self.parent(lf, dim)
                bits = (lf[1][0] & 1) | ((lf[1][1] & 1) << 1) | (((lf[1][2] & 1) << 2) if dim == 3 else 0)
                plan.append(('child', self.index[par], bits))
        return new, plan
