"""The precision design of the tensor-core residual (Q2 3D FP32), emulated in numpy on the
oracle's assembled SIPG matrix: for every element, r_e = A_e u over its own and its face
neighbours' values, computed from

  * the operand shifted by the element mean c (A_e 1 = 0 row by row, so r_e is unchanged),
  * each row of the operand scaled by a power of two that brings max |y| to [2^13, 2^14),
    the operator scaled by 2^t into the FP16 range,
  * both split into two FP16 terms, hi = fp16(x) and lo = fp16(x - hi), and the three products
    U_hi B_hi + U_hi B_lo + U_lo B_hi accumulated in FP32,

agrees with the FP64 product to FP32-accumulation accuracy relative to sum_j |A_ij y_j|,
while one TF32-like term per operand (10-bit significand), or the same split without the
mean shift, is far less accurate on the same data.  FP16 products are exact in FP32 (11 + 11 significant bits), so the emulation is exact
up to the order of the FP32 sums.  Test infrastructure only: nothing here is shared with the
CUDA path."""
import numpy as np

import workloads as W
from oracle.forest import Forest
from oracle.sipg import Disc


def _problem():
    return W.Problem(dim=3, order=2, extent=(0.3, 0.2, 0.15), base=(6, 4, 3), sigma_l=1.2, sigma_t=0.3,
                     fibre=(0.48, 0.64, 0.6), gamma=40.0, precision=64)


def _state(X):
    # a steep front on top of an offset of about 1: the regime where the mean shift matters
    r = np.sqrt(np.sum((X - np.array([0.0, 0.0, 0.0])) ** 2, axis=1))
    return 1.0 + 0.002 * np.tanh((r - 0.12) / 0.01) + 1e-4 * np.sin(40.0 * X[:, 0])


def _pow2_scale(mx):
    """2^s with mx 2^s in [2^13, 2^14) (mx > 0)."""
    return 2.0 ** (13 - np.floor(np.log2(mx)))


def _split16(x32):
    hi = x32.astype(np.float16)
    lo = (x32 - hi.astype(np.float32)).astype(np.float16)
    return hi.astype(np.float32), lo.astype(np.float32)


def _tf32(x32):
    """Round an FP32 array to a 10-bit significand (round to nearest)."""
    b = x32.astype(np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x1000) & ~np.uint64(0x1FFF)).astype(np.uint32)
    return b.view(np.float32)


def _element_systems():
    prob = _problem()
    f = Forest(3, prob.base, 0, prob.extent)
    disc = Disc(prob, f)
    A = disc.assemble().tocsr()
    u = _state(disc.node_coords())
    n_p = disc.n_p
    for e in range(disc.ne):
        rows = np.arange(e * n_p, (e + 1) * n_p)
        sub = A[rows]
        cols = np.unique(sub.indices)
        yield A[rows][:, cols].toarray(), u[cols], u[rows]


def test_element_rows_annihilate_constants():
    for Ae, _, _ in _element_systems():
        assert np.all(np.abs(Ae.sum(axis=1)) <= 1e-12 * np.abs(Ae).sum(axis=1))


def test_fp16_hi_lo_split_reaches_fp32_accuracy():
    worst_split, worst_tf32, worst_noshift = 0.0, 0.0, 0.0
    for Ae, ucols, uown in _element_systems():
        # the state is FP32 on the device: the FP64 reference takes the same FP32 values
        u32 = ucols.astype(np.float32)
        c = np.float32(np.mean(uown.astype(np.float32)))
        y = (u32 - c).astype(np.float32)                   # exact (Sterbenz): values near c
        ref = Ae @ (u32.astype(np.float64) - float(c))     # FP64, equal to Ae u32 (rows sum to zero)
        bound = np.abs(Ae) @ np.abs(y.astype(np.float64))  # sum_j |A_ij y_j|
        sy = np.float32(_pow2_scale(np.max(np.abs(y))))
        sb = np.float32(_pow2_scale(np.max(np.abs(Ae))))
        yh, yl = _split16(y * sy)
        Bh, Bl = _split16((Ae * sb).astype(np.float32))
        D = (Bh @ yh).astype(np.float32) + (Bl @ yh).astype(np.float32) + (Bh @ yl).astype(np.float32)
        r = D.astype(np.float64) / (float(sy) * float(sb))
        err = np.abs(r - ref) / bound
        worst_split = max(worst_split, float(err.max()))
        # one TF32-like term per operand
        r1 = (_tf32((Ae * sb).astype(np.float32)) @ _tf32(y * sy)).astype(np.float64) / (float(sy) * float(sb))
        worst_tf32 = max(worst_tf32, float((np.abs(r1 - ref) / bound).max()))
        # the same split without the mean shift: the operand carries the offset of ~1
        su = np.float32(_pow2_scale(np.max(np.abs(u32))))
        uh, ul = _split16(u32 * su)
        D2 = (Bh @ uh).astype(np.float32) + (Bl @ uh).astype(np.float32) + (Bh @ ul).astype(np.float32)
        r2 = D2.astype(np.float64) / (float(su) * float(sb))
        worst_noshift = max(worst_noshift, float((np.abs(r2 - ref) / bound).max()))
    # FP32 accumulation over <= 189 products of three terms, plus the split's 2^-22
    assert worst_split <= 3 * 189 * 2.0 ** -24 + 4 * 2.0 ** -22, worst_split
    assert worst_tf32 >= 30 * worst_split, (worst_tf32, worst_split)
    assert worst_noshift >= 30 * worst_split, (worst_noshift, worst_split)


def test_level_blocks_scale_by_power_of_two():
    """On box elements every SIPG block of level l is 2^((2-d) l) times its level-0 block
    (volume: (2/h)^2 h^d; faces: h^(d-1) / h), the exact row scale that lets one level-0
    operator serve every level of the tensor-core residual."""
    prob = _problem()
    disc = Disc(prob, Forest(3, prob.base, 3, prob.extent))
    for level in (1, 2, 3):
        scale = 2.0 ** ((2 - 3) * level)
        V0, Vl = disc.volume_block(0), disc.volume_block(level)
        assert np.allclose(Vl, scale * V0, rtol=1e-13, atol=1e-15 * np.abs(V0).max())
        for k in range(3):
            F0, Fl = disc.face_block(k, (0, 0, ())), disc.face_block(k, (level, level, ()))
            assert np.allclose(Fl, scale * F0, rtol=1e-13, atol=1e-15 * np.abs(F0).max())
    # the same relation with one level of refinement across the face (coarse side at level l)
    for level in (0, 1, 2):
        scale = 2.0 ** ((2 - 3) * level)
        for k in range(3):
            for pos in ((0, 0), (1, 0), (0, 1), (1, 1)):
                H0 = disc.face_block(k, (0, 1, pos))
                Hl = disc.face_block(k, (level, level + 1, pos))
                assert np.allclose(Hl, scale * H0, rtol=1e-13, atol=1e-15 * np.abs(H0).max())
