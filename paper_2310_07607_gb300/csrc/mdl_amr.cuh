// mdl_amr.cuh -- device-side forest adaptation, mesh tables and level ordering.
//
// One refine-then-coarsen step of Alg. 1 on the device, bit-identical to the
// forest bookkeeping it replaces:
//   k_amr_mark     refine flag r_e = (eta_e >= tau_refine && level < max_refine)
//   k_amr_close    2:1 closure: a refined leaf forces its coarser face neighbours;
//                  run max_refine times (forced chains only go coarser)
//   k_amr_family   complete families of consecutive siblings with every eta <= tau_coarsen,
//                  none refined, no outside face neighbour finer or refined -> coarsen
//   k_amr_count    new leaves per old leaf (2^d, 1 or 0), then an exclusive scan
//   k_amr_emit     new leaf coordinates in (root, Morton) order and the transfer plan
//   k_leaf_keys    sort key of every leaf of the new mesh (its lower corner on the finest
//                  grid: root id, then Morton index inside the root) for neighbour search
//   k_mesh_tables  face kinds/positions, neighbours, hanging lists, levels, probe and
//                  stimulus data, CFL class levels of the new mesh
// and the level ordering (a stable multi-split by b descending) with the due counts
// of every tick.  Every kernel loops over the device-resident element count, so the
// barrier runs without a host round trip.
#pragma once

#include <cuda_runtime.h>

#include "mdl_kernels.cuh"

namespace mdl {

// Geometry of the base grid and the finest grid.
struct Grid {
    int32_t base[3];
    int64_t fine[3];
    int32_t L;
    int32_t dim;
};

// Stimulus boxes with the inclusion slack already applied, and the GL nodes.
struct StimBoxes {
    int n;
    double lo[MDL_MAX_STIM][3], hi[MDL_MAX_STIM][3];
    double xi[3];
};

// --------------------------------------------------------------------------
template <int DIM>
__global__ void k_amr_mark(const int4* coord, const double* eta, uint8_t* r, uint8_t* c0, DevMeta* m,
                           double tau_r, int L) {
    pdl_enter();
    if (m->err) return;
    const int64_t ne = m->ne;
    for (int64_t e = gtid(); e < ne; e += gstride()) {
        r[e] = (eta[e] >= tau_r && coord[e].w < L) ? 1 : 0;
        c0[e] = 0;
    }
    if (gtid() == 0) m->changed = 0;
}

template <int DIM>
__global__ void k_amr_close(const uint32_t* info, const int32_t* nbr, uint8_t* r, DevMeta* m) {
    pdl_enter();
    if (m->err) return;
    constexpr int NF = 2 * DIM;
    const int64_t ne = m->ne;
    for (int64_t e = gtid(); e < ne; e += gstride()) {
        if (!r[e]) continue;
        const uint32_t inf = info[e];
        for (int f = 0; f < NF; ++f)
            if (((inf >> (4 * f)) & 3u) == 2u) r[nbr[e * NF + f]] = 1;
    }
}

template <int DIM>
__global__ void k_amr_family(const int4* coord, const uint32_t* info, const int32_t* nbr, const double* eta,
                             const uint8_t* r, uint8_t* c0, DevMeta* m, double tau_c) {
    pdl_enter();
    if (m->err) return;
    constexpr int NF = 2 * DIM, NC = 1 << DIM;
    const int64_t ne = m->ne;
    for (int64_t e = gtid(); e < ne; e += gstride()) {
        const int4 a = coord[e];
        if (a.w == 0 || (a.x & 1) || (a.y & 1) || (DIM == 3 && (a.z & 1))) continue;
        if (e + NC > ne) continue;
        bool ok = true;
        for (int b = 0; b < NC && ok; ++b) {
            const int64_t c = e + b;
            const int4 s = coord[c];
            if (s.w != a.w || s.x != a.x + (b & 1) || s.y != a.y + ((b >> 1) & 1) ||
                (DIM == 3 && s.z != a.z + ((b >> 2) & 1)))
                ok = false;
            else if (r[c] || !(eta[c] <= tau_c))
                ok = false;
            else {
                const uint32_t ic = info[c];
                for (int f = 0; f < NF && ok; ++f) {
                    const int axis = f >> 1, side = (f & 1) ? 1 : -1;
                    const int cb = (b >> axis) & 1;
                    if ((side > 0 && cb == 0) || (side < 0 && cb == 1)) continue;
                    const unsigned kind = (ic >> (4 * f)) & 3u;
                    if (kind == 3u) ok = false;
                    else if (kind == 1u && r[nbr[c * NF + f]]) ok = false;
                }
            }
        }
        if (ok) c0[e] = 1;
    }
}

// Exclusive scan of cnt[0..ne) in chunks of SCAN_CHUNK per block: block sums, a one-block
// scan of the sums, then per-block scans with the block offset.  Writes the total to ne_new.
constexpr int SCAN_THREADS = 256, SCAN_ITEMS = 2, SCAN_CHUNK = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t* sh, int64_t* total) {
    // inclusive warp scans then a scan over warp totals
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        int64_t t = lane < nw ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) sh[lane] = t;
    }
    __syncthreads();
    const int64_t woff = w > 0 ? sh[w - 1] : 0;
    *total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return woff + x - v;
}

// New leaves per old leaf: 2^d if refined, 1 if kept or child 0 of a coarsened family
// (which becomes the parent), 0 for the other children of a coarsened family.
template <int DIM>
__device__ __forceinline__ int new_count(const int4* coord, const uint8_t* r, const uint8_t* c0, int64_t e) {
    if (r[e]) return 1 << DIM;
    if (c0[e]) return 1;
    const int4 a = coord[e];
    if (a.w > 0) {
        const int b = (a.x & 1) | ((a.y & 1) << 1) | (DIM == 3 ? ((a.z & 1) << 2) : 0);
        if (b > 0 && e - b >= 0 && c0[e - b]) return 0;
    }
    return 1;
}

template <int DIM>
__global__ void k_scan_blocks(const int4* coord, const uint8_t* r, const uint8_t* c0, int64_t* bsum,
                              DevMeta* m) {
    pdl_enter();
    if (m->err) return;
    __shared__ int64_t sh[32];
    const int64_t ne = m->ne;
    const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK;
    if (base >= ne) return;
    int64_t s = 0;
    bool ch = false;
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        const int64_t e = base + (int64_t)threadIdx.x * SCAN_ITEMS + i;
        if (e < ne) {
            const int n = new_count<DIM>(coord, r, c0, e);
            s += n;
            ch = ch || n != 1 || c0[e];
        }
    }
    if (ch) m->changed = 1;
    int64_t tot;
    block_excl_scan(s, sh, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

static __global__ void k_scan_top(int64_t* bsum, DevMeta* m, int64_t cap) {
    pdl_enter();
    if (m->err) return;
    __shared__ int64_t sh[32];
    const int64_t ne = m->ne;
    const int64_t nb = (ne + SCAN_CHUNK - 1) / SCAN_CHUNK;
    int64_t carry = 0;
    for (int64_t s0 = 0; s0 < nb; s0 += blockDim.x) {
        const int64_t i = s0 + threadIdx.x;
        const int64_t v = i < nb ? bsum[i] : 0;
        int64_t tot;
        const int64_t ex = block_excl_scan(v, sh, &tot);
        if (i < nb) bsum[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        if (carry > cap) {
            m->need = carry;
            atomicOr(&m->err, ERR_CAPACITY);
        } else {
            // commit: the new count becomes current, the other set becomes current
            m->ne_new = ne;          // old count, read by the emit pass
            m->ne = carry;
            m->cur_set ^= 1u;
            m->nfac = 0u;
            if (m->changed) m->rebuilds++;
        }
    }
}

// Exclusive offsets of the new leaves, written directly as the new coordinates and the
// transfer plan (0 keep, 1 child, 2 parent).  Runs after the commit: the old count is
// in ne_new.
template <int DIM>
__global__ void k_scan_emit(const int4* coord, const uint8_t* r, const uint8_t* c0, const int64_t* bsum,
                            int4* ncoord, int8_t* pkind, int32_t* psrc, int8_t* pbits, const DevMeta* m) {
    pdl_enter();
    if (m->err) return;
    constexpr int NC = 1 << DIM;
    __shared__ int64_t sh[32];
    const int64_t ne = m->ne_new;
    const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK;
    if (base >= ne) return;
    int v[SCAN_ITEMS];
    int64_t s = 0;
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        const int64_t e = base + (int64_t)threadIdx.x * SCAN_ITEMS + i;
        v[i] = e < ne ? new_count<DIM>(coord, r, c0, e) : 0;
        s += v[i];
    }
    int64_t tot;
    int64_t o = block_excl_scan(s, sh, &tot) + bsum[blockIdx.x];
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        const int64_t e = base + (int64_t)threadIdx.x * SCAN_ITEMS + i;
        if (e >= ne) break;
        const int4 a = coord[e];
        if (v[i] == NC) {
            for (int b = 0; b < NC; ++b) {
                ncoord[o + b] = make_int4(2 * a.x + (b & 1), 2 * a.y + ((b >> 1) & 1),
                                          DIM == 3 ? 2 * a.z + ((b >> 2) & 1) : 0, a.w + 1);
                pkind[o + b] = 1;
                psrc[o + b] = (int32_t)e;
                pbits[o + b] = (int8_t)b;
            }
        } else if (v[i] == 1) {
            if (c0[e]) {
                ncoord[o] = make_int4(a.x >> 1, a.y >> 1, DIM == 3 ? a.z >> 1 : 0, a.w - 1);
                pkind[o] = 2;
            } else {
                ncoord[o] = a;
                pkind[o] = 0;
            }
            psrc[o] = (int32_t)e;
            pbits[o] = 0;
        }
        o += v[i];
    }
}

// Sort key of a finest-grid cell: its root's id (x fastest over the base grid) above the
// Morton index of the cell inside the root (x bit lowest).  Leaves are stored in this order
// (their lower corner's key), so the leaf holding a cell is the last leaf whose key does not
// exceed the cell's: a search over 8 bytes per leaf instead of an owner map of 4 bytes per
// finest cell (2^(d L) per root).
template <int DIM>
__device__ __forceinline__ uint64_t cell_key(const Grid& g, int64_t fx, int64_t fy, int64_t fz) {
    const int L = g.L;
    const int64_t rx = fx >> L, ry = fy >> L, rz = DIM == 3 ? (fz >> L) : 0;
    const uint64_t rid = (uint64_t)(rx + g.base[0] * (ry + (int64_t)g.base[1] * rz));
    const uint32_t lx = (uint32_t)(fx - (rx << L)), ly = (uint32_t)(fy - (ry << L)),
                   lz = DIM == 3 ? (uint32_t)(fz - (rz << L)) : 0u;
    uint64_t mort = 0;
    for (int b = 0; b < L; ++b) {
        mort |= (uint64_t)((lx >> b) & 1u) << (DIM * b);
        mort |= (uint64_t)((ly >> b) & 1u) << (DIM * b + 1);
        if (DIM == 3) mort |= (uint64_t)((lz >> b) & 1u) << (DIM * b + 2);
    }
    return (rid << (DIM * L)) | mort;
}

template <int DIM>
__global__ void k_leaf_keys(const int4* coord, uint64_t* lkey, Grid g, const DevMeta* m, int force) {
    pdl_enter();
    if (m->err || !(force || m->changed)) return;
    const int64_t ne = m->ne;
    for (int64_t e = gtid(); e < ne; e += gstride()) {
        const int4 a = coord[e];
        const int sh = g.L - a.w;
        lkey[e] = cell_key<DIM>(g, (int64_t)a.x << sh, (int64_t)a.y << sh, (int64_t)a.z << sh);
    }
}

// The leaf holding the cell of key k: the last e with lkey[e] <= k (lkey[0] = 0), found by a
// galloping search from `hint` (face neighbours are mostly near in the Morton order), then
// bisection.
__device__ __forceinline__ int32_t find_leaf(const uint64_t* __restrict__ lkey, int64_t ne, int64_t hint,
                                             uint64_t k) {
    int64_t lo, hi;   // lkey[lo] <= k < lkey[hi] (hi == ne: past the end)
    if (lkey[hint] <= k) {
        lo = hint;
        hi = ne;
        for (int64_t step = 1;; step <<= 1) {
            const int64_t j = lo + step;
            if (j >= ne) break;
            if (lkey[j] <= k) {
                lo = j;
            } else {
                hi = j;
                break;
            }
        }
    } else {
        hi = hint;
        lo = 0;
        for (int64_t step = 1;; step <<= 1) {
            const int64_t j = hi - step;
            if (j <= 0) break;
            if (lkey[j] <= k) {
                lo = j;
                break;
            }
            hi = j;
        }
    }
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (lkey[mid] <= k) lo = mid;
        else hi = mid;
    }
    return (int32_t)lo;
}

// Face tables of the mesh in `coord` from the leaf keys (same rules as the forest
// bookkeeping: neighbour at the same level, one coarser with the tangential position
// bits, or the 2^(d-1) finer children touching the face).
template <typename R, int DIM, int P>
__global__ void k_mesh_tables(const int4* coord, const uint64_t* lkey, Grid g, uint32_t* info, int32_t* nbr,
                              int32_t* hang, int32_t* root, uint32_t* loc, uint8_t* bcfl,
                              const uint8_t* class_b, uint32_t* smask0, uint32_t* smask1, uint32_t* smask2,
                              uint32_t* smask3, StimBoxes sb, Phys<double> phd, DevMeta* m, int force) {
    // element extents per level in FP32 for the stimulus-box pre-test below
    __shared__ float hf[8][3];
    if (threadIdx.x < 24) hf[threadIdx.x / 3][threadIdx.x % 3] = (float)phd.h[threadIdx.x / 3][threadIdx.x % 3];
    __syncthreads();
    pdl_enter();
    if (m->err || !(force || m->changed)) return;
    using S = Shape<DIM, P>;
    constexpr int N1 = S::N1, NP = S::NP, NF = S::NF, NSUB = S::NSUB;
    const int64_t ne = m->ne;
    uint32_t* smask[4] = {smask0, smask1, smask2, smask3};
    for (int64_t e = gtid(); e < ne; e += gstride()) {
        const int4 a = coord[e];
        const int l = a.w, sh = g.L - l;
        const int c[3] = {a.x, a.y, a.z};
        uint32_t inf = (uint32_t)l << 24;
        uint32_t cfg = 0;
        for (int f = 0; f < NF; ++f) {
            const int axis = f >> 1, side = (f & 1) ? 1 : -1;
            int64_t cn[3] = {c[0], c[1], DIM == 3 ? c[2] : 0};
            cn[axis] += side;
            const int64_t ncell = (int64_t)g.base[axis] << l;
            int kind = 0, pos = 0;
            int32_t nb = -1;
            if (cn[axis] >= 0 && cn[axis] < ncell) {
                int64_t fc[3];
                for (int k = 0; k < 3; ++k) fc[k] = (k < DIM) ? (cn[k] << sh) : 0;
                if (side < 0) fc[axis] = ((cn[axis] + 1) << sh) - 1;
                const int32_t o = find_leaf(lkey, ne, e, cell_key<DIM>(g, fc[0], fc[1], fc[2]));
                const int lo = coord[o].w;
                int tg[2] = {0, 0}, nt = 0;
                for (int k = 0; k < DIM; ++k)
                    if (k != axis) tg[nt++] = k;
                if (lo == l) {
                    kind = 1;
                    nb = o;
                } else if (lo != l - 1 && lo != l + 1) {
                    atomicOr(&m->err, ERR_MESH);
                } else if (lo == l - 1) {
                    kind = 2;
                    nb = o;
                    for (int t = 0; t < nt; ++t) pos |= (c[tg[t]] & 1) << t;
                } else {
                    kind = 3;
                    nb = (int32_t)((e * NF + f) * NSUB);
                    for (int b = 0; b < NSUB; ++b) {
                        int64_t ch[3] = {0, 0, 0};
                        ch[axis] = 2 * cn[axis] + (side > 0 ? 0 : 1);
                        for (int t = 0; t < nt; ++t) ch[tg[t]] = 2 * (int64_t)c[tg[t]] + ((b >> t) & 1);
                        int64_t f2[3];
                        for (int k = 0; k < 3; ++k) f2[k] = (k < DIM) ? (ch[k] << (sh - 1)) : 0;
                        hang[nb + b] = find_leaf(lkey, ne, o, cell_key<DIM>(g, f2[0], f2[1], f2[2]));
                    }
                }
            }
            inf |= (uint32_t)(kind | (pos << 2)) << (4 * f);
            cfg |= (uint32_t)kind << (2 * f);
            nbr[e * NF + f] = nb;
        }
        // probes and root
        int32_t rt[3] = {0, 0, 0};
        uint32_t lc = (uint32_t)l << 24;
        for (int k = 0; k < DIM; ++k) {
            rt[k] = c[k] >> l;
            lc |= (uint32_t)(c[k] - (rt[k] << l)) << (8 * k);
        }
        root[e] = rt[0] + g.base[0] * (rt[1] + g.base[1] * rt[2]);
        loc[e] = lc;
        bcfl[e] = class_b[(size_t)l * (1u << (2 * NF)) + cfg];
        // stimulus masks: node coordinates in FP64 without contraction (same bits as the host).
        // GL nodes lie at least 0.11 h inside the element along each axis, so an element whose
        // extent misses the box by 0.05 h (FP32 test: its rounding is below 1e-4 h) holds no
        // node of the box and skips the FP64 evaluation (a slow pipe on this part).
        bool any = false;
        for (int s = 0; s < sb.n; ++s) {
            uint32_t msk = 0;
            bool may = true;
            for (int k = 0; k < DIM; ++k) {
                const float h = hf[l][k], x0 = (float)c[k] * h;
                if (x0 + h < (float)sb.lo[s][k] - 0.05f * h || x0 > (float)sb.hi[s][k] + 0.05f * h) may = false;
            }
            for (int q = 0; may && q < NP; ++q) {
                bool in = true;
                for (int k = 0; k < DIM; ++k) {
                    const double h = phd.h[l][k];
                    const double xi = sb.xi[digit<N1>(q, k)];
                    const double x = __dadd_rn(__dmul_rn((double)c[k], h), __dmul_rn(__dmul_rn(__dadd_rn(xi, 1.0), 0.5), h));
                    if (x < sb.lo[s][k] || x > sb.hi[s][k]) in = false;
                }
                if (in) msk |= 1u << q;
            }
            smask[s][e] = msk;
            any = any || msk;
        }
        if (any) inf |= INFO_STIM;
        info[e] = inf;
    }
}

// --------------------------------------------------------------------------
// Level ordering: stable multi-split of the element ids by b descending, with the
// due count of every tick (tick 0: all; tick i > 0: b >= B - ctz(i)).
constexpr int ORD_THREADS = 256;

// Substep levels b_e = max(b^CFL_e, b^cell_e) (Eq. num-substeps), or the replayed
// levels, fused with the per-block level counts of the ordering.
template <typename R>
__global__ void k_levels_count(const DevArrays<R> d, const int8_t* ovr, const double* eta_t, double tau_cell,
                               int bcell, int B, int lts, int32_t* bcnt) {
    pdl_enter();
    if (d.meta->err) return;
    __shared__ int sc[8];
    if (threadIdx.x < 8) sc[threadIdx.x] = 0;
    __syncthreads();
    const int64_t e = (int64_t)blockIdx.x * ORD_THREADS + threadIdx.x;
    if (e < d.meta->ne) {
        int b;
        if (ovr) b = ovr[e];
        else if (!lts) b = 0;
        else {
            b = d.bcfl[e];
            const int bt = (eta_t[e] > tau_cell) ? bcell : 0;
            b = bt > b ? bt : b;
        }
        if (b > B || b < 0) {
            atomicOr(&d.meta->err, ERR_CFL);
            b = b < 0 ? 0 : B;
        }
        const uint8_t old = d.lvl[e];
        d.lvl[e] = (uint8_t)(b | (old & 8));
        atomicAdd(&sc[b], 1);
    }
    __syncthreads();
    if (threadIdx.x < 8) bcnt[(int64_t)blockIdx.x * 8 + threadIdx.x] = sc[threadIdx.x];
}

// Exclusive scan over blocks of the per-block level counts, all 8 levels at once (each
// thread holds one block's 8 counts; warp scans, then a scan of the warp totals), then the
// level base offsets (b descending) and the due counts of every tick.
static __global__ void k_order_top(int32_t* bcnt, DevMeta* m, int B) {
    pdl_enter();
    if (m->err) return;
    __shared__ int32_t ws[32][8];
    const int64_t ne = m->ne;
    const int64_t nb = (ne + ORD_THREADS - 1) / ORD_THREADS;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int32_t carry[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) carry[b] = 0;
    for (int64_t s0 = 0; s0 < nb; s0 += blockDim.x) {
        const int64_t i = s0 + threadIdx.x;
        int32_t v[8];
        if (i < nb) {
            const int4 lo = reinterpret_cast<const int4*>(bcnt)[2 * i];
            const int4 hi = reinterpret_cast<const int4*>(bcnt)[2 * i + 1];
            v[0] = lo.x; v[1] = lo.y; v[2] = lo.z; v[3] = lo.w;
            v[4] = hi.x; v[5] = hi.y; v[6] = hi.z; v[7] = hi.w;
        } else {
#pragma unroll
            for (int b = 0; b < 8; ++b) v[b] = 0;
        }
        int32_t x[8];
#pragma unroll
        for (int b = 0; b < 8; ++b) x[b] = v[b];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const int32_t y = __shfl_up_sync(0xffffffffu, x[b], o);
                if (lane >= o) x[b] += y;
            }
        }
        if (lane == 31) {
#pragma unroll
            for (int b = 0; b < 8; ++b) ws[w][b] = x[b];
        }
        __syncthreads();
        if (w == 0) {
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                int32_t t = lane < nw ? ws[lane][b] : 0;
                for (int o = 1; o < 32; o <<= 1) {
                    const int32_t y = __shfl_up_sync(0xffffffffu, t, o);
                    if (lane >= o) t += y;
                }
                if (lane < nw) ws[lane][b] = t;
            }
        }
        __syncthreads();
        int32_t ex[8];
#pragma unroll
        for (int b = 0; b < 8; ++b) ex[b] = carry[b] + (w > 0 ? ws[w - 1][b] : 0) + x[b] - v[b];
        if (i < nb) {
            reinterpret_cast<int4*>(bcnt)[2 * i] = make_int4(ex[0], ex[1], ex[2], ex[3]);
            reinterpret_cast<int4*>(bcnt)[2 * i + 1] = make_int4(ex[4], ex[5], ex[6], ex[7]);
        }
#pragma unroll
        for (int b = 0; b < 8; ++b) carry[b] += ws[nw - 1][b];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        // level base offsets in b-descending order, stored after the block table
        int64_t off = 0;
        int32_t* lo = bcnt + nb * 8;
        for (int b = 7; b >= 0; --b) {
            lo[b] = (int32_t)off;
            off += carry[b];
            m->cnt[b] = (unsigned)carry[b];
        }
        const int nt = 1 << B;
        int64_t eu = 0;
        for (int i = 0; i < nt; ++i) {
            int64_t na = 0;
            if (i == 0) na = ne;
            else {
                const int tz = __ffs(i) - 1;
                for (int b = B - tz; b <= B; ++b) na += carry[b];
            }
            m->nact[i] = (int32_t)na;
            eu += na;
        }
        m->elem_updates += eu;
    }
}

static __global__ void k_order_scatter(const uint8_t* lvl, const int32_t* bcnt, int32_t* order, const DevMeta* m) {
    pdl_enter();
    if (m->err) return;
    __shared__ int wc[ORD_THREADS / 32][8];
    const int64_t ne = m->ne;
    const int64_t nb = (ne + ORD_THREADS - 1) / ORD_THREADS;
    const int64_t e = (int64_t)blockIdx.x * ORD_THREADS + threadIdx.x;
    if ((int64_t)blockIdx.x >= nb) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const bool valid = e < ne;
    const int b = valid ? (lvl[e] & 7) : 8;
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    if (lane < 8) wc[w][lane] = 0;
    __syncwarp();
    if (valid && rank == 0) wc[w][b] = __popc(peers);
    __syncthreads();
    if (!valid) return;
    int woff = 0;
    for (int x = 0; x < w; ++x) woff += wc[x][b];
    const int32_t* lo = bcnt + nb * 8;
    order[lo[b] + bcnt[blockIdx.x * 8 + b] + woff + rank] = (int32_t)e;
}

}  // namespace mdl
