// mdl_kernels.cuh -- CUDA kernels of one barrier step (Alg. 1) for one (precision, dim, order).
//
// Data layout in HBM (structure of arrays, element-blocked DOFs):
//   V0, V1  [ne * NPS] two slots of V; element e's current value is in slot
//                      par_e ^ (updates this barrier & 1) -- a per-element ping-pong,
//                      so a tick reads the values at its start and writes the other slot
//   v       [ne * NPS] Aliev-Panfilov recovery variable (element-local, in place)
//   Ia, ga  [ne * NPS] I(u_a, t_a) and g(u_a) at the barrier start (only for S_e > 1)
//                      (NPS: the row stride, NP rounded up to 28 for Q2 3D; pad value 0)
//   lvl     [ne]       b_e (bits 0-2) | parity par_e (bit 3)
//   info    [ne]       4 bits per face: kind (0 bnd, 1 same, 2 coarser, 3 finer) | pos << 2;
//                      bits 24-27 refinement level; bit 28 in a stimulus box; bit 29 probes pending
//   nbr     [ne * 2d]  neighbour element (same/coarser) or first hang[] index (finer)
//   hang    [*]        2^(d-1) fine neighbours per hanging face
//   order   [ne]       element ids sorted by b descending: tick i updates a prefix
//   acc     [ne]       FP64 RV-T accumulator; eta_t, eta_s [ne] FP64
//   lat     [n_probe]  FP64 activation time per probe (+INF pending)
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "../../include/mdl.h"
#include "mdl_element.cuh"

namespace mdl {

constexpr uint32_t INFO_STIM = 1u << 28;
constexpr uint32_t INFO_PENDING = 1u << 29;

// Device-resident bookkeeping of one context: every kernel reads its element count
// and the sticky error word from here, so a barrier needs no host round trip.
struct DevMeta {
    int64_t ne;              // elements of the current mesh
    int64_t ne_new;          // elements after this barrier's adaptation
    int64_t nbar;            // completed barriers
    int64_t need;            // element capacity requested on overflow
    unsigned int err;        // sticky: 1 non-finite, 2 CFL, 4 capacity, 8 mesh
    unsigned int changed;    // the adaptation changed the mesh
    unsigned int nf_pending; // non-finite values seen by this barrier's epilogue
    unsigned int cur_set;    // index of the state set holding the current values
    unsigned int done_blocks;// epilogue blocks finished (last-block reduction)
    unsigned int cnt[8];     // elements per level b in this barrier
    int32_t nact[128];       // due elements per tick
    int64_t elem_updates;    // accumulated element steps
    int64_t rebuilds;        // barriers whose mesh changed
    int64_t fac_updates;     // curved meshes: elements whose factors were computed
    double integral;         // FP64 int V after the last barrier
    unsigned int nfac;       // curved meshes: elements whose factors the adaptation recomputes
    unsigned int gbar;       // cooperative sweep: arrivals at its grid barriers (zeroed before each launch)
};

// ERR_WAIT: a bounded wait of a kernel gave up (tensor-core mbarrier, cooperative grid barrier)
constexpr unsigned ERR_NONFINITE = 1u, ERR_CFL = 2u, ERR_CAPACITY = 4u, ERR_MESH = 8u, ERR_WAIT = 16u;

// Programmatic dependent launch: wait until the preceding grid on the stream has completed
// and its writes are visible, then let the following grid be scheduled.  Each kernel of a
// barrier step calls this first; launched without the attribute it returns at once.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ int64_t gstride() { return (int64_t)gridDim.x * blockDim.x; }
__device__ __forceinline__ int64_t gtid() { return blockIdx.x * (int64_t)blockDim.x + threadIdx.x; }

template <typename R>
struct DevArrays {
    R* V0;
    R* V1;
    R* v;
    R* Ia;
    R* ga;
    double* acc;
    double* eta_t;
    double* eta_s;
    double* lat;
    double* partial;
    uint8_t* lvl;
    const uint8_t* bcfl;
    uint32_t* info;
    const int32_t* nbr;
    const int32_t* hang;
    const int32_t* order;
    const int32_t* root;
    const uint32_t* loc;
    const uint32_t* smask[MDL_MAX_STIM];
    DevMeta* meta;
    const R* qvol;      // Q1 class blocks (see q1_blocks): volume, face, Kelly
    const R* qface;
    const R* qkelly;
    const R* gvol;      // mapped meshes: per-element geometric factors (mdl_mapped.cuh)
    const R* gface;
    const double* mq;   // mapped meshes: per-element GL masses (null on boxes)
};

// Vector width for rows of NP values of type R: 16-byte loads when a row is a whole number
// of them (every table block and element vector below starts on a 16-byte boundary).
template <typename R, int NP>
struct Vec {
    static constexpr int W = (16 / (int)sizeof(R));
    static constexpr bool ok = (NP % W) == 0;
};

// out[0..n) = p[0..n), 16-byte loads where the width allows (p 16-byte aligned then).
template <typename R, int N>
__device__ __forceinline__ void ld_row(const R* __restrict__ p, R* out) {
    if constexpr (Vec<R, N>::ok && sizeof(R) == 4) {
#pragma unroll
        for (int i = 0; i < N / 4; ++i) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(p) + i);
            out[4 * i] = v.x; out[4 * i + 1] = v.y; out[4 * i + 2] = v.z; out[4 * i + 3] = v.w;
        }
    } else if constexpr (Vec<R, N>::ok && sizeof(R) == 8) {
#pragma unroll
        for (int i = 0; i < N / 2; ++i) {
            const double2 v = __ldg(reinterpret_cast<const double2*>(p) + i);
            out[2 * i] = v.x; out[2 * i + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) out[i] = __ldg(p + i);
    }
}

// Plain (coherent) vector load / store of an element's N values.
template <typename R, int N>
__device__ __forceinline__ void ld_vec(const R* p, R* out) {
    if constexpr (Vec<R, N>::ok && sizeof(R) == 4) {
#pragma unroll
        for (int i = 0; i < N / 4; ++i) {
            const float4 v = reinterpret_cast<const float4*>(p)[i];
            out[4 * i] = v.x; out[4 * i + 1] = v.y; out[4 * i + 2] = v.z; out[4 * i + 3] = v.w;
        }
    } else if constexpr (Vec<R, N>::ok && sizeof(R) == 8) {
#pragma unroll
        for (int i = 0; i < N / 2; ++i) {
            const double2 v = reinterpret_cast<const double2*>(p)[i];
            out[2 * i] = v.x; out[2 * i + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) out[i] = p[i];
    }
}

template <typename R, int N>
__device__ __forceinline__ void st_vec(R* p, const R* x) {
    if constexpr (Vec<R, N>::ok && sizeof(R) == 4) {
#pragma unroll
        for (int i = 0; i < N / 4; ++i)
            reinterpret_cast<float4*>(p)[i] = make_float4(x[4 * i], x[4 * i + 1], x[4 * i + 2], x[4 * i + 3]);
    } else if constexpr (Vec<R, N>::ok && sizeof(R) == 8) {
#pragma unroll
        for (int i = 0; i < N / 2; ++i) reinterpret_cast<double2*>(p)[i] = make_double2(x[2 * i], x[2 * i + 1]);
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) p[i] = x[i];
    }
}

// One element row of a per-DOF state array: NP values at row stride NPS.  With NPS a whole
// number of 16-byte vectors the row moves in vectors (the pad value read is dropped; a
// store writes the pad as 0), else value by value.
template <typename R, int NP, int NPS>
__device__ __forceinline__ void ld_dofs(const R* p, R* out) {
    if constexpr (NPS == NP) {
        ld_vec<R, NP>(p, out);
    } else {
        R t[NPS];
        ld_vec<R, NPS>(p, t);
#pragma unroll
        for (int q = 0; q < NP; ++q) out[q] = t[q];
    }
}

template <typename R, int NP, int NPS>
__device__ __forceinline__ void st_dofs(R* p, const R* x) {
    if constexpr (NPS == NP) {
        st_vec<R, NP>(p, x);
    } else {
        R t[NPS];
#pragma unroll
        for (int q = 0; q < NPS; ++q) t[q] = q < NP ? x[q] : R(0);
        st_vec<R, NPS>(p, t);
    }
}

// j[t] += sum_q K[t][q] x[q] for a row-major NT x NP block (read-only path).
template <typename R, int NT, int NP>
__device__ __forceinline__ void block_jump(const R* __restrict__ K, const R* x, R* j) {
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        R row[NP];
        ld_row<R, NP>(K + t * NP, row);
        R acc = j[t];
#pragma unroll
        for (int q = 0; q < NP; ++q) acc += row[q] * x[q];
        j[t] = acc;
    }
}

// r[q] += sum_j A[q][j] x[j] for a row-major NP x NP block in global memory (read-only path).
template <typename R, int NP>
__device__ __forceinline__ void block_mv(const R* __restrict__ A, const R* x, R* r) {
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        R row[NP];
        ld_row<R, NP>(A + q * NP, row);
        R acc = r[q];
#pragma unroll
        for (int j = 0; j < NP; ++j) acc += row[j] * x[j];
        r[q] = acc;
    }
}

// 2^-sh exactly, for 0 <= sh < 64 (built from the IEEE-754 exponent field).
template <typename R>
__device__ __forceinline__ R pow2_neg(int sh);
template <>
__device__ __forceinline__ float pow2_neg<float>(int sh) { return __int_as_float((127 - sh) << 23); }
template <>
__device__ __forceinline__ double pow2_neg<double>(int sh) {
    return __longlong_as_double((long long)(1023 - sh) << 52);
}

struct StimArgs {
    int n;
    double t0[MDL_MAX_STIM], t1[MDL_MAX_STIM], amp[MDL_MAX_STIM];
};

template <typename R>
__device__ __forceinline__ R r_exp(R x);
template <>
__device__ __forceinline__ float r_exp<float>(float x) { return expf(x); }
template <>
__device__ __forceinline__ double r_exp<double>(double x) { return exp(x); }

// a / b: FP32 through the fast reciprocal (within 2 ulp; b >= 1e-6 here), FP64 exact.
template <typename R>
__device__ __forceinline__ R r_div(R a, R b);
template <>
__device__ __forceinline__ float r_div<float>(float a, float b) { return __fdividef(a, b); }
template <>
__device__ __forceinline__ double r_div<double>(double a, double b) { return a / b; }

// e^x - 1 in FP32 without the cancellation of expf(x) - 1: for |x| < 1/16 the Taylor series
// of the exponential through x^6 (truncation below 1e-12 relative), else expf(x) - 1.
__device__ __forceinline__ float expm1_f32(float x) {
    if (fabsf(x) < 0.0625f)
        return x * (1.0f + x * (0.5f + x * (1.0f / 6.0f + x * (1.0f / 24.0f + x * (1.0f / 120.0f + x * (1.0f / 720.0f))))));
    return expf(x) - 1.0f;
}

template <typename R>
__device__ __forceinline__ R ap_iion(const Phys<R>& ph, R V, R w) {
    if (ph.ionic < 0) return R(0);
    return (ph.k * V * (V - ph.a) * (V - R(1)) + V * w) * ph.inv_ts;
}

template <typename R>
__device__ __forceinline__ R ap_eps(const Phys<R>& ph, R V, R w) {
    R den = V + ph.mu2;
    den = den > R(1e-6) ? den : R(1e-6);
    return ph.eps0 + r_div<R>(ph.mu1 * w, den);
}

template <typename R>
__device__ __forceinline__ R ap_g(const Phys<R>& ph, R V, R w) {
    if (ph.ionic < 0) return R(0);
    const R vinf = -ph.k * V * (V - ph.a - R(1));
    return ap_eps(ph, V, w) * (vinf - w) * ph.inv_ts;
}

// One step of the state: forward Euler, or the exponential step v_inf + (v - v_inf) e^(-eps dt)
// with eps and v_inf frozen at the step start.  In FP32 the exponential step is evaluated as
// v + (v - v_inf) (e^(-eps dt) - 1): on explicit substeps eps dt is far below 1 (about
// 1e-8 .. 1e-4 for substeps of 1e-6 .. 1e-2 ms), where e^(-eps dt) rounded to FP32 would
// lose most of the increment.
template <typename R>
__device__ __forceinline__ R ap_step_state(const Phys<R>& ph, R V, R w, R dt) {
    if (ph.ionic < 0) return w;
    const R vinf = -ph.k * V * (V - ph.a - R(1));
    const R eps = ap_eps(ph, V, w);
    if (ph.integrator == 0) return w + dt * eps * (vinf - w) * ph.inv_ts;
    if constexpr (sizeof(R) == 4) return w + (w - vinf) * expm1_f32(-eps * dt * ph.inv_ts);
    return vinf + (w - vinf) * r_exp<R>(-eps * dt * ph.inv_ts);
}

// Values of element nb as seen at tick `tick`, given its level byte: its current value if
// it is due (or finer), else the linear time interpolant of its last step (Alg. 1).
template <typename R, int NP, int NPS = NP>
__device__ __forceinline__ void load_seen_lv(const DevArrays<R>& d, int tick, int B, int nb, uint8_t lv, R* un) {
    const int b = lv & 7, par = (lv >> 3) & 1;
    const int sh = B - b;
    const int j = tick >> sh;
    const int rem = tick & ((1 << sh) - 1);
    const int nw = par ^ ((j + (rem ? 1 : 0)) & 1);
    ld_dofs<R, NP, NPS>((nw ? d.V1 : d.V0) + (size_t)nb * NPS, un);
    if (rem) {
        R so[NP];
        ld_dofs<R, NP, NPS>((nw ? d.V0 : d.V1) + (size_t)nb * NPS, so);
        const R th = R(rem) * pow2_neg<R>(sh);
#pragma unroll
        for (int q = 0; q < NP; ++q) un[q] = so[q] + th * (un[q] - so[q]);
    }
}

template <typename R, int NP, int NPS = NP>
__device__ __forceinline__ void load_seen(const DevArrays<R>& d, int tick, int B, int nb, R* un) {
    load_seen_lv<R, NP, NPS>(d, tick, B, nb, d.lvl[nb], un);
}

// Residual r = (A u)_e with the neighbours seen at tick `tick`.  All same-level and
// coarser neighbours are gathered before any face arithmetic (their ids, then their
// level bytes, then their values), so the dependent loads of the faces overlap;
// hanging faces (finer neighbours) follow on a separate path.
template <typename R, int DIM, int P>
__device__ __forceinline__ void element_residual(const DevArrays<R>& d, const Tables<R>& T,
                                                 const Phys<R>& ph, int tick, int B, int e,
                                                 uint32_t inf, int lev, const R* u, R* r) {
    using S = Shape<DIM, P>;
    constexpr int NP = S::NP, NF = S::NF, NSUB = S::NSUB, NPS = S::NPS;
#pragma unroll
    for (int q = 0; q < NP; ++q) r[q] = R(0);
    if constexpr (P > 1) {
        // Q2: one face at a time (holding every neighbour's 27 values would spill)
        volume_term<R, DIM, P>(T, ph, lev, u, r);
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            const int kind = (inf >> (4 * f)) & 3;
            if (kind == 0) continue;
            const int k = f >> 1, s = (f & 1) ? 1 : -1;
            const int nbi = d.nbr[(size_t)e * NF + f];
            if (kind != 3) {
                R un[NP];
                load_seen<R, NP, NPS>(d, tick, B, nbi, un);
                const int pos = (inf >> (4 * f + 2)) & 3;
                face_term<R, DIM, P>(T, ph, k, s, lev, -1, u, kind == 1 ? lev : lev - 1,
                                     kind == 1 ? -1 : pos, un, lev, r);
            } else {
                for (int sb = 0; sb < NSUB; ++sb) {
                    R un[NP];
                    load_seen<R, NP, NPS>(d, tick, B, d.hang[nbi + sb], un);
                    face_term<R, DIM, P>(T, ph, k, s, lev, sb, u, lev + 1, -1, un, lev + 1, r);
                }
            }
        }
        return;
    }
    int nbf[NF], src[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) nbf[f] = d.nbr[(size_t)e * NF + f];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        const int kind = (inf >> (4 * f)) & 3;
        src[f] = (kind == 1 || kind == 2) ? nbf[f] : e;
    }
    uint8_t lvn[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) lvn[f] = d.lvl[src[f]];
    R un[NF][NP];
#pragma unroll
    for (int f = 0; f < NF; ++f) load_seen_lv<R, NP>(d, tick, B, src[f], lvn[f], un[f]);
    // Q1: precomputed class blocks, r = A_vol u + sum_f (A_own u + A_nb u_nb)
    constexpr int NREL = 1 + 2 * NSUB;
    block_mv<R, NP>(d.qvol + (size_t)lev * NP * NP, u, r);
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        const int kind = (inf >> (4 * f)) & 3;
        if (kind == 1 || kind == 2) {
            const int rel = kind == 1 ? 0 : 1 + ((inf >> (4 * f + 2)) & 3);
            const R* A = d.qface + ((((size_t)f * 8 + lev) * NREL + rel) * 2) * NP * NP;
            block_mv<R, NP>(A, u, r);
            block_mv<R, NP>(A + NP * NP, un[f], r);
        }
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        const int kind = (inf >> (4 * f)) & 3;
        if (kind != 3) continue;
        for (int sb = 0; sb < NSUB; ++sb) {
            R uh[NP];
            load_seen<R, NP>(d, tick, B, d.hang[nbf[f] + sb], uh);
            const R* A = d.qface + ((((size_t)f * 8 + lev) * NREL + 1 + NSUB + sb) * 2) * NP * NP;
            block_mv<R, NP>(A, u, r);
            block_mv<R, NP>(A + NP * NP, uh, r);
        }
    }
}

// Probe activation check for element e after a step from u (at t_old) to un (t_old + dte).
// The probes inside the leaf are the root GL nodes a with pfl[lev][a_k] == the leaf's cell
// in every direction k; a pending probe's values before and after the step are the leaf
// polynomial at its position, evaluated by sum factorisation.
// lc, rid: the leaf's cell in its root and the root id (loc[e], root[e]).
// pend: bit q set if probe q of the root may still be pending (from a read of lat before
// the step; a probe it marks that has meanwhile activated fails the crossing test below).
template <typename R, int DIM, int P>
__device__ void lat_check_at(const DevArrays<R>& d, const Tables<R>& T, const Phys<R>& ph, int e, uint32_t inf,
                             int lev, uint32_t lc, int64_t rid, const R* u, const R* un, double t_old, double dte,
                             uint32_t pend = 0xffffffffu, bool known = false) {
    using S = Shape<DIM, P>;
    constexpr int N1 = S::N1, NP = S::NP;
    const int lx[3] = {(int)(lc & 255u), (int)((lc >> 8) & 255u), (int)((lc >> 16) & 255u)};
    unsigned inside_k[3] = {1u, 1u, 1u};
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        inside_k[k] = 0u;
#pragma unroll
        for (int a = 0; a < N1; ++a)
            if (T.pfl[lev][a] == lx[k]) inside_k[k] |= 1u << a;
    }
    uint32_t im = 0u;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        bool in = true;
#pragma unroll
        for (int k = 0; k < DIM; ++k) in = in && ((inside_k[k] >> digit<N1>(q, k)) & 1u);
        if (in) im |= 1u << q;
    }
    bool pending = false;
    im &= pend;
    while (im) {
        const int q = __ffs(im) - 1;
        im &= im - 1u;
        double* lp = d.lat + rid * NP + q;
        if (!known && !isinf(*lp)) continue;
        R Pk[3][3];
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int j = 0; j < N1; ++j) Pk[k][j] = (k < DIM) ? T.pphi[lev][digit<N1>(q, k)][j] : R(1);
        R po = 0, pn = 0;
#pragma unroll
        for (int j2 = 0; j2 < (DIM == 3 ? N1 : 1); ++j2) {
            R t1o = 0, t1n = 0;
#pragma unroll
            for (int j1 = 0; j1 < N1; ++j1) {
                R t0o = 0, t0n = 0;
#pragma unroll
                for (int j0 = 0; j0 < N1; ++j0) {
                    const int idx = j0 + N1 * j1 + N1 * N1 * j2;
                    t0o += Pk[0][j0] * u[idx];
                    t0n += Pk[0][j0] * un[idx];
                }
                t1o += Pk[1][j1] * t0o;
                t1n += Pk[1][j1] * t0n;
            }
            po += Pk[2][j2] * t1o;
            pn += Pk[2][j2] * t1n;
        }
        if (po <= ph.act && pn > ph.act) {
            *lp = t_old + dte * (double)((ph.act - po) / (pn - po));
        } else {
            pending = true;
        }
    }
    if (!pending) d.info[e] = inf & ~INFO_PENDING;
}

template <typename R, int DIM, int P>
__device__ void lat_check(const DevArrays<R>& d, const Tables<R>& T, const Phys<R>& ph, int e,
                          uint32_t inf, int lev, const R* u, const R* un, double t_old, double dte) {
    lat_check_at<R, DIM, P>(d, T, ph, e, inf, lev, d.loc[e], (int64_t)d.root[e], u, un, t_old, dte);
}

template <typename R>
struct TickArgs {
    DevArrays<R> d;
    StimArgs stim;
    double dt;         // barrier step
    double tscale;     // dt * 2^-B: t at tick i of barrier n is (n 2^B + i) * tscale (exact)
    double dte[8];     // dt * 2^-b per level b (exact), and the same rounded to R
    R dteR[8];
    int tick, B;
};

// Canonical time of tick `tick` in the current barrier, ((n 2^B + i) dt) / 2^B (the
// division by 2^B is exact, so scaling dt first gives the same value).  Evaluated only
// where a time is needed (stimulus windows, activation times): FP64 is slow on this part.
template <typename R>
__device__ __forceinline__ double tick_time(const TickArgs<R>& a, int tick) {
    return ((double)a.d.meta->nbar * (double)(1 << a.B) + (double)tick) * a.tscale;
}

// Per-element data that stays fixed during a sweep: the element, its level byte and face
// info, its face neighbours and (Q1) their level bytes.  A tick reads it before waiting for
// the previous tick (programmatic dependent launch), so after the wait only the values are
// loaded, all at once.  (info's probe-pending bit may be cleared by an earlier tick of the
// sweep; a stale bit only repeats a probe check that finds nothing left to do.)
template <int NF, bool NB>
struct TickMeta {
    static constexpr bool HP = NF == 4;   // 2D: the finer neighbours of hanging faces too
    int e;
    uint32_t inf;
    uint8_t lv;
    int nbf[NF];
    uint8_t lvn[NF];
    int hg[HP ? NF : 1][2];               // fine neighbours of a hanging face and their level bytes
    uint8_t hgl[HP ? NF : 1][2];
    uint32_t lc;                          // probe lookup: cell in the root, root id
    int rid;
    uint32_t pend;                        // probes of the root with no activation time yet
};
// Q2: the neighbours are read face by face inside the residual (holding them would spill)
template <int NF>
struct TickMeta<NF, false> {
    int e;
    uint32_t inf;
    uint8_t lv;
};
template <int DIM, int P>
using TickMetaT = TickMeta<2 * DIM, P == 1>;

template <typename R, int DIM, int P>
__device__ __forceinline__ void tick_fetch(const DevArrays<R>& d, int idx, TickMetaT<DIM, P>& m) {
    constexpr int NF = 2 * DIM;
    m.e = d.order[idx];
    m.lv = d.lvl[m.e];
    m.inf = d.info[m.e];
    if constexpr (P != 1) {
    } else if constexpr (DIM == 2) {
        const int4 n = *reinterpret_cast<const int4*>(d.nbr + (size_t)m.e * 4);
        m.nbf[0] = n.x; m.nbf[1] = n.y; m.nbf[2] = n.z; m.nbf[3] = n.w;
    } else {
#pragma unroll
        for (int f = 0; f < NF; f += 2) {
            const int2 n = *reinterpret_cast<const int2*>(d.nbr + (size_t)m.e * NF + f);
            m.nbf[f] = n.x;
            m.nbf[f + 1] = n.y;
        }
    }
    if constexpr (P == 1) {
        m.lc = d.loc[m.e];
        m.rid = d.root[m.e];
        // activation times of the root's probes (only this leaf writes those inside it, at its
        // own steps; a value read before the previous tick's write only repeats a check)
        m.pend = 0u;
        if (m.inf & INFO_PENDING) {
            constexpr int NP = Shape<DIM, P>::NP;
#pragma unroll
            for (int q = 0; q < NP; ++q)
                if (isinf(d.lat[(int64_t)m.rid * NP + q])) m.pend |= 1u << q;
        }
        if constexpr (TickMetaT<DIM, P>::HP) {
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                const bool hanging = ((m.inf >> (4 * f)) & 3) == 3;
#pragma unroll
                for (int sb = 0; sb < 2; ++sb) {
                    m.hg[f][sb] = hanging ? d.hang[m.nbf[f] + sb] : m.e;
                    m.hgl[f][sb] = d.lvl[m.hg[f][sb]];
                }
            }
        }
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            const int kind = (m.inf >> (4 * f)) & 3;
            m.lvn[f] = d.lvl[(kind == 1 || kind == 2) ? m.nbf[f] : m.e];
        }
    }
}

// Q1 residual r = (A u)_e from the class blocks, with the face neighbours and their level
// bytes already known: r = A_vol u + sum_f (A_own u + A_nb u_nb); hanging faces after.
template <typename R, int DIM>
__device__ __forceinline__ void residual_q1(const DevArrays<R>& d, int tick, int B, const TickMetaT<DIM, 1>& m,
                                            int lev, const R* u, R* r) {
    using S = Shape<DIM, 1>;
    constexpr int NP = S::NP, NF = S::NF, NSUB = S::NSUB, NREL = 1 + 2 * NSUB;
    R un[NF][NP];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        const int kind = (m.inf >> (4 * f)) & 3;
        load_seen_lv<R, NP>(d, tick, B, (kind == 1 || kind == 2) ? m.nbf[f] : m.e, m.lvn[f], un[f]);
    }
#pragma unroll
    for (int q = 0; q < NP; ++q) r[q] = R(0);
    block_mv<R, NP>(d.qvol + (size_t)lev * NP * NP, u, r);
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        const int kind = (m.inf >> (4 * f)) & 3;
        if (kind == 1 || kind == 2) {
            const int rel = kind == 1 ? 0 : 1 + ((m.inf >> (4 * f + 2)) & 3);
            const R* A = d.qface + ((((size_t)f * 8 + lev) * NREL + rel) * 2) * NP * NP;
            block_mv<R, NP>(A, u, r);
            block_mv<R, NP>(A + NP * NP, un[f], r);
        }
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        const int kind = (m.inf >> (4 * f)) & 3;
        if (kind != 3) continue;
        for (int sb = 0; sb < NSUB; ++sb) {
            R uh[NP];
            if constexpr (TickMetaT<DIM, 1>::HP) load_seen_lv<R, NP>(d, tick, B, m.hg[f][sb], m.hgl[f][sb], uh);
            else load_seen<R, NP>(d, tick, B, d.hang[m.nbf[f] + sb], uh);
            const R* A = d.qface + ((((size_t)f * 8 + lev) * NREL + 1 + NSUB + sb) * 2) * NP * NP;
            block_mv<R, NP>(A, u, r);
            block_mv<R, NP>(A + NP * NP, uh, r);
        }
    }
}

// Stimulus currents of DOF q of element e at the step start (so) and at the step midpoint
// (sm): -amplitude for every stimulus box holding the node whose window [t0, t1) holds the
// time (the midpoint value enters the RV-T term).
template <typename R>
__device__ __forceinline__ void dof_stim(const TickArgs<R>& a, int e, int tick, double dte_d, int q, R& so, R& sm) {
    so = sm = R(0);
    const double t_i = tick_time(a, tick);
    const double t_mid = t_i + 0.5 * dte_d;
    for (int s = 0; s < a.stim.n; ++s) {
        const bool on_o = (a.stim.t0[s] <= t_i) && (t_i < a.stim.t1[s]);
        const bool on_m = (a.stim.t0[s] <= t_mid) && (t_mid < a.stim.t1[s]);
        if (!on_o && !on_m) continue;
        if (!((a.d.smask[s][e] >> q) & 1u)) continue;
        const R amp = (R)a.stim.amp[s];
        if (on_o) so -= amp;
        if (on_m) sm -= amp;
    }
}

// Update of one DOF given its residual r = (A u)_q, its GL mass Mq = w_q det J and the
// inverse Minv: forward Euler on V, the exponential/FE step on v, and the DOF's share
// Mq [dI^2 + dg^2] of the RV-T midpoint term (returned).  At the element's first step of
// the barrier (ke == 0), Ia/ga receive I and g at the barrier start.
template <typename R>
__device__ __forceinline__ R dof_update(const Phys<R>& ph, R Mq, R Minv, int ke, R dte, R so, R sm, R u, R w, R r,
                                        R& Ia, R& ga, R& un, R& wn) {
    if (ke == 0) {
        Ia = ap_iion(ph, u, w) + so;
        ga = ap_g(ph, u, w);
    }
    const R I = ap_iion(ph, u, w) + so;
    un = u + dte * (-r * Minv - I);
    wn = ap_step_state(ph, u, w, dte);
    const R Vm = R(0.5) * (u + un);
    const R wm = R(0.5) * (w + wn);
    const R dI = ap_iion(ph, Vm, wm) + sm - Ia;
    const R dg = ap_g(ph, Vm, wm) - ga;
    return Mq * (dI * dI + dg * dg);
}

// dof_update for an element without stimulus under the Aliev-Panfilov model (ionic 0) with
// the exponential state step (integrator 1): the same expressions as ap_iion, ap_g and
// ap_step_state without their model and integrator branches, and e^x - 1 as a select of both
// forms, so that the code is straight-line and the items of a thread can interleave.  FIRST:
// the element's first step of the barrier (ke == 0), which sets Ia and ga to I and g at the
// step start; otherwise they are inputs.
template <bool FIRST>
__device__ __forceinline__ float dof_update_ap(const Phys<float>& ph, float Mq, float Minv, float dte, float u, float w,
                                               float r, float& Ia, float& ga, float& un, float& wn) {
    const float I = (ph.k * u * (u - ph.a) * (u - 1.0f) + u * w) * ph.inv_ts;
    un = u + dte * (-r * Minv - I);
    const float vinf = -ph.k * u * (u - ph.a - 1.0f);
    const float den = fmaxf(u + ph.mu2, 1e-6f);
    const float eps = ph.eps0 + __fdividef(ph.mu1 * w, den);
    if (FIRST) {
        Ia = I;
        ga = eps * (vinf - w) * ph.inv_ts;
    }
    const float x = -eps * dte * ph.inv_ts;
    const float em1_t =
        x * (1.0f + x * (0.5f + x * (1.0f / 6.0f + x * (1.0f / 24.0f + x * (1.0f / 120.0f + x * (1.0f / 720.0f))))));
    const float em1_e = expf(x) - 1.0f;
    wn = w + (w - vinf) * (fabsf(x) < 0.0625f ? em1_t : em1_e);
    const float Vm = 0.5f * (u + un);
    const float wm = 0.5f * (w + wn);
    const float dI = (ph.k * Vm * (Vm - ph.a) * (Vm - 1.0f) + Vm * wm) * ph.inv_ts - Ia;
    const float vinf_m = -ph.k * Vm * (Vm - ph.a - 1.0f);
    const float den_m = fmaxf(Vm + ph.mu2, 1e-6f);
    const float dg = (ph.eps0 + __fdividef(ph.mu1 * wm, den_m)) * (vinf_m - wm) * ph.inv_ts - ga;
    return Mq * (dI * dI + dg * dg);
}

// dof_update for DOF q of an element of refinement level lev (mass from the tables).
template <typename R, int DIM, int P>
__device__ __forceinline__ R dof_step(const Tables<R>& T, const Phys<R>& ph, int lev, int q, int ke, R dte, R so,
                                      R sm, R u, R w, R r, R& Ia, R& ga, R& un, R& wn) {
    constexpr int N1 = P + 1;
    R Mq = ph.Wvol[lev];
#pragma unroll
    for (int k = 0; k < DIM; ++k) Mq *= T.w[digit<N1>(q, k)];
    return dof_update<R>(ph, Mq, ph.Minv[lev][q], ke, dte, so, sm, u, w, r, Ia, ga, un, wn);
}

// Pointwise part of one element step (Alg. 1) given the residual r = (A u)_e (dof_step for
// every DOF); returns the element's RV-T term, vmax = max_q |V_new|.
template <typename R, int DIM, int P>
__device__ __forceinline__ R elem_pointwise(const TickArgs<R>& a, const Tables<R>& T, const Phys<R>& ph, int tick,
                                            int e, uint32_t inf, int b, int ke, int lev, const R* u, const R* w,
                                            const R* r, R* Ia, R* ga, R* un, R* wn, R& vmax) {
    constexpr int NP = Shape<DIM, P>::NP;
    const double dte_d = a.dte[b];
    const R dte = a.dteR[b];
    R term = R(0);
    vmax = R(0);
    if constexpr (sizeof(R) == 4) {
        // no stimulus, Aliev-Panfilov, exponential state step: the straight-line update, so
        // that the element's DOFs interleave
        if (!(inf & INFO_STIM) && ph.ionic == 0 && ph.integrator == 1) {
            auto run = [&](auto first) {
                constexpr bool FIRST = decltype(first)::value;
#pragma unroll
                for (int q = 0; q < NP; ++q) {
                    constexpr int N1 = P + 1;
                    R Mq = ph.Wvol[lev];
#pragma unroll
                    for (int kk = 0; kk < DIM; ++kk) Mq *= T.w[digit<N1>(q, kk)];
                    term += dof_update_ap<FIRST>(ph, Mq, ph.Minv[lev][q], dte, u[q], w[q], r[q], Ia[q], ga[q], un[q],
                                                 wn[q]);
                    const R av = un[q] < R(0) ? -un[q] : un[q];
                    vmax = av > vmax ? av : vmax;
                }
            };
            if (ke == 0) run(std::true_type{});
            else run(std::false_type{});
            return term;
        }
    }
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        R so = R(0), sm = R(0);
        if (inf & INFO_STIM) dof_stim<R>(a, e, tick, dte_d, q, so, sm);
        term += dof_step<R, DIM, P>(T, ph, lev, q, ke, dte, so, sm, u[q], w[q], r[q], Ia[q], ga[q], un[q], wn[q]);
        const R av = un[q] < R(0) ? -un[q] : un[q];
        vmax = av > vmax ? av : vmax;
    }
    return term;
}

// One element step of Alg. 1 at tick `tick`: forward Euler on V, exponential/FE step on
// v, the RV-T accumulation and the element's probe check.
template <typename R, int DIM, int P>
__device__ __forceinline__ void tick_elem(const TickArgs<R>& a, const Tables<R>& T, const Phys<R>& ph, int tick,
                                          const TickMetaT<DIM, P>& m, double t_tick) {
    using S = Shape<DIM, P>;
    constexpr int NP = S::NP;
    const DevArrays<R>& d = a.d;
    const int e = m.e;
    const uint32_t inf = m.inf;
    const int b = m.lv & 7, par = (m.lv >> 3) & 1;
    const int ke = tick >> (a.B - b);
    const int cur = par ^ (ke & 1);
    const int lev = (inf >> 24) & 15;
    constexpr int NPS = S::NPS;
    const R* Vc = (cur ? d.V1 : d.V0) + (size_t)e * NPS;
    R* Vd = (cur ? d.V0 : d.V1) + (size_t)e * NPS;
    R* vp = d.v + (size_t)e * NPS;
    // every value this step needs is addressed by now: issue the loads together
    R u[NP], w[NP], r[NP], Ia[NP], ga[NP];
    ld_dofs<R, NP, NPS>(Vc, u);
    ld_dofs<R, NP, NPS>(vp, w);
    double acc0 = 0.0;
    if constexpr (P == 1) {
        if (ke != 0) {
            ld_dofs<R, NP, NPS>(d.Ia + (size_t)e * NPS, Ia);
            ld_dofs<R, NP, NPS>(d.ga + (size_t)e * NPS, ga);
            acc0 = d.acc[e];
        }
        residual_q1<R, DIM>(d, tick, a.B, m, lev, u, r);
    } else {
        // Q2: the barrier-start terms are loaded after the residual (register pressure)
        element_residual<R, DIM, P>(d, T, ph, tick, a.B, e, inf, lev, u, r);
        if (ke != 0) {
            ld_dofs<R, NP, NPS>(d.Ia + (size_t)e * NPS, Ia);
            ld_dofs<R, NP, NPS>(d.ga + (size_t)e * NPS, ga);
            acc0 = d.acc[e];
        }
    }

    R un[NP], wn[NP], vmax;
    const R term = elem_pointwise<R, DIM, P>(a, T, ph, tick, e, inf, b, ke, lev, u, w, r, Ia, ga, un, wn, vmax);
    const double dte_d = a.dte[b];
    if (ke == 0 && b > 0) {
        st_dofs<R, NP, NPS>(d.Ia + (size_t)e * NPS, Ia);
        st_dofs<R, NP, NPS>(d.ga + (size_t)e * NPS, ga);
    }
    st_dofs<R, NP, NPS>(Vd, un);
    st_dofs<R, NP, NPS>(vp, wn);
    d.acc[e] = acc0 + dte_d * (double)term;
    if ((inf & INFO_PENDING) && vmax >= ph.lat_gate)
    {
        const double tt = t_tick >= 0.0 ? t_tick : tick_time(a, tick);
        if constexpr (P == 1)
            lat_check_at<R, DIM, P>(d, T, ph, e, inf, lev, m.lc, m.rid, u, un, tt, dte_d, m.pend, true);
        else lat_check<R, DIM, P>(d, T, ph, e, inf, lev, u, un, tt, dte_d);
    }
}

// One tick of Alg. 1 over the due elements (a prefix of `order`), for callers that
// already waited for the previous tick.
template <typename R, int DIM, int P>
__device__ __forceinline__ void tick_work(const TickArgs<R>& a, const Tables<R>& T, const Phys<R>& ph, int tick) {
    const int n_act = a.d.meta->nact[tick];
    const double t_tick = -1.0;   // computed where a probe check needs it
    for (int idx = (int)gtid(); idx < n_act; idx += (int)gstride()) {
        TickMetaT<DIM, P> m;
        tick_fetch<R, DIM, P>(a.d, idx, m);
        tick_elem<R, DIM, P>(a, T, ph, tick, m, t_tick);
    }
}

// (The bound's "1" lets the Q1 2D FP32 step keep its 168 registers: under the default heuristic
// the compiler held it to 128 and spilled 40 bytes, and the C2 sweep ran 11% slower.)
template <typename R, int DIM, int P>
__global__ void __launch_bounds__(256, 1) k_tick(const TickArgs<R> a, const Tables<R> T, const Phys<R> ph) {
    // the due count and the first element's metadata are fixed during the sweep: read them
    // while the previous tick drains, then wait for its values (the first tick of a sweep
    // is launched without overlap, after the ordering that writes them)
    // (so are the tick's time and the error word: ticks do not set errors)
    const int n_act = a.d.meta->nact[a.tick];
    const bool bad = a.d.meta->err != 0;
    const int idx0 = (int)gtid();
    TickMetaT<DIM, P> m;
    if (idx0 < n_act) tick_fetch<R, DIM, P>(a.d, idx0, m);
    // the tick's time (FP64, a slow pipe here) only where a probe check may need it
    const double t_tick = (idx0 < n_act && (m.inf & INFO_PENDING)) ? tick_time(a, a.tick) : -1.0;
    pdl_enter();
    if (bad) return;
    for (int idx = idx0; idx < n_act; idx += (int)gstride()) {
        if (idx != idx0) tick_fetch<R, DIM, P>(a.d, idx, m);
        tick_elem<R, DIM, P>(a, T, ph, a.tick, m, t_tick);
    }
}

// Kelly-type spatial indicator per element (Eq. dg-error-estimate) on the barrier-start
// values; same-level and coarser neighbours are gathered before the face arithmetic.  In
// FP32 the face-point sums are FP32 and the faces accumulate in FP64 (FP64 arithmetic per
// face point would bound the kernel by the FP64 pipe).
template <typename R, int DIM, int P>
__global__ void k_eta_s(const DevArrays<R> d, const Tables<R> T, const Phys<R> ph) {
    pdl_enter();
    using S = Shape<DIM, P>;
    constexpr int NP = S::NP, NF = S::NF, NSUB = S::NSUB, NPS = S::NPS;
    if (d.meta->err) return;
    const int64_t ne = d.meta->ne;
    for (int64_t e = gtid(); e < ne; e += gstride()) {
        const uint32_t inf = d.info[e];
        const int lev = (inf >> 24) & 15;
        const int par = (d.lvl[e] >> 3) & 1;
        const R* Vc = (par ? d.V1 : d.V0) + (size_t)e * NPS;
        R u[NP];
        ld_dofs<R, NP, NPS>(Vc, u);
        // squared face jumps in the working precision, summed in FP64 (the indicator decides
        // refinement, so its reduction keeps FP64 as on the host)
        double acc = 0.0;
        int nbf[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) nbf[f] = d.nbr[(size_t)e * NF + f];
        if constexpr (P == 1) {
            int src[NF];
            uint8_t lvn[NF];
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                const int kind = (inf >> (4 * f)) & 3;
                src[f] = (kind == 1 || kind == 2) ? nbf[f] : (int)e;
            }
#pragma unroll
            for (int f = 0; f < NF; ++f) lvn[f] = d.lvl[src[f]];
            R un[NF][NP];
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                const R* srcp = (((lvn[f] >> 3) & 1) ? d.V1 : d.V0) + (size_t)src[f] * NPS;
                ld_dofs<R, NP, NPS>(srcp, un[f]);
            }
            constexpr int NT = S::NT, NREL = 1 + 2 * NSUB;
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                const int kind = (inf >> (4 * f)) & 3;
                if (kind != 1 && kind != 2) continue;
                const int rel = kind == 1 ? 0 : 1 + ((inf >> (4 * f + 2)) & 3);
                const R* K = d.qkelly + ((((size_t)f * 8 + lev) * NREL + rel) * 2) * NT * NP;
                R j[NT];
#pragma unroll
                for (int t = 0; t < NT; ++t) j[t] = R(0);
                block_jump<R, NT, NP>(K, u, j);
                block_jump<R, NT, NP>(K + NT * NP, un[f], j);
                R fsum = R(0);
#pragma unroll
                for (int t = 0; t < NT; ++t) fsum += j[t] * j[t];
                acc += (double)fsum;
            }
        } else {
            // Q2: the axis unrolled, the side a loop (half the code of a fully unrolled face
            // loop; the kernel's size bounded it by instruction fetch)
#pragma unroll
            for (int k = 0; k < DIM; ++k)
#pragma unroll 1
            for (int side = 0; side < 2; ++side) {
                const int f = 2 * k + side;
                const int kind = (inf >> (4 * f)) & 3;
                if (kind != 1 && kind != 2) continue;
                const int s = side ? 1 : -1;
                const int nbi = d.nbr[(size_t)e * NF + f];
                const int pn = (d.lvl[nbi] >> 3) & 1;
                const R* src = (pn ? d.V1 : d.V0) + (size_t)nbi * NPS;
                R un[NP];
                ld_dofs<R, NP, NPS>(src, un);
                const int pos = (inf >> (4 * f + 2)) & 3;
                if constexpr (sizeof(R) == 4)
                    acc += ph.kfac[lev][k] * (double)face_kelly_sum<R, DIM, P>(T, ph, k, s, lev, -1, u,
                                                                             kind == 1 ? lev : lev - 1,
                                                                             kind == 1 ? -1 : pos, un, lev);
                else
                    acc += face_kelly<R, DIM, P>(T, ph, k, s, lev, -1, u, kind == 1 ? lev : lev - 1,
                                                 kind == 1 ? -1 : pos, un, lev);
            }
        }
        if constexpr (P == 1) {
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                const int kind = (inf >> (4 * f)) & 3;
                if (kind != 3) continue;
                for (int sb = 0; sb < NSUB; ++sb) {
                    const int nb = d.hang[nbf[f] + sb];
                    const int pn = (d.lvl[nb] >> 3) & 1;
                    const R* src = (pn ? d.V1 : d.V0) + (size_t)nb * NPS;
                    R un[NP];
                    ld_dofs<R, NP, NPS>(src, un);
                    constexpr int NT = S::NT, NREL = 1 + 2 * NSUB;
                    const R* K = d.qkelly + ((((size_t)f * 8 + lev) * NREL + 1 + NSUB + sb) * 2) * NT * NP;
                    R j[NT];
#pragma unroll
                    for (int t = 0; t < NT; ++t) j[t] = R(0);
                    block_jump<R, NT, NP>(K, u, j);
                    block_jump<R, NT, NP>(K + NT * NP, un, j);
                    R fsum = R(0);
#pragma unroll
                    for (int t = 0; t < NT; ++t) fsum += j[t] * j[t];
                    acc += (double)fsum;
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < DIM; ++k)
#pragma unroll 1
            for (int side = 0; side < 2; ++side) {
                const int f = 2 * k + side;
                const int kind = (inf >> (4 * f)) & 3;
                if (kind != 3) continue;
                const int s = side ? 1 : -1;
                const int h0 = d.nbr[(size_t)e * NF + f];
                for (int sb = 0; sb < NSUB; ++sb) {
                    const int nb = d.hang[h0 + sb];
                    const int pn = (d.lvl[nb] >> 3) & 1;
                    const R* src = (pn ? d.V1 : d.V0) + (size_t)nb * NPS;
                    R un[NP];
                    ld_dofs<R, NP, NPS>(src, un);
                    if constexpr (sizeof(R) == 4)
                        acc += ph.kfac[lev + 1][k] *
                               (double)face_kelly_sum<R, DIM, P>(T, ph, k, s, lev, sb, u, lev + 1, -1, un, lev + 1);
                    else
                        acc += face_kelly<R, DIM, P>(T, ph, k, s, lev, sb, u, lev + 1, -1, un, lev + 1);
                }
            }
        }
        d.eta_s[e] = sqrt(acc);
    }
}

// Barrier epilogue: eta^t = sqrt(acc)/dt, parity flip of single-step elements, non-finite
// check, per-block partial sums of int V = sum_q M_q V_q (FP64).
template <typename R, int DIM, int P>
__global__ void __launch_bounds__(256) k_epilogue(const DevArrays<R> d, const double* __restrict__ mtab,
                                                 double dt, double inv_dt, int inv_dt_exact, int mass_per_elem) {
    pdl_enter();
    using S = Shape<DIM, P>;
    constexpr int NP = S::NP;
    __shared__ double red[256];
    if (d.meta->err) return;
    const int64_t ne = d.meta->ne;
    double loc = 0.0;
    bool bad = false;
    for (int64_t e = gtid(); e < ne; e += gstride()) {
        // eta^t = sqrt(acc) / dt in FP64 (it sets b^cell); the product with 1/dt equals the
        // quotient whenever dt is a power of two, as the automatic barrier step is
        d.eta_t[e] = inv_dt_exact ? sqrt(d.acc[e]) * inv_dt : sqrt(d.acc[e]) / dt;
        uint8_t lv = d.lvl[e];
        if ((lv & 7) == 0) {
            lv ^= 8;
            d.lvl[e] = lv;
        }
        const int par = (lv >> 3) & 1;
        const R* Vc = (par ? d.V1 : d.V0) + (size_t)e * S::NPS;
        const R* w = d.v + (size_t)e * S::NPS;
        const int lev = (d.info[e] >> 24) & 15;
        // GL masses: per (level, node) on box elements, per (element, node) on mapped ones
        const double* Mq = mtab + (mass_per_elem ? (size_t)e * NP : (size_t)lev * NP);
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            const R x = Vc[q];
            loc += Mq[q] * (double)x;
            bad = bad || !isfinite(x) || !isfinite(w[q]);
        }
    }
    if (bad) atomicOr(&d.meta->nf_pending, 1u);
    red[threadIdx.x] = loc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    __shared__ bool last;
    if (threadIdx.x == 0) {
        d.partial[blockIdx.x] = red[0];
        __threadfence();
        last = atomicAdd(&d.meta->done_blocks, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    // the last block: fixed-order sum of the partials, barrier count, non-finite flag
    __threadfence();
    double s2 = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) s2 += ((volatile double*)d.partial)[i];
    red[threadIdx.x] = s2;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        DevMeta* m = d.meta;
        m->integral = red[0];
        m->nbar += 1;
        m->done_blocks = 0;
        if (m->nf_pending) {
            m->err |= ERR_NONFINITE;
            m->nf_pending = 0;
        }
    }
}



// Q1 tick with a group of G = (p+1)^d lanes per element (4 in 2D, 8 in 3D), lane g owning
// DOF g: it computes row g of the residual from the class blocks (r_g = A_vol[g] u +
// sum_f A_own,f[g] u + A_nb,f[g] u_nb,f) and the pointwise step of DOF g, so G times more
// threads are in flight than with a thread per element and each runs a short chain.
// Everything fixed during the sweep -- the element, its level byte and face info, its
// neighbours and their level bytes, and in 2D the block rows -- is read before waiting for
// the previous tick; after the wait every value load is issued at once.
template <typename R, int DIM>
struct GroupMeta {
    static constexpr int NP = Shape<DIM, 1>::NP, NF = 2 * DIM;
    static constexpr bool ROWS = DIM == 2;     // block rows held in registers (2D only)
    int e;
    uint32_t inf;
    uint8_t lv;
    int nbf[NF];
    uint8_t lvn[NF];
    R vrow[NP];
    R orow[ROWS ? NF : 1][NP];
    R nrow[ROWS ? NF : 1][NP];
};

template <typename R, int DIM>
__device__ __forceinline__ void group_fetch(const DevArrays<R>& d, int64_t idx, int g, GroupMeta<R, DIM>& m) {
    using M = GroupMeta<R, DIM>;
    constexpr int NP = M::NP, NF = M::NF, NREL = 1 + 2 * Shape<DIM, 1>::NSUB;
    m.e = d.order[idx];
    m.lv = d.lvl[m.e];
    m.inf = d.info[m.e];
#pragma unroll
    for (int f = 0; f < NF; ++f) m.nbf[f] = d.nbr[(size_t)m.e * NF + f];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        const int kind = (m.inf >> (4 * f)) & 3;
        m.lvn[f] = d.lvl[(kind == 1 || kind == 2) ? m.nbf[f] : m.e];
    }
    const int lev = (m.inf >> 24) & 15;
    ld_row<R, NP>(d.qvol + ((size_t)lev * NP + g) * NP, m.vrow);
    if constexpr (M::ROWS) {
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            const int kind = (m.inf >> (4 * f)) & 3;
            const int rel = kind == 2 ? 1 + ((m.inf >> (4 * f + 2)) & 3) : 0;
            const R* A = d.qface + ((((size_t)f * 8 + lev) * NREL + rel) * 2) * NP * NP;
            ld_row<R, NP>(A + g * NP, m.orow[f]);
            ld_row<R, NP>(A + NP * NP + g * NP, m.nrow[f]);
        }
    }
}

template <typename R, int DIM>
__global__ void __launch_bounds__(256) k_tick_group(const TickArgs<R> a, const Phys<R> ph, const Tables<R> T) {
    using S = Shape<DIM, 1>;
    using M = GroupMeta<R, DIM>;
    constexpr int N1 = S::N1, NP = S::NP, NF = S::NF, NSUB = S::NSUB, NREL = 1 + 2 * NSUB;
    constexpr int G = NP;
    const DevArrays<R>& d = a.d;
    const int tick = a.tick, B = a.B;
    const int lane = threadIdx.x & 31;
    const int g = lane % G;
    const unsigned gmask = ((1u << G) - 1u) << (lane - g);
    const int64_t gsz = gstride() / G;
    // per (level, node) GL mass and inverse in shared memory (lanes read different nodes)
    __shared__ R sMq[8 * NP], sMinv[8 * NP];
    for (int i = threadIdx.x; i < 8 * NP; i += blockDim.x) {
        const int l = i / NP, q = i - l * NP;
        R w = ph.Wvol[l];
#pragma unroll
        for (int k = 0; k < DIM; ++k) w *= T.w[digit<N1>(q, k)];
        sMq[i] = w;
        sMinv[i] = ph.Minv[l][q];
    }
    // the due count, the element order and the error word do not change during a sweep
    // (the first tick of a sweep is launched without overlap, after the ordering)
    const int n_act = d.meta->nact[tick];
    const bool bad = d.meta->err != 0;
    int64_t idx = gtid() / G;
    M m;
    if (idx < n_act) group_fetch<R, DIM>(d, idx, g, m);
    __syncthreads();
    pdl_enter();
    if (bad) return;
    for (bool first = true; idx < n_act; idx += gsz, first = false) {
        if (!first) group_fetch<R, DIM>(d, idx, g, m);
        const int e = m.e;
        const uint32_t inf = m.inf;
        const int b = m.lv & 7, par = (m.lv >> 3) & 1;
        const int ke = tick >> (B - b);
        const int cur = par ^ (ke & 1);
        const int lev = (inf >> 24) & 15;
        // every value this step needs: own row, neighbours as seen, state, barrier-start terms
        R u[NP];
        constexpr int NPS = S::NPS;
        ld_dofs<R, NP, NPS>((cur ? d.V1 : d.V0) + (size_t)e * NPS, u);
        const R w = d.v[(size_t)e * NPS + g];
        R un[NF][NP];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            const int kind = (inf >> (4 * f)) & 3;
            load_seen_lv<R, NP>(d, tick, B, (kind == 1 || kind == 2) ? m.nbf[f] : e, m.lvn[f], un[f]);
        }
        R Ia = R(0), ga = R(0);
        double acc0 = 0.0;
        if (ke != 0) {
            Ia = d.Ia[(size_t)e * NPS + g];
            ga = d.ga[(size_t)e * NPS + g];
            if (g == 0) acc0 = d.acc[e];
        }
        // row g of the residual
        R rg = R(0);
#pragma unroll
        for (int j = 0; j < NP; ++j) rg += m.vrow[j] * u[j];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            const int kind = (inf >> (4 * f)) & 3;
            if (kind == 1 || kind == 2) {
                if constexpr (M::ROWS) {
#pragma unroll
                    for (int j = 0; j < NP; ++j) rg += m.orow[f][j] * u[j] + m.nrow[f][j] * un[f][j];
                } else {
                    const int rel = kind == 2 ? 1 + ((inf >> (4 * f + 2)) & 3) : 0;
                    const R* A = d.qface + ((((size_t)f * 8 + lev) * NREL + rel) * 2) * NP * NP;
                    R ro[NP], rn[NP];
                    ld_row<R, NP>(A + g * NP, ro);
                    ld_row<R, NP>(A + NP * NP + g * NP, rn);
#pragma unroll
                    for (int j = 0; j < NP; ++j) rg += ro[j] * u[j] + rn[j] * un[f][j];
                }
            }
        }
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            const int kind = (inf >> (4 * f)) & 3;
            if (kind != 3) continue;
            for (int sb = 0; sb < NSUB; ++sb) {
                R uh[NP], ro[NP], rn[NP];
                load_seen<R, NP>(d, tick, B, d.hang[m.nbf[f] + sb], uh);
                const R* A = d.qface + ((((size_t)f * 8 + lev) * NREL + 1 + NSUB + sb) * 2) * NP * NP;
                ld_row<R, NP>(A + g * NP, ro);
                ld_row<R, NP>(A + NP * NP + g * NP, rn);
#pragma unroll
                for (int j = 0; j < NP; ++j) rg += ro[j] * u[j] + rn[j] * uh[j];
            }
        }
        // pointwise step of DOF g
        const double dte_d = a.dte[b];
        R so = R(0), smd = R(0);
        if (inf & INFO_STIM) dof_stim<R>(a, e, tick, dte_d, g, so, smd);
        R my_u = u[0];
#pragma unroll
        for (int q = 1; q < NP; ++q)
            if (q == g) my_u = u[q];
        R un_g, wn_g;
        R term = dof_update<R>(ph, sMq[lev * NP + g], sMinv[lev * NP + g], ke, a.dteR[b], so, smd, my_u, w, rg, Ia,
                               ga, un_g, wn_g);
        R vmax = un_g < R(0) ? -un_g : un_g;
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            term += __shfl_xor_sync(gmask, term, o, G);
            const R om = __shfl_xor_sync(gmask, vmax, o, G);
            vmax = om > vmax ? om : vmax;
        }
        ((cur ? d.V0 : d.V1) + (size_t)e * NPS)[g] = un_g;
        d.v[(size_t)e * NPS + g] = wn_g;
        if (ke == 0 && b > 0) {
            d.Ia[(size_t)e * NPS + g] = Ia;
            d.ga[(size_t)e * NPS + g] = ga;
        }
        if (g == 0) d.acc[e] = acc0 + dte_d * (double)term;
        if ((inf & INFO_PENDING) && vmax >= ph.lat_gate) {
            R unv[NP];
#pragma unroll
            for (int q = 0; q < NP; ++q) unv[q] = __shfl_sync(gmask, un_g, q, G);
            if (g == 0) lat_check<R, DIM, 1>(d, T, ph, e, inf, lev, u, unv, tick_time(a, tick), dte_d);
        }
    }
}

// Grid-wide barrier number `round` (1, 2, ...) of a cooperative launch (every block resident):
// each block's thread 0 counts its arrival in m->gbar (zeroed before the launch) and waits,
// with at most `limit` polls 64 ns apart (~1 s by default), until every block of the round has
// arrived.  A wait that gives up sets ERR_WAIT (the host reports it) and lets the block go on:
// no hang.
constexpr uint32_t GRID_WAIT_LIMIT = 1u << 24;
__device__ __forceinline__ void grid_barrier(DevMeta* m, unsigned round, uint32_t limit = GRID_WAIT_LIMIT) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned target = round * gridDim.x;
        __threadfence();
        atomicAdd(&m->gbar, 1u);
        uint32_t it = 0;
        while (*(volatile unsigned*)&m->gbar < target) {
            if (++it > limit) {
                atomicOr(&m->err, ERR_WAIT);
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
    }
    __syncthreads();
}

// The whole sweep of a barrier in one cooperative launch: every tick of Alg. 1 with a
// grid-wide barrier between ticks (the Jacobi reading needs all of tick i before tick
// i+1), then the epilogue with a fixed-order final reduction by block 0.  The grid is
// sized from the occupancy API so that every block is resident.
template <typename R, int DIM, int P>
__global__ void __launch_bounds__(256) k_sweep(const TickArgs<R> a, const Tables<R> T, const Phys<R> ph,
                                              const double* __restrict__ mtab) {
    using S = Shape<DIM, P>;
    constexpr int NP = S::NP;
    const DevArrays<R>& d = a.d;
    if (d.meta->err) return;             // uniform: nothing below changes err before the end
    const int nt = 1 << a.B;
    for (int i = 0; i < nt; ++i) {
        tick_work<R, DIM, P>(a, T, ph, i);
        grid_barrier(d.meta, (unsigned)(i + 1));
    }
    __shared__ double red[256];
    const int64_t ne = d.meta->ne;
    double loc = 0.0;
    bool bad = false;
    for (int64_t e = gtid(); e < ne; e += gstride()) {
        d.eta_t[e] = sqrt(d.acc[e]) / a.dt;
        uint8_t lv = d.lvl[e];
        if ((lv & 7) == 0) {
            lv ^= 8;
            d.lvl[e] = lv;
        }
        const int par = (lv >> 3) & 1;
        const R* Vc = (par ? d.V1 : d.V0) + (size_t)e * S::NPS;
        const R* w = d.v + (size_t)e * S::NPS;
        const int lev = (d.info[e] >> 24) & 15;
        const double* Mq = mtab + lev * NP;
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            const R x = Vc[q];
            loc += Mq[q] * (double)x;
            bad = bad || !isfinite(x) || !isfinite(w[q]);
        }
    }
    if (bad) atomicOr(&d.meta->nf_pending, 1u);
    red[threadIdx.x] = loc;
    __syncthreads();
    for (int s2 = blockDim.x / 2; s2 > 0; s2 >>= 1) {
        if (threadIdx.x < s2) red[threadIdx.x] += red[threadIdx.x + s2];
        __syncthreads();
    }
    if (threadIdx.x == 0) d.partial[blockIdx.x] = red[0];
    grid_barrier(d.meta, (unsigned)(nt + 1));
    if (blockIdx.x != 0) return;
    double s3 = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) s3 += d.partial[i];
    red[threadIdx.x] = s3;
    __syncthreads();
    for (int s2 = blockDim.x / 2; s2 > 0; s2 >>= 1) {
        if (threadIdx.x < s2) red[threadIdx.x] += red[threadIdx.x + s2];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        DevMeta* m = d.meta;
        m->integral = red[0];
        m->nbar += 1;
        if (m->nf_pending) {
            m->err |= ERR_NONFINITE;
            m->nf_pending = 0;
        }
    }
}

// Copy V (current slot by parity) or v to a compact output (NP values per element).
template <typename R, int NP, int NPS, typename Out>
__global__ void k_gather(const DevArrays<R> d, int64_t ne, int which, Out* out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= ne * NP) return;
    const int64_t e = i / NP, j = e * NPS + (i - e * NP);
    if (which == 0) {
        const int par = (d.lvl[e] >> 3) & 1;
        out[i] = (Out)((par ? d.V1 : d.V0)[j]);
    } else {
        out[i] = (Out)d.v[j];
    }
}

// V (current slot) and the state variable into one compact FP32 buffer [V | v].
template <typename R, int NP, int NPS>
__global__ void k_gather_f32(const DevArrays<R> d, int64_t ne, float* outV, float* outS) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= ne * NP) return;
    const int64_t e = i / NP, j = e * NPS + (i - e * NP);
    const int par = (d.lvl[e] >> 3) & 1;
    if (outV) outV[i] = (float)((par ? d.V1 : d.V0)[j]);
    if (outS) outS[i] = (float)d.v[j];
}

// The same for page-locked host buffers read or written over the host link: four consecutive
// compact values per thread as one 16-byte access (buffers 16-byte aligned; the last partial
// group value by value), which keeps more bytes in flight per request than 4-byte accesses.
template <typename R, int NP, int NPS>
__global__ void k_gather_f32x4(const DevArrays<R> d, int64_t ne, float* outV, float* outS) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, n = ne * NP, i0 = 4 * t;
    if (i0 >= n) return;
    float va[4] = {0.0f, 0.0f, 0.0f, 0.0f}, sa[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int64_t i = i0 + k;
        if (i < n) {
            const int64_t e = i / NP, j = e * NPS + (i - e * NP);
            const int par = (d.lvl[e] >> 3) & 1;
            va[k] = (float)((par ? d.V1 : d.V0)[j]);
            sa[k] = (float)d.v[j];
        }
    }
    if (i0 + 3 < n) {
        if (outV) reinterpret_cast<float4*>(outV)[t] = make_float4(va[0], va[1], va[2], va[3]);
        if (outS) reinterpret_cast<float4*>(outS)[t] = make_float4(sa[0], sa[1], sa[2], sa[3]);
    } else {
        for (int k = 0; i0 + k < n; ++k) {
            if (outV) outV[i0 + k] = va[k];
            if (outS) outS[i0 + k] = sa[k];
        }
    }
}

template <typename R, int NP, int NPS>
__global__ void k_scatter_initial_x4(DevArrays<R> d, int64_t ne, const float* V, const float* w) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, n = ne * NP, i0 = 4 * t;
    if (i0 < n) {
        float va[4] = {0.0f, 0.0f, 0.0f, 0.0f}, wa[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (i0 + 3 < n) {
            const float4 a = reinterpret_cast<const float4*>(V)[t];
            va[0] = a.x; va[1] = a.y; va[2] = a.z; va[3] = a.w;
            if (w) {
                const float4 b = reinterpret_cast<const float4*>(w)[t];
                wa[0] = b.x; wa[1] = b.y; wa[2] = b.z; wa[3] = b.w;
            }
        } else {
            for (int k = 0; i0 + k < n; ++k) {
                va[k] = V[i0 + k];
                if (w) wa[k] = w[i0 + k];
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t i = i0 + k;
            if (i < n) {
                const int64_t e = i / NP, j = e * NPS + (i - e * NP);
                d.V0[j] = (R)va[k];
                if (w) d.v[j] = (R)wa[k];
            }
        }
    }
    // element t: the pad values of its padded rows, and its level byte's parity reset
    if (t < ne) {
#pragma unroll
        for (int q = NP; q < NPS; ++q) {
            d.V0[t * NPS + q] = R(0);
            if (w) d.v[t * NPS + q] = R(0);
        }
        d.lvl[t] &= 7;
    }
}

// Set V (into slot 0, parity reset) and optionally v from compact FP64 or FP32 input; the
// pad values of padded rows are set to 0.
template <typename R, int NP, int NPS, typename In>
__global__ void k_scatter_initial(DevArrays<R> d, int64_t ne, const In* V, const In* w) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= ne * NPS) return;
    const int64_t e = j / NPS, q = j - e * NPS, i = e * NP + q;
    const bool pad = q >= NP;
    d.V0[j] = pad ? R(0) : (R)V[i];
    if (w) d.v[j] = pad ? R(0) : (R)w[i];
    if (q == 0) d.lvl[e] &= 7;
}

// Activation at the current time for probes already above threshold, and the
// per-element pending flag (any probe of the element not yet activated).
template <typename R, int DIM, int P>
__global__ void k_lat_refresh(DevArrays<R> d, const Tables<R> T, const Phys<R> ph, double t, int mark_now,
                              int force) {
    pdl_enter();
    using S = Shape<DIM, P>;
    constexpr int N1 = S::N1, NP = S::NP;
    if (d.meta->err || !(force || d.meta->changed)) return;
    const int64_t ne = d.meta->ne;
    for (int64_t e = gtid(); e < ne; e += gstride()) {
    uint32_t inf = d.info[e];
    const int lev = (inf >> 24) & 15;
    const int par = (d.lvl[e] >> 3) & 1;
    const R* Vc = (par ? d.V1 : d.V0) + (size_t)e * S::NPS;
    R u[NP];
    ld_dofs<R, NP, S::NPS>(Vc, u);
    const uint32_t lc = d.loc[e];
    const int lx[3] = {(int)(lc & 255u), (int)((lc >> 8) & 255u), (int)((lc >> 16) & 255u)};
    const int64_t rid = d.root[e];
    bool pending = false;
    for (int q = 0; q < NP; ++q) {
        bool inside = true;
#pragma unroll
        for (int k = 0; k < DIM; ++k) inside = inside && (T.pfl[lev][digit<N1>(q, k)] == lx[k]);
        if (!inside) continue;
        double* lp = d.lat + rid * NP + q;
        if (!isinf(*lp)) continue;
        if (mark_now) {
            R pv = 0;
            for (int j = 0; j < NP; ++j) {
                R w = R(1);
#pragma unroll
                for (int k = 0; k < DIM; ++k) w *= T.pphi[lev][digit<N1>(q, k)][digit<N1>(j, k)];
                pv += w * u[j];
            }
            if (pv > ph.act) {
                *lp = t;
                continue;
            }
        }
        pending = true;
    }
    inf = pending ? (inf | INFO_PENDING) : (inf & ~INFO_PENDING);
    d.info[e] = inf;
    }
}

// Solution transfer after adaptation (Alg. 1 adapt steps): keep, prolong (parent
// polynomial at the child nodes) or restrict (L2 projection with the children's GL
// rule, exact for the diagonal GL mass).  Old arrays in `o`, new in `n` (slot 0).  Kept
// elements (most of them) with rows of 27 values are copied by whole warps: a warp takes 32
// consecutive new elements and copies their rows lane-parallel over the values, the old row
// of each element broadcast from its lane; shorter rows, refined and coarsened elements take
// a thread each.
template <typename R, int DIM, int P>
__global__ void k_transfer(const DevArrays<R> o, DevArrays<R> n, const int8_t* pkind, const int32_t* psrc,
                           const int8_t* pbits, const Tables<R> T) {
    pdl_enter();
    using S = Shape<DIM, P>;
    constexpr int N1 = S::N1, NP = S::NP, NC = 1 << DIM, NPS = S::NPS;
    if (n.meta->err) return;
    const int64_t nne = n.meta->ne;
    if constexpr (NP < 27) {
        // short rows (Q1, 2D Q2): a thread per kept element
        for (int64_t i = gtid(); i < nne; i += gstride()) {
            if (pkind[i] != 0) continue;
            const int src = psrc[i];
            const int par = (o.lvl[src] >> 3) & 1;
            const R* Vo = (par ? o.V1 : o.V0) + (size_t)src * NPS;
            const R* wo = o.v + (size_t)src * NPS;
#pragma unroll
            for (int q = 0; q < NPS; ++q) {
                n.V0[(size_t)i * NPS + q] = Vo[q];
                n.v[(size_t)i * NPS + q] = wo[q];
            }
            n.eta_t[i] = o.eta_t[src];
            n.lvl[i] = 0;
        }
    } else {
        const int lane = threadIdx.x & 31;
        const int64_t nwarp = gstride() >> 5;
        for (int64_t base = (gtid() >> 5) * 32; base < nne; base += nwarp * 32) {
            const int64_t i = base + lane;
            long long vrow = 0, wrow = 0;   // old rows of a kept element (0: not kept)
            if (i < nne && pkind[i] == 0) {
                const int src = psrc[i];
                const int par = (o.lvl[src] >> 3) & 1;
                vrow = (long long)((par ? o.V1 : o.V0) + (size_t)src * NPS);
                wrow = (long long)(o.v + (size_t)src * NPS);
                n.eta_t[i] = o.eta_t[src];
                n.lvl[i] = 0;
            }
            // value idx = lane + 32 j of the warp's block of padded rows: row r = idx / NPS,
            // column q (the pad copied too); every load of the block is issued before the
            // first store
            R xv[NPS], xw[NPS];
            bool keep[NPS];
            int r = lane / NPS, q = lane - (lane / NPS) * NPS;
#pragma unroll
            for (int j = 0; j < NPS; ++j) {
                const long long vr = __shfl_sync(0xffffffffu, vrow, r);
                const long long wr = __shfl_sync(0xffffffffu, wrow, r);
                keep[j] = vr != 0;
                xv[j] = keep[j] ? reinterpret_cast<const R*>(vr)[q] : R(0);
                xw[j] = keep[j] ? reinterpret_cast<const R*>(wr)[q] : R(0);
                q += 32 % NPS;
                r += 32 / NPS;
                if (q >= NPS) {
                    q -= NPS;
                    ++r;
                }
            }
            const size_t o0 = (size_t)base * NPS + lane;
#pragma unroll
            for (int j = 0; j < NPS; ++j) {
                if (keep[j]) {
                    n.V0[o0 + 32 * j] = xv[j];
                    n.v[o0 + 32 * j] = xw[j];
                }
            }
        }
    }
    for (int64_t i = gtid(); i < nne; i += gstride()) {
    const int kd = pkind[i];
    if (kd == 0) continue;
    const int src = psrc[i];
    R* Vn = n.V0 + (size_t)i * NPS;
    R* wn = n.v + (size_t)i * NPS;
#pragma unroll
    for (int q = NP; q < NPS; ++q) Vn[q] = wn[q] = R(0);
    if (kd == 1) {
        const int bits = pbits[i];
        const int par = (o.lvl[src] >> 3) & 1;
        const R* Vo = (par ? o.V1 : o.V0) + (size_t)src * NPS;
        const R* wo = o.v + (size_t)src * NPS;
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            R a = 0, c = 0;
            for (int j = 0; j < NP; ++j) {
                R w = R(1);
#pragma unroll
                for (int k = 0; k < DIM; ++k) w *= T.Pi[(bits >> k) & 1][digit<N1>(q, k)][digit<N1>(j, k)];
                a += w * Vo[j];
                c += w * wo[j];
            }
            Vn[q] = a;
            wn[q] = c;
        }
        n.eta_t[i] = o.eta_t[src];
    } else {
        R a[NP], c[NP];
#pragma unroll
        for (int q = 0; q < NP; ++q) a[q] = c[q] = R(0);
        double et = 0.0;
        for (int cb = 0; cb < NC; ++cb) {
            const int ch = src + cb;
            const int par = (o.lvl[ch] >> 3) & 1;
            const R* Vo = (par ? o.V1 : o.V0) + (size_t)ch * NPS;
            const R* wo = o.v + (size_t)ch * NPS;
            et += o.eta_t[ch];
            for (int qc = 0; qc < NP; ++qc) {
                // the child's GL weight in the parent's measure; on a mapped mesh the child's
                // own GL mass (divided by the parent's below)
                R wc = R(1);
                if (o.mq) {
                    wc = (R)o.mq[(size_t)ch * NP + qc];
                } else {
#pragma unroll
                    for (int k = 0; k < DIM; ++k) wc *= T.w[digit<N1>(qc, k)] * R(0.5);
                }
                const R xv = wc * Vo[qc], xw = wc * wo[qc];
#pragma unroll
                for (int q = 0; q < NP; ++q) {
                    R w = R(1);
#pragma unroll
                    for (int k = 0; k < DIM; ++k) w *= T.Pi[(cb >> k) & 1][digit<N1>(qc, k)][digit<N1>(q, k)];
                    a[q] += w * xv;
                    c[q] += w * xw;
                }
            }
        }
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            R wq = R(1);
            if (n.mq) {
                wq = (R)n.mq[(size_t)i * NP + q];
            } else {
#pragma unroll
                for (int k = 0; k < DIM; ++k) wq *= T.w[digit<N1>(q, k)];
            }
            Vn[q] = a[q] / wq;
            wn[q] = c[q] / wq;
        }
        n.eta_t[i] = et / NC;
    }
    n.lvl[i] = 0;
    }
}

}  // namespace mdl

