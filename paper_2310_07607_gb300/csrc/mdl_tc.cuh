// mdl_tc.cuh -- tensor-core (tcgen05) element residual for the Q2 3D FP32 sweep.
//
// For an element whose six faces all have a same-level neighbour, the SIPG residual
// (Eq. monodomain-primal-formulation with the flux of Eq. monodomain-numerical-flux) is
//   r_e = A_self(l) u_e + sum_f A_nb,f(l) u_nb,f,   A_self = A_vol + sum_f A_own,f,
// and on box elements every one of these blocks scales with the level as
// A(l) = 2^((2-d) l) A(0) (volume: (2/h)^2 h^d; faces: h^(d-1) (1/h)), so a single set of
// level-0 blocks serves every element up to an exact power-of-two row scale.  A tile of
// 64 due elements is one tcgen05 MMA problem
//   D[64 x 32] = U[64 x 192] B^T,   U row i = [u_e | u_nb,1 | ... | u_nb,6] (7 x 27 values),
//   B[32 x 192] = [A_self(0) | A_nb,1(0) | ... | A_nb,6(0)],
// with D in tensor memory (one TMEM lane per element, one column per output DOF).
//
// Precision.  A has zero row sums (A 1 = 0), so r_e is unchanged when the element mean c of
// u_e is subtracted from every gathered value: the operand is y = x - c, whose size is the
// local variation of V.  Both operands are split into two FP16 terms (y = y_hi + y_lo,
// B = B_hi + B_lo, each term with an 11-bit significand; B scaled by 2^t, each row of U by
// its own power of two that brings max |y| to [2^13, 2^14)) and the product is
// U_hi B_hi + U_hi B_lo + U_lo B_hi with FP32 accumulation: about 22 significant bits
// relative to the row's variation, as FP32 arithmetic on the CUDA cores.  (One TF32 term per
// operand loses ~2^-11 of y per step; the temporal indicator, a sum of squared small
// differences, then drifts by up to ~10% on a front.  Two TF32 terms of U would need
// 192 KB of shared memory per tile; FP16 terms of the same significand take half.)
//
// Faces that are not same-level interior faces (boundary, coarser or finer neighbours) are
// zero slots in U; their exact contribution minus the same-level own block that A_self
// assumed is added on the CUDA cores in FP32 from precomputed level-0 correction blocks
// (same power-of-two level scaling), on the same mean-shifted values.
//
// Shared-memory operands use the 128-byte swizzled K-major layout: 8-row x 128-byte atoms
// (64 FP16 values per row), atoms of one 64-value K block stacked over the rows, K blocks
// outermost.  The MMA of K step j (16 values) starts 32 j bytes into its atom.  With M = 64
// the accumulator row 16 w + t sits in TMEM lane 32 w + t (w = 0..3).
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

#include "mdl_kernels.cuh"

namespace mdl {
namespace tc {

constexpr int M = 64;           // elements per tile (M = 64 MMA: row 16 w + t in TMEM lane 32 w + t)
constexpr int N = 32;           // output DOFs per element (27 used)
constexpr int K = 192;          // 7 slots x 27 input DOFs (189 used, 3 zero)
constexpr int KU = 189;         // used K
constexpr int NP = 27;
constexpr int NPS = 28;         // row stride of the per-DOF state arrays (27 values and a pad)
constexpr int SLOTS = 7;
constexpr int THREADS = 256;    // 8 warps; two CTAs per SM overlap each other's latencies
constexpr int RST = 29;         // row stride of the residual staging array (odd: no bank conflicts)
constexpr uint32_t TMEM_COLS = 32;
constexpr int KSTEP = 16;       // K per kind::f16 MMA

// Shared-memory plan (bytes from a 1024-aligned base).
constexpr int B_BYTES = N * K * 2;                    // one FP16 term of B
constexpr int U_BYTES = M * K * 2;                    // one FP16 term of U
constexpr int OFF_BHI = 0;
constexpr int OFF_BLO = OFF_BHI + B_BYTES;
constexpr int OFF_UHI = OFF_BLO + B_BYTES;
constexpr int OFF_ULO = OFF_UHI + U_BYTES;
constexpr int OFF_R = OFF_ULO + U_BYTES;              // float [M][RST] scaled residual
constexpr int OFF_SCR = OFF_R + M * RST * 4;          // float [8 warps][2][32] per-warp scratch
constexpr int OFF_PTR = OFF_SCR + 8 * 2 * 32 * 4;     // const float* [8][M]: row of slot s (seen value)
constexpr int OFF_PTRO = OFF_PTR + M * 8 * 8;         // const float* [8][M]: other V slot (interpolated slots only)
constexpr int OFF_E = OFF_PTRO + M * 8 * 8;           // int32 [2][M] element id (-1: padding row)
constexpr int OFF_INF = OFF_E + 2 * M * 4;            // uint32 [2][M] face info
constexpr int OFF_NB = OFF_INF + 2 * M * 4;           // int32 [6][M] face neighbours
constexpr int OFF_TH = OFF_NB + M * 6 * 4;            // float [8][M] time-interpolation weight (interpolated slots only)
constexpr int OFF_RS = OFF_TH + M * 8 * 4;            // float 2^-sc: undoes the row's operand scale
constexpr int OFF_C = OFF_RS + M * 4;                 // float operand mean c of the row
constexpr int OFF_LV = OFF_C + M * 4;                 // uint8 [2][M] level byte
constexpr int OFF_LIVE = OFF_LV + 2 * M;              // uint8 bit s: slot s holds values
constexpr int OFF_INTP = OFF_LIVE + M;                // uint8 bit s: slot s is interpolated in time
constexpr int OFF_IRR = OFF_INTP + M;                 // uint8 [2][M] element has a non-regular face
constexpr int OFF_CORR = ((OFF_IRR + 2 * M + 15) / 16) * 16;  // float [M][RST] residual corrections
constexpr int OFF_MTAB = OFF_CORR + M * RST * 4;      // float [8][27] GL mass, [8][27] inverse, [8] dt_e
constexpr int OFF_MBAR = ((OFF_MTAB + (2 * 8 * NP + 8) * 4 + 7) / 8) * 8;
constexpr int OFF_FLAG = OFF_MBAR + 8;
constexpr int OFF_TMEM = OFF_FLAG + 8;
constexpr int SMEM_BYTES = OFF_TMEM + 16 + 1024;      // + alignment slack of the dynamic base
static_assert(OFF_UHI % 1024 == 0 && OFF_ULO % 1024 == 0 && OFF_BLO % 1024 == 0, "operand alignment");
static_assert(2 * (SMEM_BYTES + 1024) <= 228 * 1024, "two CTAs per SM");

constexpr unsigned ERR_TIMEOUT = ERR_WAIT;            // a bounded wait of the sweep gave up
constexpr uint32_t WAIT_LIMIT = 1u << 26;             // mbarrier polls before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of FP16 element (row, k) in a 128-byte swizzled K-major operand of `rows` rows.
__host__ __device__ __forceinline__ uint32_t sw128h(int row, int k, int rows) {
    return (uint32_t)((k >> 6) * rows * 128 + (row >> 3) * 1024 + (row & 7) * 128 +
                      ((((k >> 3) & 7) ^ (row & 7)) << 4) + ((k & 7) << 1));
}

// Shared-memory matrix descriptor: 128-byte swizzle, 1024-byte stride between 8-row groups,
// start address in 16-byte units; bits 46-48 hold the descriptor version (1).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1u << 16) | ((uint64_t)(1024u >> 4) << 32) |
           ((uint64_t)1u << 46) | ((uint64_t)2u << 61);
}

// Instruction descriptor of kind::f16: D FP32, A and B FP16, both K-major, M x N shape.
__host__ __device__ constexpr uint32_t idesc_f16(int m, int n) {
    return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes become visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mma_f16(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}
// arrive on the mbarrier once every MMA issued so far by this thread has completed
__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(mbar))
                 : "memory");
}
__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase of the given parity (at most `limit` polls); false if it did not
// complete.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, uint32_t limit = WAIT_LIMIT) {
    for (uint32_t it = 0; it < limit; ++it)
        if (mbar_test(mbar, parity)) return true;
    return false;
}

// 32 consecutive FP32 columns of this thread's TMEM lane (32x32b shape: warp w reads
// lanes 32 (w % 4) .. + 31); the wait is in the same asm so no use precedes it.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// y (already scaled) as two FP16 terms: hi = fp16(y), lo = fp16(y - hi).
__device__ __forceinline__ void split_half(float y, __half& hi, __half& lo) {
    hi = __float2half_rn(y);
    lo = __float2half_rn(y - __half2float(hi));
}

// Issue the 3 x 12 MMAs of one tile (U_hi B_hi, U_hi B_lo, U_lo B_hi per K step) and
// commit to mbar.
__device__ __forceinline__ void issue_tile_mma(uint32_t tmem, uint32_t sUhi, uint32_t sUlo, uint32_t sBhi,
                                               uint32_t sBlo, uint64_t* mbar) {
    constexpr uint32_t idesc = idesc_f16(M, N);
#pragma unroll 1
    for (int ks = 0; ks < K / KSTEP; ++ks) {
        const int k0 = ks * KSTEP;
        const uint32_t offA = (uint32_t)((k0 >> 6) * M * 128 + (k0 & 63) * 2);
        const uint32_t offB = (uint32_t)((k0 >> 6) * N * 128 + (k0 & 63) * 2);
        const uint64_t ahi = sdesc(sUhi + offA), bhi = sdesc(sBhi + offB);
        mma_f16(tmem, ahi, bhi, idesc, ks > 0 ? 1u : 0u);
        mma_f16(tmem, ahi, sdesc(sBlo + offB), idesc, 1u);
        mma_f16(tmem, sdesc(sUlo + offA), bhi, idesc, 1u);
    }
    mma_commit(mbar);
}


}  // namespace tc

// Values of DOF q of element nb as seen at tick `tick` (Alg. 1): its current value if due,
// else the linear time interpolant of its last step.
__device__ __forceinline__ float seen_dof(const DevArrays<float>& d, int tick, int B, int nb, int q) {
    const int lv = d.lvl[nb], sh = B - (lv & 7), par = (lv >> 3) & 1;
    const int j = tick >> sh, rem = tick & ((1 << sh) - 1);
    const int nw = par ^ ((j + (rem ? 1 : 0)) & 1);
    const size_t o = (size_t)nb * tc::NPS + q;
    const float x = (nw ? d.V1 : d.V0)[o];
    if (!rem) return x;
    const float xo = (nw ? d.V0 : d.V1)[o];
    return xo + (float)rem * pow2_neg<float>(sh) * (x - xo);
}

// Row q of a 27 x 28 correction block (16-byte aligned) times the 27 values in s.
__device__ __forceinline__ float block_row_dot(const float* __restrict__ row, const float* s) {
    float acc = 0.0f;
#pragma unroll
    for (int m = 0; m < 6; ++m) {
        const float4 r4 = __ldg(reinterpret_cast<const float4*>(row) + m);
        acc += r4.x * s[4 * m] + r4.y * s[4 * m + 1] + r4.z * s[4 * m + 2] + r4.w * s[4 * m + 3];
    }
    acc += __ldg(row + 24) * s[24] + __ldg(row + 25) * s[25] + __ldg(row + 26) * s[26];
    return acc;
}

// One tick of Alg. 1 for a Q2 3D FP32 context with the element residual on the tensor
// cores.  Persistent, two CTAs per SM (each hides the other's memory latency), each CTA
// walking tiles of 64 due elements (the first tile's records are built before the loop):
//   1  warp w = 8-row group w, lane = 4 ii + kk: row ii, column pairs k = 2 kk + 8 jj +
//      {0, 1}; all loads issued at once, then the row mean c, y = x - c, the row's
//      power-of-two scale and the FP16 hi/lo terms in the swizzled operand layout
//   2  one thread of warp 0 issues the MMAs and commits to an mbarrier; threads 0..63 fetch
//      the next tile's face info, neighbours and level bytes
//   3  while they run: corrections of non-regular faces (warps 1-7, warp per element, lane =
//      row) and the loads of the pointwise step: thread 4 i + p takes DOFs p + 4 m of element i
//   4  warps 0-3: D row -> scaled residual in shared memory
//   5  the pointwise step of the thread's DOFs (element metadata read once per thread):
//      straight-line (dof_update_ap) for a tile without stimulus or padding rows, else
//      dof_update; the element's RV-T sum and max |V_new| over its four threads by shuffles,
//      the accumulation and a due probe check; then threads 0..63 build the next tile's
//      records: per operand slot the row that holds the value the element sees (Alg. 1: a
//      coarser LTS neighbour mid-interval is seen through the linear interpolant of its last
//      step), the interpolation weights, live and interpolated slots
// unscale = 2^-t undoes the scaling of B by 2^t; each row's scale of y is undone by 2^-sc.
template <int DIM, int P>
__global__ void __launch_bounds__(tc::THREADS, 2)
    k_tick_tc(const TickArgs<float> a, const Tables<float> T, const Phys<float> ph,
              const uint16_t* __restrict__ Bg, const float unscale, const float* __restrict__ Cg) {
    static_assert(DIM == 3 && P == 2, "tensor-core sweep: Q2 3D only");
    using namespace tc;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    float* sR = reinterpret_cast<float*>(sm + OFF_R);
    float* sScr = reinterpret_cast<float*>(sm + OFF_SCR);
    const float** sPtr = reinterpret_cast<const float**>(sm + OFF_PTR);
    const float** sPtrO = reinterpret_cast<const float**>(sm + OFF_PTRO);
    int* const bE = reinterpret_cast<int*>(sm + OFF_E);          // [2][M]: this tile's and the next's
    uint32_t* const bInf = reinterpret_cast<uint32_t*>(sm + OFF_INF);
    int* sNb = reinterpret_cast<int*>(sm + OFF_NB);
    float* sTh = reinterpret_cast<float*>(sm + OFF_TH);
    float* sRs = reinterpret_cast<float*>(sm + OFF_RS);
    float* sC = reinterpret_cast<float*>(sm + OFF_C);
    uint8_t* const bLv = sm + OFF_LV;
    uint8_t* sLive = sm + OFF_LIVE;
    uint8_t* sIntp = sm + OFF_INTP;
    uint8_t* const bIrr = sm + OFF_IRR;
    float* sCorr = reinterpret_cast<float*>(sm + OFF_CORR);
    float* sMq = reinterpret_cast<float*>(sm + OFF_MTAB);
    float* sMinv = sMq + 8 * NP;
    float* sDte = sMinv + 8 * NP;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + OFF_MBAR);
    unsigned* sFlag = reinterpret_cast<unsigned*>(sm + OFF_FLAG);
    uint32_t* sTmem = reinterpret_cast<uint32_t*>(sm + OFF_TMEM);

    const DevArrays<float>& d = a.d;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tick = a.tick, B = a.B;
    // due count and element order are fixed during the sweep; a block without a tile of this
    // tick skips the set-up and leaves its SM to other work (a small instance's fine ticks)
    const int n_act = d.meta->nact[tick];
    const int ntiles = (n_act + M - 1) / M;
    if ((int)blockIdx.x >= ntiles) return;

    // --- set-up that reads nothing the previous tick writes (before the dependent wait)
    // the operator's FP16 terms, stored in global memory as the image of their swizzled shared-
    // memory layout (B_hi then B_lo): a straight 16-byte copy
    for (int i = tid; i < 2 * B_BYTES / 16; i += THREADS)
        reinterpret_cast<uint4*>(sm + OFF_BHI)[i] = __ldg(reinterpret_cast<const uint4*>(Bg) + i);
    // per (level, node) GL mass and its inverse: lanes read different nodes, which kernel-
    // parameter arrays would serve one address at a time
    for (int i = tid; i < 8 * NP; i += THREADS) {
        const int l = i / NP, q = i - l * NP;
        sMq[i] = ph.Wvol[l] * T.w[q % 3] * T.w[(q / 3) % 3] * T.w[q / 9];
        sMinv[i] = ph.Minv[l][q];
    }
    if (tid < 8) sDte[tid] = a.dteR[tid];
    if (warp == 0) tmem_alloc(sTmem, TMEM_COLS);
    if (tid == 0) {
        mbar_init(mbar, 1);
        *sFlag = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *sTmem;
    const int G = (int)gridDim.x;
    int e_cur = -1, e_next = -1;   // threads 0..63: element of this CTA's first tile, of the next one
    if (tid < M && (int)blockIdx.x * M + tid < n_act) e_cur = d.order[blockIdx.x * M + tid];
    if (tid < M && ((int)blockIdx.x + G) * M + tid < n_act) e_next = d.order[(blockIdx.x + G) * M + tid];
    // Metadata of a tile's element (threads 0..63) is fetched one tile ahead: its face info,
    // neighbours and level byte while the previous tile's gather and MMAs run, the neighbours'
    // level bytes while its pointwise step runs, and the tile's records are built at the end of
    // that step (the records read by phases 2 and 5 are double-buffered).
    auto fetch_raw = [&](int e, int* nx) {
        const int es = e >= 0 ? e : 0;
        nx[0] = e >= 0 ? (int)d.info[es] : 0;
#pragma unroll
        for (int f = 0; f < 6; f += 2) {
            const int2 n2 = *reinterpret_cast<const int2*>(d.nbr + (size_t)es * 6 + f);
            nx[1 + f] = n2.x;
            nx[2 + f] = n2.y;
        }
        nx[7] = e >= 0 ? (int)d.lvl[es] : 0;
    };
    auto fetch_lvn = [&](int e, const int* nx, uint32_t& lo, uint32_t& hi) {
        const int es = e >= 0 ? e : 0;
        lo = 0u;
        hi = 0u;
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            const uint32_t v = d.lvl[(((nx[0] >> (4 * f)) & 3) == 1) ? nx[1 + f] : es];
            if (f < 3) lo |= v << (8 * f);
            else hi |= v << (8 * (f - 3));
        }
    };
    // The records of element e (row tid of a tile) from its raw metadata: per operand slot the row
    // holding the value the element sees (Alg. 1: a coarser LTS neighbour mid-interval is seen
    // through the linear interpolant of its last step), the interpolation weights, live and
    // interpolated slots; into buffer nb of the double-buffered records.  Returns whether the
    // element needs the general pointwise step (padding row or stimulus).
    auto build_meta = [&](int e, const int* nx, uint32_t lo, uint32_t hi, int nb) -> bool {
        const int es = e >= 0 ? e : 0;                    // any valid row for padding slots
        uint8_t live = 0, intp = 0;
        const uint32_t inf = (uint32_t)nx[0];
        const uint8_t lv = (uint8_t)(nx[7] & 255);
        const int b = lv & 7, par = (lv >> 3) & 1;
        const int cur = par ^ ((tick >> (B - b)) & 1);
        sPtr[tid] = (cur ? d.V1 : d.V0) + (size_t)es * NPS;
        if (e >= 0) live = 1;
        bool irr = false;
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            const uint32_t lvn = (f < 3 ? (lo >> (8 * f)) : (hi >> (8 * (f - 3)))) & 255u;
            const bool same = e >= 0 && ((inf >> (4 * f)) & 3) == 1;
            const int sh = B - (int)(lvn & 7), pn = (lvn >> 3) & 1;
            const int j = tick >> sh, rem = same ? (tick & ((1 << sh) - 1)) : 0;
            const int nw = pn ^ ((j + (rem ? 1 : 0)) & 1);
            const size_t o = (size_t)(same ? nx[1 + f] : es) * NPS;
            sPtr[(1 + f) * M + tid] = (nw ? d.V1 : d.V0) + o;
            if (rem) {
                sPtrO[(1 + f) * M + tid] = (nw ? d.V0 : d.V1) + o;
                sTh[(1 + f) * M + tid] = (float)rem * pow2_neg<float>(sh);
            }
            if (same) live |= (uint8_t)(2u << f);
            if (rem) intp |= (uint8_t)(2u << f);
            irr = irr || (((inf >> (4 * f)) & 3) != 1);
            sNb[f * M + tid] = nx[1 + f];
        }
        bE[nb * M + tid] = e;
        bInf[nb * M + tid] = inf;
        bLv[nb * M + tid] = lv;
        bIrr[nb * M + tid] = (e >= 0 && irr) ? 1 : 0;
        sLive[tid] = live;
        sIntp[tid] = intp;
        return e < 0 || (inf & INFO_STIM);
    };
    bool slow0 = false;
    if (tid < M && (int)blockIdx.x < ntiles) {
        int nx[8];
        uint32_t lo, hi;
        fetch_raw(e_cur, nx);
        fetch_lvn(e_cur, nx, lo, hi);
        slow0 = build_meta(e_cur, nx, lo, hi, 0);
    }
    // a tile without padding rows or stimulus, under the Aliev-Panfilov model with the
    // exponential state step, takes the straight-line pointwise step (phase 5)
    const bool ap_exp = ph.ionic == 0 && ph.integrator == 1;
    bool fast = !__syncthreads_or(slow0) && ap_exp;
    // everything above reads only what is fixed during the sweep (order, due counts, face info,
    // neighbours, level bytes): it overlaps the previous tick's tail; the values from here on
    pdl_enter();
    uint32_t parity = 0;
    bool ok = d.meta->err == 0;
    const double t_tick = tick_time(a, tick);
    int nxr[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // threads 0..63: next tile's raw metadata in flight
    uint32_t nlo = 0u, nhi = 0u;
    int buf = 0;                             // buffer of this tile's records

    for (int t = blockIdx.x; ok && t < ntiles; t += gridDim.x) {
        int* const sE = bE + buf * M;
        uint32_t* const sInf = bInf + buf * M;
        uint8_t* const sLv = bLv + buf * M;
        uint8_t* const sIrr = bIrr + buf * M;

        // ---- 1: gather, mean shift, FP16 split (warp w: rows 8 w .. 8 w + 7; lane = 4 ii + kk:
        //      row ii, column pairs k = 2 kk + 8 jj + {0, 1})
        {
            const int ii = lane >> 2, kk = lane & 3, i = warp * 8 + ii;
            const float* pr[SLOTS];
#pragma unroll
            for (int s = 0; s < SLOTS; ++s) pr[s] = sPtr[s * M + i];
            const unsigned live = sLive[i], intp = sIntp[i];
            float x[48];
            // column k lies in slot s0 = floor(8 jj / 27) or the next one
#pragma unroll
            for (int jj = 0; jj < 24; ++jj) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int s0 = (8 * jj) / NP, s1 = s0 + 1 < SLOTS ? s0 + 1 : s0;
                    const int k = 2 * kk + 8 * jj + h;
                    const bool nxt = k >= NP * (s0 + 1) && s1 != s0;
                    const int q = (k < KU ? k : KU - 1) - NP * (nxt ? s1 : s0);
                    x[2 * jj + h] = __ldg((nxt ? pr[s1] : pr[s0]) + q);
                }
            }
            if (intp) {
                // coarser LTS neighbours mid-interval: linear interpolant in time (Alg. 1)
#pragma unroll
                for (int m = 0; m < 48; ++m) {
                    const int k = 2 * kk + 8 * (m >> 1) + (m & 1);
                    const int s = (k < KU ? k : KU - 1) / NP;
                    if (k < KU && ((intp >> s) & 1u)) {
                        const float xo = __ldg(sPtrO[s * M + i] + (k - NP * s));
                        x[m] = xo + sTh[s * M + i] * (x[m] - xo);
                    }
                }
            }
            float cs = 0.0f;
#pragma unroll
            for (int m = 0; m < 8; ++m)
                if (2 * kk + 8 * (m >> 1) + (m & 1) < NP) cs += x[m];
            cs += __shfl_xor_sync(0xffffffffu, cs, 1);
            cs += __shfl_xor_sync(0xffffffffu, cs, 2);
            const float c = cs * (1.0f / NP);
            float mx = 0.0f;
#pragma unroll
            for (int m = 0; m < 48; ++m) {
                const int k = 2 * kk + 8 * (m >> 1) + (m & 1);
                const int s = (k < KU ? k : KU - 1) / NP;
                x[m] = (k < KU && ((live >> s) & 1u)) ? x[m] - c : 0.0f;
                mx = fmaxf(mx, fabsf(x[m]));
            }
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
            // row scale 2^sc with max |y| 2^sc in [2^13, 2^14): the FP16 terms keep 22 bits
            // relative to the row's own variation (exact power of two, undone after the MMA)
            const int ex = (mx > 0.0f) ? (int)((__float_as_uint(mx) >> 23) & 255u) - 126 : 14;
            const int sc = min(max(14 - ex, -100), 100);
            const float up = __int_as_float((127 + sc) << 23);
            if (kk == 0) {
                sRs[i] = __int_as_float((127 - sc) << 23);
                sC[i] = c;
            }
#pragma unroll
            for (int jj = 0; jj < 24; ++jj) {
                const int k = 2 * kk + 8 * jj;
                const float a0 = x[2 * jj] * up, a1 = x[2 * jj + 1] * up;
                const __half2 hi = __floats2half2_rn(a0, a1);
                const __half2 lo = __floats2half2_rn(a0 - __low2float(hi), a1 - __high2float(hi));
                *reinterpret_cast<__half2*>(sm + OFF_UHI + sw128h(i, k, M)) = hi;
                *reinterpret_cast<__half2*>(sm + OFF_ULO + sw128h(i, k, M)) = lo;
            }
        }
        fence_async_smem();
        __syncthreads();

        // ---- 2: MMAs (the tensor cores run while the corrections and the item loads below run)
        if (tid == 0) {
            fence_after();
            issue_tile_mma(tmem, smem_u32(sm + OFF_UHI), smem_u32(sm + OFF_ULO), smem_u32(sm + OFF_BHI),
                           smem_u32(sm + OFF_BLO), mbar);
        }

        if (tid < M) fetch_raw(e_next, nxr);

        // ---- 3: non-regular faces (boundary, coarser, finer neighbours): exact face terms minus
        //      the same-level own blocks the tensor product assumed, from level-0 correction
        //      blocks; warp w >= 1 takes elements w - 1, w + 6, ... (warp 0 issues the MMAs),
        //      lane q = row q, on the operand's mean-shifted values (the same c as the MMA)
        {
            const int q = lane < NP ? lane : NP - 1;
            float* su = sScr + warp * 64;
            float* sn = su + 32;
#pragma unroll 1
            for (int i = warp - 1; warp > 0 && i < M; i += 7) {
                if (!sIrr[i]) continue;
                const uint32_t inf = sInf[i];
                const float c = sC[i];
                su[lane] = __ldg(sPtr[i] + q) - c;
                __syncwarp();
                float corr = 0.0f;
                for (int f = 0; f < 6; ++f) {
                    const int kind = (inf >> (4 * f)) & 3;
                    if (kind == 1) continue;
                    const float* Bf = Cg + (size_t)f * 14 * NP * 28 + (size_t)q * 28;
                    if (kind == 0) {
                        corr += block_row_dot(Bf, su);
                    } else if (kind == 2) {
                        const int pos = (inf >> (4 * f + 2)) & 3;
                        corr += block_row_dot(Bf + (1 + pos) * NP * 28, su);
                        sn[lane] = seen_dof(d, tick, B, sNb[f * M + i], q) - c;
                        __syncwarp();
                        corr += block_row_dot(Bf + (5 + pos) * NP * 28, sn);
                        __syncwarp();
                    } else {
                        corr += block_row_dot(Bf + 9 * NP * 28, su);
                        for (int sb = 0; sb < 4; ++sb) {
                            sn[lane] = seen_dof(d, tick, B, d.hang[sNb[f * M + i] + sb], q) - c;
                            __syncwarp();
                            corr += block_row_dot(Bf + (10 + sb) * NP * 28, sn);
                            __syncwarp();
                        }
                    }
                }
                if (lane < NP) sCorr[i * RST + q] = corr * pow2_neg<float>((DIM - 2) * ((inf >> 24) & 15));
                __syncwarp();
            }
        }

        // element i = tid / 4, DOFs q = p + 4 m (p = tid % 4): the loads of the thread's DOFs
        constexpr int NIT = (NP + 3) / 4;
        float u[NIT], w[NIT], Ia[NIT], ga[NIT];
        {
            const int i = tid >> 2, p = tid & 3;
            const int e = sE[i], es = e >= 0 ? e : 0;
            const int ke = tick >> (B - (sLv[i] & 7));
            const bool need = e >= 0 && ke != 0;
            const float* up = sPtr[i];
#pragma unroll
            for (int m = 0; m < NIT; ++m) {
                const int q = min(p + 4 * m, NP - 1);
                u[m] = __ldg(up + q);
                w[m] = d.v[(size_t)es * NPS + q];
                Ia[m] = need ? d.Ia[(size_t)es * NPS + q] : 0.0f;
                ga[m] = need ? d.ga[(size_t)es * NPS + q] : 0.0f;
            }
        }
        // thread 4 i: the RV-T accumulator of element i, needed at the end of the tile (ke != 0)
        double acc0 = 0.0;
        if ((tid & 3) == 0) {
            const int e = sE[tid >> 2];
            if (e >= 0 && (tick >> (B - (sLv[tid >> 2] & 7))) != 0) acc0 = d.acc[e];
        }

        // ---- 4: residual rows (warps 0-3; thread t < 16 of warp w holds row 16 w + t)
        if (warp < 4) {
            const bool done = mbar_wait(mbar, parity);
            fence_after();
            float acc[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16), acc);
            if (!done) {
                atomicOr(sFlag, 1u);
            } else if (lane < 16) {
                const int i = warp * 16 + lane;
                const float scale = unscale * sRs[i] * pow2_neg<float>((DIM - 2) * ((sInf[i] >> 24) & 15));
#pragma unroll
                for (int q = 0; q < NP; ++q) sR[i * RST + q] = acc[q] * scale;
            }
        }
        parity ^= 1u;
        fence_before();
        __syncthreads();
        if (*sFlag) {
            ok = false;
            if (tid == 0) atomicOr(&d.meta->err, ERR_TIMEOUT);
            break;
        }

        if (tid < M) fetch_lvn(e_next, nxr, nlo, nhi);

        // ---- 5: the pointwise step of element i = tid / 4, DOFs q = p + 4 m; the RV-T sum and
        //      max |V_new| of its four threads by shuffles, the accumulation and the record of a
        //      due probe check (the values before and after the step of elements with a pending
        //      probe go to shared memory for it)
        {
            const int i = tid >> 2, p = tid & 3;
            const int e = sE[i];
            const uint32_t inf = sInf[i];
            const int b = sLv[i] & 7, lev = (inf >> 24) & 15, ke = tick >> (B - b);
            const bool irr = sIrr[i] != 0, pend = (inf & INFO_PENDING) != 0;
            const int par = (sLv[i] >> 3) & 1, cur = par ^ (ke & 1);
            float* vrow = (cur ? d.V0 : d.V1) + (size_t)(e >= 0 ? e : 0) * NPS;   // the row the step writes
            float* sUo = reinterpret_cast<float*>(sm + OFF_UHI) + M * NP;
            float* sUn = sUo + M * NP;
            float term = 0.0f, vmax = 0.0f;
            auto fast_dofs = [&](auto first) {
                constexpr bool FIRST = decltype(first)::value;
                const float dte = sDte[b];
#pragma unroll
                for (int m = 0; m < NIT; ++m) {
                    const int q = p + 4 * m;
                    if (q < NP) {
                        const float r = sR[i * RST + q] + (irr ? sCorr[i * RST + q] : 0.0f);
                        float un, wn;
                        term += dof_update_ap<FIRST>(ph, sMq[lev * NP + q], sMinv[lev * NP + q], dte, u[m], w[m], r,
                                                     Ia[m], ga[m], un, wn);
                        vmax = fmaxf(vmax, fabsf(un));
                        vrow[q] = un;
                        d.v[(size_t)e * NPS + q] = wn;
                        if (FIRST && b > 0) {
                            d.Ia[(size_t)e * NPS + q] = Ia[m];
                            d.ga[(size_t)e * NPS + q] = ga[m];
                        }
                        if (pend) {
                            sUo[i * NP + q] = u[m];
                            sUn[i * NP + q] = un;
                        }
                    }
                }
            };
            if (fast) {
                if (tick == 0) fast_dofs(std::true_type{});
                else fast_dofs(std::false_type{});
            } else if (e >= 0) {
#pragma unroll
                for (int m = 0; m < NIT; ++m) {
                    const int q = p + 4 * m;
                    if (q < NP) {
                        float so = 0.0f, smd = 0.0f;
                        if (inf & INFO_STIM) dof_stim<float>(a, e, tick, a.dte[b], q, so, smd);
                        const float r = sR[i * RST + q] + (irr ? sCorr[i * RST + q] : 0.0f);
                        float un, wn;
                        term += dof_update<float>(ph, sMq[lev * NP + q], sMinv[lev * NP + q], ke, a.dteR[b], so, smd,
                                                  u[m], w[m], r, Ia[m], ga[m], un, wn);
                        vmax = fmaxf(vmax, fabsf(un));
                        const size_t o = (size_t)e * NPS + q;
                        vrow[q] = un;
                        d.v[o] = wn;
                        if (ke == 0 && b > 0) {
                            d.Ia[o] = Ia[m];
                            d.ga[o] = ga[m];
                        }
                        if (pend) {
                            sUo[i * NP + q] = u[m];
                            sUn[i * NP + q] = un;
                        }
                    }
                }
            }
            term += __shfl_xor_sync(0xffffffffu, term, 1);
            vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, 1));
            term += __shfl_xor_sync(0xffffffffu, term, 2);
            vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, 2));
            __syncwarp();   // the element's values before and after the step, for its probe check
            if (p == 0) {
                if (e >= 0) d.acc[e] = acc0 + a.dte[b] * (double)term;
                if (e >= 0 && pend && vmax >= ph.lat_gate)
                    lat_check<float, DIM, P>(d, T, ph, e, inf, lev, sUo + i * NP, sUn + i * NP, t_tick, a.dte[b]);
            }
        }
        // the next tile's records (threads 0..63), then the next tile's element ids
        bool slow = false;
        if (tid < M) {
            slow = build_meta(e_next, nxr, nlo, nhi, buf ^ 1);
            const int idx_n = (t + 2 * G) * M + tid;
            e_next = idx_n < n_act ? d.order[idx_n] : -1;
        }
        fast = !__syncthreads_or(slow) && ap_exp;
        buf ^= 1;
    }
    if (*sFlag) {
        // a wait gave up: give the MMAs in flight one more bounded wait before freeing TMEM
        if (tid == 0) mbar_wait(mbar, parity ^ 1u);
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}

}  // namespace mdl
