// mdl_fused.cu -- the fused multi-simulation sweep (see mdl_fused.h).
#include "mdl_fused.h"

namespace mdl {

namespace {

// Elements [lo, hi) of the slot's due order at its tick `tick`, one thread per element
// (the element step of the thread-per-element sweep, Alg. 1).
template <typename R, int DIM, int P>
__device__ __forceinline__ void fused_range(const FusedSlot<R>& fs, int tick, int lo, int hi) {
    for (int idx = lo + (int)threadIdx.x; idx < hi; idx += (int)blockDim.x) {
        TickMetaT<DIM, P> m;
        tick_fetch<R, DIM, P>(fs.ta.d, idx, m);
        tick_elem<R, DIM, P>(fs.ta, *fs.T, *fs.ph, tick, m, -1.0);
    }
}

// One global tick g of a fused round.  Every block first finds, per slot, whether g is one
// of the slot's ticks, its tick there and its due count (fixed during the sweep: written by
// the slot's ordering phase before the round's first tick), and the prefix sums of the work
// items; then walks work items t = block, block + grid, ...
template <typename R, int CLS>
__global__ void __launch_bounds__(256) k_tick_fused(const FusedSlot<R>* __restrict__ slots, int nslot, int g,
                                                   int tile) {
    __shared__ int sOff[FUSED_MAX_SLOTS + 1];
    __shared__ int sTick[FUSED_MAX_SLOTS];
    __shared__ int sCnt[FUSED_MAX_SLOTS];
    for (int s = threadIdx.x; s < nslot; s += blockDim.x) {
        const FusedSlot<R>& fs = slots[s];
        int n = 0, tk = 0;
        if ((g & ((1 << fs.shift) - 1)) == 0) {
            tk = g >> fs.shift;
            const DevMeta* m = fs.ta.d.meta;
            n = m->err ? 0 : m->nact[tk];
        }
        sTick[s] = tk;
        sCnt[s] = n;
        sOff[s + 1] = (n + tile - 1) / tile;
    }
    __syncthreads();
    // prefix sums of the work items by warp 0, 32 slots at a time
    if (threadIdx.x < 32) {
        const int lane = (int)threadIdx.x;
        int carry = 0;
        for (int base = 0; base < nslot; base += 32) {
            const int s = base + lane;
            int v = s < nslot ? sOff[s + 1] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += y;
            }
            if (s < nslot) sOff[s + 1] = carry + v;
            carry += __shfl_sync(0xffffffffu, v, 31);
        }
        if (lane == 0) sOff[0] = 0;
    }
    __syncthreads();
    // the values of the previous global tick are needed from here on
    pdl_enter();
    const int total = sOff[nslot];
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        int lo = 0, hi = nslot;   // slot s with sOff[s] <= t < sOff[s + 1]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (sOff[mid] <= t) lo = mid;
            else hi = mid;
        }
        const int s = lo;
        const int e0 = (t - sOff[s]) * tile;
        const int e1 = min(e0 + tile, sCnt[s]);
        constexpr int DIM = (CLS == FC_3_1 || CLS == FC_3_2) ? 3 : 2;
        constexpr int P = (CLS == FC_2_2 || CLS == FC_3_2) ? 2 : 1;
        fused_range<R, DIM, P>(slots[s], sTick[s], e0, e1);
    }
}

template <typename R, int CLS>
cudaError_t launch_round(const void* d_slots, int nslot, int Bmax, FusedShape sh, cudaStream_t st) {
    const FusedSlot<R>* p = static_cast<const FusedSlot<R>*>(d_slots);
    for (int g = 0; g < (1 << Bmax); ++g) {
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3((unsigned)sh.blocks);
        cfg.blockDim = dim3((unsigned)sh.threads);
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = g > 0 ? 1 : 0;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        cudaError_t e = cudaLaunchKernelEx(&cfg, k_tick_fused<R, CLS>, p, nslot, g, sh.tile);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

size_t fused_slot_bytes(int precision) {
    return precision == 64 ? sizeof(FusedSlot<double>) : sizeof(FusedSlot<float>);
}

void fused_set_shift(void* record, int precision, int shift) {
    if (precision == 64) static_cast<FusedSlot<double>*>(record)->shift = shift;
    else static_cast<FusedSlot<float>*>(record)->shift = shift;
}

int fused_class(int dim, int order) {
    return dim == 2 ? (order == 1 ? FC_2_1 : FC_2_2) : (order == 1 ? FC_3_1 : FC_3_2);
}

namespace {

template <typename R>
int blocks_per_sm(int cls, int threads) {
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (cls) {
        case FC_2_1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_tick_fused<R, FC_2_1>, threads, 0); break;
        case FC_2_2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_tick_fused<R, FC_2_2>, threads, 0); break;
        case FC_3_1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_tick_fused<R, FC_3_1>, threads, 0); break;
        case FC_3_2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_tick_fused<R, FC_3_2>, threads, 0); break;
        default: break;
    }
    return e == cudaSuccess && n > 0 ? n : 1;
}

template <typename R>
cudaError_t sweep(int cls, const void* d_slots, int nslot, int Bmax, FusedShape sh, cudaStream_t st) {
    switch (cls) {
        case FC_2_1: return launch_round<R, FC_2_1>(d_slots, nslot, Bmax, sh, st);
        case FC_2_2: return launch_round<R, FC_2_2>(d_slots, nslot, Bmax, sh, st);
        case FC_3_1: return launch_round<R, FC_3_1>(d_slots, nslot, Bmax, sh, st);
        case FC_3_2: return launch_round<R, FC_3_2>(d_slots, nslot, Bmax, sh, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

int fused_blocks_per_sm(int precision, int cls, int threads) {
    return precision == 64 ? blocks_per_sm<double>(cls, threads) : blocks_per_sm<float>(cls, threads);
}

cudaError_t fused_sweep(int precision, int cls, const void* d_slots, int nslot, int Bmax, FusedShape shape,
                        cudaStream_t st) {
    if (nslot <= 0 || nslot > FUSED_MAX_SLOTS || Bmax < 0 || Bmax > 7 || shape.threads <= 0 ||
        shape.threads > 256 || shape.tile <= 0 || shape.blocks <= 0 || cls < FC_2_1 || cls > FC_3_2)
        return cudaErrorInvalidValue;
    return precision == 64 ? sweep<double>(cls, d_slots, nslot, Bmax, shape, st)
                           : sweep<float>(cls, d_slots, nslot, Bmax, shape, st);
}

}  // namespace mdl
