// mdl_noalloc.cu -- FP64 integral of a DOF field without any device allocation.
//
// The same reduction as the barrier diagnostic (int V = sum_e sum_q w_q det J_e V_eq in
// FP64, block partials then a fixed-order final sum), for callers that must not
// allocate device memory: code that runs inside a stream capture or a real-time loop,
// or a host application whose device memory is fully pre-partitioned by another
// allocator.  The block partials live in a file-scope static device array of
// MDL_NOALLOC_MAX_PARTIALS doubles, which every GPU that loads the library holds until
// the process exits.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>

#include <mutex>

#include "../../include/mdl.h"

namespace {

static __device__ __align__(256) double g_partials[MDL_NOALLOC_MAX_PARTIALS];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
double* g_addr[MAX_DEVICES] = {nullptr};

struct MassTable {
    double m[8][27];   // w_q prod_k h_k(level)/2
};

template <typename R>
__global__ void k_integral_partials(const R* __restrict__ V, const int8_t* __restrict__ level, int64_t n_e,
                                    int n_p, MassTable mt, double* partials) {
    __shared__ double red[256];
    double s = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_e;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int l = level[e];
        if (l < 0 || l > 7) {
            s += __longlong_as_double(0x7ff8000000000000ll);   // a level outside 0..7: NaN result
            continue;
        }
        for (int q = 0; q < n_p; ++q) s += mt.m[l][q] * (double)V[e * n_p + q];
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

__global__ void k_integral_final(const double* partials, int n, double* out) {
    __shared__ double red[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += partials[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

thread_local char g_err[256];

int fail(int code, const char* msg) {
    snprintf(g_err, sizeof(g_err), "%s", msg);
    return code;
}

// Device address of the scratch array on the current device (looked up once per device).
int scratch_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(MDL_E_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= MAX_DEVICES) return fail(MDL_E_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_partials);
        if (e != cudaSuccess) return fail(MDL_E_CUDA, cudaGetErrorString(e));
        g_addr[dev] = (double*)p;
    }
    *out = g_addr[dev];
    return MDL_OK;
}

}  // namespace

extern "C" const char* mdl_noalloc_last_error(void) { return g_err; }

extern "C" int mdl_integral_noalloc(int32_t dim, int32_t order, const double* extent, const int32_t* base,
                                    int32_t precision, const void* V_dev, const int8_t* level_dev, int64_t n_e,
                                    double* out_dev, void* stream) {
    g_err[0] = 0;
    if (dim != 2 && dim != 3) return fail(MDL_E_ARG, "dim must be 2 or 3");
    if (order != 1 && order != 2) return fail(MDL_E_ARG, "order must be 1 or 2");
    if (precision != 32 && precision != 64) return fail(MDL_E_ARG, "precision must be 32 or 64");
    if (!extent || !base || !out_dev) return fail(MDL_E_ARG, "extent, base and out_dev are required");
    if (n_e < 0) return fail(MDL_E_ARG, "n_e must be >= 0");
    if (n_e > 0 && (!V_dev || !level_dev)) return fail(MDL_E_ARG, "V_dev and level_dev are required");
    const int n1 = order + 1;
    const int n_p = dim == 2 ? n1 * n1 : n1 * n1 * n1;
    if (n_e > MDL_NOALLOC_MAX_ELEMENTS)
        return fail(MDL_E_ARG, "n_e exceeds MDL_NOALLOC_MAX_ELEMENTS");
    for (int k = 0; k < dim; ++k)
        if (!(extent[k] > 0) || base[k] < 1) return fail(MDL_E_ARG, "extent must be > 0 and base >= 1");
    cudaStream_t st = (cudaStream_t)stream;
    if (n_e == 0) {
        cudaError_t e = cudaMemsetAsync(out_dev, 0, sizeof(double), st);
        return e == cudaSuccess ? MDL_OK : fail(MDL_E_CUDA, cudaGetErrorString(e));
    }
    // an error left pending by the caller's own CUDA work is reported as such (and left in
    // place) instead of being taken for a failure of this call's launches
    const cudaError_t pending = cudaPeekAtLastError();
    if (pending != cudaSuccess)
        return fail(MDL_E_CUDA, "a CUDA error from earlier work was pending before this call");
    double* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    // FP64 GL mass per (level, node): closed-form nodes/weights of the (p+1)-point rule
    double w[3];
    if (order == 1) {
        w[0] = w[1] = 1.0;
    } else {
        w[0] = w[2] = 5.0 / 9.0;
        w[1] = 8.0 / 9.0;
    }
    MassTable mt{};
    for (int l = 0; l < 8; ++l)
        for (int q = 0; q < n_p; ++q) {
            double m = 1.0;
            int r = q;
            for (int k = 0; k < dim; ++k) {
                m *= w[r % n1] * extent[k] / ((double)base[k] * (double)(1 << l)) * 0.5;
                r /= n1;
            }
            mt.m[l][q] = m;
        }
    int64_t nb = (n_e + 255) / 256;
    if (nb > MDL_NOALLOC_MAX_PARTIALS) nb = MDL_NOALLOC_MAX_PARTIALS;
    if (precision == 32)
        k_integral_partials<float><<<(int)nb, 256, 0, st>>>((const float*)V_dev, level_dev, n_e, n_p, mt, scratch);
    else
        k_integral_partials<double><<<(int)nb, 256, 0, st>>>((const double*)V_dev, level_dev, n_e, n_p, mt, scratch);
    k_integral_final<<<1, 256, 0, st>>>(scratch, (int)nb, out_dev);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MDL_OK : fail(MDL_E_CUDA, cudaGetErrorString(e));
}
