// mdl_selftest.cu -- the bounded device waits of the sweeps, made to run out on purpose.
//
// The tensor-core sweep waits on an mbarrier for its MMAs and the cooperative sweep on a grid
// barrier between ticks; each wait has a poll limit after which the kernel records ERR_WAIT and
// returns instead of hanging, and the stepping call reports MDL_E_TIMEOUT.  Here a one-block
// kernel runs the same wait helpers on a phase or a count that nothing completes (a flag that
// nothing sets), so that the give-up path is exercised on the device without any fault.
#include <cuda_runtime.h>

#include <chrono>

#include "../../include/mdl.h"
#include "mdl_tc.cuh"

namespace mdl {
namespace {

// which 0: the grid barrier, whose count can never reach two rounds of a one-block grid;
// which 1: the mbarrier wait on a phase with no arrival, `limit` polls.
__global__ void k_selftest_wait(int which, uint32_t limit, DevMeta* m) {
    __shared__ __align__(8) uint64_t mbar;
    if (which == 0) {
        grid_barrier(m, 2u, limit);
        return;
    }
    if (threadIdx.x == 0) {
        tc::mbar_init(&mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0 && !tc::mbar_wait(&mbar, 0u, limit)) atomicOr(&m->err, ERR_WAIT);
}

}  // namespace
}  // namespace mdl

extern "C" int mdl_selftest_wait(int32_t which, int32_t* status, double* elapsed_ms) {
    if (!status || (which != 0 && which != 1)) return MDL_E_ARG;
    mdl::DevMeta* m = nullptr;
    if (cudaMalloc(&m, sizeof(mdl::DevMeta)) != cudaSuccess) return MDL_E_CUDA;
    int rc = MDL_OK;
    const auto t0 = std::chrono::steady_clock::now();
    if (cudaMemset(m, 0, sizeof(mdl::DevMeta)) != cudaSuccess) rc = MDL_E_CUDA;
    if (rc == MDL_OK) {
        // the grid barrier at its production limit; the mbarrier wait at 2^16 polls (its
        // production limit of 2^26 polls would take far longer than a test should)
        const uint32_t limit = which == 0 ? mdl::GRID_WAIT_LIMIT : (1u << 16);
        mdl::k_selftest_wait<<<1, 32>>>(which, limit, m);
        if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) rc = MDL_E_CUDA;
    }
    unsigned err = 0;
    if (rc == MDL_OK &&
        cudaMemcpy(&err, (char*)m + offsetof(mdl::DevMeta, err), sizeof(err), cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = MDL_E_CUDA;
    const auto t1 = std::chrono::steady_clock::now();
    cudaFree(m);
    if (rc != MDL_OK) return rc;
    *status = (err & mdl::ERR_WAIT) ? MDL_E_TIMEOUT : MDL_OK;
    if (elapsed_ms) *elapsed_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    return MDL_OK;
}
