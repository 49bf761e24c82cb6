// selftest.cu -- diagnostics with no counterpart in the paper: the bounded-wait path that every
// pipelined kernel of the library relies on, exercised on purpose, and the f_k path query.
//
// The statistics and GEMM kernels wait on mbarriers (copies landing, MMAs committing, stages being
// released) with a bound: a wait that runs past kTimeoutNs gives up, raises the CTA's abort flag
// (so the CTA's other roles stop waiting too), records BMM_ERR_TIMEOUT in the caller's status word
// and returns, instead of hanging the GPU.  That path cannot be reached by a correct problem, so
// bmm_wait_selftest reaches it directly: one CTA waits, with the library's own wait routine, on an
// mbarrier that nothing will ever complete, and a second warp waits on another such barrier and
// must give up through the abort flag.  Nothing is in flight (no copy, no MMA, no TMEM), so giving
// up is safe by construction.
#include "internal.h"
#include "tc_ptx.cuh"

#define BMM_API extern "C" __attribute__((visibility("default")))

namespace bmm {
namespace {

using namespace ptx;

__global__ void __launch_bounds__(64) wait_selftest_kernel(DevStatus* st) {
    __shared__ __align__(8) uint64_t bar_never[2];
    __shared__ volatile int s_abort;
    __shared__ int s_gave_up;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar_never[0]), 1);  // one arrival expected, none will come
        mbar_init(smem_u32(&bar_never[1]), 1);
        s_abort = 0;
        s_gave_up = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        // warp 0 gives up on the time bound and raises the flag; warp 1 gives up on the flag
        if (!mbar_wait<true>(smem_u32(&bar_never[warp]), 0u, &s_abort)) atomicAdd(&s_gave_up, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_abort) set_status(st, BMM_ERR_TIMEOUT, s_gave_up);
}

}  // namespace
}  // namespace bmm

using namespace bmm;

BMM_API bmm_status bmm_wait_selftest(void* ws, size_t ws_bytes, bmm_stream_t stream) {
    if (ws == nullptr || (reinterpret_cast<uintptr_t>(ws) & 255) || ws_bytes < 256) return BMM_ERR_WORKSPACE;
    if (!tc_gemm_supported()) return BMM_ERR_UNSUPPORTED;
    (count_launch(), wait_selftest_kernel<<<1, 64, 0, reinterpret_cast<cudaStream_t>(stream)>>>(static_cast<DevStatus*>(ws)));
    return cudaGetLastError() == cudaSuccess ? BMM_OK : BMM_ERR_CUDA;
}

BMM_API bmm_status bmm_f_tc_supported(const bmm_mat* M, const bmm_mat* N, const bmm_blocks* B, int32_t* uses_tc) {
    bmm_status s = check_problem(M, N, B);
    if (s != BMM_OK) return s;
    if (uses_tc == nullptr) return BMM_ERR_ARG;
    *uses_tc = blockstats_tc_supported(vecset_of_M(M), vecset_of_N(N), B->max_nk) ? 1 : 0;
    return BMM_OK;
}
