// static_scratch.cu -- bmm_probs_static: the statistics pass and probabilities without a workspace.
//
// Some callers cannot allocate device memory when they call us: a plugin inside a host program
// that hands out all GPU memory from its own fixed pool and forbids any other allocation, or a
// latency-critical loop that must not pay for cudaMalloc's implicit device synchronisation.
// For them this entry point keeps the only scratch the statistics pass needs -- the per-slice
// partial column sums of a row-major M (or column-major N) -- in a fixed array compiled into
// the library.  The array is kStaticScratchBytes (16 MiB) on every GPU that loads the library
// and stays allocated until the process exits.
//
// Notes for callers
//  - The first call on each device looks up the array's device address (cudaGetSymbolAddress)
//    with that device current; make that first call before any stream capture begins.
//  - All calls share the one array and it keeps the last call's contents.  Every element the
//    pass reads is written earlier in the same call, so nothing has to start at zero; but two
//    calls whose work overlaps on the GPU (different streams, no ordering) race on the array.
//  - Problems whose partial sums need more than kStaticScratchBytes are rejected with
//    BMM_ERR_WORKSPACE before anything is launched; use bmm_probs with a workspace instead.
//  - The address is cached per device for the life of the process.  Resetting a device after the
//    first call (cudaDeviceReset, or anything else that tears its primary context down) leaves a
//    stale address behind, so it is not supported; every other use of the device is unaffected.
//  - Arguments are checked exactly as bmm_probs checks them (same tests, same order, same codes),
//    plus the status word: non-null and 4-byte aligned (it is updated with 32-bit atomics).
#include <mutex>

#include "internal.h"

#define BMM_API extern "C" __attribute__((visibility("default")))

namespace bmm {
namespace {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device, looked up once per device.
cudaError_t static_scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (g_scratch_addr[dev] == nullptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace bmm

using namespace bmm;

BMM_API bmm_status bmm_probs_static(const bmm_mat* M, const bmm_mat* N, const bmm_blocks* B, int32_t pkind,
                                    double* p_out, const bmm_stats* st, int32_t* status_out, bmm_stream_t stream) {
    // the order of bmm_probs: the kind, then the problem, then the statistics
    if (pkind != BMM_P_COL_OPT && pkind != BMM_P_COL_UNIFORM && pkind != BMM_P_BLK_NORMPROD) return BMM_ERR_ARG;
    bmm_status s = check_problem(M, N, B);
    if (s != BMM_OK) return s;
    if (st == nullptr || !st->x || !st->y || !st->a || !st->s || !st->mf || !st->nf) return BMM_ERR_ARG;
    if (status_out == nullptr || (reinterpret_cast<uintptr_t>(status_out) & 3)) return BMM_ERR_ARG;
    const VecSet vM = vecset_of_M(M), vN = vecset_of_N(N);
    const int64_t partial_elems = imax(vec_sqnorms_partial_elems(vM), vec_sqnorms_partial_elems(vN));
    if ((size_t)partial_elems * sizeof(double) > kStaticScratchBytes) return BMM_ERR_WORKSPACE;
    void* scratch = nullptr;
    if (static_scratch_address(&scratch) != cudaSuccess) return BMM_ERR_CUDA;
    double* partial = static_cast<double*>(scratch);
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    DevStatus* dst = reinterpret_cast<DevStatus*>(status_out);
    cudaError_t e = launch_vec_sqnorms(vM, st->x, partial, partial_elems, cs);
    if (e == cudaSuccess) e = launch_vec_sqnorms(vN, st->y, partial, partial_elems, cs);
    if (e == cudaSuccess)
        e = launch_block_stats(st->x, st->y, B->offsets, B->K, B->n, st->a, st->s, st->mf, st->nf, dst, cs);
    if (e == cudaSuccess && p_out != nullptr)
        e = launch_probs(pkind, st->x, st->y, st->a, st->mf, st->nf, nullptr, B->offsets, B->K, B->n, p_out, dst, cs);
    return e == cudaSuccess ? BMM_OK : BMM_ERR_CUDA;
}
