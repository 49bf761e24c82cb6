// frob.cu -- ||sum_t w_t u_t v_t^T||_F^2 per block, through the trace identity
// ||A B||_F^2 = <A^T A, B B^T>_F  (A = [w_t u_t], B = [v_t]).
//
// Used for f_k = ||M^k N_k||_F^2 (eq. 1.2, eq. 3.9; every column of block k, w = 1) and for
// the Alg. 3 pilot ||C^{0k} D_{0k}||_F^2 (eq. 4.7; the [c0/K] drawn columns, w = 1/(c0' p0)).
// The Gram form needs 2 (m + p) n_k^2 flops per block instead of 2 m p n_k for the product
// itself.  Each CTA owns one 32 x 32 tile of index pairs (t, t') of one block, stages 32
// coordinates of its 64 vectors in shared memory and accumulates the dot products with
// FP64-accurate float-float sums (FP64 for FP64 data).
#include "internal.h"

namespace bmm {

template <typename T> struct AccT { using type = float; };
template <> struct AccT<double> { using type = double; };

struct DotAcc32 {
    FF ff;
    double d;
    __device__ __forceinline__ void init() { ff.zero(); d = 0.0; }
    __device__ __forceinline__ void add(float a, float b) { ff.add_prod(a, b); }
    __device__ __forceinline__ void add(double a, double b) { d = fma(a, b, d); }
    __device__ __forceinline__ void fold() { d += ff.value(); ff.zero(); }
    __device__ __forceinline__ double value() const { return d + ff.value(); }
};

__device__ __forceinline__ float ld_as(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ld_as(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ double ld_as(const double* p) { return __ldg(p); }

constexpr int kTile = 32;   // pairs tile edge
constexpr int kChunk = 32;  // coordinates staged per step

// Gram tile of one vector set: G[a][b] = <vec_{ia}, vec_{jb}> for a, b < 32, over all coordinates.
// Each of the 256 threads owns pairs (a, b) = (q*8 + tid/32, tid%32) for q < 4.
template <typename T>
__device__ void gram_tile(const T* __restrict__ X, int64_t len, int64_t ld, int mode,
                          const int64_t* vi, const int64_t* vj, bool same,
                          typename AccT<T>::type (*sA)[kTile + 1], typename AccT<T>::type (*sB)[kTile + 1],
                          double out[4]) {
    using A = typename AccT<T>::type;
    const int tid = threadIdx.x;
    DotAcc32 acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q].init();
    for (int64_t h0 = 0; h0 < len; h0 += kChunk) {
        __syncthreads();
        // stage sA[h][a] = vec_{vi[a]}[h0 + h] (and sB for the second index set)
        for (int e = tid; e < kChunk * kTile * 2; e += blockDim.x) {
            const int which = e / (kChunk * kTile);
            if (which == 1 && same) break;
            const int r = e % (kChunk * kTile);
            int h, a;
            if (mode == VEC_CONTIG) { a = r / kChunk; h = r % kChunk; }   // contiguous along h
            else { h = r / kTile; a = r % kTile; }                         // contiguous along the index
            const int64_t idx = which ? vj[a] : vi[a];
            A v = A(0);
            if (idx >= 0 && h0 + h < len) {
                const T* p = (mode == VEC_CONTIG) ? X + idx * ld + (h0 + h) : X + (h0 + h) * ld + idx;
                v = (A)ld_as(p);
            }
            if (which) sB[h][a] = v; else sA[h][a] = v;
        }
        __syncthreads();
        A (*tB)[kTile + 1] = same ? sA : sB;
#pragma unroll 4
        for (int h = 0; h < kChunk; ++h) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int a = q * 8 + (tid >> 5), b = tid & 31;
                acc[q].add(sA[h][a], tB[h][b]);
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q].fold();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) out[q] = acc[q].value();
}

template <typename T>
__global__ void __launch_bounds__(256) gram_frob_kernel(const T* __restrict__ U, int64_t lenU, int64_t ldU, int modeU,
                                                        const T* __restrict__ V, int64_t lenV, int64_t ldV, int modeV,
                                                        int64_t n_vec, const int64_t* __restrict__ off, int64_t K,
                                                        const int32_t* __restrict__ cols,
                                                        const double* __restrict__ wts, int64_t per, int tiles,
                                                        double* __restrict__ partial, DevStatus* st) {
    using A = typename AccT<T>::type;
    __shared__ A sA[kChunk][kTile + 1];
    __shared__ A sB[kChunk][kTile + 1];
    __shared__ int64_t vi[kTile], vj[kTile];
    __shared__ double wi[kTile], wj[kTile];
    __shared__ double red[8];
    const int64_t k = blockIdx.x;
    const int pairs = tiles * (tiles + 1) / 2;
    // decode the upper-triangular pair (ti <= tj) of this CTA
    int q = blockIdx.y, ti = 0;
    while (q >= tiles - ti) { q -= tiles - ti; ++ti; }
    const int tj = ti + q;
    int64_t base = 0, len = 0;
    bool ok = true;
    if (cols == nullptr) {
        base = off[k];
        len = off[k + 1] - base;
        ok = base >= 0 && len > 0 && base + len <= n_vec;
    } else {
        base = k * per;
        len = per;
    }
    double* outp = partial + k * pairs + blockIdx.y;
    if (!ok) {
        if (threadIdx.x == 0) { set_status(st, BMM_ERR_SHAPE, (int)k); *outp = 0.0; }
        return;
    }
    if ((int64_t)ti * kTile >= len || (int64_t)tj * kTile >= len) {
        if (threadIdx.x == 0) *outp = 0.0;
        return;
    }
    if (threadIdx.x < 2 * kTile) {
        const int which = threadIdx.x / kTile, a = threadIdx.x % kTile;
        const int64_t t = (int64_t)(which ? tj : ti) * kTile + a;
        int64_t idx = -1;
        double w = 0.0;
        if (t < len) {
            if (cols == nullptr) { idx = base + t; w = 1.0; }
            else {
                idx = cols[base + t];
                w = wts[base + t];
                if (idx < 0 || idx >= n_vec) { set_status(st, BMM_ERR_ARG, (int)k); idx = -1; w = 0.0; }
            }
        }
        if (which) { vj[a] = idx; wj[a] = w; } else { vi[a] = idx; wi[a] = w; }
    }
    __syncthreads();
    const bool same = (ti == tj);
    double gu[4], gv[4];
    gram_tile<T>(U, lenU, ldU, modeU, vi, vj, same, sA, sB, gu);
    gram_tile<T>(V, lenV, ldV, modeV, vi, vj, same, sA, sB, gv);
    double part = 0.0;
#pragma unroll
    for (int qq = 0; qq < 4; ++qq) {
        const int a = qq * 8 + (threadIdx.x >> 5), b = threadIdx.x & 31;
        part += wi[a] * wj[b] * gu[qq] * gv[qq];
    }
    part = warp_sum(part);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += red[w];
        *outp = same ? s : 2.0 * s;
    }
}

__global__ void sum_pairs_kernel(const double* __restrict__ partial, int64_t K, int pairs, double* __restrict__ f) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    double s = 0.0;
    for (int q = 0; q < pairs; ++q) s += partial[k * pairs + q];
    f[k] = s;
}

static int tiles_for(int64_t max_len) { return (int)ceil_div(imax(max_len, 1), kTile); }

int64_t gram_frob_partial_elems(int64_t K, int64_t max_len) {
    const int t = tiles_for(max_len);
    return K * (int64_t)(t * (t + 1) / 2);
}

template <typename T>
static cudaError_t gram_frob_t(const VecSet& U, const VecSet& V, const int64_t* off, int64_t K, int64_t max_len,
                               const int32_t* cols, const double* wts, int64_t per, double* f, double* partial,
                               DevStatus* st, cudaStream_t s) {
    const int tiles = tiles_for(cols ? per : max_len);
    const int pairs = tiles * (tiles + 1) / 2;
    dim3 grid((unsigned)K, (unsigned)pairs);
    (count_launch(), gram_frob_kernel<T><<<grid, 256, 0, s>>>(static_cast<const T*>(U.data), U.len, U.ld, U.mode,
                                             static_cast<const T*>(V.data), V.len, V.ld, V.mode, U.count, off, K,
                                             cols, wts, per, tiles, partial, st));
    (count_launch(), sum_pairs_kernel<<<(unsigned)ceil_div(K, 256), 256, 0, s>>>(partial, K, pairs, f));
    return cudaGetLastError();
}

cudaError_t launch_gram_frob(const VecSet& U, const VecSet& V, const int64_t* off, int64_t K, int64_t max_len,
                             const int32_t* cols, const double* wts, int64_t per, double* f, double* partial,
                             int64_t partial_cap, DevStatus* st, cudaStream_t s) {
    if (K <= 0) return cudaSuccess;
    if (partial_cap < gram_frob_partial_elems(K, cols ? per : max_len)) return cudaErrorInvalidValue;
    if (K > 2147483647LL || tiles_for(cols ? per : max_len) > 362) return cudaErrorInvalidValue;
    switch (U.dtype) {
        case BMM_F64: return gram_frob_t<double>(U, V, off, K, max_len, cols, wts, per, f, partial, st, s);
        case BMM_F32: return gram_frob_t<float>(U, V, off, K, max_len, cols, wts, per, f, partial, st, s);
        default: return gram_frob_t<__nv_bfloat16>(U, V, off, K, max_len, cols, wts, per, f, partial, st, s);
    }
}

}  // namespace bmm
