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

// ---------------------------------------------------------------- direct form
// For small m p the product itself is cheaper than the Grams: f = ||sum_t w_t u_t v_t^T||_F^2 costs
// 2 m p len flops directly against 2 (m + p) len^2 through the trace identity (eq. 1.2 and eq. 3.9 with
// blocks of thousands of vectors and m, p of a few dozen, as in the paper's experiments).  CTA
// (k, s, r) accumulates the rectangle r (kDirTH rows x kDirTF columns) of block k's product over
// the s-th slice of its vectors in FP64 (each term (w_t u_h) v_f one FMA), and writes it to a
// partial buffer; direct_reduce_kernel sums the slices in slice order, squares and sums the entries.
constexpr int kDirThreads = 256;
constexpr int kDirTH = 32;                     // product rows per rectangle
constexpr int kDirTF = 64;                     // product columns per rectangle
constexpr int kDirPer = kDirTH * kDirTF / kDirThreads;  // 8 entries per thread: row t / 8, columns t % 8 + 8 j
constexpr int kDirChunk = 32;                  // vectors staged per step
constexpr int64_t kDirMaxEntries = 1 << 16;    // m p limit of the direct form (partial buffer size)

static int64_t dir_rects(int64_t m, int64_t p) { return ceil_div(m, kDirTH) * ceil_div(p, kDirTF); }
static int64_t dir_slices(int64_t K, int64_t len, int64_t m, int64_t p) {
    // about four CTAs per SM over the launch, slices of at least kDirChunk vectors
    const int64_t want = ceil_div(4 * 152, imax(K * dir_rects(m, p), 1));
    return imax(1, imin(want, ceil_div(imax(len, 1), kDirChunk)));
}

bool frob_use_direct(int64_t m, int64_t p, int64_t len) {
    if (m < 1 || p < 1 || m * p > kDirMaxEntries) return false;
    return m * p <= (m + p) * len || ceil_div(imax(len, 1), kTile) > 362;
}

template <typename T>
__global__ void __launch_bounds__(kDirThreads)
    direct_frob_kernel(const T* __restrict__ U, int64_t m, int64_t ldU, int modeU, const T* __restrict__ V, int64_t p,
                       int64_t ldV, int modeV, int64_t n_vec, const int64_t* __restrict__ off,
                       const int32_t* __restrict__ cols, const double* __restrict__ wts, int64_t per, int64_t slices,
                       double* __restrict__ partial, DevStatus* st) {
    __shared__ double su[kDirChunk][kDirTH];
    __shared__ double sv[kDirChunk][kDirTF];
    __shared__ double sw[kDirChunk];
    __shared__ int64_t sidx[kDirChunk];
    const int64_t k = blockIdx.x, sl = blockIdx.y, rect = blockIdx.z;
    const int64_t rf = ceil_div(p, kDirTF);
    const int64_t h0 = (rect / rf) * kDirTH, f0 = (rect % rf) * kDirTF;
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
    const int tid = threadIdx.x;
    const int hh = tid / 8, fc = tid % 8;
    double acc[kDirPer];
#pragma unroll
    for (int j = 0; j < kDirPer; ++j) acc[j] = 0.0;
    if (!ok) {
        if (tid == 0 && sl == 0 && rect == 0) set_status(st, BMM_ERR_SHAPE, (int)k);
        len = 0;
    }
    const int64_t chunk = ceil_div(imax(len, 1), slices);
    const int64_t t_lo = sl * chunk, t_hi = imin(len, t_lo + chunk);
    for (int64_t t0 = t_lo; t0 < t_hi; t0 += kDirChunk) {
        __syncthreads();
        if (tid < kDirChunk) {
            const int64_t t = t0 + tid;
            int64_t idx = -1;
            double w = 0.0;
            if (t < t_hi) {
                if (cols == nullptr) { idx = base + t; w = 1.0; }
                else {
                    idx = cols[base + t];
                    w = wts[base + t];
                    if (idx < 0 || idx >= n_vec) { set_status(st, BMM_ERR_ARG, (int)k); idx = -1; w = 0.0; }
                }
            }
            sidx[tid] = idx;
            sw[tid] = w;
        }
        __syncthreads();
        // stage u_t[h0 .. h0 + 32) (times w_t) and v_t[f0 .. f0 + 64) of the chunk's vectors
        for (int e = tid; e < kDirChunk * kDirTH; e += kDirThreads) {
            const int c = e / kDirTH, h = e % kDirTH;
            const int64_t idx = sidx[c], hg = h0 + h;
            double v = 0.0;
            if (idx >= 0 && hg < m) v = sw[c] * (double)Elem<T>::to_f64(modeU == VEC_CONTIG ? U[idx * ldU + hg] : U[hg * ldU + idx]);
            su[c][h] = v;
        }
        for (int e = tid; e < kDirChunk * kDirTF; e += kDirThreads) {
            const int c = e / kDirTF, f = e % kDirTF;
            const int64_t idx = sidx[c], fg = f0 + f;
            double v = 0.0;
            if (idx >= 0 && fg < p) v = (double)Elem<T>::to_f64(modeV == VEC_CONTIG ? V[idx * ldV + fg] : V[fg * ldV + idx]);
            sv[c][f] = v;
        }
        __syncthreads();
        const int nc = (int)imin(kDirChunk, t_hi - t0);
        for (int c = 0; c < nc; ++c) {
            const double a = su[c][hh];
#pragma unroll
            for (int j = 0; j < kDirPer; ++j) acc[j] = fma(a, sv[c][fc + 8 * j], acc[j]);
        }
    }
    double* out = partial + (k * slices + sl) * (m * p);
#pragma unroll
    for (int j = 0; j < kDirPer; ++j) {
        const int64_t h = h0 + hh, f = f0 + fc + 8 * j;
        if (h < m && f < p) out[h * p + f] = acc[j];
    }
}

// f[k] = sum over entries of (sum over slices of the partial products)^2, in a fixed order.
__global__ void __launch_bounds__(256) direct_reduce_kernel(const double* __restrict__ partial, int64_t mp, int64_t slices,
                                                            double* __restrict__ f) {
    __shared__ double red[8];
    const int64_t k = blockIdx.x;
    double s2 = 0.0;
    for (int64_t e = threadIdx.x; e < mp; e += blockDim.x) {
        double pe = 0.0;
        for (int64_t sl = 0; sl < slices; ++sl) pe += partial[(k * slices + sl) * mp + e];
        s2 = fma(pe, pe, s2);
    }
    s2 = warp_sum(s2);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < 8; ++w) tot += red[w];
        f[k] = tot;
    }
}

template <typename T>
static cudaError_t direct_frob_t(const VecSet& U, const VecSet& V, const int64_t* off, int64_t K, int64_t max_len,
                                 const int32_t* cols, const double* wts, int64_t per, double* f, double* partial,
                                 DevStatus* st, cudaStream_t s) {
    const int64_t m = U.len, p = V.len;
    const int64_t len = cols ? per : max_len;
    const int64_t slices = dir_slices(K, len, m, p);
    const int64_t rects = dir_rects(m, p);
    if (K > 2147483647LL || slices > 65535 || rects > 65535) return cudaErrorInvalidValue;
    dim3 grid((unsigned)K, (unsigned)slices, (unsigned)rects);
    (count_launch(), direct_frob_kernel<T><<<grid, kDirThreads, 0, s>>>(
                         static_cast<const T*>(U.data), m, U.ld, U.mode, static_cast<const T*>(V.data), p, V.ld, V.mode,
                         U.count, off, cols, wts, per, slices, partial, st));
    (count_launch(), direct_reduce_kernel<<<(unsigned)K, 256, 0, s>>>(partial, m * p, slices, f));
    return cudaGetLastError();
}

// ---------------------------------------------------------------- small pilots
// The Alg. 3 pilot with few draws per block (per <= kPilotMax, e.g. c0 = 4 K): one CTA per block
// k keeps every pair product <u_a, u_b>, <v_a, v_b> (a <= b < P) of its drawn vectors in registers,
// each thread summing a strided share of the coordinates in float-float (FP64 for FP64 data) and
// folding into FP64 every kPilotFold coordinates; the shares are summed in FP64 across the CTA and
// thread 0 forms f^_k = sum_{a,b} w_a w_b <u_a, u_b> <v_a, v_b>.  Rounding per up to P, so draws
// past per are empty vectors of weight 0.  Reads only the drawn vectors, once.
constexpr int kPilotMax = 8;
constexpr int kPilotThreads = 256;
constexpr int kPilotFold = 64;

template <int P> struct PilotPairs { static constexpr int n = P * (P + 1) / 2; };

template <typename T, int P>
__device__ __forceinline__ void pilot_gram(const T* __restrict__ X, int64_t len, int64_t ld, int mode,
                                           const int64_t* idx, double (*red)[kPilotThreads / 32], double* out) {
    constexpr int NP = PilotPairs<P>::n;
    DotAcc32 acc[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) acc[q].init();
    int since = 0;
    for (int64_t h = threadIdx.x; h < len; h += kPilotThreads) {
        typename AccT<T>::type v[P];
#pragma unroll
        for (int a = 0; a < P; ++a) {
            v[a] = 0;
            if (idx[a] >= 0) v[a] = ld_as(mode == VEC_CONTIG ? X + idx[a] * ld + h : X + h * ld + idx[a]);
        }
        int q = 0;
#pragma unroll
        for (int a = 0; a < P; ++a)
#pragma unroll
            for (int b = a; b < P; ++b) acc[q++].add(v[a], v[b]);
        if (++since == kPilotFold) {
#pragma unroll
            for (int qq = 0; qq < NP; ++qq) acc[qq].fold();
            since = 0;
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        const double w = warp_sum(acc[q].value());
        if (lane == 0) red[q][warp] = w;
    }
    __syncthreads();
    if (threadIdx.x < NP) {
        double s = 0.0;
        for (int w = 0; w < kPilotThreads / 32; ++w) s += red[threadIdx.x][w];
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

template <typename T, int P>
__global__ void __launch_bounds__(kPilotThreads)
    pilot_frob_kernel(const T* __restrict__ U, int64_t lenU, int64_t ldU, int modeU, const T* __restrict__ V,
                      int64_t lenV, int64_t ldV, int modeV, int64_t n_vec, const int32_t* __restrict__ cols,
                      const double* __restrict__ wts, int per, double* __restrict__ f, DevStatus* st) {
    constexpr int NP = PilotPairs<P>::n;
    __shared__ int64_t s_idx[P];
    __shared__ double s_w[P];
    __shared__ double red[NP][kPilotThreads / 32];
    __shared__ double gu[NP], gv[NP];
    const int64_t k = blockIdx.x;
    if (threadIdx.x < P) {
        int64_t id = -1;
        double w = 0.0;
        if ((int)threadIdx.x < per) {
            id = cols[k * per + threadIdx.x];
            w = wts[k * per + threadIdx.x];
            if (id < 0 || id >= n_vec) { set_status(st, BMM_ERR_ARG, (int)k); id = -1; w = 0.0; }
        }
        s_idx[threadIdx.x] = id;
        s_w[threadIdx.x] = w;
    }
    __syncthreads();
    pilot_gram<T, P>(U, lenU, ldU, modeU, s_idx, red, gu);
    pilot_gram<T, P>(V, lenV, ldV, modeV, s_idx, red, gv);
    if (threadIdx.x == 0) {
        double s = 0.0;
        int q = 0;
        for (int a = 0; a < P; ++a)
            for (int b = a; b < P; ++b, ++q) s += (a == b ? 1.0 : 2.0) * s_w[a] * s_w[b] * gu[q] * gv[q];
        f[k] = s;
    }
}

template <typename T, int P>
static cudaError_t pilot_frob_t(const VecSet& U, const VecSet& V, int64_t K, const int32_t* cols, const double* wts,
                                int per, double* f, DevStatus* st, cudaStream_t s) {
    (count_launch(), pilot_frob_kernel<T, P><<<(unsigned)K, kPilotThreads, 0, s>>>(
                         static_cast<const T*>(U.data), U.len, U.ld, U.mode, static_cast<const T*>(V.data), V.len, V.ld,
                         V.mode, U.count, cols, wts, per, f, st));
    return cudaGetLastError();
}

template <typename T>
static cudaError_t pilot_frob_any(const VecSet& U, const VecSet& V, int64_t K, const int32_t* cols, const double* wts,
                                  int per, double* f, DevStatus* st, cudaStream_t s) {
    if (per <= 1) return pilot_frob_t<T, 1>(U, V, K, cols, wts, per, f, st, s);
    if (per <= 2) return pilot_frob_t<T, 2>(U, V, K, cols, wts, per, f, st, s);
    if (per <= 4) return pilot_frob_t<T, 4>(U, V, K, cols, wts, per, f, st, s);
    return pilot_frob_t<T, kPilotMax>(U, V, K, cols, wts, per, f, st, s);
}

int64_t frob_partial_elems(int64_t K, int64_t len, int64_t m, int64_t p) {
    if (frob_use_direct(m, p, len)) return K * dir_slices(K, len, m, p) * m * p;
    return gram_frob_partial_elems(K, len);
}

cudaError_t launch_gram_frob(const VecSet& U, const VecSet& V, const int64_t* off, int64_t K, int64_t max_len,
                             const int32_t* cols, const double* wts, int64_t per, double* f, double* partial,
                             int64_t partial_cap, DevStatus* st, cudaStream_t s) {
    if (K <= 0) return cudaSuccess;
    if (cols != nullptr && per >= 1 && per <= kPilotMax && K <= 2147483647LL) {
        switch (U.dtype) {
            case BMM_F64: return pilot_frob_any<double>(U, V, K, cols, wts, (int)per, f, st, s);
            case BMM_F32: return pilot_frob_any<float>(U, V, K, cols, wts, (int)per, f, st, s);
            default: return pilot_frob_any<__nv_bfloat16>(U, V, K, cols, wts, (int)per, f, st, s);
        }
    }
    const int64_t len = cols ? per : max_len;
    if (frob_use_direct(U.len, V.len, len)) {
        if (partial_cap < frob_partial_elems(K, len, U.len, V.len)) return cudaErrorInvalidValue;
        switch (U.dtype) {
            case BMM_F64: return direct_frob_t<double>(U, V, off, K, max_len, cols, wts, per, f, partial, st, s);
            case BMM_F32: return direct_frob_t<float>(U, V, off, K, max_len, cols, wts, per, f, partial, st, s);
            default: return direct_frob_t<__nv_bfloat16>(U, V, off, K, max_len, cols, wts, per, f, partial, st, s);
        }
    }
    if (partial_cap < gram_frob_partial_elems(K, cols ? per : max_len)) return cudaErrorInvalidValue;
    if (K > 2147483647LL || tiles_for(cols ? per : max_len) > 362) return cudaErrorInvalidValue;
    switch (U.dtype) {
        case BMM_F64: return gram_frob_t<double>(U, V, off, K, max_len, cols, wts, per, f, partial, st, s);
        case BMM_F32: return gram_frob_t<float>(U, V, off, K, max_len, cols, wts, per, f, partial, st, s);
        default: return gram_frob_t<__nv_bfloat16>(U, V, off, K, max_len, cols, wts, per, f, partial, st, s);
    }
}

}  // namespace bmm
