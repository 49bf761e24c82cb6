// norms.cu -- the statistics pass (Sec. 2, eq. 3.8; eq. 1.4; eq. 4.2).
//
// One read of M and N gives x_i = ||M^{(i)}||_2^2 and y_i = ||N_{(i)}||_2^2; a second,
// tiny kernel folds them into the per-block a_k, s_k, ||M^k||_F^2, ||N_k||_F^2.
// The pass is HBM-bound: 16-byte vector loads, many loads in flight per thread,
// FP64-accurate sums built from FP32 float-float pairs (GB300's FP64 rate is too
// low to square every element in FP64 at HBM speed), renormalised every 32 terms and folded
// into FP64 every 128 (one warp-wide FP64 instruction costs about 64 FP32 ones on GB300).
#include "internal.h"

namespace bmm {

template <typename T> struct VecTraits;
template <> struct VecTraits<float> { static constexpr int E = 4; };
template <> struct VecTraits<double> { static constexpr int E = 2; };
template <> struct VecTraits<__nv_bfloat16> { static constexpr int E = 8; };

__device__ __forceinline__ uint4 ldg16(const void* p) {
    return __ldg(reinterpret_cast<const uint4*>(p));
}

// FP64-accurate running sum of squares.
struct SqAcc {
    FF ff;
    double d;
    __device__ __forceinline__ void init() { ff.zero(); d = 0.0; }
    __device__ __forceinline__ void add(float v) { ff.add_prod(v, v); }
    __device__ __forceinline__ void add(double v) { d = fma(v, v, d); }
    __device__ __forceinline__ void fold() { d += ff.value(); ff.zero(); }
    __device__ __forceinline__ void renorm() { ff.renorm(); }
    __device__ __forceinline__ double value() const { return d + ff.value(); }
};

// 16 bytes -> E values of the accumulation type
__device__ __forceinline__ void acc16(SqAcc& a, uint4 r, float) {
    a.add(__uint_as_float(r.x)); a.add(__uint_as_float(r.y));
    a.add(__uint_as_float(r.z)); a.add(__uint_as_float(r.w));
}
__device__ __forceinline__ void acc16(SqAcc& a, uint4 r, double) {
    a.add(__hiloint2double((int)r.y, (int)r.x));
    a.add(__hiloint2double((int)r.w, (int)r.z));
}
__device__ __forceinline__ void acc16(SqAcc& a, uint4 r, __nv_bfloat16) {
    const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        a.add(__uint_as_float(w[q] << 16));
        a.add(__uint_as_float(w[q] & 0xffff0000u));
    }
}
// per-lane E accumulators, element e of the 16 bytes into acc[e]
__device__ __forceinline__ void acc16_split(SqAcc* a, uint4 r, float) {
    a[0].add(__uint_as_float(r.x)); a[1].add(__uint_as_float(r.y));
    a[2].add(__uint_as_float(r.z)); a[3].add(__uint_as_float(r.w));
}
__device__ __forceinline__ void acc16_split(SqAcc* a, uint4 r, double) {
    a[0].add(__hiloint2double((int)r.y, (int)r.x));
    a[1].add(__hiloint2double((int)r.w, (int)r.z));
}
__device__ __forceinline__ void acc16_split(SqAcc* a, uint4 r, __nv_bfloat16) {
    const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        a[2 * q].add(__uint_as_float(w[q] << 16));
        a[2 * q + 1].add(__uint_as_float(w[q] & 0xffff0000u));
    }
}
__device__ __forceinline__ void acc1(SqAcc& a, float v) { a.add(v); }
__device__ __forceinline__ void acc1(SqAcc& a, double v) { a.add(v); }
__device__ __forceinline__ void acc1(SqAcc& a, __nv_bfloat16 v) { a.add(__bfloat162float(v)); }

// Vectors stored as rows: one warp per vector, lanes stride the row with 16-byte loads.
template <typename T>
__global__ void __launch_bounds__(256) sqnorm_rows_kernel(const T* __restrict__ X, int64_t count, int64_t len,
                                                          int64_t ld, int vec_ok, double* __restrict__ out) {
    constexpr int E = VecTraits<T>::E;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = w0; r < count; r += nw) {
        const T* row = X + r * ld;
        SqAcc acc;
        acc.init();
        int64_t done = 0;
        if (vec_ok) {
            const int64_t nvec = len / E;
            int64_t it = lane;
            int batches = 0;
            for (; it + 7 * 32 < nvec; it += 8 * 32) {
                uint4 raw[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) raw[u] = ldg16(row + (it + u * 32) * E);
#pragma unroll
                for (int u = 0; u < 8; ++u) acc16(acc, raw[u], T());
                acc.renorm();
                if (++batches == 4) {
                    acc.fold();
                    batches = 0;
                }
            }
            for (; it < nvec; it += 32) acc16(acc, ldg16(row + it * E), T());
            acc.fold();
            done = nvec * E;
        }
        for (int64_t q = done + lane; q < len; q += 32) acc1(acc, row[q]);
        acc.fold();
        const double v = warp_sum(acc.value());
        if (lane == 0) out[r] = v;
    }
}

// Vectors stored as columns: thread owns E adjacent columns of a row slice.
template <typename T>
__global__ void __launch_bounds__(128) sqnorm_cols_kernel(const T* __restrict__ X, int64_t rows, int64_t cols,
                                                          int64_t ld, int64_t rows_per_slice, int vec_ok,
                                                          double* __restrict__ out) {
    constexpr int E = VecTraits<T>::E;
    const int64_t c0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * E;
    if (c0 >= cols) return;
    const int64_t r0 = (int64_t)blockIdx.y * rows_per_slice;
    const int64_t r1 = min(rows, r0 + rows_per_slice);
    SqAcc acc[E];
#pragma unroll
    for (int e = 0; e < E; ++e) acc[e].init();
    if (vec_ok && c0 + E <= cols) {
        int64_t r = r0;
        int batches = 0;
        for (; r + 8 <= r1; r += 8) {
            uint4 raw[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) raw[u] = ldg16(X + (r + u) * ld + c0);
#pragma unroll
            for (int u = 0; u < 8; ++u) acc16_split(acc, raw[u], T());
            if ((++batches & 3) == 0) {
#pragma unroll
                for (int e = 0; e < E; ++e) acc[e].renorm();
            }
            if (batches == 16) {
#pragma unroll
                for (int e = 0; e < E; ++e) acc[e].fold();
                batches = 0;
            }
        }
        for (; r < r1; ++r) acc16_split(acc, ldg16(X + r * ld + c0), T());
    } else {
        const int64_t ne = min((int64_t)E, cols - c0);
        for (int64_t r = r0; r < r1; ++r) {
            for (int e = 0; e < ne; ++e) acc1(acc[e], X[r * ld + c0 + e]);
            if (((r - r0) & 31) == 31)
                for (int e = 0; e < E; ++e) acc[e].fold();
        }
    }
    double* o = out + (int64_t)blockIdx.y * cols + c0;
#pragma unroll
    for (int e = 0; e < E; ++e)
        if (c0 + e < cols) o[e] = acc[e].value();
}

__global__ void sum_slices_kernel(const double* __restrict__ partial, int64_t slices, int64_t cols,
                                  double* __restrict__ out) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    double s = 0.0;
    for (int64_t q = 0; q < slices; ++q) s += partial[q * cols + c];
    out[c] = s;
}

static int elems_per_16(int dtype) { return dtype == BMM_F64 ? 2 : (dtype == BMM_F32 ? 4 : 8); }

static void col_geometry(const VecSet& v, int64_t* gx, int64_t* slices, int64_t* rps) {
    const int64_t E = elems_per_16(v.dtype);
    *gx = ceil_div(v.count, 128 * E);
    int64_t S = ceil_div(2048, *gx);
    S = imax(1, imin(S, ceil_div(v.len, 64)));
    S = imin(S, 65535);
    *rps = round_up(ceil_div(v.len, S), 32);
    *slices = ceil_div(v.len, *rps);
}

int64_t vec_sqnorms_partial_elems(const VecSet& v) {
    if (v.mode != VEC_STRIDED) return 0;
    int64_t gx, S, rps;
    col_geometry(v, &gx, &S, &rps);
    return S > 1 ? S * v.count : 0;
}

template <typename T>
static cudaError_t sqnorms_t(const VecSet& v, double* out, double* partial, int64_t partial_cap, cudaStream_t s) {
    const T* X = static_cast<const T*>(v.data);
    constexpr int E = VecTraits<T>::E;
    const int vec_ok = ((reinterpret_cast<uintptr_t>(X) & 15) == 0) && (v.ld % E == 0);
    if (v.count == 0) return cudaSuccess;
    if (v.mode == VEC_CONTIG) {
        const int64_t warps_needed = v.count;
        int64_t blocks = imin(ceil_div(warps_needed, 8), 152 * 64);
        (count_launch(), sqnorm_rows_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(X, v.count, v.len, v.ld, vec_ok, out));
        return cudaGetLastError();
    }
    int64_t gx, S, rps;
    col_geometry(v, &gx, &S, &rps);
    if (S > 1 && (partial == nullptr || partial_cap < S * v.count)) {
        S = 1;
        rps = v.len;
    }
    if (S <= 1) {
        dim3 grid((unsigned)gx, 1);
        (count_launch(), sqnorm_cols_kernel<T><<<grid, 128, 0, s>>>(X, v.len, v.count, v.ld, imax(v.len, 1), vec_ok, out));
        return cudaGetLastError();
    }
    dim3 grid((unsigned)gx, (unsigned)S);
    (count_launch(), sqnorm_cols_kernel<T><<<grid, 128, 0, s>>>(X, v.len, v.count, v.ld, rps, vec_ok, partial));
    (count_launch(), sum_slices_kernel<<<(unsigned)ceil_div(v.count, 256), 256, 0, s>>>(partial, S, v.count, out));
    return cudaGetLastError();
}

cudaError_t launch_vec_sqnorms(const VecSet& v, double* out, double* partial, int64_t partial_cap, cudaStream_t s) {
    switch (v.dtype) {
        case BMM_F64: return sqnorms_t<double>(v, out, partial, partial_cap, s);
        case BMM_F32: return sqnorms_t<float>(v, out, partial, partial_cap, s);
        default: return sqnorms_t<__nv_bfloat16>(v, out, partial, partial_cap, s);
    }
}

// One warp per block: a_k, s_k, mf_k, nf_k; validates offsets and finiteness.
__global__ void block_stats_kernel(const double* __restrict__ x, const double* __restrict__ y,
                                   const int64_t* __restrict__ off, int64_t K, int64_t n, double* a, double* ssum,
                                   double* mf, double* nf, DevStatus* st) {
    const int lane = threadIdx.x & 31;
    const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (k >= K) return;
    const int64_t lo = off[k], hi = off[k + 1];
    if ((k == 0 && lo != 0) || (k == K - 1 && hi != n) || hi <= lo || lo < 0 || hi > n) {
        if (lane == 0) set_status(st, BMM_ERR_SHAPE, (int)k);
        if (lane == 0) { a[k] = 0; ssum[k] = 0; mf[k] = 0; nf[k] = 0; }
        return;
    }
    double sa = 0, ss = 0, sx = 0, sy = 0;
    bool bad = false;
    for (int64_t i = lo + lane; i < hi; i += 32) {
        const double xi = x[i], yi = y[i];
        const double xy = __dmul_rn(xi, yi);
        bad |= !isfinite(xi) || !isfinite(yi);
        sa += sqrt(xy);
        ss += xy;
        sx += xi;
        sy += yi;
    }
    sa = warp_sum(sa);
    ss = warp_sum(ss);
    sx = warp_sum(sx);
    sy = warp_sum(sy);
    bad = __any_sync(0xffffffffu, bad);
    if (lane == 0) {
        a[k] = sa;
        ssum[k] = ss;
        mf[k] = sx;
        nf[k] = sy;
        if (bad) set_status(st, BMM_ERR_NONFINITE, (int)k);
    }
}

cudaError_t launch_block_stats(const double* x, const double* y, const int64_t* off, int64_t K, int64_t n,
                               double* a, double* ssum, double* mf, double* nf, DevStatus* st, cudaStream_t s) {
    (count_launch(), block_stats_kernel<<<(unsigned)ceil_div(K * 32, 256), 256, 0, s>>>(x, y, off, K, n, a, ssum, mf, nf, st));
    return cudaGetLastError();
}

}  // namespace bmm
