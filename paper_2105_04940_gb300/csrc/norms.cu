// norms.cu -- the statistics pass (Sec. 2, eq. 3.8; eq. 1.4; eq. 4.2).
//
// One read of M and N gives x_i = ||M^{(i)}||_2^2 and y_i = ||N_{(i)}||_2^2; a second,
// tiny kernel folds them into the per-block a_k, s_k, ||M^k||_F^2, ||N_k||_F^2.
// The pass is HBM-bound: 16-byte vector loads, many loads in flight per thread,
// FP64-accurate sums built from FP32 float-float pairs (GB300's FP64 rate is too
// low to square every element in FP64 at HBM speed), renormalised every 32 terms and folded
// into FP64 every 128 (one warp-wide FP64 instruction costs about 64 FP32 ones on GB300).
#include <algorithm>
#include <type_traits>
#include <vector>

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

// ---------------------------------------------------------------- grouped norm pass
// x_i or y_i of the vector sets of many products in one launch per kernel kind and element type
// (bmm_probs_batched): a table of jobs travels as a __grid_constant__ kernel parameter, the CTAs of
// job j follow those of job j - 1 along blockIdx.x, and a CTA finds its job by binary search.  With
// many products in flight the slices of rows are taken only where the product's partial buffer
// holds them.  Two sums share paired FP32 instructions (FF2); BF16 squares are exact in FP32, so
// their TwoProd residual is left out; sums stay float-float (a second float-float level every 128
// terms or fewer) and reach FP64 once per vector, because on GB300 one warp-wide FP64 instruction
// costs about as much issue time as 64 FP32 ones.
struct NormJob {
    const void* X;
    int64_t len, count, ld;
    double* out;      // [count]
    double* partial;  // strided jobs with slices > 1: [slices][count] float-float (float2) slice sums
    int64_t rps;      // rows per slice
    int cta_begin;
    int vec_ok;
    int gx;           // CTAs across the vectors (strided)
    int slices;
};
constexpr int kMaxNormJobs = 384;  // 80-byte jobs: under the 32 KB kernel-parameter limit
constexpr int64_t kGroupedSliceRows = 512;  // strided sets in grouped launches: rows per slice, at least
struct NormTable {
    int count;
    int total;
    NormJob job[kMaxNormJobs];
};
static_assert(sizeof(NormTable) <= 32764, "norm table exceeds the kernel-parameter limit");

template <typename T> struct SqPair;
template <> struct SqPair<float> {
    static __device__ __forceinline__ void add(FF2& a, float2 v) { a.add_sq(v); }
};
template <> struct SqPair<__nv_bfloat16> {
    static __device__ __forceinline__ void add(FF2& a, float2 v) { a.add_sq_exact(v); }
};
// 16 bytes as pairs of FP32 values: FP32 (x, y), (z, w); BF16 the two halves of each word
template <typename T> __device__ __forceinline__ float2 pair_of(const uint4& r, int q);
template <> __device__ __forceinline__ float2 pair_of<float>(const uint4& r, int q) {
    return q == 0 ? make_float2(__uint_as_float(r.x), __uint_as_float(r.y))
                  : make_float2(__uint_as_float(r.z), __uint_as_float(r.w));
}
template <> __device__ __forceinline__ float2 pair_of<__nv_bfloat16>(const uint4& r, int q) {
    const uint32_t w = q == 0 ? r.x : (q == 1 ? r.y : (q == 2 ? r.z : r.w));
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}

__device__ __forceinline__ int norm_job_of(const NormTable& tab) {
    const int b = (int)blockIdx.x;
    int lo = 0, hi = tab.count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tab.job[mid].cta_begin <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Strided vectors (element r of vector c at X[r * ld + c]): a thread owns E adjacent vectors over
// one slice of rows.  Sums stay float-float (FP32 pipe): paired running sums renormalised every 32
// rows and added into a second float-float level every 128; a slice's sums go out as float-float
// pairs (partial buffer) or, without slices, as FP64.
template <typename T>
__global__ void __launch_bounds__(128) sqnorm_cols_grouped_kernel(const __grid_constant__ NormTable tab) {
    constexpr int E = VecTraits<T>::E, P = E / 2;
    const NormJob& jb = tab.job[norm_job_of(tab)];
    const T* X = static_cast<const T*>(jb.X);
    const int local = (int)blockIdx.x - jb.cta_begin;
    const int bx = local % jb.gx, by = local / jb.gx;
    const int64_t c0 = ((int64_t)bx * blockDim.x + threadIdx.x) * E;
    if (c0 >= jb.count) return;
    const int64_t r_lo = (int64_t)by * jb.rps, r_hi = imin(jb.len, r_lo + jb.rps);
    FF2 tot[P];
#pragma unroll
    for (int q = 0; q < P; ++q) tot[q].zero();
    if (jb.vec_ok && c0 + E <= jb.count) {
        FF2 acc[P];
#pragma unroll
        for (int q = 0; q < P; ++q) acc[q].zero();
        int64_t r = r_lo;
        int batches = 0;
        for (; r + 8 <= r_hi; r += 8) {
            uint4 raw[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) raw[u] = ldg16(X + (r + u) * jb.ld + c0);
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int q = 0; q < P; ++q) SqPair<T>::add(acc[q], pair_of<T>(raw[u], q));
            if ((++batches & 3) == 0) {
#pragma unroll
                for (int q = 0; q < P; ++q) acc[q].renorm();
            }
            if (batches == 16) {
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    tot[q].add(acc[q]);
                    tot[q].renorm();
                    acc[q].zero();
                }
                batches = 0;
            }
        }
        for (; r < r_hi; ++r) {
            const uint4 raw = ldg16(X + r * jb.ld + c0);
#pragma unroll
            for (int q = 0; q < P; ++q) SqPair<T>::add(acc[q], pair_of<T>(raw, q));
        }
#pragma unroll
        for (int q = 0; q < P; ++q) {
            acc[q].renorm();
            tot[q].add(acc[q]);
            tot[q].renorm();
        }
    } else {  // the ragged edge, one element at a time (pairs of one element each)
        const int64_t ne = imin((int64_t)E, jb.count - c0);
        FF2 acc[P];
#pragma unroll
        for (int q = 0; q < P; ++q) acc[q].zero();
        for (int64_t r = r_lo; r < r_hi; ++r) {
#pragma unroll
            for (int q = 0; q < P; ++q) {
                const float a = 2 * q < ne ? to_f32(X[r * jb.ld + c0 + 2 * q]) : 0.f;
                const float b = 2 * q + 1 < ne ? to_f32(X[r * jb.ld + c0 + 2 * q + 1]) : 0.f;
                SqPair<T>::add(acc[q], make_float2(a, b));
            }
            if (((r - r_lo) & 31) == 31) {
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    acc[q].renorm();
                    tot[q].add(acc[q]);
                    tot[q].renorm();
                    acc[q].zero();
                }
            }
        }
#pragma unroll
        for (int q = 0; q < P; ++q) {
            acc[q].renorm();
            tot[q].add(acc[q]);
            tot[q].renorm();
        }
    }
    if (jb.slices > 1) {
        float2* o = reinterpret_cast<float2*>(jb.partial) + (int64_t)by * jb.count;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const FF f = tot[e >> 1].half(e & 1);
            if (c0 + e < jb.count) o[c0 + e] = make_float2(f.hi, f.lo);
        }
    } else {
#pragma unroll
        for (int e = 0; e < E; ++e)
            if (c0 + e < jb.count) jb.out[c0 + e] = tot[e >> 1].half(e & 1).value();
    }
}

// out[c] = the sum of the slices' float-float partial sums of strided jobs, in slice order (one
// thread per vector), converted to FP64 once
__global__ void __launch_bounds__(256) sum_slices_grouped_kernel(const __grid_constant__ NormTable tab) {
    const NormJob& jb = tab.job[norm_job_of(tab)];
    const int64_t c = (int64_t)(blockIdx.x - jb.cta_begin) * blockDim.x + threadIdx.x;
    if (c >= jb.count) return;
    const float2* part = reinterpret_cast<const float2*>(jb.partial);
    FF v;
    v.zero();
    for (int q = 0; q < jb.slices; ++q) {
        const float2 t = part[(int64_t)q * jb.count + c];
        FF o;
        o.hi = t.x;
        o.lo = t.y;
        v.add(o);
        v.renorm();
    }
    jb.out[c] = v.value();
}

// Contiguous vectors (element r of vector c at X[c * ld + r]): a warp takes 32 consecutive vectors,
// four at a time with eight lanes each (short vectors keep more loads in flight that way), and the
// sum of vector 4 s + j is handed to lane 4 s + j, so that the 32 results are converted to FP64 by
// one instruction and stored together.  Sums stay float-float on the FP32 pipe.
template <typename T>
__global__ void __launch_bounds__(256) sqnorm_rows_grouped_kernel(const __grid_constant__ NormTable tab) {
    constexpr int E = VecTraits<T>::E, P = E / 2;
    const NormJob& jb = tab.job[norm_job_of(tab)];
    const T* X = static_cast<const T*>(jb.X);
    const int lane = threadIdx.x & 31, sub = lane >> 3, sl = lane & 7;
    const int64_t v0 = ((int64_t)(blockIdx.x - jb.cta_begin) * 8 + (threadIdx.x >> 5)) * 32;
    if (v0 >= jb.count) return;
    const int64_t nvec = jb.vec_ok ? jb.len / E : 0;  // 16-byte chunks per vector
    FF mine;  // the sum of vector v0 + lane
    mine.zero();
    for (int step = 0; step < 8; ++step) {
        const int64_t v = v0 + 4 * step + sub;
        FF f;
        f.zero();
        if (v < jb.count) {
            const T* row = X + v * jb.ld;
            FF2 acc, tot;
            acc.zero();
            tot.zero();
            int64_t it = sl;
            int batches = 0;
            for (; it + 7 * 8 < nvec; it += 8 * 8) {
                uint4 raw[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) raw[u] = ldg16(row + (it + u * 8) * E);
#pragma unroll
                for (int u = 0; u < 8; ++u)
#pragma unroll
                    for (int q = 0; q < P; ++q) SqPair<T>::add(acc, pair_of<T>(raw[u], q));
                acc.renorm();
                if (++batches * 8 * E >= 128) {  // a second float-float level every >= 128 terms
                    tot.add(acc);
                    tot.renorm();
                    acc.zero();
                    batches = 0;
                }
            }
            for (; it < nvec; it += 8) {
                const uint4 raw = ldg16(row + it * E);
#pragma unroll
                for (int q = 0; q < P; ++q) SqPair<T>::add(acc, pair_of<T>(raw, q));
            }
            // the rest (unaligned rows: all of it), one element at a time, 16 pairs per fold
            int pairs = 0;
            for (int64_t q = nvec * E + sl; q < jb.len; q += 16) {
                const float a = to_f32(row[q]);
                const float b = q + 8 < jb.len ? to_f32(row[q + 8]) : 0.f;
                SqPair<T>::add(acc, make_float2(a, b));
                if (++pairs == 16) {
                    acc.renorm();
                    tot.add(acc);
                    tot.renorm();
                    acc.zero();
                    pairs = 0;
                }
            }
            acc.renorm();
            tot.add(acc);
            tot.renorm();
            f = tot.both();
        }
        // the eight lanes of each vector combine their sums
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            FF other;
            other.hi = __shfl_xor_sync(0xffffffffu, f.hi, o);
            other.lo = __shfl_xor_sync(0xffffffffu, f.lo, o);
            f.add(other);
            f.renorm();
        }
        // vector 4 step + j sits in lanes 8 j .. 8 j + 7; lane 4 step + j takes it
        const int src = 8 * (lane & 3);
        const float hi = __shfl_sync(0xffffffffu, f.hi, src), lo = __shfl_sync(0xffffffffu, f.lo, src);
        if ((lane >> 2) == step) {
            mine.hi = hi;
            mine.lo = lo;
        }
    }
    if (v0 + lane < jb.count) jb.out[v0 + lane] = mine.value();
}

template <typename T, bool STRIDED>
static cudaError_t norm_grouped_t(const NormJobArgs* jobs, int64_t count, cudaStream_t s) {
    static thread_local NormTable tab;  // host-side staging of the kernel parameter, one per host thread (~37 KB below the limit)
    static thread_local NormTable sums;  // the slice sums of the same jobs
    constexpr int E = VecTraits<T>::E;
    const int dt = std::is_same<T, float>::value ? BMM_F32 : BMM_BF16;
    tab.count = tab.total = 0;
    sums.count = sums.total = 0;
    auto flush = [&]() -> cudaError_t {
        if (tab.count > 0 && tab.total > 0) {
            if (STRIDED)
                (count_launch(), sqnorm_cols_grouped_kernel<T><<<(unsigned)tab.total, 128, 0, s>>>(tab));
            else
                (count_launch(), sqnorm_rows_grouped_kernel<T><<<(unsigned)tab.total, 256, 0, s>>>(tab));
        }
        if (sums.count > 0 && sums.total > 0)
            (count_launch(), sum_slices_grouped_kernel<<<(unsigned)sums.total, 256, 0, s>>>(sums));
        tab.count = tab.total = 0;
        sums.count = sums.total = 0;
        return cudaGetLastError();
    };
    // the longest CTAs first (rows per CTA for strided sets, vector length for contiguous ones), so
    // that short ones fill the tail of the launch
    std::vector<int64_t> order;
    std::vector<int64_t> work;
    for (int64_t i = 0; i < count; ++i) {
        const VecSet& v = jobs[i].v;
        if (v.dtype != dt || (v.mode == VEC_STRIDED) != STRIDED || v.count <= 0) continue;
        order.push_back(i);
    }
    auto geometry = [&](int64_t i, int64_t* gx, int64_t* S, int64_t* rps) {
        const VecSet& v = jobs[i].v;
        *gx = ceil_div(v.count, 256);  // contiguous: 256 vectors per CTA
        *S = 1;
        *rps = imax(v.len, 1);
        if (STRIDED) {
            // slices of rows where the product's partial buffer holds them; with many products in the
            // launch there is no need for the single-product kernel's thin slices: at least
            // kGroupedSliceRows rows each keeps the partial sums' traffic under 1% of the input
            col_geometry(v, gx, S, rps);
            if (*rps < kGroupedSliceRows) {
                *rps = round_up(imin(imax(v.len, 1), kGroupedSliceRows), 32);
                *S = ceil_div(v.len, *rps);
            }
            if (*S > 1 && (jobs[i].partial == nullptr || jobs[i].partial_cap < *S * v.count)) {
                *S = 1;
                *rps = imax(v.len, 1);
            }
        }
    };
    for (const int64_t i : order) {
        int64_t gx, S, rps;
        geometry(i, &gx, &S, &rps);
        work.push_back(rps);
    }
    std::vector<int64_t> perm(order.size());
    for (size_t q = 0; q < perm.size(); ++q) perm[q] = (int64_t)q;
    std::stable_sort(perm.begin(), perm.end(), [&](int64_t a, int64_t b) { return work[a] > work[b]; });
    for (const int64_t pi : perm) {
        const int64_t i = order[pi];
        const VecSet& v = jobs[i].v;
        int64_t gx, S, rps;
        geometry(i, &gx, &S, &rps);
        const int64_t ctas = gx * S;
        if (tab.count == kMaxNormJobs || sums.count == kMaxNormJobs || (int64_t)tab.total + ctas > 0x7fffffffLL) {
            cudaError_t e = flush();
            if (e != cudaSuccess) return e;
        }
        NormJob& j = tab.job[tab.count++];
        j.X = v.data;
        j.len = v.len;
        j.count = v.count;
        j.ld = v.ld;
        j.out = jobs[i].out;
        j.partial = S > 1 ? jobs[i].partial : nullptr;
        j.rps = rps;
        j.cta_begin = tab.total;
        j.vec_ok = ((reinterpret_cast<uintptr_t>(v.data) & 15) == 0) && (v.ld % E == 0);
        j.gx = (int)gx;
        j.slices = (int)S;
        tab.total += (int)ctas;
        if (S > 1) {
            NormJob& q = sums.job[sums.count++];
            q = j;
            q.cta_begin = sums.total;
            sums.total += (int)ceil_div(v.count, 256);
        }
    }
    return flush();
}

cudaError_t launch_vec_sqnorms_grouped(const NormJobArgs* jobs, int64_t count, cudaStream_t s) {
    for (int64_t i = 0; i < count; ++i)
        if (jobs[i].v.dtype != BMM_F32 && jobs[i].v.dtype != BMM_BF16) return cudaErrorInvalidValue;
    cudaError_t e;
    if ((e = norm_grouped_t<float, true>(jobs, count, s)) != cudaSuccess) return e;
    if ((e = norm_grouped_t<float, false>(jobs, count, s)) != cudaSuccess) return e;
    if ((e = norm_grouped_t<__nv_bfloat16, true>(jobs, count, s)) != cudaSuccess) return e;
    return norm_grouped_t<__nv_bfloat16, false>(jobs, count, s);
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

// block_stats_kernel for many products in one launch (one warp per block, the CTAs of product j after
// those of product j - 1), and, where p is given, the eq. 3.8 probabilities p_i = sqrt(x_i y_i) / a_k
// of the block's columns with the same FP64 operations as probs_col_kernel (uniform 1/n_k when
// a_k = 0), reusing the square roots of the block sum: one kernel over all products' blocks instead
// of a probability launch per product.
struct BlockStatsJob {
    const double *x, *y;
    const int64_t* off;
    int64_t K, n;
    double *a, *s, *mf, *nf;
    DevStatus* st;
    double* p;
    int cta_begin;
};
constexpr int kMaxBlockStatsJobs = 336;
struct BlockStatsTable {
    int count;
    int total;
    BlockStatsJob job[kMaxBlockStatsJobs];
};
static_assert(sizeof(BlockStatsTable) <= 32764, "block-stats table exceeds the kernel-parameter limit");

__global__ void __launch_bounds__(256) block_stats_grouped_kernel(const __grid_constant__ BlockStatsTable tab) {
    const int b = (int)blockIdx.x;
    int lo = 0, hi = tab.count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tab.job[mid].cta_begin <= b) lo = mid;
        else hi = mid - 1;
    }
    const BlockStatsJob& jb = tab.job[lo];
    const int lane = threadIdx.x & 31;
    const int64_t k = ((int64_t)(b - jb.cta_begin) * blockDim.x + threadIdx.x) >> 5;
    if (k >= jb.K) return;
    const int64_t a0 = jb.off[k], a1 = jb.off[k + 1];
    if ((k == 0 && a0 != 0) || (k == jb.K - 1 && a1 != jb.n) || a1 <= a0 || a0 < 0 || a1 > jb.n) {
        if (lane == 0) {
            set_status(jb.st, BMM_ERR_SHAPE, (int)k);
            jb.a[k] = 0; jb.s[k] = 0; jb.mf[k] = 0; jb.nf[k] = 0;
        }
        return;
    }
    constexpr int kKeep = 4;  // square roots kept in registers for the probabilities (blocks <= 128)
    double root[kKeep];
    double sa = 0, ss = 0, sx = 0, sy = 0;
    bool bad = false;
    int q = 0;
    for (int64_t i = a0 + lane; i < a1; i += 32, ++q) {
        const double xi = jb.x[i], yi = jb.y[i];
        const double xy = __dmul_rn(xi, yi);
        bad |= !isfinite(xi) || !isfinite(yi);
        const double r = sqrt(xy);
        if (q < kKeep) root[q] = r;
        sa += r;
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
        jb.a[k] = sa;
        jb.s[k] = ss;
        jb.mf[k] = sx;
        jb.nf[k] = sy;
        if (bad) set_status(jb.st, BMM_ERR_NONFINITE, (int)k);
    }
    if (jb.p != nullptr) {
        const double uni = __ddiv_rn(1.0, (double)(a1 - a0));
        q = 0;
        for (int64_t i = a0 + lane; i < a1; i += 32, ++q) {
            double v = uni;
            if (sa > 0.0) v = __ddiv_rn(q < kKeep ? root[q] : sqrt(__dmul_rn(jb.x[i], jb.y[i])), sa);
            jb.p[i] = v;
        }
    }
}

cudaError_t launch_block_stats_grouped(const BlockStatsArgs* args, int64_t count, cudaStream_t s) {
    static thread_local BlockStatsTable tab;  // host-side staging of the kernel parameter, one per host thread
    tab.count = 0;
    tab.total = 0;
    auto flush = [&]() -> cudaError_t {
        if (tab.count > 0 && tab.total > 0)
            (count_launch(), block_stats_grouped_kernel<<<(unsigned)tab.total, 256, 0, s>>>(tab));
        tab.count = 0;
        tab.total = 0;
        return cudaGetLastError();
    };
    for (int64_t i = 0; i < count; ++i) {
        const BlockStatsArgs& g = args[i];
        if (g.K <= 0) continue;
        const int64_t ctas = ceil_div(g.K * 32, 256);
        if (tab.count == kMaxBlockStatsJobs || (int64_t)tab.total + ctas > 0x7fffffffLL) {
            cudaError_t e = flush();
            if (e != cudaSuccess) return e;
        }
        BlockStatsJob& j = tab.job[tab.count++];
        j.x = g.x; j.y = g.y; j.off = g.off; j.K = g.K; j.n = g.n;
        j.a = g.a; j.s = g.s; j.mf = g.mf; j.nf = g.nf; j.st = g.st; j.p = g.p;
        j.cta_begin = tab.total;
        tab.total += (int)ctas;
    }
    return flush();
}

}  // namespace bmm
