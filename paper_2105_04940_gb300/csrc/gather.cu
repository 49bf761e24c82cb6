// gather.cu -- building the operands C and D of Alg. 2 (Alg. 1 step 1(b)).
//
// C^{(t)} = M^{(i_t)} sqrt(scale_t) and D_{(t)} = N_{(i_t)} sqrt(scale_t) are written as K-major
// rows for the tensor-core GEMM: operand A holds m rows of length L (row h = (C_{h,1..L})),
// operand B holds p rows of length L (row f = (D_{1..L,f})).  Block sampling first expands
// every drawn block into its run of contraction indices.
#include <cuda_fp8.h>

#include <type_traits>

#include "internal.h"

namespace bmm {

// ---------------------------------------------------------------- block expansion
// length of block k, or -1 when its offsets are invalid (then nothing is read or written for it)
__device__ __forceinline__ int64_t block_len(const int64_t* off, int64_t k, int64_t K, int64_t n, int64_t max_nk) {
    if (k < 0 || k >= K) return -1;
    const int64_t a = off[k], b = off[k + 1];
    if (a < 0 || b > n || b <= a || b - a > max_nk) return -1;
    return b - a;
}

__global__ void __launch_bounds__(1024) expand_prefix_kernel(const int32_t* __restrict__ kidx, int64_t count,
                                                             const int64_t* __restrict__ count_dev,
                                                             const int64_t* __restrict__ off, int64_t K, int64_t n,
                                                             int64_t max_nk, int64_t* __restrict__ pos,
                                                             int64_t* __restrict__ ext, DevStatus* st) {
    __shared__ long long sm[32];
    __shared__ long long carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (count_dev != nullptr) count = imin(count, *count_dev);
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b0 = 0; b0 < count; b0 += 1024) {
        const int64_t t = b0 + threadIdx.x;
        long long len = 0;
        if (t < count) {
            const int64_t k = kidx[t];
            len = block_len(off, k, K, n, max_nk);
            if (len < 0) {
                set_status(st, (k < 0 || k >= K) ? BMM_ERR_ARG : BMM_ERR_SHAPE, (int)t);
                len = 0;
            }
        }
        long long inc = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        if (lane == 31) sm[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            long long w = sm[lane], wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                long long v = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += v;
            }
            sm[lane] = wi - w;
        }
        __syncthreads();
        const long long c0 = carry;
        const long long excl = c0 + sm[warp] + inc - len;
        if (t < count) pos[t] = excl;
        __syncthreads();
        if (threadIdx.x == 1023) carry = excl + len;
        __syncthreads();
    }
    if (threadIdx.x == 0) *ext = carry;
}

__global__ void expand_fill_kernel(const int32_t* __restrict__ kidx, const double* __restrict__ kscale, int64_t count,
                                   const int64_t* __restrict__ count_dev, const int64_t* __restrict__ off, int64_t K,
                                   int64_t n, int64_t max_nk, const int64_t* __restrict__ pos,
                                   int32_t* __restrict__ col, double* __restrict__ w) {
    const int64_t t = blockIdx.x;
    if (count_dev != nullptr) count = imin(count, *count_dev);
    if (t >= count) return;
    const int64_t k = kidx[t];
    const int64_t len = block_len(off, k, K, n, max_nk);
    if (len <= 0) return;
    const int64_t a = off[k], p0 = pos[t];
    const double sc = kscale[t];
    for (int64_t q = threadIdx.x; q < len; q += blockDim.x) {
        col[p0 + q] = (int32_t)(a + q);
        w[p0 + q] = sc;
    }
}

cudaError_t launch_expand_blocks(const int32_t* kidx, const double* kscale, int64_t count, const int64_t* count_dev,
                                 const int64_t* off, int64_t K, int64_t n, int64_t max_nk, int32_t* col, double* w,
                                 int64_t* ext_dev, int64_t* prefix_scratch, DevStatus* st, cudaStream_t s) {
    (count_launch(), expand_prefix_kernel<<<1, 1024, 0, s>>>(kidx, count, count_dev, off, K, n, max_nk, prefix_scratch, ext_dev, st));
    if (count > 0)
        (count_launch(), expand_fill_kernel<<<(unsigned)count, 128, 0, s>>>(kidx, kscale, count, count_dev, off, K, n, max_nk,
                                                           prefix_scratch, col, w));
    return cudaGetLastError();
}


// ---------------------------------------------------------------- operand writers
// V is the arithmetic type of the scaled value: float for the BF16 modes, double for F64.
template <typename T, typename V> __device__ __forceinline__ V ldv(const T* p);
template <> __device__ __forceinline__ float ldv<float, float>(const float* p) { return __ldg(p); }
template <> __device__ __forceinline__ float ldv<__nv_bfloat16, float>(const __nv_bfloat16* p) { return __bfloat162float(*p); }
template <> __device__ __forceinline__ float ldv<double, float>(const double* p) { return (float)__ldg(p); }
template <> __device__ __forceinline__ double ldv<float, double>(const float* p) { return (double)__ldg(p); }
template <> __device__ __forceinline__ double ldv<__nv_bfloat16, double>(const __nv_bfloat16* p) { return (double)__bfloat162float(*p); }
template <> __device__ __forceinline__ double ldv<double, double>(const double* p) { return __ldg(p); }

// write the value of (row r, column j) into the operand layout of `mode`
struct OpWriter {
    void* out;
    int64_t ldo, kseg;
    int mode, role;
    int kunit;              // padded extent: a multiple of 64 (128 for e4m3)
    const float* colscale;  // per-column factor replacing sqrt(w_j), or null
    __device__ __forceinline__ void put(int64_t r, int64_t j, double v) const {
        static_cast<double*>(out)[r * ldo + j] = v;
    }
    __device__ __forceinline__ void put(int64_t r, int64_t j, float v) const {
        if (mode == BMM_GEMM_E4M3) {
            static_cast<__nv_fp8_storage_t*>(out)[r * ldo + j] = __nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
            return;
        }
        __nv_bfloat16* o = static_cast<__nv_bfloat16*>(out) + r * ldo;
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        if (mode == BMM_GEMM_BF16) {
            o[j] = hi;
            return;
        }
        const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
        o[j] = hi;
        o[kseg + j] = role == 0 ? hi : lo;
        o[2 * kseg + j] = role == 0 ? lo : hi;
    }
};

// vectors are storage columns: element r of vector i at X[r*ld + i].  One thread per column j and
// a run of kGatherRows rows, so the weight's square root is taken once per run.
constexpr int kGatherRows = 64;

// One CTA's share of a strided gather: operand columns j = 128 bx + thread, rows from 64 by in
// steps of 64 gy (bx, by, gy: the CTA's place in a (gx, gy) grid of this gather).
template <typename T, typename V>
__device__ __forceinline__ void gather_strided_body(const T* __restrict__ X, int64_t len, int64_t ld, int64_t nvec,
                                                    const int32_t* __restrict__ col, const double* __restrict__ w,
                                                    int64_t ext, bool apply_weight, OpWriter wr, DevStatus* st,
                                                    int64_t bx, int64_t by, int64_t gy) {
    const int64_t kseg = round_up(ext, wr.kunit);
    const int64_t j = bx * blockDim.x + threadIdx.x;
    if (j >= kseg) return;
    wr.kseg = kseg;
    int64_t c = -1;
    V sw = V(0);
    if (j < ext) {
        c = col[j];
        sw = wr.colscale != nullptr ? (V)wr.colscale[j] : (apply_weight ? (V)sqrt(w[j]) : V(1));
        if (c < 0 || c >= nvec) { set_status(st, BMM_ERR_ARG, (int)j); c = -1; }
    }
    for (int64_t r0 = by * kGatherRows; r0 < len; r0 += gy * kGatherRows) {
        const int64_t r1 = imin(len, r0 + kGatherRows);
        if (c < 0) {
            for (int64_t r = r0; r < r1; ++r) wr.put(r, j, V(0));
            continue;
        }
        int64_t r = r0;
        for (; r + 4 <= r1; r += 4) {
            V v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = ldv<T, V>(X + (r + u) * ld + c);
#pragma unroll
            for (int u = 0; u < 4; ++u) wr.put(r + u, j, v[u] * sw);
        }
        for (; r < r1; ++r) wr.put(r, j, ldv<T, V>(X + r * ld + c) * sw);
    }
}

template <typename T, typename V>
__global__ void gather_strided_kernel(const T* __restrict__ X, int64_t len, int64_t ld, int64_t nvec,
                                      const int32_t* __restrict__ col, const double* __restrict__ w,
                                      const int64_t* __restrict__ ext_dev, bool apply_weight, OpWriter wr,
                                      DevStatus* st) {
    gather_strided_body<T, V>(X, len, ld, nvec, col, w, *ext_dev, apply_weight, wr, st, blockIdx.x, blockIdx.y,
                              gridDim.y);
}

// vectors are storage rows: element r of vector i at X[i*ld + r]; 32(j) x 64(r) transpose tiles
template <typename T, typename V>
__global__ void __launch_bounds__(256) gather_contig_kernel(const T* __restrict__ X, int64_t len, int64_t ld,
                                                            int64_t nvec, const int32_t* __restrict__ col,
                                                            const double* __restrict__ w,
                                                            const int64_t* __restrict__ ext_dev, bool apply_weight,
                                                            OpWriter wr, DevStatus* st) {
    __shared__ V tile[32][65];
    __shared__ int64_t cidx[32];
    __shared__ V csw[32];
    const int64_t ext = *ext_dev;
    const int64_t kseg = round_up(ext, wr.kunit);
    const int64_t j0 = (int64_t)blockIdx.x * 32;
    if (j0 >= kseg) return;
    wr.kseg = kseg;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x < 32) {
        const int64_t j = j0 + threadIdx.x;
        int64_t c = -1;
        V sw = V(0);
        if (j < ext) {
            c = col[j];
            sw = apply_weight ? (V)sqrt(w[j]) : V(1);
            if (c < 0 || c >= nvec) { set_status(st, BMM_ERR_ARG, (int)j); c = -1; }
        }
        cidx[threadIdx.x] = c;
        csw[threadIdx.x] = sw;
    }
    __syncthreads();
    for (int64_t r0 = (int64_t)blockIdx.y * 64; r0 < len; r0 += (int64_t)gridDim.y * 64) {
        for (int jj = warp; jj < 32; jj += 8) {
            const int64_t c = cidx[jj];
            for (int rr = lane; rr < 64; rr += 32) {
                const int64_t r = r0 + rr;
                tile[jj][rr] = (c >= 0 && r < len) ? ldv<T, V>(X + c * ld + r) * csw[jj] : V(0);
            }
        }
        __syncthreads();
        for (int rr = warp; rr < 64; rr += 8) {
            const int64_t r = r0 + rr;
            if (r < len && j0 + lane < kseg) wr.put(r, j0 + lane, tile[lane][rr]);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- BF16 operands, vector stores
// hi (and, for split BF16, lo) parts of n consecutive values, written as 8- or 16-byte stores
// (n = 4, 8) into the segments of the operand row: [hi] for BF16; [hi | hi | lo] (A, role 0)
// or [hi | lo | hi] (B, role 1) for split BF16, whose K-concatenated product is hi hi + hi lo + lo hi.
template <int NV>
struct Bf16Pack;
template <> struct Bf16Pack<4> { using type = uint2; };
template <> struct Bf16Pack<8> { using type = uint4; };

template <int NV>
__device__ __forceinline__ void put_bf16(const OpWriter& wr, int64_t r, int64_t j, const float* v) {
    using P = typename Bf16Pack<NV>::type;
    __align__(16) __nv_bfloat16 hi[NV], lo[NV];
#pragma unroll
    for (int u = 0; u < NV; ++u) {
        hi[u] = __float2bfloat16_rn(v[u]);
        lo[u] = __float2bfloat16_rn(v[u] - __bfloat162float(hi[u]));
    }
    __nv_bfloat16* o = static_cast<__nv_bfloat16*>(wr.out) + r * wr.ldo + j;
    *reinterpret_cast<P*>(o) = *reinterpret_cast<const P*>(hi);
    if (wr.mode == BMM_GEMM_SPLIT_BF16) {
        *reinterpret_cast<P*>(o + wr.kseg) = *reinterpret_cast<const P*>(wr.role == 0 ? hi : lo);
        *reinterpret_cast<P*>(o + 2 * wr.kseg) = *reinterpret_cast<const P*>(wr.role == 0 ? lo : hi);
    }
}

// 8 consecutive values as e4m3 bytes (saturating), one 8-byte store
__device__ __forceinline__ void put_fp8x8(const OpWriter& wr, int64_t r, int64_t j, const float* v) {
    __align__(8) __nv_fp8_storage_t q[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) q[u] = __nv_cvt_float_to_fp8(v[u], __NV_SATFINITE, __NV_E4M3);
    *reinterpret_cast<uint2*>(static_cast<__nv_fp8_storage_t*>(wr.out) + r * wr.ldo + j) = *reinterpret_cast<const uint2*>(q);
}

// Vectors are storage rows (row-major N): 64 (contraction index j) x S (coordinate r) tiles through
// shared memory, S = 16 elements of 16 bytes (64 FP32, 128 BF16, 32 FP64 coordinates); rows are read
// 16 bytes at a time when aligned and the transposed operand is written 8 BF16 (16 bytes) or 8 e4m3
// at a time.  One CTA (256 threads) handles operand columns 64 bx .. 64 bx + 63 and coordinates from
// S by in steps of S gy; the next step's loads are issued before this step's transposed stores, so
// each CTA keeps a tile of loads (16 KB) in flight while it writes.
template <typename T> constexpr int contig_step() { return 16 * (16 / (int)sizeof(T)); }
template <typename T>
__device__ __forceinline__ void gather_contig_bf16_body(const T* __restrict__ X, int64_t len, int64_t ld, int64_t nvec,
                                                        const int32_t* __restrict__ col, const double* __restrict__ w,
                                                        int64_t ext, bool apply_weight, bool vec16, OpWriter wr,
                                                        DevStatus* st, int64_t bx, int64_t by, int64_t gy) {
    constexpr int EPL = 16 / (int)sizeof(T);    // elements per 16-byte load
    constexpr int kStep = contig_step<T>();     // coordinates per step
    constexpr int LPR = kStep / EPL;            // loads per draw per step (16)
    constexpr int NL = 64 * LPR / 256;          // loads per thread per step (4)
    __shared__ float tile[64][kStep + 1];
    __shared__ int64_t cidx[64];
    __shared__ float csw[64];
    const int64_t kseg = round_up(ext, wr.kunit);
    const int64_t j0 = bx * 64;
    if (j0 >= kseg) return;
    wr.kseg = kseg;
    const int t = threadIdx.x;
    if (t < 64) {
        const int64_t j = j0 + t;
        int64_t c = -1;
        float sw = 0.f;
        if (j < ext) {
            c = col[j];
            sw = wr.colscale != nullptr ? wr.colscale[j] : (apply_weight ? (float)sqrt(w[j]) : 1.f);
            if (c < 0 || c >= nvec) { set_status(st, BMM_ERR_ARG, (int)j); c = -1; }
        }
        cidx[t] = c;
        csw[t] = sw;
    }
    __syncthreads();
    float e[NL][EPL];
    auto load_tile = [&](int64_t r0) {
#pragma unroll
        for (int u = 0; u < NL; ++u) {
            const int idx = t + 256 * u;
            const int jj = idx / LPR, q = idx % LPR;
            const int64_t c = cidx[jj];
            const int64_t r = r0 + EPL * q;
#pragma unroll
            for (int k = 0; k < EPL; ++k) e[u][k] = 0.f;
            if (c >= 0) {
                const T* src = X + c * ld + r;
                if (vec16 && r + EPL <= len) {
                    const uint4 raw = __ldg(reinterpret_cast<const uint4*>(src));
                    if constexpr (std::is_same<T, float>::value) {
                        e[u][0] = __uint_as_float(raw.x); e[u][1] = __uint_as_float(raw.y);
                        e[u][2] = __uint_as_float(raw.z); e[u][3] = __uint_as_float(raw.w);
                    } else if constexpr (std::is_same<T, double>::value) {
                        e[u][0] = (float)__hiloint2double((int)raw.y, (int)raw.x);
                        e[u][1] = (float)__hiloint2double((int)raw.w, (int)raw.z);
                    } else {
                        const uint32_t wd[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            e[u][2 * k] = __uint_as_float(wd[k] << 16);
                            e[u][2 * k + 1] = __uint_as_float(wd[k] & 0xffff0000u);
                        }
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < EPL; ++k)
                        if (r + k < len) e[u][k] = ldv<T, float>(src + k);
                }
            }
        }
    };
    int64_t r0 = by * kStep;
    if (r0 < len) load_tile(r0);
    for (; r0 < len; r0 += gy * kStep) {
#pragma unroll
        for (int u = 0; u < NL; ++u) {
            const int idx = t + 256 * u;
            const int jj = idx / LPR, q = idx % LPR;
            const float sw = csw[jj];
#pragma unroll
            for (int k = 0; k < EPL; ++k) tile[jj][EPL * q + k] = e[u][k] * sw;
        }
        __syncthreads();
        if (r0 + gy * kStep < len) load_tile(r0 + gy * kStep);
#pragma unroll
        for (int u = 0; u < kStep / 32; ++u) {
            const int rr = (t >> 3) + 32 * u, jj8 = (t & 7) * 8;
            if (r0 + rr < len) {
                float v[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) v[k] = tile[jj8 + k][rr];
                if (wr.mode == BMM_GEMM_E4M3)
                    put_fp8x8(wr, r0 + rr, j0 + jj8, v);
                else
                    put_bf16<8>(wr, r0 + rr, j0 + jj8, v);
            }
        }
        __syncthreads();
    }
}


template <typename T>
__global__ void __launch_bounds__(256) gather_contig_bf16_kernel(
    const T* __restrict__ X, int64_t len, int64_t ld, int64_t nvec, const int32_t* __restrict__ col,
    const double* __restrict__ w, const int64_t* __restrict__ ext_dev, bool apply_weight, bool vec16, OpWriter wr,
    DevStatus* st) {
    gather_contig_bf16_body<T>(X, len, ld, nvec, col, w, *ext_dev, apply_weight, vec16, wr, st, blockIdx.x, blockIdx.y,
                               gridDim.y);
}

// CTAs along the coordinates of a contiguous BF16 / e4m3 gather: each takes up to four steps of
// contig_step<T>() coordinates, so that its loads for one step overlap its stores of the previous one
template <typename T>
static int64_t contig_gy(int64_t len) { return imin(imax(ceil_div(ceil_div(len, contig_step<T>()), 4), 1), 2048); }

template <typename T> constexpr int dtype_of();
template <> constexpr int dtype_of<float>() { return BMM_F32; }
template <> constexpr int dtype_of<__nv_bfloat16>() { return BMM_BF16; }
template <> constexpr int dtype_of<double>() { return BMM_F64; }

// rows of X can be read 16 bytes at a time: every row starts on a 16-byte boundary
template <typename T>
static bool contig_vec16(const VecSet& v) {
    return (v.ld % (int64_t)(16 / sizeof(T))) == 0 && (reinterpret_cast<uintptr_t>(v.data) % 16) == 0;
}

template <typename T, typename V>
static cudaError_t gather_t(const VecSet& v, const int32_t* col, const double* w, const int64_t* ext_dev,
                            int64_t ext_max, int mode, int role, bool apply_weight, void* out, int64_t ldo,
                            DevStatus* st, cudaStream_t s, const float* colscale) {
    const int kunit = mode == BMM_GEMM_E4M3 ? 128 : 64;
    OpWriter wr{out, ldo, 0, mode, role, kunit, colscale};
    const int64_t kmax = round_up(imax(ext_max, 1), kunit);
    const T* X = static_cast<const T*>(v.data);
    if constexpr (std::is_same<V, float>::value) {
        // BF16 / e4m3 operand rows: 8- and 16-byte stores need ldo and the output 16-byte aligned
        if ((ldo % 16) != 0 || (reinterpret_cast<uintptr_t>(out) & 15) != 0) return cudaErrorInvalidValue;
        if (v.mode == VEC_STRIDED) {
            // one operand column per lane keeps every warp load one contiguous 128-byte span; wider
            // per-lane column groups spread a load over several spans and re-fetch sectors
            dim3 grid((unsigned)ceil_div(kmax, 128), (unsigned)imin(imax(ceil_div(v.len, kGatherRows), 1), 4096));
            (count_launch(), gather_strided_kernel<T, V><<<grid, 128, 0, s>>>(X, v.len, v.ld, v.count, col, w, ext_dev,
                                                                              apply_weight, wr, st));
        } else {
            const bool vec16 = contig_vec16<T>(v);
            dim3 grid((unsigned)ceil_div(kmax, 64), (unsigned)contig_gy<T>(v.len));
            (count_launch(), gather_contig_bf16_kernel<T><<<grid, 256, 0, s>>>(X, v.len, v.ld, v.count, col, w, ext_dev,
                                                                               apply_weight, vec16, wr, st));
        }
        return cudaGetLastError();
    } else {
    if (v.mode == VEC_STRIDED) {
        dim3 grid((unsigned)ceil_div(kmax, 128), (unsigned)imin(imax(ceil_div(v.len, kGatherRows), 1), 4096));
        (count_launch(), gather_strided_kernel<T, V><<<grid, 128, 0, s>>>(X, v.len, v.ld, v.count, col, w, ext_dev, apply_weight, wr, st));
    } else {
        dim3 grid((unsigned)ceil_div(kmax, 32), (unsigned)imin(imax(ceil_div(v.len, 64), 1), 2048));
        (count_launch(), gather_contig_kernel<T, V><<<grid, 256, 0, s>>>(X, v.len, v.ld, v.count, col, w, ext_dev, apply_weight, wr, st));
    }
    return cudaGetLastError();
    }
}

template <typename V>
static cudaError_t gather_v(const VecSet& v, const int32_t* col, const double* w, const int64_t* ext_dev,
                            int64_t ext_max, int mode, int role, bool apply_weight, void* out, int64_t ldo,
                            DevStatus* st, cudaStream_t s, const float* colscale) {
    switch (v.dtype) {
        case BMM_F64: return gather_t<double, V>(v, col, w, ext_dev, ext_max, mode, role, apply_weight, out, ldo, st, s, colscale);
        case BMM_F32: return gather_t<float, V>(v, col, w, ext_dev, ext_max, mode, role, apply_weight, out, ldo, st, s, colscale);
        default: return gather_t<__nv_bfloat16, V>(v, col, w, ext_dev, ext_max, mode, role, apply_weight, out, ldo, st, s, colscale);
    }
}

cudaError_t launch_gather_operand(const VecSet& v, const int32_t* col, const double* w, const int64_t* ext_dev,
                                  int64_t ext_max, int mode, int split_role, bool apply_weight, void* out, int64_t ldo,
                                  DevStatus* st, cudaStream_t s, const float* colscale) {
    if (mode == BMM_GEMM_F64)
        return gather_v<double>(v, col, w, ext_dev, ext_max, mode, split_role, apply_weight, out, ldo, st, s, colscale);
    return gather_v<float>(v, col, w, ext_dev, ext_max, mode, split_role, apply_weight, out, ldo, st, s, colscale);
}

// ---------------------------------------------------------------- grouped gathers
// The gathers of many products in one launch (bmm_apply_batched): a table of jobs travels as a
// __grid_constant__ kernel parameter, each job a (gx, gy) grid of the single-product kernel laid out
// one after another along blockIdx.x; a CTA finds its job by binary search over the jobs' first CTAs
// and runs the same body as the single-product kernel.  Extents are host values here.
struct GatherJobDev {
    const void* X;
    int64_t len, ld, nvec;
    const int32_t* col;
    const double* w;
    int64_t ext;                // draws, or their upper bound (the grid) when ext_dev is set
    const int64_t* ext_dev;     // device count of draws, or null
    OpWriter wr;
    DevStatus* st;
    int gx, gy;
    int cta_begin;
    int vec16;  // rows readable 16 bytes at a time
};
constexpr int kMaxGatherJobs = 224;  // 144-byte jobs: the table stays under the 32 KB parameter limit
struct GatherTable {
    int count;
    int total;
    GatherJobDev job[kMaxGatherJobs];
};
static_assert(sizeof(GatherTable) <= 32764, "gather table exceeds the kernel-parameter limit");

template <typename T, bool STRIDED>
__global__ void __launch_bounds__(STRIDED ? 128 : 256) gather_grouped_kernel(const __grid_constant__ GatherTable tab) {
    const int b = (int)blockIdx.x;
    int lo = 0, hi = tab.count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tab.job[mid].cta_begin <= b) lo = mid;
        else hi = mid - 1;
    }
    const GatherJobDev& jb = tab.job[lo];
    const int local = b - jb.cta_begin;
    const int64_t bx = local % jb.gx, by = local / jb.gx;
    const T* X = static_cast<const T*>(jb.X);
    const int64_t ext = jb.ext_dev != nullptr ? imin(*jb.ext_dev, jb.ext) : jb.ext;
    if constexpr (STRIDED)
        gather_strided_body<T, float>(X, jb.len, jb.ld, jb.nvec, jb.col, jb.w, ext, true, jb.wr, jb.st, bx, by, jb.gy);
    else
        gather_contig_bf16_body<T>(X, jb.len, jb.ld, jb.nvec, jb.col, jb.w, ext, true, jb.vec16 != 0, jb.wr, jb.st, bx,
                                   by, jb.gy);
}

template <typename T, bool STRIDED>
static cudaError_t launch_gather_table(const GatherTable& tab, cudaStream_t s) {
    if (tab.count == 0 || tab.total == 0) return cudaSuccess;
    (count_launch(), gather_grouped_kernel<T, STRIDED><<<(unsigned)tab.total, STRIDED ? 128 : 256, 0, s>>>(tab));
    return cudaGetLastError();
}

template <typename T, bool STRIDED>
static cudaError_t gather_grouped_t(const GatherJob* jobs, int64_t count, cudaStream_t s) {
    static thread_local GatherTable tab;  // host-side staging of the kernel parameter, one per host thread (~31 KB)
    tab.count = 0;
    tab.total = 0;
    for (int64_t i = 0; i <= count; ++i) {
        const bool flush = i == count || tab.count == kMaxGatherJobs;
        if (flush) {
            cudaError_t e = launch_gather_table<T, STRIDED>(tab, s);
            if (e != cudaSuccess) return e;
            tab.count = 0;
            tab.total = 0;
        }
        if (i == count) break;
        const GatherJob& g = jobs[i];
        const bool strided = g.v.mode == VEC_STRIDED;
        if (strided != STRIDED || g.v.dtype != dtype_of<T>()) continue;
        const int kunit = g.mode == BMM_GEMM_E4M3 ? 128 : 64;
        const int64_t kmax = round_up(imax(g.ext, 1), kunit);
        const int64_t gx = ceil_div(kmax, STRIDED ? 128 : 64);
        const int64_t gy = STRIDED ? imin(imax(ceil_div(g.v.len, kGatherRows), 1), 4096) : contig_gy<T>(g.v.len);
        if ((int64_t)tab.total + gx * gy > 0x7fffffffLL) {  // keep every launch's grid within 2^31 CTAs
            cudaError_t e = launch_gather_table<T, STRIDED>(tab, s);
            if (e != cudaSuccess) return e;
            tab.count = 0;
            tab.total = 0;
        }
        GatherJobDev& d = tab.job[tab.count++];
        d.X = g.v.data;
        d.len = g.v.len;
        d.ld = g.v.ld;
        d.nvec = g.v.count;
        d.col = g.col;
        d.w = g.w;
        d.ext = g.ext;
        d.ext_dev = g.ext_dev;
        d.wr = OpWriter{g.out, g.ldo, 0, g.mode, g.role, kunit, nullptr};
        d.st = g.st;
        d.gx = (int)gx;
        d.gy = (int)gy;
        d.cta_begin = tab.total;
        d.vec16 = contig_vec16<T>(g.v) ? 1 : 0;
        tab.total += (int)(gx * gy);
    }
    return cudaSuccess;
}

cudaError_t launch_gather_grouped(const GatherJob* jobs, int64_t count, cudaStream_t s) {
    for (int64_t i = 0; i < count; ++i) {
        const GatherJob& g = jobs[i];
        if (g.mode == BMM_GEMM_F64 || g.ext < 0 || (g.v.dtype != BMM_F32 && g.v.dtype != BMM_BF16 && g.v.dtype != BMM_F64))
            return cudaErrorInvalidValue;
        // BF16 / e4m3 operand rows: 8- and 16-byte stores need ldo and the output 16-byte aligned
        if ((g.ldo % 16) != 0 || (reinterpret_cast<uintptr_t>(g.out) & 15) != 0) return cudaErrorInvalidValue;
    }
    cudaError_t e;
    if ((e = gather_grouped_t<float, true>(jobs, count, s)) != cudaSuccess) return e;
    if ((e = gather_grouped_t<float, false>(jobs, count, s)) != cudaSuccess) return e;
    if ((e = gather_grouped_t<__nv_bfloat16, true>(jobs, count, s)) != cudaSuccess) return e;
    if ((e = gather_grouped_t<__nv_bfloat16, false>(jobs, count, s)) != cudaSuccess) return e;
    if ((e = gather_grouped_t<double, true>(jobs, count, s)) != cudaSuccess) return e;
    return gather_grouped_t<double, false>(jobs, count, s);
}

// ---------------------------------------------------------------- FP8 operand scales
// amax[j] = sqrt(w_j) max_r |vec_{col_j}[r]| as the bit pattern of a non-negative float, so that
// partial maxima combine with integer atomicMax.  Vectors are storage columns: a thread per j and a
// run of rows (as the strided gather); storage rows: a warp per j.
template <typename T>
__global__ void absmax_strided_kernel(const T* __restrict__ X, int64_t len, int64_t ld, int64_t nvec,
                                      const int32_t* __restrict__ col, const double* __restrict__ w,
                                      const int64_t* __restrict__ ext_dev, float* __restrict__ amax) {
    const int64_t ext = *ext_dev;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ext) return;
    const int64_t c = col[j];
    if (c < 0 || c >= nvec) return;
    float m = 0.f;
    const int64_t r1 = imin(len, ((int64_t)blockIdx.y + 1) * kGatherRows * 4);
    for (int64_t r = (int64_t)blockIdx.y * kGatherRows * 4; r < r1; ++r) m = fmaxf(m, fabsf(ldv<T, float>(X + r * ld + c)));
    m *= (float)sqrt(w[j]);
    if (m > 0.f) atomicMax(reinterpret_cast<int*>(amax) + j, __float_as_int(m));
}

template <typename T>
__global__ void absmax_contig_kernel(const T* __restrict__ X, int64_t len, int64_t ld, int64_t nvec,
                                     const int32_t* __restrict__ col, const double* __restrict__ w,
                                     const int64_t* __restrict__ ext_dev, float* __restrict__ amax) {
    const int64_t ext = *ext_dev;
    const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= ext) return;
    const int64_t c = col[j];
    if (c < 0 || c >= nvec) return;
    float m = 0.f;
    for (int64_t r = lane; r < len; r += 32) m = fmaxf(m, fabsf(ldv<T, float>(X + c * ld + r)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    m *= (float)sqrt(w[j]);
    if (lane == 0 && m > 0.f) atomicMax(reinterpret_cast<int*>(amax) + j, __float_as_int(m));
}

template <typename T>
static cudaError_t absmax_t(const VecSet& v, const int32_t* col, const double* w, const int64_t* ext_dev,
                            int64_t ext_max, float* amax, cudaStream_t s) {
    const T* X = static_cast<const T*>(v.data);
    if (v.mode == VEC_STRIDED) {
        dim3 grid((unsigned)ceil_div(imax(ext_max, 1), 128), (unsigned)imax(ceil_div(v.len, kGatherRows * 4), 1));
        (count_launch(), absmax_strided_kernel<T><<<grid, 128, 0, s>>>(X, v.len, v.ld, v.count, col, w, ext_dev, amax));
    } else {
        (count_launch(), absmax_contig_kernel<T><<<(unsigned)ceil_div(imax(ext_max, 1) * 32, 256), 256, 0, s>>>(
            X, v.len, v.ld, v.count, col, w, ext_dev, amax));
    }
    return cudaGetLastError();
}

cudaError_t launch_vec_absmax(const VecSet& v, const int32_t* col, const double* w, const int64_t* ext_dev,
                              int64_t ext_max, float* amax, cudaStream_t s) {
    if (v.len > 0x7fffffffLL / 2) return cudaErrorInvalidValue;  // grid.y of the strided form
    switch (v.dtype) {
        case BMM_F64: return absmax_t<double>(v, col, w, ext_dev, ext_max, amax, s);
        case BMM_F32: return absmax_t<float>(v, col, w, ext_dev, ext_max, amax, s);
        default: return absmax_t<__nv_bfloat16>(v, col, w, ext_dev, ext_max, amax, s);
    }
}

// One CTA.  e_j = round(log2(sqrt(b_j / a_j))) makes a_j 2^(e_j) and b_j 2^(-e_j) about equal (the
// product a_j b_j is unchanged); gA, gB are the largest exponents keeping every scaled maximum of
// their operand at most 448.  All factors are powers of two (exact).
__global__ void __launch_bounds__(1024) fp8_scales_kernel(const float* __restrict__ amaxA, const float* __restrict__ amaxB,
                                                          const double* __restrict__ w, const int64_t* __restrict__ ext_dev,
                                                          float* __restrict__ sa, float* __restrict__ sb,
                                                          float* __restrict__ out_scale) {
    __shared__ float red[2][32];
    const int64_t ext = *ext_dev;
    float ma = 0.f, mb = 0.f;
    for (int64_t j = threadIdx.x; j < ext; j += blockDim.x) {
        const float a = amaxA[j], b = amaxB[j];
        int e = 0;
        if (a > 0.f && b > 0.f) e = (int)fminf(fmaxf(rintf(0.5f * log2f(b / a)), -60.f), 60.f);
        ma = fmaxf(ma, ldexpf(a, e));
        mb = fmaxf(mb, ldexpf(b, -e));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ma = fmaxf(ma, __shfl_xor_sync(0xffffffffu, ma, o));
        mb = fmaxf(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    }
    if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = ma; red[1][threadIdx.x >> 5] = mb; }
    __syncthreads();
    if (threadIdx.x < 32) {
        ma = threadIdx.x < (blockDim.x >> 5) ? red[0][threadIdx.x] : 0.f;
        mb = threadIdx.x < (blockDim.x >> 5) ? red[1][threadIdx.x] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ma = fmaxf(ma, __shfl_xor_sync(0xffffffffu, ma, o));
            mb = fmaxf(mb, __shfl_xor_sync(0xffffffffu, mb, o));
        }
        if (threadIdx.x == 0) { red[0][0] = ma; red[1][0] = mb; }
    }
    __syncthreads();
    // largest g with max * 2^g <= 448: g = floor(log2(448 / max)), corrected for log2f rounding
    auto gexp = [](float mx) {
        if (!(mx > 0.f)) return 0;
        int g = (int)floorf(log2f(448.f / mx));
        g = max(-100, min(100, g));
        while (g > -100 && ldexpf(mx, g) > 448.f) --g;
        while (g < 100 && ldexpf(mx, g + 1) <= 448.f) ++g;
        return g;
    };
    const int gA = gexp(red[0][0]), gB = gexp(red[1][0]);
    for (int64_t j = threadIdx.x; j < ext; j += blockDim.x) {
        const float a = amaxA[j], b = amaxB[j];
        int e = 0;
        if (a > 0.f && b > 0.f) e = (int)fminf(fmaxf(rintf(0.5f * log2f(b / a)), -60.f), 60.f);
        // factors stay finite: the largest scaled value is at most 448, so only a column of values
        // below ~1e-36 could ask for more than 2^100
        const float r = (float)sqrt(w[j]);
        sa[j] = ldexpf(r, max(-140, min(100, e + gA)));
        sb[j] = ldexpf(r, max(-140, min(100, gB - e)));
    }
    if (threadIdx.x == 0) *out_scale = ldexpf(1.f, -(gA + gB));
}

cudaError_t launch_fp8_scales(const float* amaxA, const float* amaxB, const double* w, const int64_t* ext_dev,
                              float* sa, float* sb, float* out_scale, cudaStream_t s) {
    (count_launch(), fp8_scales_kernel<<<1, 1024, 0, s>>>(amaxA, amaxB, w, ext_dev, sa, sb, out_scale));
    return cudaGetLastError();
}

}  // namespace bmm
