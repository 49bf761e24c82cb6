// gather.cu -- building the operands C and D of Alg. 2 (Alg. 1 step 1(b)).
//
// C^{(t)} = M^{(i_t)} sqrt(scale_t) and D_{(t)} = N_{(i_t)} sqrt(scale_t) are written as K-major
// rows for the tensor-core GEMM: operand A holds m rows of length L (row h = (C_{h,1..L})),
// operand B holds p rows of length L (row f = (D_{1..L,f})).  Block sampling first expands
// every drawn block into its run of contraction indices.
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

__global__ void set_extent_kernel(int64_t* ext, int64_t v) { *ext = v; }

cudaError_t launch_set_extent(int64_t* ext_dev, int64_t value, cudaStream_t s) {
    (count_launch(), set_extent_kernel<<<1, 1, 0, s>>>(ext_dev, value));
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
    __device__ __forceinline__ void put(int64_t r, int64_t j, double v) const {
        static_cast<double*>(out)[r * ldo + j] = v;
    }
    __device__ __forceinline__ void put(int64_t r, int64_t j, float v) const {
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

template <typename T, typename V>
__global__ void gather_strided_kernel(const T* __restrict__ X, int64_t len, int64_t ld, int64_t nvec,
                                      const int32_t* __restrict__ col, const double* __restrict__ w,
                                      const int64_t* __restrict__ ext_dev, bool apply_weight, OpWriter wr,
                                      DevStatus* st) {
    const int64_t ext = *ext_dev;
    const int64_t kseg = round_up(ext, 64);
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= kseg) return;
    wr.kseg = kseg;
    int64_t c = -1;
    V sw = V(0);
    if (j < ext) {
        c = col[j];
        sw = apply_weight ? (V)sqrt(w[j]) : V(1);
        if (c < 0 || c >= nvec) { set_status(st, BMM_ERR_ARG, (int)j); c = -1; }
    }
    for (int64_t r0 = (int64_t)blockIdx.y * kGatherRows; r0 < len; r0 += (int64_t)gridDim.y * kGatherRows) {
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
    const int64_t kseg = round_up(ext, 64);
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

// Vectors are storage rows (row-major N): 64 (contraction index j) x 64 (r) tiles through shared
// memory; rows are read 16 bytes at a time when aligned and the transposed operand is written 8
// BF16 (16 bytes) at a time.
template <typename T>
__global__ void __launch_bounds__(256) gather_contig_bf16_kernel(
    const T* __restrict__ X, int64_t len, int64_t ld, int64_t nvec, const int32_t* __restrict__ col,
    const double* __restrict__ w, const int64_t* __restrict__ ext_dev, bool apply_weight, bool vec4, OpWriter wr,
    DevStatus* st) {
    __shared__ float tile[64][65];
    __shared__ int64_t cidx[64];
    __shared__ float csw[64];
    const int64_t ext = *ext_dev;
    const int64_t kseg = round_up(ext, 64);
    const int64_t j0 = (int64_t)blockIdx.x * 64;
    if (j0 >= kseg) return;
    wr.kseg = kseg;
    const int t = threadIdx.x;
    if (t < 64) {
        const int64_t j = j0 + t;
        int64_t c = -1;
        float sw = 0.f;
        if (j < ext) {
            c = col[j];
            sw = apply_weight ? (float)sqrt(w[j]) : 1.f;
            if (c < 0 || c >= nvec) { set_status(st, BMM_ERR_ARG, (int)j); c = -1; }
        }
        cidx[t] = c;
        csw[t] = sw;
    }
    __syncthreads();
    for (int64_t r0 = (int64_t)blockIdx.y * 64; r0 < len; r0 += (int64_t)gridDim.y * 64) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int idx = t + 256 * u;
            const int jj = idx >> 4, q = idx & 15;
            const int64_t c = cidx[jj];
            const int64_t r = r0 + 4 * q;
            float e[4] = {0.f, 0.f, 0.f, 0.f};
            if (c >= 0) {
                const T* src = X + c * ld + r;
                if (vec4 && r + 4 <= len) {
                    const float4 f4 = __ldg(reinterpret_cast<const float4*>(src));
                    e[0] = f4.x; e[1] = f4.y; e[2] = f4.z; e[3] = f4.w;
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (r + k < len) e[k] = ldv<T, float>(src + k);
                }
            }
            const float sw = csw[jj];
#pragma unroll
            for (int k = 0; k < 4; ++k) tile[jj][4 * q + k] = e[k] * sw;
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int rr = (t >> 3) + 32 * u, jj8 = (t & 7) * 8;
            if (r0 + rr < len) {
                float v[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) v[k] = tile[jj8 + k][rr];
                put_bf16<8>(wr, r0 + rr, j0 + jj8, v);
            }
        }
        __syncthreads();
    }
}

template <typename T, typename V>
static cudaError_t gather_t(const VecSet& v, const int32_t* col, const double* w, const int64_t* ext_dev,
                            int64_t ext_max, int mode, int role, bool apply_weight, void* out, int64_t ldo,
                            DevStatus* st, cudaStream_t s) {
    OpWriter wr{out, ldo, 0, mode, role};
    const int64_t kmax = round_up(imax(ext_max, 1), 64);
    const T* X = static_cast<const T*>(v.data);
    if constexpr (std::is_same<V, float>::value) {
        // BF16 operand rows: 8- and 16-byte stores need ldo and the output 16-byte aligned
        if ((ldo % 8) != 0 || (reinterpret_cast<uintptr_t>(out) & 15) != 0) return cudaErrorInvalidValue;
        if (v.mode == VEC_STRIDED) {
            // one operand column per lane keeps every warp load one contiguous 128-byte span; wider
            // per-lane column groups spread a load over several spans and re-fetch sectors
            dim3 grid((unsigned)ceil_div(kmax, 128), (unsigned)imin(imax(ceil_div(v.len, kGatherRows), 1), 4096));
            (count_launch(), gather_strided_kernel<T, V><<<grid, 128, 0, s>>>(X, v.len, v.ld, v.count, col, w, ext_dev,
                                                                              apply_weight, wr, st));
        } else {
            const bool vec4 = sizeof(T) == 4 && std::is_same<T, float>::value && (v.ld % 4) == 0 &&
                              (reinterpret_cast<uintptr_t>(v.data) & 15) == 0;
            dim3 grid((unsigned)ceil_div(kmax, 64), (unsigned)imin(imax(ceil_div(v.len, 64), 1), 2048));
            (count_launch(), gather_contig_bf16_kernel<T><<<grid, 256, 0, s>>>(X, v.len, v.ld, v.count, col, w, ext_dev,
                                                                               apply_weight, vec4, wr, st));
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
                            DevStatus* st, cudaStream_t s) {
    switch (v.dtype) {
        case BMM_F64: return gather_t<double, V>(v, col, w, ext_dev, ext_max, mode, role, apply_weight, out, ldo, st, s);
        case BMM_F32: return gather_t<float, V>(v, col, w, ext_dev, ext_max, mode, role, apply_weight, out, ldo, st, s);
        default: return gather_t<__nv_bfloat16, V>(v, col, w, ext_dev, ext_max, mode, role, apply_weight, out, ldo, st, s);
    }
}

cudaError_t launch_gather_operand(const VecSet& v, const int32_t* col, const double* w, const int64_t* ext_dev,
                                  int64_t ext_max, int mode, int split_role, bool apply_weight, void* out, int64_t ldo,
                                  DevStatus* st, cudaStream_t s) {
    if (mode == BMM_GEMM_F64)
        return gather_v<double>(v, col, w, ext_dev, ext_max, mode, split_role, apply_weight, out, ldo, st, s);
    return gather_v<float>(v, col, w, ext_dev, ext_max, mode, split_role, apply_weight, out, ldo, st, s);
}

}  // namespace bmm
