// backward.cu -- adjoint of the sampled product (dM^{(i)} += w_i G N_{(i)}^T, dN_{(i)} += w_i M^{(i)T} G).
//
// The redrawn indices are reduced to their distinct values (ascending) with multiplicities, so the
// gradient scatter writes every touched column/row exactly once: no float atomics, deterministic.
// Duplicate draws of index i carry the same scale 1/(c_k p_i), hence w_i = mult_i * scale_i.
#include <type_traits>

#include "internal.h"

namespace bmm {

constexpr int kTileScan = 1024;

__device__ __forceinline__ unsigned long long warp_scan_incl(unsigned long long v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}
__device__ unsigned long long block_scan_incl(unsigned long long v, unsigned long long* sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long inc = warp_scan_incl(v);
    if (lane == 31) sm[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = sm[lane];
        sm[lane] = warp_scan_incl(w) - w;
    }
    __syncthreads();
    const unsigned long long r = inc + sm[warp];
    __syncthreads();
    return r;
}

int64_t unique_scratch_bytes(int64_t space, int64_t count) {
    (void)count;
    const int64_t ntiles = ceil_div(imax(space, 1), kTileScan);
    return round_up(space * 4, 256) + round_up(space * 8, 256) + round_up(space * 8, 256) + round_up(ntiles * 8, 256);
}

// ---------------------------------------------------------------- distinct draws, many products
// The same reduction for a table of products in five launches whatever their number: clear the
// counts, count the draws, scan the per-tile flags, scan each product's tile totals, compact.  Each
// CTA finds its product by binary search over the table's running offsets.
struct UniqueJobDev {
    const int32_t* idx;
    const double* scale;
    int64_t count, space;
    int* cnt;
    double* sval;
    unsigned long long* pos;
    unsigned long long* tot;
    int32_t* uidx;
    double* uw;
    int64_t* ucount;
    DevStatus* st;
    long long draw_begin, space_begin, tile_begin;
};
constexpr int kMaxUniqueJobs = 256;
struct UniqueTable {
    int count;
    long long draws, spaces, tiles;
    UniqueJobDev job[kMaxUniqueJobs];
};
static_assert(sizeof(UniqueTable) <= 32764, "distinct-draw table exceeds the kernel-parameter limit");

template <int WHICH>  // 0: draws, 1: space elements, 2: scan tiles
__device__ __forceinline__ int find_unique_job(const UniqueTable& tab, long long v) {
    int lo = 0, hi = tab.count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const long long b = WHICH == 0 ? tab.job[mid].draw_begin
                                       : (WHICH == 1 ? tab.job[mid].space_begin : tab.job[mid].tile_begin);
        if (b <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void unique_clear_grouped(const __grid_constant__ UniqueTable tab) {
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= tab.spaces) return;
    const UniqueJobDev& jb = tab.job[find_unique_job<1>(tab, v)];
    const long long i = v - jb.space_begin;
    jb.cnt[i] = 0;
    reinterpret_cast<unsigned long long*>(jb.sval)[i] = ~0ull;
}

__global__ void unique_hist_grouped(const __grid_constant__ UniqueTable tab) {
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= tab.draws) return;
    const UniqueJobDev& jb = tab.job[find_unique_job<0>(tab, v)];
    const long long t = v - jb.draw_begin;
    const int64_t i = jb.idx[t];
    if (i < 0 || i >= jb.space) {
        set_status(jb.st, BMM_ERR_ARG, (int)t);
        return;
    }
    atomicAdd(&jb.cnt[i], 1);
    const unsigned long long val = (unsigned long long)__double_as_longlong(jb.scale[t]);
    const unsigned long long old = atomicCAS(reinterpret_cast<unsigned long long*>(jb.sval) + i, ~0ull, val);
    if (old != ~0ull && old != val) set_status(jb.st, BMM_ERR_ARG, (int)t);
}

__global__ void __launch_bounds__(kTileScan) unique_flags_grouped(const __grid_constant__ UniqueTable tab) {
    __shared__ unsigned long long sm[32];
    const UniqueJobDev& jb = tab.job[find_unique_job<2>(tab, (long long)blockIdx.x)];
    const long long tile = (long long)blockIdx.x - jb.tile_begin;
    const int64_t i = tile * kTileScan + threadIdx.x;
    const unsigned long long f = (i < jb.space && jb.cnt[i] > 0) ? 1ull : 0ull;
    const unsigned long long inc = block_scan_incl(f, sm);
    if (i < jb.space) jb.pos[i] = inc - f;
    if (threadIdx.x == kTileScan - 1) jb.tot[tile] = inc;
}

__global__ void __launch_bounds__(kTileScan) unique_tiles_grouped(const __grid_constant__ UniqueTable tab) {
    __shared__ unsigned long long sm[32];
    __shared__ unsigned long long carry;
    const UniqueJobDev& jb = tab.job[blockIdx.x];
    const int64_t ntiles = ceil_div(jb.space, kTileScan);
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b = 0; b < ntiles; b += kTileScan) {
        const int64_t i = b + threadIdx.x;
        const unsigned long long v = i < ntiles ? jb.tot[i] : 0ull;
        const unsigned long long inc = block_scan_incl(v, sm);
        const unsigned long long c0 = carry;
        if (i < ntiles) jb.tot[i] = c0 + inc - v;
        __syncthreads();
        if (threadIdx.x == kTileScan - 1) carry = c0 + inc;
        __syncthreads();
    }
}

__global__ void unique_compact_grouped(const __grid_constant__ UniqueTable tab) {
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= tab.spaces) return;
    const UniqueJobDev& jb = tab.job[find_unique_job<1>(tab, v)];
    const int64_t i = v - jb.space_begin;
    const unsigned long long q = jb.pos[i] + jb.tot[i / kTileScan];
    const int c = jb.cnt[i];
    if (c > 0) {
        jb.uidx[q] = (int32_t)i;
        jb.uw[q] = __dmul_rn((double)c, jb.sval[i]);
    }
    if (i == jb.space - 1) *jb.ucount = (int64_t)(q + (c > 0 ? 1 : 0));
}

static cudaError_t launch_unique_table(const UniqueTable& tab, cudaStream_t s) {
    if (tab.count == 0) return cudaSuccess;
    (count_launch(), unique_clear_grouped<<<(unsigned)ceil_div(tab.spaces, 256), 256, 0, s>>>(tab));
    if (tab.draws > 0) (count_launch(), unique_hist_grouped<<<(unsigned)ceil_div(tab.draws, 256), 256, 0, s>>>(tab));
    (count_launch(), unique_flags_grouped<<<(unsigned)tab.tiles, kTileScan, 0, s>>>(tab));
    (count_launch(), unique_tiles_grouped<<<(unsigned)tab.count, kTileScan, 0, s>>>(tab));
    (count_launch(), unique_compact_grouped<<<(unsigned)ceil_div(tab.spaces, 256), 256, 0, s>>>(tab));
    return cudaGetLastError();
}

cudaError_t launch_unique_grouped(const UniqueJob* jobs, int64_t n, cudaStream_t s) {
    static thread_local UniqueTable tab;  // host-side staging of the kernel parameter, one per host thread (~31 KB)
    tab.count = 0;
    tab.draws = tab.spaces = tab.tiles = 0;
    for (int64_t k = 0; k <= n; ++k) {
        const bool full = tab.count == kMaxUniqueJobs ||
                          (k < n && (tab.spaces + jobs[k].space > 0x7fffffffLL * 128 ||
                                     tab.tiles + ceil_div(jobs[k].space, kTileScan) > 0x7fffffffLL));
        if (k == n || full) {
            cudaError_t e = launch_unique_table(tab, s);
            if (e != cudaSuccess) return e;
            tab.count = 0;
            tab.draws = tab.spaces = tab.tiles = 0;
        }
        if (k == n) break;
        const UniqueJob& u = jobs[k];
        if (u.space <= 0) return cudaErrorInvalidValue;
        UniqueJobDev& d = tab.job[tab.count++];
        char* w = static_cast<char*>(u.scratch);
        d.idx = u.idx;
        d.scale = u.scale;
        d.count = u.count;
        d.space = u.space;
        d.cnt = reinterpret_cast<int*>(w);
        w += round_up(u.space * 4, 256);
        d.sval = reinterpret_cast<double*>(w);
        w += round_up(u.space * 8, 256);
        d.pos = reinterpret_cast<unsigned long long*>(w);
        w += round_up(u.space * 8, 256);
        d.tot = reinterpret_cast<unsigned long long*>(w);
        d.uidx = u.uidx;
        d.uw = u.uw;
        d.ucount = u.ucount;
        d.st = u.st;
        d.draw_begin = tab.draws;
        d.space_begin = tab.spaces;
        d.tile_begin = tab.tiles;
        tab.draws += u.count;
        tab.spaces += u.space;
        tab.tiles += ceil_div(u.space, kTileScan);
    }
    return cudaSuccess;
}

cudaError_t launch_unique(const int32_t* idx, const double* scale, int64_t count, int64_t space, int32_t* uidx,
                          double* uw, int64_t* ucount_dev, void* scratch, DevStatus* st, cudaStream_t s) {
    const UniqueJob job{idx, scale, count, space, scratch, uidx, uw, ucount_dev, st};
    return launch_unique_grouped(&job, 1, s);
}

// ---------------------------------------------------------------- conversions of G
__global__ void convert_f32_bf16_kernel(const float* __restrict__ G, int64_t rows, int64_t cols, int64_t ldg,
                                        __nv_bfloat16* __restrict__ out, int64_t ldo) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t r = blockIdx.y; r < rows; r += gridDim.y)
        if (c < cols) out[r * ldo + c] = __float2bfloat16_rn(G[r * ldg + c]);
}

// eight elements per thread: two 16-byte loads, one 16-byte store (rows of 16-byte multiples)
__global__ void convert_f32_bf16_vec_kernel(const float* __restrict__ G, int64_t rows, int64_t cols8, int64_t ldg,
                                            __nv_bfloat16* __restrict__ out, int64_t ldo) {
    const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 8;
    if (c >= cols8 * 8) return;
    for (int64_t r = blockIdx.y; r < rows; r += gridDim.y) {
        const float4 a = *reinterpret_cast<const float4*>(G + r * ldg + c);
        const float4 b = *reinterpret_cast<const float4*>(G + r * ldg + c + 4);
        __nv_bfloat162 o[4] = {__floats2bfloat162_rn(a.x, a.y), __floats2bfloat162_rn(a.z, a.w),
                               __floats2bfloat162_rn(b.x, b.y), __floats2bfloat162_rn(b.z, b.w)};
        *reinterpret_cast<uint4*>(out + r * ldo + c) = *reinterpret_cast<const uint4*>(o);
    }
}

__global__ void convert_f64_kernel(const double* __restrict__ G, int64_t rows, int64_t cols, int64_t ldg,
                                   bool transpose, double* __restrict__ out, int64_t ldo) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t r = blockIdx.y; r < rows; r += gridDim.y) {
        if (c >= cols) continue;
        const double v = G[r * ldg + c];
        if (transpose) out[c * ldo + r] = v; else out[r * ldo + c] = v;
    }
}

cudaError_t launch_convert_f32_to_bf16(const float* G, int64_t rows, int64_t cols, int64_t ldg, __nv_bfloat16* out,
                                       int64_t ldo, cudaStream_t s) {
    if (cols % 8 == 0 && ldg % 4 == 0 && ldo % 8 == 0 && (reinterpret_cast<uintptr_t>(G) & 15) == 0 &&
        (reinterpret_cast<uintptr_t>(out) & 15) == 0) {
        dim3 grid((unsigned)ceil_div(cols / 8, 256), (unsigned)imin(imax(rows, 1), 8192));
        (count_launch(), convert_f32_bf16_vec_kernel<<<grid, 256, 0, s>>>(G, rows, cols / 8, ldg, out, ldo));
        return cudaGetLastError();
    }
    dim3 grid((unsigned)ceil_div(cols, 256), (unsigned)imin(imax(rows, 1), 8192));
    (count_launch(), convert_f32_bf16_kernel<<<grid, 256, 0, s>>>(G, rows, cols, ldg, out, ldo));
    return cudaGetLastError();
}

cudaError_t launch_convert_to_f64(const void* G, int dtype, int64_t rows, int64_t cols, int64_t ldg, bool transpose,
                                  double* out, int64_t ldo, cudaStream_t s) {
    if (dtype != BMM_F64) return cudaErrorInvalidValue;
    dim3 grid((unsigned)ceil_div(cols, 256), (unsigned)imin(imax(rows, 1), 8192));
    (count_launch(), convert_f64_kernel<<<grid, 256, 0, s>>>(static_cast<const double*>(G), rows, cols, ldg, transpose, out, ldo));
    return cudaGetLastError();
}

// ---------------------------------------------------------------- gathered vectors as rows
// out[j][r] = vec_{col_j}[r] for j < ext (zero rows for ext <= j < jmax)
template <typename T, typename O>
__global__ void gather_rows_kernel(const T* __restrict__ X, int64_t len, int64_t ld, int mode, int64_t nvec,
                                   const int32_t* __restrict__ col, const int64_t* __restrict__ ext_dev, int64_t jmax,
                                   O* __restrict__ out, int64_t ldo, int64_t r_begin) {
    __shared__ float t[32][33];
    const int64_t ext = *ext_dev;
    const int64_t j0 = (int64_t)blockIdx.x * 32, r0 = r_begin + (int64_t)blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    if (mode == VEC_CONTIG) {  // vector j is a storage row: copy along r
        for (int jj = ty; jj < 32; jj += blockDim.y) {
            const int64_t j = j0 + jj, r = r0 + tx;
            if (j >= jmax || r >= len) continue;
            O v = O(0.f);
            if (j < ext) {
                const int64_t c = col[j];
                if (c >= 0 && c < nvec) v = (O)(float)X[c * ld + r];
            }
            out[j * ldo + r] = v;
        }
        return;
    }
    // vector j is a storage column: read X[r*ld + col_j] along j, write along r
    for (int rr = ty; rr < 32; rr += blockDim.y) {
        const int64_t r = r0 + rr, j = j0 + tx;
        float v = 0.f;
        if (r < len && j < ext) {
            const int64_t c = col[j];
            if (c >= 0 && c < nvec) v = (float)X[r * ld + c];
        }
        t[rr][tx] = v;
    }
    __syncthreads();
    for (int jj = ty; jj < 32; jj += blockDim.y) {
        const int64_t j = j0 + jj, r = r0 + tx;
        if (j < jmax && r < len) out[j * ldo + r] = (O)t[tx][jj];
    }
}

template <typename T>
__global__ void gather_rows_f64_kernel(const T* __restrict__ X, int64_t len, int64_t ld, int mode, int64_t nvec,
                                       const int32_t* __restrict__ col, const int64_t* __restrict__ ext_dev,
                                       int64_t jmax, double* __restrict__ out, int64_t ldo) {
    const int64_t ext = *ext_dev;
    const int64_t j = blockIdx.x;
    if (j >= jmax) return;
    const int64_t c = (j < ext) ? (int64_t)col[j] : -1;
    for (int64_t r = threadIdx.x; r < len; r += blockDim.x) {
        double v = 0.0;
        if (c >= 0 && c < nvec) v = (double)((mode == VEC_CONTIG) ? X[c * ld + r] : X[r * ld + c]);
        out[j * ldo + r] = v;
    }
}

// Contiguous vectors, eight elements per thread (16-byte BF16 stores): row j of out is storage row
// col_j of X converted to BF16, or zeros for j >= ext; elements r < len8 * 8 only (the caller copies
// the tail with the general kernel)
template <typename T>
__global__ void gather_rows_contig_vec_kernel(const T* __restrict__ X, int64_t len8, int64_t ld, int64_t nvec,
                                              const int32_t* __restrict__ col, const int64_t* __restrict__ ext_dev,
                                              __nv_bfloat16* __restrict__ out, int64_t ldo) {
    const int64_t j = blockIdx.y;
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 8;
    if (r >= len8 * 8) return;
    const int64_t c = j < *ext_dev ? (int64_t)col[j] : -1;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (c >= 0 && c < nvec) {
        if constexpr (sizeof(T) == 2) {
            v = *reinterpret_cast<const uint4*>(X + c * ld + r);
        } else {
            const float4 a = *reinterpret_cast<const float4*>(X + c * ld + r);
            const float4 b = *reinterpret_cast<const float4*>(X + c * ld + r + 4);
            __nv_bfloat162 o[4] = {__floats2bfloat162_rn(a.x, a.y), __floats2bfloat162_rn(a.z, a.w),
                                   __floats2bfloat162_rn(b.x, b.y), __floats2bfloat162_rn(b.z, b.w)};
            v = *reinterpret_cast<const uint4*>(o);
        }
    }
    *reinterpret_cast<uint4*>(out + j * ldo + r) = v;
}

template <typename T>
static cudaError_t gather_rows_t(const VecSet& v, const int32_t* col, const int64_t* ext_dev, int64_t jmax, void* out,
                                 int64_t ldo, bool f64, cudaStream_t s) {
    const T* X = static_cast<const T*>(v.data);
    if (f64) {
        (count_launch(), gather_rows_f64_kernel<T><<<(unsigned)jmax, 256, 0, s>>>(X, v.len, v.ld, v.mode, v.count, col, ext_dev, jmax,
                                                               static_cast<double*>(out), ldo));
    } else {
        if (ceil_div(v.len, 32) > 65535) return cudaErrorInvalidValue;
        constexpr int64_t per16 = 16 / (int64_t)sizeof(T);
        const bool vec = (std::is_same<T, float>::value || std::is_same<T, __nv_bfloat16>::value) &&
                         v.mode == VEC_CONTIG && v.len >= 8 && v.ld % per16 == 0 && ldo % 8 == 0 &&
                         jmax <= 65535 && (reinterpret_cast<uintptr_t>(X) & 15) == 0 &&
                         (reinterpret_cast<uintptr_t>(out) & 15) == 0;
        if (vec) {
            const int64_t len8 = v.len / 8;
            dim3 g((unsigned)ceil_div(len8, 256), (unsigned)jmax);
            (count_launch(), gather_rows_contig_vec_kernel<T><<<g, 256, 0, s>>>(X, len8, v.ld, v.count, col, ext_dev,
                                                                                 static_cast<__nv_bfloat16*>(out), ldo));
            if (v.len % 8 == 0) return cudaGetLastError();
        }
        // the general kernel: everything, or the tail past the vectorised part (r0 at a multiple of 32)
        const int64_t done = vec ? (v.len / 8) * 8 / 32 * 32 : 0;
        dim3 grid((unsigned)ceil_div(jmax, 32), (unsigned)ceil_div(v.len - done, 32));
        (count_launch(), gather_rows_kernel<T, __nv_bfloat16><<<grid, dim3(32, 8), 0, s>>>(
            X, v.len, v.ld, v.mode, v.count, col, ext_dev, jmax, static_cast<__nv_bfloat16*>(out), ldo, done));
    }
    return cudaGetLastError();
}

cudaError_t launch_gather_rows(const VecSet& v, const int32_t* col, const int64_t* ext_dev, int64_t jmax, void* out,
                               int64_t ldo, bool f64, cudaStream_t s) {
    if (jmax <= 0) return cudaSuccess;
    switch (v.dtype) {
        case BMM_F64: return gather_rows_t<double>(v, col, ext_dev, jmax, out, ldo, f64, s);
        case BMM_F32: return gather_rows_t<float>(v, col, ext_dev, jmax, out, ldo, f64, s);
        default: return gather_rows_t<__nv_bfloat16>(v, col, ext_dev, jmax, out, ldo, f64, s);
    }
}

// ---------------------------------------------------------------- scatter
template <typename D, typename S>
__global__ void scatter_kernel(D* __restrict__ dst, int64_t dst_ld, int dst_mode, int64_t len,
                               const S* __restrict__ src, int64_t src_ld, bool src_rows,
                               const int32_t* __restrict__ col, const double* __restrict__ w,
                               const int64_t* __restrict__ ext_dev, int64_t r_begin) {
    const int64_t ext = *ext_dev;
    const int64_t j0 = (int64_t)blockIdx.x * 32;
    if (j0 >= ext) return;
    const int64_t r0 = r_begin + (int64_t)blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    // dst_mode CONTIG: element r of vector c at dst[c*ld + r] -> let tx run along r
    // dst_mode STRIDED: at dst[r*ld + c] -> let tx run along j (adjacent columns)
    for (int q = ty; q < 32; q += blockDim.y) {
        int64_t j, r;
        if (dst_mode == VEC_CONTIG) { j = j0 + q; r = r0 + tx; }
        else { j = j0 + tx; r = r0 + q; }
        if (j >= ext || r >= len) continue;
        const int64_t c = col[j];
        const double sv = src_rows ? (double)src[j * src_ld + r] : (double)src[r * src_ld + j];
        D* d = (dst_mode == VEC_CONTIG) ? dst + c * dst_ld + r : dst + r * dst_ld + c;
        *d = (D)((double)*d + w[j] * sv);
    }
}

template <>
__global__ void scatter_kernel<float, float>(float* __restrict__ dst, int64_t dst_ld, int dst_mode, int64_t len,
                                             const float* __restrict__ src, int64_t src_ld, bool src_rows,
                                             const int32_t* __restrict__ col, const double* __restrict__ w,
                                             const int64_t* __restrict__ ext_dev, int64_t r_begin) {
    const int64_t ext = *ext_dev;
    const int64_t j0 = (int64_t)blockIdx.x * 32;
    if (j0 >= ext) return;
    const int64_t r0 = r_begin + (int64_t)blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int q = ty; q < 32; q += blockDim.y) {
        int64_t j, r;
        if (dst_mode == VEC_CONTIG) { j = j0 + q; r = r0 + tx; }
        else { j = j0 + tx; r = r0 + q; }
        if (j >= ext || r >= len) continue;
        const int64_t c = col[j];
        const float sv = src_rows ? src[j * src_ld + r] : src[r * src_ld + j];
        float* d = (dst_mode == VEC_CONTIG) ? dst + c * dst_ld + r : dst + r * dst_ld + c;
        *d = __fmaf_rn((float)w[j], sv, *d);
    }
}

// BF16 gradient from FP32 products: each touched element is w_j * src rounded to FP32, added to the
// stored value in FP32 and rounded to BF16 once (with a zeroed gradient: the FP32 value rounded)
template <>
__global__ void scatter_kernel<__nv_bfloat16, float>(__nv_bfloat16* __restrict__ dst, int64_t dst_ld, int dst_mode,
                                                     int64_t len, const float* __restrict__ src, int64_t src_ld,
                                                     bool src_rows, const int32_t* __restrict__ col,
                                                     const double* __restrict__ w,
                                                     const int64_t* __restrict__ ext_dev, int64_t r_begin) {
    const int64_t ext = *ext_dev;
    const int64_t j0 = (int64_t)blockIdx.x * 32;
    if (j0 >= ext) return;
    const int64_t r0 = r_begin + (int64_t)blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int q = ty; q < 32; q += blockDim.y) {
        int64_t j, r;
        if (dst_mode == VEC_CONTIG) { j = j0 + q; r = r0 + tx; }
        else { j = j0 + tx; r = r0 + q; }
        if (j >= ext || r >= len) continue;
        const int64_t c = col[j];
        const float sv = src_rows ? src[j * src_ld + r] : src[r * src_ld + j];
        __nv_bfloat16* d = (dst_mode == VEC_CONTIG) ? dst + c * dst_ld + r : dst + r * dst_ld + c;
        *d = __float2bfloat16_rn(__fmaf_rn((float)w[j], sv, __bfloat162float(*d)));
    }
}

// The BF16 gradient's drawn rows (contiguous vectors) from FP32 product rows, eight elements per
// thread with 16-byte accesses: element for element the operations of scatter_kernel<bf16, float>
// (w_j * src rounded to FP32, added to the stored value, rounded to BF16 once); r < len8 * 8 only
__global__ void scatter_rows_bf16_vec_kernel(__nv_bfloat16* __restrict__ dst, int64_t dst_ld, int64_t len8,
                                             const float* __restrict__ src, int64_t src_ld,
                                             const int32_t* __restrict__ col, const double* __restrict__ w,
                                             const int64_t* __restrict__ ext_dev) {
    const int64_t j = blockIdx.y;
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 8;
    if (j >= *ext_dev || r >= len8 * 8) return;
    const int64_t c = col[j];
    const float wj = (float)w[j];
    const float4 a = *reinterpret_cast<const float4*>(src + j * src_ld + r);
    const float4 b = *reinterpret_cast<const float4*>(src + j * src_ld + r + 4);
    const float sv[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    uint4* d = reinterpret_cast<uint4*>(dst + c * dst_ld + r);
    uint4 raw = *d;
    __nv_bfloat16* e = reinterpret_cast<__nv_bfloat16*>(&raw);
#pragma unroll
    for (int u = 0; u < 8; ++u) e[u] = __float2bfloat16_rn(__fmaf_rn(wj, sv[u], __bfloat162float(e[u])));
    *d = raw;
}

cudaError_t launch_scatter_grad(void* dst, int dst_dtype, int64_t dst_ld, int dst_mode, int64_t len, const void* src,
                                int src_dtype, int64_t src_ld, bool src_rows, const int32_t* col, const double* w,
                                const int64_t* ext_dev, int64_t ext_max, cudaStream_t s) {
    if (ext_max <= 0 || len <= 0) return cudaSuccess;
    if (ceil_div(len, 32) > 65535) return cudaErrorInvalidValue;
    int64_t done = 0;  // elements of each vector the vectorised kernel covers (a multiple of 32)
    if (dst_dtype == BMM_BF16 && src_dtype == BMM_F32 && dst_mode == VEC_CONTIG && src_rows && len >= 32 &&
        ext_max <= 65535 && dst_ld % 8 == 0 && src_ld % 4 == 0 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0 &&
        (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
        const int64_t len8 = len / 32 * 4;  // whole 32-element tiles, so that the rest starts at a tile
        dim3 g((unsigned)ceil_div(len8, 256), (unsigned)ext_max);
        (count_launch(), scatter_rows_bf16_vec_kernel<<<g, 256, 0, s>>>(static_cast<__nv_bfloat16*>(dst), dst_ld, len8,
                                                                        static_cast<const float*>(src), src_ld, col, w,
                                                                        ext_dev));
        done = len8 * 8;
        if (done == len) return cudaGetLastError();
    }
    dim3 grid((unsigned)ceil_div(ext_max, 32), (unsigned)ceil_div(len - done, 32));
    dim3 block(32, 8);
    if (dst_dtype == BMM_F64 && src_dtype == BMM_F64)
        (count_launch(), scatter_kernel<double, double><<<grid, block, 0, s>>>(static_cast<double*>(dst), dst_ld, dst_mode, len,
                                                             static_cast<const double*>(src), src_ld, src_rows, col, w,
                                                             ext_dev, done));
    else if (dst_dtype == BMM_F32 && src_dtype == BMM_F32)
        (count_launch(), scatter_kernel<float, float><<<grid, block, 0, s>>>(static_cast<float*>(dst), dst_ld, dst_mode, len,
                                                           static_cast<const float*>(src), src_ld, src_rows, col, w,
                                                           ext_dev, done));
    else if (dst_dtype == BMM_BF16 && src_dtype == BMM_F32)
        (count_launch(), scatter_kernel<__nv_bfloat16, float><<<grid, block, 0, s>>>(
                             static_cast<__nv_bfloat16*>(dst), dst_ld, dst_mode, len, static_cast<const float*>(src),
                             src_ld, src_rows, col, w, ext_dev, done));
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_zero_matrix(void* dst, int dtype, int64_t rows, int64_t cols, int64_t ld, cudaStream_t s) {
    const size_t es = dtype == BMM_F64 ? 8 : (dtype == BMM_F32 ? 4 : 2);
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    return cudaMemset2DAsync(dst, (size_t)ld * es, 0, (size_t)cols * es, (size_t)rows, s);
}

}  // namespace bmm
