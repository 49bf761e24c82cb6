// sampler.cu -- i.i.d. draws with replacement (Alg. 1 step 1(a), Alg. 2 step 1).
//
// W_j = floor(p_j 2^62) is an exact integer, so the inclusive prefix S is exact and the
// same in any summation order (uint64 arithmetic; differences within a segment are taken
// modulo 2^64, which is exact because a segment's mass is at most ~2^62).  Draw t of its
// segment uses r = Philox4x32-10(counter = (t, stream id), key = seed) and picks the
// smallest j with S_j > floor(r T / 2^64) by binary search.
#include "internal.h"

namespace bmm {

constexpr int kScanTile = 1024;

__device__ __forceinline__ unsigned long long warp_incl_scan_u64(unsigned long long v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// inclusive scan of one u64 per thread over a 1024-thread block; returns inclusive value
__device__ unsigned long long block_incl_scan_u64(unsigned long long v, unsigned long long* sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long inc = warp_incl_scan_u64(v);
    if (lane == 31) sm[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = sm[lane];
        unsigned long long wi = warp_incl_scan_u64(w);
        sm[lane] = wi - w;
    }
    __syncthreads();
    const unsigned long long res = inc + sm[warp];
    __syncthreads();
    return res;
}

// W, local inclusive scan per 1024-tile, tile totals
__global__ void __launch_bounds__(kScanTile) weights_scan_kernel(const double* __restrict__ p, int64_t len,
                                                                 unsigned long long* __restrict__ G,
                                                                 unsigned long long* __restrict__ tile_tot,
                                                                 DevStatus* st) {
    __shared__ unsigned long long sm[32];
    const int64_t j = (int64_t)blockIdx.x * kScanTile + threadIdx.x;
    unsigned long long W = 0;
    if (j < len) {
        const double pj = p[j];
        if (!(pj >= 0.0 && pj <= 1.0)) set_status(st, BMM_ERR_ARG, (int)(j & 0x7fffffff));
        else W = __double2ull_rz(floor(ldexp(pj, 62)));
    }
    const unsigned long long inc = block_incl_scan_u64(W, sm);
    if (j < len) G[j] = inc;
    if (threadIdx.x == kScanTile - 1) tile_tot[blockIdx.x] = inc;
}

// exclusive scan of the tile totals (one CTA, sequential over 1024-chunks)
__global__ void __launch_bounds__(kScanTile) tile_prefix_kernel(unsigned long long* __restrict__ tot, int64_t ntiles) {
    __shared__ unsigned long long sm[32];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b = 0; b < ntiles; b += kScanTile) {
        const int64_t i = b + threadIdx.x;
        const unsigned long long v = i < ntiles ? tot[i] : 0ull;
        const unsigned long long inc = block_incl_scan_u64(v, sm);
        const unsigned long long c0 = carry;
        if (i < ntiles) tot[i] = c0 + inc - v;
        __syncthreads();
        if (threadIdx.x == kScanTile - 1) carry = c0 + inc;
        __syncthreads();
    }
}

__global__ void add_tile_prefix_kernel(unsigned long long* __restrict__ G, const unsigned long long* __restrict__ tot,
                                       int64_t len) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < len) G[j] += tot[j / kScanTile];
}

// draw offsets D[k] = sum_{j<k} ck[j] (one CTA), with validation of ck and sum ck = c
__global__ void __launch_bounds__(kScanTile) draw_offsets_kernel(const int64_t* __restrict__ ck, int64_t K, int64_t c,
                                                                 int64_t* __restrict__ D, DevStatus* st) {
    __shared__ unsigned long long sm[32];
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b = 0; b < K; b += kScanTile) {
        const int64_t i = b + threadIdx.x;
        long long v = i < K ? ck[i] : 0;
        if (v < 0) { set_status(st, BMM_ERR_ARG, (int)i); v = 0; }
        const unsigned long long inc = block_incl_scan_u64((unsigned long long)v, sm);
        const long long c0 = carry;
        if (i < K) D[i] = c0 + (long long)inc - v;
        __syncthreads();
        if (threadIdx.x == kScanTile - 1) carry = c0 + (long long)inc;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        D[K] = carry;
        if (carry != c) set_status(st, BMM_ERR_INFEASIBLE, 3);
    }
}

// one thread per draw
__global__ void draw_kernel(const double* __restrict__ p, int unit, const int64_t* __restrict__ off, int64_t K,
                            int64_t len, const int64_t* __restrict__ D, const int64_t* __restrict__ ck, int64_t c,
                            uint64_t seed, uint64_t sid, const unsigned long long* __restrict__ G,
                            int32_t* __restrict__ idx, double* __restrict__ scale, DevStatus* st) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= c) return;
    int64_t a = 0, b = len, cnt = c;
    if (unit == BMM_UNIT_COLUMN) {
        // segment k with D[k] <= t < D[k+1] (D is non-decreasing)
        int64_t lo = 0, hi = K;  // invariant: D[lo] <= t < D[hi]
        if (!(D[K] > t)) {
            set_status(st, BMM_ERR_INFEASIBLE, 4);
            idx[t] = 0; scale[t] = 0.0;
            return;
        }
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (D[mid] <= t) lo = mid; else hi = mid;
        }
        a = off[lo];
        b = off[lo + 1];
        cnt = ck[lo];
        if (a < 0 || b <= a || b > len) {
            set_status(st, BMM_ERR_SHAPE, (int)lo);
            idx[t] = 0; scale[t] = 0.0;
            return;
        }
    }
    const unsigned long long base = (a == 0) ? 0ull : G[a - 1];
    const unsigned long long T = G[b - 1] - base;
    if (T == 0ull) {
        set_status(st, BMM_ERR_ARG, (int)(a & 0x7fffffff));
        idx[t] = (int32_t)a; scale[t] = 0.0;
        return;
    }
    const uint64_t r = draw_bits(seed, sid, (uint64_t)t);
    const unsigned long long target = __umul64hi(r, T);
    // smallest j in [a, b) with G[j] - base > target
    int64_t lo = a, hi = b - 1;  // answer in [lo, hi]; G[b-1] - base = T > target
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (G[mid] - base > target) hi = mid; else lo = mid + 1;
    }
    idx[t] = (int32_t)lo;
    scale[t] = __ddiv_rn(1.0, __dmul_rn((double)cnt, p[lo]));
}

// ---- many products per launch (bmm_sample_batched): the same integers, hence the same draws, as
// one launch sequence per product.  Three launches for up to kMaxSampleJobs products: the weights
// and per-tile scans of every product's tiles, one CTA per product for its tile prefix and draw
// offsets, and one thread per draw (the tile prefix added inside the binary search).
namespace {

struct SampleJob {
    const double* p;
    const int64_t* off;
    const int64_t* ck;
    int32_t* idx;
    double* scale;
    unsigned long long* G;    // [len] tile-local inclusive prefix of W
    unsigned long long* tot;  // [ntiles] tile totals, then their exclusive prefix
    int64_t* D;               // [K + 1] draw offsets (column unit)
    DevStatus* st;
    long long K, len, c;
    unsigned long long seed, sid;
    int unit;
    int tiles_before;   // tiles of the launch's earlier jobs
    int blocks_before;  // 128-draw blocks of the launch's earlier jobs
};
constexpr int kMaxSampleJobs = 200;  // 152-byte jobs under the kernel-parameter limit
template <int G> struct SampleTable {
    int count;
    SampleJob job[G];
};
static_assert(sizeof(SampleTable<kMaxSampleJobs>) <= 32760, "sampler table exceeds the kernel-parameter limit");

// the job whose range [before[j], before[j + 1]) holds x (before is non-decreasing over jobs)
template <int G, typename F>
__device__ __forceinline__ int job_of(const SampleTable<G>& tab, long long x, F before) {
    int lo = 0, hi = tab.count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (before(tab.job[mid]) <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <int G>
__global__ void __launch_bounds__(kScanTile) weights_scan_grouped_kernel(const __grid_constant__ SampleTable<G> tab) {
    __shared__ unsigned long long sm[32];
    const int q = job_of(tab, blockIdx.x, [](const SampleJob& j) { return (long long)j.tiles_before; });
    const SampleJob& jb = tab.job[q];
    const long long tile = (long long)blockIdx.x - jb.tiles_before;
    const long long j = tile * kScanTile + threadIdx.x;
    unsigned long long W = 0;
    if (j < jb.len) {
        const double pj = jb.p[j];
        if (!(pj >= 0.0 && pj <= 1.0)) set_status(jb.st, BMM_ERR_ARG, (int)(j & 0x7fffffff));
        else W = __double2ull_rz(floor(ldexp(pj, 62)));
    }
    const unsigned long long inc = block_incl_scan_u64(W, sm);
    if (j < jb.len) jb.G[j] = inc;
    if (threadIdx.x == kScanTile - 1) jb.tot[tile] = inc;
}

// one CTA per job: exclusive prefix of its tile totals, and its draw offsets (column unit)
template <int G>
__global__ void __launch_bounds__(kScanTile) prefix_grouped_kernel(const __grid_constant__ SampleTable<G> tab) {
    __shared__ unsigned long long sm[32];
    __shared__ unsigned long long carry;
    const SampleJob& jb = tab.job[blockIdx.x];
    const long long ntiles = (jb.len + kScanTile - 1) / kScanTile;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (long long b = 0; b < ntiles; b += kScanTile) {
        const long long i = b + threadIdx.x;
        const unsigned long long v = i < ntiles ? jb.tot[i] : 0ull;
        const unsigned long long inc = block_incl_scan_u64(v, sm);
        const unsigned long long c0 = carry;
        if (i < ntiles) jb.tot[i] = c0 + inc - v;
        __syncthreads();
        if (threadIdx.x == kScanTile - 1) carry = c0 + inc;
        __syncthreads();
    }
    if (jb.unit != BMM_UNIT_COLUMN) return;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (long long b = 0; b < jb.K; b += kScanTile) {
        const long long i = b + threadIdx.x;
        long long v = i < jb.K ? jb.ck[i] : 0;
        if (v < 0) { set_status(jb.st, BMM_ERR_ARG, (int)i); v = 0; }
        const unsigned long long inc = block_incl_scan_u64((unsigned long long)v, sm);
        const long long c0 = (long long)carry;
        if (i < jb.K) jb.D[i] = c0 + (long long)inc - v;
        __syncthreads();
        if (threadIdx.x == kScanTile - 1) carry = (unsigned long long)(c0 + (long long)inc);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        jb.D[jb.K] = (long long)carry;
        if ((long long)carry != jb.c) set_status(jb.st, BMM_ERR_INFEASIBLE, 3);
    }
}

template <int G>
__global__ void __launch_bounds__(128) draw_grouped_kernel(const __grid_constant__ SampleTable<G> tab) {
    const int q = job_of(tab, blockIdx.x, [](const SampleJob& j) { return (long long)j.blocks_before; });
    const SampleJob& jb = tab.job[q];
    const long long t = ((long long)blockIdx.x - jb.blocks_before) * 128 + threadIdx.x;
    if (t >= jb.c) return;
    const unsigned long long* pre = jb.G;
    const unsigned long long* tot = jb.tot;
    auto S = [&](long long j) { return pre[j] + tot[j / kScanTile]; };  // the full inclusive prefix
    long long a = 0, b = jb.len, cnt = jb.c;
    if (jb.unit == BMM_UNIT_COLUMN) {
        long long lo = 0, hi = jb.K;  // invariant: D[lo] <= t < D[hi]
        if (!(jb.D[jb.K] > t)) {
            set_status(jb.st, BMM_ERR_INFEASIBLE, 4);
            jb.idx[t] = 0; jb.scale[t] = 0.0;
            return;
        }
        while (hi - lo > 1) {
            const long long mid = (lo + hi) >> 1;
            if (jb.D[mid] <= t) lo = mid; else hi = mid;
        }
        a = jb.off[lo];
        b = jb.off[lo + 1];
        cnt = jb.ck[lo];
        if (a < 0 || b <= a || b > jb.len) {
            set_status(jb.st, BMM_ERR_SHAPE, (int)lo);
            jb.idx[t] = 0; jb.scale[t] = 0.0;
            return;
        }
    }
    const unsigned long long base = (a == 0) ? 0ull : S(a - 1);
    const unsigned long long T = S(b - 1) - base;
    if (T == 0ull) {
        set_status(jb.st, BMM_ERR_ARG, (int)(a & 0x7fffffff));
        jb.idx[t] = (int32_t)a; jb.scale[t] = 0.0;
        return;
    }
    const uint64_t r = draw_bits(jb.seed, jb.sid, (uint64_t)t);
    const unsigned long long target = __umul64hi(r, T);
    long long lo = a, hi = b - 1;  // smallest j in [a, b) with S(j) - base > target
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if (S(mid) - base > target) hi = mid; else lo = mid + 1;
    }
    jb.idx[t] = (int32_t)lo;
    jb.scale[t] = __ddiv_rn(1.0, __dmul_rn((double)cnt, jb.p[lo]));
}

}  // namespace

cudaError_t launch_sample_grouped(const SampleArgs* args, int64_t count, cudaStream_t s) {
    static thread_local SampleTable<kMaxSampleJobs> tab;  // host-side staging of the kernel parameter, one per host thread
    int64_t i = 0;
    while (i < count) {
        tab.count = 0;
        long long tiles = 0, blocks = 0;
        for (; i < count && tab.count < kMaxSampleJobs; ++i) {
            const SampleArgs& a = args[i];
            if (a.c == 0) continue;
            const int64_t len = a.unit == BMM_UNIT_COLUMN ? a.n : a.K;
            const int64_t ntiles = ceil_div(len, kScanTile);
            char* w = static_cast<char*>(a.scratch);
            SampleJob& jb = tab.job[tab.count++];
            jb.p = a.p; jb.off = a.off; jb.ck = a.ck; jb.idx = a.idx; jb.scale = a.scale;
            jb.G = reinterpret_cast<unsigned long long*>(w);
            w += round_up(len * 8, 256);
            jb.tot = reinterpret_cast<unsigned long long*>(w);
            w += round_up(ntiles * 8, 256);
            jb.D = reinterpret_cast<int64_t*>(w);
            jb.st = a.st;
            jb.K = a.K; jb.len = len; jb.c = a.c; jb.seed = a.seed; jb.sid = a.sid; jb.unit = a.unit;
            jb.tiles_before = (int)tiles;
            jb.blocks_before = (int)blocks;
            tiles += ntiles;
            blocks += ceil_div(a.c, 128);
        }
        if (tab.count == 0) continue;
        if (tiles > 0x7fffffffLL || blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
        (count_launch(), weights_scan_grouped_kernel<kMaxSampleJobs><<<(unsigned)tiles, kScanTile, 0, s>>>(tab));
        (count_launch(), prefix_grouped_kernel<kMaxSampleJobs><<<(unsigned)tab.count, kScanTile, 0, s>>>(tab));
        (count_launch(), draw_grouped_kernel<kMaxSampleJobs><<<(unsigned)blocks, 128, 0, s>>>(tab));
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int64_t sampler_scratch_bytes(int64_t len, int64_t K) {
    const int64_t ntiles = ceil_div(imax(len, 1), kScanTile);
    return round_up(len * 8, 256) + round_up(ntiles * 8, 256) + round_up((K + 1) * 8, 256);
}

cudaError_t launch_sample(const double* p, int unit, const int64_t* off, int64_t K, int64_t n, const int64_t* ck,
                          int64_t c, uint64_t seed, uint64_t sid, int32_t* idx, double* scale, void* scratch,
                          DevStatus* st, cudaStream_t s) {
    const int64_t len = (unit == BMM_UNIT_COLUMN) ? n : K;
    const int64_t ntiles = ceil_div(len, kScanTile);
    char* w = static_cast<char*>(scratch);
    unsigned long long* G = reinterpret_cast<unsigned long long*>(w);
    w += round_up(len * 8, 256);
    unsigned long long* tot = reinterpret_cast<unsigned long long*>(w);
    w += round_up(ntiles * 8, 256);
    int64_t* D = reinterpret_cast<int64_t*>(w);
    if (c == 0) return cudaSuccess;
    (count_launch(), weights_scan_kernel<<<(unsigned)ntiles, kScanTile, 0, s>>>(p, len, G, tot, st));
    if (ntiles > 1) {
        (count_launch(), tile_prefix_kernel<<<1, kScanTile, 0, s>>>(tot, ntiles));
        (count_launch(), add_tile_prefix_kernel<<<(unsigned)ceil_div(len, 256), 256, 0, s>>>(G, tot, len));
    }
    if (unit == BMM_UNIT_COLUMN) (count_launch(), draw_offsets_kernel<<<1, kScanTile, 0, s>>>(ck, K, c, D, st));
    (count_launch(), draw_kernel<<<(unsigned)ceil_div(c, 128), 128, 0, s>>>(p, unit, off, K, len, D, ck, c, seed, sid, G, idx, scale, st));
    return cudaGetLastError();
}

}  // namespace bmm
