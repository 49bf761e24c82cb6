// blockstats_tc.cu -- the statistics pass and ||M^k N_k||_F^2 in one read of M and N.
//
// f_k = ||M^k N_k||_F^2 = <G_M, G_N>_F with G_M = M^kT M^k and G_N = N_k N_kT (n_k x n_k Grams;
// eq. 1.2, eq. 3.9).  Its diagonal is s_k = sum_i x_i y_i, which this kernel accumulates exactly
// (float-float folded into FP64) together with x_i = ||M^(i)||^2 and y_i = ||N_(i)||^2; the
// off-diagonal part sum_{i != j} G_M[i,j] G_N[i,j] comes from TF32 tensor-core Grams in TMEM.
//
// One CTA per SM pulls blocks from a global counter.  For block k it streams the vectors of the
// block -- columns of M (length m), then rows of N (length p) -- in chunks of 32 coordinates:
//   warp 0      one lane: TMA loads of 32 x 32 FP32 boxes into an 8-deep ring (128-byte swizzle,
//               in 32-byte atoms for strided storage);
//   warp 1      one lane: tcgen05.mma kind::tf32 (M = 128, N = the block's operand rows rounded to
//               16, K = 8) with the same operand tile as A and B, G_M and G_N in two TMEM
//               accumulators, double buffered across blocks (512 columns).  A tile whose vectors
//               are its rows (contiguous storage) is a K-major operand, one whose vectors are its
//               columns (strided storage: row-major M, column-major N) an MN-major operand; both are
//               read where TMA put them;
//   warps 2-9   sum squares of every element they see (exact norms) and, at the end of a block,
//               fold the norms into a_k, s_k, ||M^k||_F^2, ||N_k||_F^2 and reduce the off-diagonal
//               Gram products from TMEM.
// A strided operand's first box starts at the 16-byte boundary at or below the block's first
// column (TMA needs a 16-byte-aligned inner coordinate), so its vectors are operand rows
// d .. d + n_k - 1 with d = off_k mod 4; the contiguous operand of the same block is loaded d rows
// early to match.  When d + n_k exceeds the MMA's 128 rows (n_k > 125) the strided tiles are
// transposed by warps 2-9 into a 2-deep ring of K-major tiles instead, with the block at row 0.
// Operand rows outside the block hold neighbouring data or zeros and are masked out of every
// sum.  All waits are bounded; on expiry the CTA records BMM_ERR_TIMEOUT, lets its copies and
// MMAs in flight land, frees TMEM and returns.
#include "internal.h"
#include "tc_ptx.cuh"

namespace bmm {
namespace {

using namespace ptx;

constexpr int kRawStages = 8;                    // TMA ring: covers DRAM latency
constexpr int kOpStages = 2;                     // transposed operand tiles for the MMA
constexpr int kBoxBytes = 32 * 32 * 4;           // one 32 x 32 FP32 box
constexpr int kRawBoxes = 5;                     // strided operand: 3 leading columns + 128
constexpr int kRawBytes = kRawBoxes * kBoxBytes;  // 20 KB
constexpr int kOpBytes = 4 * kBoxBytes;           // 128 vectors x 32 coordinates
constexpr int kFoldEvery = 8;                    // chunks between FP64 folds of the float-float sums
constexpr int kConvWarps = 8;
constexpr int kConvThreads = 32 * kConvWarps;
constexpr int kThreads = 64 + kConvThreads;
constexpr int kSmem = kRawStages * kRawBytes + kOpStages * kOpBytes + 1024;
constexpr uint32_t kTmemCols = 512;
constexpr int kMaxBlock = 128;

// How a stage's tile reaches the MMA.
enum TileMode : int {
    TILE_KMAJOR = 0,     // vectors are tile rows (contiguous storage): K-major operand in place
    TILE_MNMAJOR = 1,    // vectors are tile columns (strided storage): MN-major operand in place
    TILE_TRANSPOSE = 2,  // strided, but the aligned window exceeds 128 vectors: transposed copy
};

struct StageInfo {
    int block;  // -1: no more work
    int phase;  // 0: columns of M, 1: rows of N
    int nk;     // block size
    int d;      // tile row (K-major) or column (strided) of the block's first vector
    int dpos;   // operand row of the block's first vector, the same in both phases of a block
    int nb;     // boxes loaded
    int first;  // first chunk of the phase
    int last;   // last chunk of the phase
    int mode;   // TileMode
};

__device__ __forceinline__ uint32_t idesc_tf32(int npad, bool mn_major) {
    // D = F32 (bits 4-5), A = B = TF32 (2 at bits 7-9, 10-12), A and B MN-major (bits 15, 16) or
    // K-major, N>>3 at 17, M>>4 at 24
    const uint32_t major = mn_major ? (3u << 15) : 0u;
    return (1u << 4) | (2u << 7) | (2u << 10) | major | ((uint32_t)(npad >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// Byte offset of element (row h, column cc) in a 32 x 32 FP32 box of a strided operand, loaded
// with the 128-byte swizzle of 32-byte atoms: chunk cc / 8 of row h sits at chunk (cc / 8) ^ (h mod 4).
__device__ __forceinline__ int strided_offset(int h, int cc) { return h * 128 + ((((cc >> 3) ^ (h & 3)) << 5) | ((cc & 7) << 2)); }

// Barrier over the converter warps built on an mbarrier, so that its wait is bounded like every
// other wait (a bar.sync could not give up if a warp left the loop after a timeout).
__device__ __forceinline__ bool conv_sync(uint32_t bar, int& uses, volatile int* abort_flag) {
    __threadfence_block();
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(bar);
    const bool ok = mbar_wait(bar, (uint32_t)(uses & 1), abort_flag);
    ++uses;
    return ok;
}

template <bool STATS>
__global__ void __launch_bounds__(kThreads, 1)
    blockstats_tc_kernel(const __grid_constant__ CUtensorMap tmM, const __grid_constant__ CUtensorMap tmN,
                         int M_strided, int N_strided, long long m, long long p, const int64_t* __restrict__ off,
                         long long K, long long n, int* __restrict__ counter, double* __restrict__ x,
                         double* __restrict__ y, double* __restrict__ a, double* __restrict__ ssum,
                         double* __restrict__ mf, double* __restrict__ nf, double* __restrict__ f, DevStatus* st) {
    extern __shared__ uint8_t dsmem[];
    __shared__ __align__(8) uint64_t bar_full[kRawStages], bar_empty[kRawStages];
    __shared__ __align__(8) uint64_t bar_opfull[kOpStages], bar_opempty[kOpStages];
    __shared__ __align__(8) uint64_t bar_tfull[2], bar_tempty[2], bar_drain, bar_cs;
    __shared__ StageInfo info[kRawStages];
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;
    __shared__ double part[2][2][kMaxBlock];  // [phase][coordinate half][vector]
    __shared__ double red[kConvWarps][5];

    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dsmem) + 1023) & ~uintptr_t(1023));
    auto raw = [&](int s) { return base + s * kRawBytes; };
    auto opt = [&](int s) { return base + kRawStages * kRawBytes + s * kOpBytes; };
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kRawStages; ++s) {
            mbar_init(smem_u32(&bar_full[s]), 1);
            // released by the 8 converter warps plus the MMA thread: its commit when the tile is used
            // in place, a plain arrival once it has read the stage's record when the tile was
            // transposed.  The MMA thread's arrival is what keeps the producer from overwriting a
            // record (or advancing bar_full by a whole phase) before the MMA has read it.
            mbar_init(smem_u32(&bar_empty[s]), kConvWarps + 1);
        }
        for (int s = 0; s < kOpStages; ++s) {
            mbar_init(smem_u32(&bar_opfull[s]), kConvWarps);
            mbar_init(smem_u32(&bar_opempty[s]), 1);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(smem_u32(&bar_tfull[q]), 1);
            mbar_init(smem_u32(&bar_tempty[q]), kConvWarps);
        }
        mbar_init(smem_u32(&bar_drain), 1);
        mbar_init(smem_u32(&bar_cs), kConvWarps);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // operand tiles start as zeros, so rows no copy ever wrote are finite
    for (int e = threadIdx.x; e < (kRawStages * kRawBytes + kOpStages * kOpBytes) / 16; e += kThreads)
        reinterpret_cast<uint4*>(base)[e] = make_uint4(0, 0, 0, 0);
    if (warp == 1) tmem_alloc(smem_u32(&s_tmem), kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    if (warp == 0) {
        if (lane == 0) {
            // ------------------------------------------------ producer
            int stage = 0;
            uint32_t ph = 0;
            uint32_t issued_mask = 0, issued_phase = 0;
            bool aborted = false;
            while (!aborted) {
                const long long k = atomicAdd(counter, 1);
                if (k >= K) {
                    if (!mbar_wait(smem_u32(&bar_empty[stage]), ph ^ 1u, &s_abort)) { aborted = true; break; }
                    info[stage].block = -1;
                    mbar_arrive(smem_u32(&bar_full[stage]));
                    break;
                }
                const long long lo = off[k], hi = off[k + 1];
                const long long nk = hi - lo;
                if (lo < 0 || hi > n || nk <= 0 || nk > kMaxBlock) {
                    set_status(st, BMM_ERR_SHAPE, (int)k);
                    if (STATS) { a[k] = 0.0; ssum[k] = 0.0; mf[k] = 0.0; nf[k] = 0.0; }
                    f[k] = 0.0;
                    continue;
                }
                // A strided tile starts at the 16-byte boundary at or below lo, so the block's vectors
                // sit at tile columns dlo .. dlo + nk - 1.  Used in place (MN-major) they are operand
                // rows dlo.., and a contiguous tile of the same block starts dlo rows early so that
                // both Grams index a vector alike.  A window wider than the MMA's 128 rows (nk > 125)
                // sends the strided tiles through the transposed copy at operand row 0 instead.
                const int dlo = (int)(lo & 3);
                const bool any_strided = M_strided || N_strided;
                const bool wide = any_strided && dlo + nk > 128;
                const int dpos = (any_strided && !wide) ? dlo : 0;
                for (int phase = 0; phase < 2 && !aborted; ++phase) {
                    const int strided = phase == 0 ? M_strided : N_strided;
                    const long long len = phase == 0 ? m : p;
                    const long long nchunks = (len + 31) / 32;
                    const int mode = !strided ? TILE_KMAJOR : (wide ? TILE_TRANSPOSE : TILE_MNMAJOR);
                    const int d = strided ? dlo : dpos;
                    const int nb = (int)((d + nk + 31) / 32);
                    const CUtensorMap* map = phase == 0 ? &tmM : &tmN;
                    for (long long c = 0; c < nchunks; ++c) {
                        if (!mbar_wait(smem_u32(&bar_empty[stage]), ph ^ 1u, &s_abort)) { aborted = true; break; }
                        StageInfo& si = info[stage];
                        si.block = (int)k;
                        si.phase = phase;
                        si.nk = (int)nk;
                        si.d = d;
                        si.dpos = dpos;
                        si.nb = nb;
                        si.first = c == 0;
                        si.last = c == nchunks - 1;
                        si.mode = mode;
                        const uint32_t fb = smem_u32(&bar_full[stage]);
                        mbar_expect_tx(fb, (uint32_t)(nb * kBoxBytes));
                        uint8_t* dst = raw(stage);  // every tile lands in the TMA ring
                        for (int b = 0; b < nb; ++b) {
                            if (strided)
                                tma_load_2d(smem_u32(dst + b * kBoxBytes), map, fb, (int32_t)(lo - d + 32 * b),
                                            (int32_t)(32 * c));
                            else
                                tma_load_2d(smem_u32(dst + b * kBoxBytes), map, fb, (int32_t)(32 * c),
                                            (int32_t)(lo - d + 32 * b));
                        }
                        issued_mask |= 1u << stage;
                        issued_phase = (issued_phase & ~(1u << stage)) | (ph << stage);
                        if (++stage == kRawStages) { stage = 0; ph ^= 1u; }
                    }
                }
            }
            if (aborted)
                for (int s = 0; s < kRawStages; ++s)
                    if (issued_mask & (1u << s)) mbar_wait(smem_u32(&bar_full[s]), (issued_phase >> s) & 1u, nullptr);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ------------------------------------------------ MMA issuer
            int stage = 0, ostage = 0;
            uint32_t ph = 0, oph = 0;
            int it = 0, acc = 0;
            bool aborted = false;
            while (true) {
                if (!mbar_wait(smem_u32(&bar_full[stage]), ph, &s_abort)) { aborted = true; break; }
                const StageInfo si = info[stage];
                if (si.block < 0) break;
                if (si.first && si.phase == 0) {
                    acc = it & 1;
                    if (!mbar_wait(smem_u32(&bar_tempty[acc]), ((uint32_t)(it >> 1) & 1u) ^ 1u, &s_abort)) {
                        aborted = true;
                        break;
                    }
                }
                const bool transposed = si.mode == TILE_TRANSPOSE;
                uint8_t* tile = raw(stage);
                if (transposed) {
                    mbar_arrive(smem_u32(&bar_empty[stage]));  // record read; the raw tile is not used here
                    if (!mbar_wait(smem_u32(&bar_opfull[ostage]), oph, &s_abort)) { aborted = true; break; }
                    tile = opt(ostage);
                }
                tc_fence_after();
                // operand rows dpos .. dpos + nk - 1 hold the block (dpos + nk <= 128 by construction)
                const int npad = (si.dpos + si.nk + 15) & ~15;
                const uint32_t d = tmem + (uint32_t)(acc * 256 + si.phase * 128);
                const bool mn = si.mode == TILE_MNMAJOR;
                // K step of 8 TF32: 32 bytes along a K-major row, one 1024-byte row group when MN-major
                const uint64_t desc = mn ? sw128_atom32_mn_desc(smem_u32(tile), kBoxBytes) : sw128_desc(smem_u32(tile));
                const uint64_t kstep = mn ? 64ull : 2ull;
                const uint32_t idesc = idesc_tf32(npad, mn);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    tc_mma_tf32(d, desc + kstep * kk, desc + kstep * kk, idesc, (!si.first || kk > 0) ? 1u : 0u);
                if (transposed) {
                    tc_commit(smem_u32(&bar_opempty[ostage]));
                    if (++ostage == kOpStages) { ostage = 0; oph ^= 1u; }
                } else {
                    tc_commit(smem_u32(&bar_empty[stage]));
                }
                if (si.last && si.phase == 1) {
                    tc_commit(smem_u32(&bar_tfull[acc]));
                    ++it;
                }
                if (++stage == kRawStages) { stage = 0; ph ^= 1u; }
            }
            if (aborted) {
                tc_commit(smem_u32(&bar_drain));
                mbar_wait(smem_u32(&bar_drain), 0u, nullptr);
            }
        }
    } else {
        // ------------------------------------------------ norms, transpose, block epilogue
        const int t = threadIdx.x - 64;
        const int i = t & 127, hh = t >> 7;
        const int cw = warp - 2;  // converter warp 0..7
        int stage = 0, ostage = 0;
        uint32_t ph = 0, oph = 0;
        int it = 0;
        FF ff;
        ff.zero();
        double dacc = 0.0;
        int since_fold = 0;
        int cs_uses = 0;
        const uint32_t cs_bar = smem_u32(&bar_cs);
        bool aborted = false;
        while (true) {
            if (!mbar_wait(smem_u32(&bar_full[stage]), ph, &s_abort)) break;
            const StageInfo si = info[stage];
            if (si.block < 0) break;
            const bool mine = STATS && i < si.nk;
            if (si.mode == TILE_MNMAJOR) {
                // vector i is tile column d + i: sum its squares, the MMA reads the tile in place
                if (mine) {
                    const int j = i + si.d;
                    const uint8_t* src = raw(stage) + (j >> 5) * kBoxBytes;
                    const int cc = j & 31;
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int h = 16 * hh + q;
                        const float v = *reinterpret_cast<const float*>(src + strided_offset(h, cc));
                        ff.add_prod(v, v);
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&bar_empty[stage]));
            } else if (si.mode == TILE_TRANSPOSE) {
                const int j = i + si.d;  // tile column of vector i
                const uint8_t* src = raw(stage) + (j >> 5) * kBoxBytes;
                const int cc = j & 31;
                float v[16];
                if (j < 32 * si.nb) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int h = 16 * hh + q;
                        v[q] = *reinterpret_cast<const float*>(src + strided_offset(h, cc));
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 16; ++q) v[q] = 0.f;
                }
                // the raw tile is read: hand it back to the producer
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&bar_empty[stage]));
                if (mine) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) ff.add_prod(v[q], v[q]);
                }
                if (!mbar_wait(smem_u32(&bar_opempty[ostage]), oph ^ 1u, &s_abort)) { aborted = true; break; }
                uint8_t* dst = opt(ostage) + i * 128;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int chunk = (4 * hh + q) ^ (i & 7);
                    *reinterpret_cast<float4*>(dst + chunk * 16) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                }
                fence_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&bar_opfull[ostage]));
                if (++ostage == kOpStages) { ostage = 0; oph ^= 1u; }
            } else {
                if (mine) {
                    const int r = i + si.d;  // tile row of vector i
                    const uint8_t* row = raw(stage) + r * 128;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 w4 = *reinterpret_cast<const float4*>(row + (((4 * hh + q) ^ (r & 7)) << 4));
                        ff.add_prod(w4.x, w4.x);
                        ff.add_prod(w4.y, w4.y);
                        ff.add_prod(w4.z, w4.z);
                        ff.add_prod(w4.w, w4.w);
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&bar_empty[stage]));
            }
            ff.renorm();
            if (++since_fold == kFoldEvery) {
                dacc += ff.value();
                ff.zero();
                since_fold = 0;
            }
            if (si.last) {
                dacc += ff.value();
                ff.zero();
                since_fold = 0;
                if (STATS) part[si.phase][hh][i] = dacc;
                dacc = 0.0;
            }
            if (++stage == kRawStages) { stage = 0; ph ^= 1u; }
            if (!(si.last && si.phase == 1)) continue;

            // ---- block epilogue
            const long long k = si.block, nk = si.nk;
            const int dpos = si.dpos;
            const long long lo = off[k];
            conv_sync(cs_bar, cs_uses, &s_abort);
            double sa = 0.0, ss = 0.0, sx = 0.0, sy = 0.0;
            if (STATS && t < 128 && i < nk) {
                const double xi = part[0][0][i] + part[0][1][i];
                const double yi = part[1][0][i] + part[1][1][i];
                x[lo + i] = xi;
                y[lo + i] = yi;
                const double xy = __dmul_rn(xi, yi);
                sa = sqrt(xy);
                ss = xy;
                sx = xi;
                sy = yi;
            }
            // off-diagonal Gram products from TMEM (rows = lanes of this warp's quadrant)
            const int acc = it & 1;
            FF offf;
            offf.zero();
            if (mbar_wait(smem_u32(&bar_tfull[acc]), (uint32_t)(it >> 1) & 1u, &s_abort)) {
                tc_fence_after();
                const int q4 = warp & 3, half = cw >> 2;
                const int r = 32 * q4 + lane - dpos;  // vector of this TMEM lane
#pragma unroll 1
                for (int u = 0; u < 2; ++u) {
                    const int c0 = 64 * half + 32 * u;
                    uint32_t gm[32], gn[32];
                    const uint32_t taddr = tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)(acc * 256 + c0);
                    TMEM_LD_32X32B_X32(taddr, gm);
                    TMEM_LD_32X32B_X32(taddr + 128, gn);
                    tmem_ld_wait();
                    if (r >= 0 && r < nk) {
#pragma unroll
                        for (int e = 0; e < 32; ++e) {
                            const int jj = c0 + e - dpos;
                            if (jj >= 0 && jj < nk && jj != r)
                                offf.add_prod(__uint_as_float(gm[e]), __uint_as_float(gn[e]));
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&bar_tempty[acc]));
            }
            ++it;
            double offd = offf.value();
            sa = warp_sum(sa);
            ss = warp_sum(ss);
            sx = warp_sum(sx);
            sy = warp_sum(sy);
            offd = warp_sum(offd);
            if (lane == 0) {
                red[cw][0] = sa; red[cw][1] = ss; red[cw][2] = sx; red[cw][3] = sy; red[cw][4] = offd;
            }
            conv_sync(cs_bar, cs_uses, &s_abort);
            if (t == 0) {
                double r5[5] = {0, 0, 0, 0, 0};
                for (int w = 0; w < kConvWarps; ++w)
                    for (int q = 0; q < 5; ++q) r5[q] += red[w][q];
                const double sk = STATS ? r5[1] : ssum[k];
                if (STATS) { a[k] = r5[0]; ssum[k] = r5[1]; mf[k] = r5[2]; nf[k] = r5[3]; }
                f[k] = sk + r5[4];
            }
            conv_sync(cs_bar, cs_uses, &s_abort);  // part[] and red[] are reused by the next block
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
    if (threadIdx.x == 0 && s_abort) set_status(st, BMM_ERR_TIMEOUT, 2);
}

// Strided operands (vectors along the storage rows' inner dimension) feed the MMA MN-major, which
// for TF32 wants 32-byte swizzle atoms; contiguous ones are K-major with the plain 128-byte swizzle.
bool make_map_f32(CUtensorMap* mp, const void* ptr, int64_t rows, int64_t cols, int64_t ld, bool strided) {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (fn == nullptr) {
        void* q = nullptr;
        cudaDriverEntryPointQueryResult r;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &q, 12000, cudaEnableDefault, &r) != cudaSuccess ||
            r != cudaDriverEntryPointSuccess)
            return false;
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(q);
    }
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * 4)};
    cuuint32_t box[2] = {32, 32};
    cuuint32_t es[2] = {1, 1};
    return fn(mp, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(ptr), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, strided ? CU_TENSOR_MAP_SWIZZLE_128B_ATOM_32B : CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool blockstats_tc_supported(const VecSet& vM, const VecSet& vN, int64_t max_nk) {
    if (vM.dtype != BMM_F32 || vN.dtype != BMM_F32 || max_nk > kMaxBlock) return false;
    if (vM.len < 1 || vN.len < 1) return false;  // every block needs chunks in both phases
    if ((vM.ld % 4) || (vN.ld % 4)) return false;
    if ((reinterpret_cast<uintptr_t>(vM.data) & 15) || (reinterpret_cast<uintptr_t>(vN.data) & 15)) return false;
    if (vM.len > 0x7fffffffLL || vN.len > 0x7fffffffLL || vM.count > 0x7fffffffLL) return false;
    return tc_gemm_supported();
}

cudaError_t launch_blockstats_tc(const VecSet& vM, const VecSet& vN, const int64_t* off, int64_t K, int64_t n,
                                 bool stats, int* counter, double* x, double* y, double* a, double* ssum, double* mf,
                                 double* nf, double* f, DevStatus* st, cudaStream_t s) {
    // storage of each operand: rows x cols with stride ld (vectors are columns when strided)
    CUtensorMap mM, mN;
    const int64_t mrows = vM.mode == VEC_STRIDED ? vM.len : vM.count;
    const int64_t mcols = vM.mode == VEC_STRIDED ? vM.count : vM.len;
    const int64_t nrows = vN.mode == VEC_STRIDED ? vN.len : vN.count;
    const int64_t ncols = vN.mode == VEC_STRIDED ? vN.count : vN.len;
    if (!make_map_f32(&mM, vM.data, mrows, mcols, vM.ld, vM.mode == VEC_STRIDED) ||
        !make_map_f32(&mN, vN.data, nrows, ncols, vN.ld, vN.mode == VEC_STRIDED))
        return cudaErrorInvalidValue;
    static bool attr[2] = {false, false};
    if (!attr[stats]) {
        cudaError_t e = stats ? cudaFuncSetAttribute(blockstats_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem)
                              : cudaFuncSetAttribute(blockstats_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
        if (e != cudaSuccess) return e;
        attr[stats] = true;
    }
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = (int)imin(K, sms);
    if (stats)
        (count_launch(), blockstats_tc_kernel<true><<<grid, kThreads, kSmem, s>>>(
            mM, mN, vM.mode == VEC_STRIDED, vN.mode == VEC_STRIDED, vM.len, vN.len, off, K, n, counter, x, y, a, ssum,
            mf, nf, f, st));
    else
        (count_launch(), blockstats_tc_kernel<false><<<grid, kThreads, kSmem, s>>>(
            mM, mN, vM.mode == VEC_STRIDED, vN.mode == VEC_STRIDED, vM.len, vN.len, off, K, n, counter, x, y, a, ssum,
            mf, nf, f, st));
    return cudaGetLastError();
}

}  // namespace bmm
