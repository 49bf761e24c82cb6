// gemm_tc.cu -- the sampled product CD = C D on the sm_103a tensor cores (Alg. 2 step 4, eq. 3.3).
//
// out[M x N] (+)= scale * A[M x K] * B[N x K]^T with A, B K-major (rows of length K), BF16 or FP8
// e4m3 (scale = 1 for BF16, a device FP32 factor for FP8, whose operands carry power-of-two scales).
// Persistent kernel, one CTA per SM, 192 threads:
//   warp 0   one lane issues TMA loads of 128-row (A) and BN-row (B) tiles of 128 bytes of K
//            (64 BF16 or 128 e4m3), 128-byte swizzled, into a ring of shared-memory stages;
//   warp 1   allocates 2*BN TMEM columns; one lane issues tcgen05.mma (kind::f16, K = 16, or
//            kind::f8f6f4, K = 32; M=128, N=BN) into one of two TMEM accumulators and commits stages
//            back;
//   warps 2-5 drain the other accumulator with tcgen05.ld (one TMEM lane quadrant per warp),
//            overlapping the next tile's MMAs: each warp stages 32 x 32 FP32 blocks in shared
//            memory (two 4 KB buffers, 128-byte swizzled) and writes them with TMA tile stores, or
//            TMA reduce-adds when accumulating (the same FP32 old + new as a load-add-store); an
//            output whose base or row stride is not 16-byte aligned is written with plain stores.
// CTA-pair form (PAIR, tile choice bn = 512): clusters of two CTAs on two SMs compute 256 x 256
// tiles with cta_group::2 MMAs (M = 256, N = 256).  Each CTA loads its own 128 rows of A and 128 of
// the tile's 256 rows of B per stage (32 KB instead of the single-CTA 48 KB for 128 x 256), both
// copies completing on the even CTA's stage barrier; that CTA's MMA lane issues for the pair and
// multicasts its commits to both CTAs' stage and accumulator barriers; each CTA's epilogue drains
// its own 128 rows and releases the accumulator on the even CTA's barrier.  Per SM the shared-memory
// traffic of one 64-deep BF16 stage drops from 96 KB (copy writes and MMA operand reads) to about
// 80 KB for the same 128 x 256 x 64 of math, and the L2 traffic per tile element halves.
// Every wait is bounded (globaltimer); on expiry the CTA records BMM_ERR_TIMEOUT, lets its
// copies and MMAs in flight finish (again bounded), frees TMEM and returns.
#include <map>
#include <mutex>
#include <vector>

#include "internal.h"
#include "tc_ptx.cuh"

namespace bmm {
namespace {

using namespace ptx;
constexpr int BM = 128;
constexpr int ROW_BYTES = 128;  // K per stage: one 128-byte swizzled row
constexpr int kMnBoxBytes = 64 * ROW_BYTES;  // an MN-major B box: 64 N x 64 K rows of 128 bytes

// EK: element kind, 0 = BF16 (kind::f16), 1 = FP8 e4m3 (kind::f8f6f4).  PAIR: CTA-pair tiles of
// TILE_M = 256 output rows (128 per CTA) by BN = 256 or 512 columns, B_ROWS = BN / 2 rows of B per
// CTA; each K step is BN / 256 pair MMAs of N = 256.  The 256 x 512 tile keeps one 512-column
// accumulator (its epilogue does not overlap the next tile's MMAs) and needs 47 B of copies per
// cycle per SM at the math rate against the 256 x 256 tile's 64.
template <int BN, int EK, bool PAIR = false> struct Cfg {
    static_assert(!PAIR || BN == 256 || BN == 512, "CTA-pair tiles are 256 x 256 or 256 x 512");
    static constexpr int ESIZE = EK ? 1 : 2;
    static constexpr int BK = ROW_BYTES / ESIZE;       // elements of K per stage
    static constexpr int KMMA = 32 / ESIZE;            // elements of K per MMA (32 bytes)
    static constexpr int TILE_M = PAIR ? 2 * BM : BM;
    static constexpr int B_ROWS = PAIR ? BN / 2 : BN;
    static constexpr int NMMA = PAIR ? BN / 256 : 1;  // MMAs per K step
    static constexpr int MMA_N = PAIR ? 256 : BN;
    static constexpr int ACCS = (PAIR && BN == 512) ? 1 : 2;  // accumulators in TMEM
    static constexpr int STAGES = PAIR ? (BN == 512 ? 4 : 6) : ((BN == 256) ? 4 : 6);
    static constexpr int A_BYTES = BM * ROW_BYTES;
    static constexpr int B_BYTES = B_ROWS * ROW_BYTES;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr uint32_t STAGE_TX = (PAIR ? 2u : 1u) * (uint32_t)STAGE_BYTES;  // bytes a full barrier awaits
    static constexpr int TMEM_COLS = ACCS * BN;
    static constexpr int EPI_BYTES = 4 * 2 * 32 * 32 * 4;  // 4 epilogue warps x 2 buffers x 32 x 32 FP32
    static constexpr int SMEM = STAGES * STAGE_BYTES + EPI_BYTES + 1024;
    // instruction descriptor: D=F32 (bits 4-5); A, B format (bits 7-9, 10-12): BF16 = 1 for
    // kind::f16, E4M3 = 0 for kind::f8f6f4; both K-major, N>>3 at bits 17-22, M>>4 at bits 24-28
    static constexpr uint32_t FMT = EK ? 0u : 1u;
    static constexpr uint32_t IDESC = (1u << 4) | (FMT << 7) | (FMT << 10) | ((uint32_t)(MMA_N >> 3) << 17) |
                                      ((uint32_t)(TILE_M >> 4) << 24);
};

// G M-tiles per raster group (4, 8 or 16, chosen per product by the autotuner), so that concurrent
// CTAs share A and B panels in L2
__device__ __forceinline__ void tile_coords(int tile, int tiles_m, int tiles_n, int G, int* tm, int* tn) {
    const int span = G * tiles_n;
    const int group = tile / span;
    const int first = group * G;
    const int gm = min(tiles_m - first, G);
    const int r = tile - group * span;
    *tm = first + r % gm;
    *tn = r / gm;
}

// One product of a (possibly grouped) launch.  The table travels as a __grid_constant__ kernel
// parameter, so the tensor maps are used in place and the whole launch can sit in a CUDA graph.
struct GemmProblem {
    CUtensorMap mapA;
    CUtensorMap mapB;
    CUtensorMap mapO;  // FP32 output, 32 x 32 boxes, 128-byte swizzle (valid when tma_out)
    float* out;
    long long ldo;
    const long long* k_dev;
    long long k_host;
    int M, N;
    int tiles_m, tiles_n;
    int tile_begin;
    int k_mult;
    int accumulate;
    int vec_ok;
    int tma_out;
    int raster;
    const float* scale;  // device factor applied to the product (FP8), or null
    int b_mn;            // B is MN-major (BF16 only): rows of K, N contiguous; boxes of 64 N x 64 K
};
template <int G> struct GemmTable {
    int count;
    int total_tiles;
    GemmProblem prob[G];
};
constexpr int kMaxGroup = 60;  // 60 x 512-byte entries keep the table under the 32 KB kernel-parameter limit
static_assert(sizeof(GemmTable<kMaxGroup>) <= 32764, "GEMM table exceeds the kernel-parameter limit");

template <int G>
__device__ __forceinline__ int find_problem(const GemmTable<G>& tab, int tile) {
    int pi = 0;
    while (pi + 1 < tab.count && tile >= tab.prob[pi + 1].tile_begin) ++pi;
    return pi;
}

// K blocks of one product: with a device extent, each of the k_mult segments is padded to BK, and
// k_host (when positive) caps the depth at the operands' capacity
template <int BK>
__device__ __forceinline__ int problem_kb(const GemmProblem& pr) {
    long long K = pr.k_host;
    if (pr.k_dev) {
        const long long e = *pr.k_dev;
        K = (long long)pr.k_mult * ((((e > 0 ? e : 0) + BK - 1) / BK) * BK);
        if (pr.k_host > 0 && K > pr.k_host) K = pr.k_host;
    }
    return (int)(K / BK);
}

// A bounded wait whose first poll is inline: on the issue path of the single MMA thread a call to
// the out-of-line wait for a phase that is already complete costs about 4% of the GEMM's time.
__device__ __forceinline__ bool wait_fast(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
    return mbar_try_wait(bar, parity) || mbar_wait(bar, parity, abort_flag);
}

__device__ __forceinline__ int ld_cluster_s32(uint32_t cluster_addr) {
    int v;
    asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(cluster_addr) : "memory");
    return v;
}

// The MMAs of one stage (BK elements of K in KMMA steps).  A is K-major (32 bytes per step); B is
// K-major (32 bytes per step) or, with BMN, MN-major (16 rows of 128 bytes per step, the transpose-B
// bit set).  In PAIR form MMA h takes B rows (or columns) 128 h .. 128 h + 127 of each CTA -- 16 KB
// into the stage either way -- into accumulator columns 256 h ...
template <class C, int EK, bool PAIR, bool BMN>
__device__ __forceinline__ void mma_stage(uint32_t d, uint64_t ad, uint64_t bd, bool accumulate) {
    constexpr uint32_t idesc = C::IDESC | (BMN ? (1u << 16) : 0u);
    constexpr uint64_t bstep = BMN ? (uint64_t)((16 * ROW_BYTES) >> 4) : 2ull;
#pragma unroll
    for (int k = 0; k < C::BK / C::KMMA; ++k) {
        const uint32_t acc_in = (accumulate || k > 0) ? 1u : 0u;
        if constexpr (PAIR) {
#pragma unroll
            for (int h = 0; h < C::NMMA; ++h) {
                const uint32_t dh = d + (uint32_t)(256 * h);
                const uint64_t bh = bd + (uint64_t)((h * 128 * ROW_BYTES) >> 4) + bstep * k;
                if (EK)
                    tc_mma_f8_pair(dh, ad + 2ull * k, bh, idesc, acc_in);
                else
                    tc_mma_bf16_pair(dh, ad + 2ull * k, bh, idesc, acc_in);
            }
        } else {
            if (EK)
                tc_mma_f8(d, ad + 2ull * k, bd + bstep * k, idesc, acc_in);
            else
                tc_mma_bf16(d, ad + 2ull * k, bd + bstep * k, idesc, acc_in);
        }
    }
}

template <int BN, int G, int EK, bool PAIR>
__global__ void __launch_bounds__(192, 1) gemm_bf16_tc_kernel(const __grid_constant__ GemmTable<G> tab, DevStatus* st) {
    using C = Cfg<BN, EK, PAIR>;
    constexpr int BK = C::BK;
    extern __shared__ uint8_t dsmem[];
    __shared__ __align__(8) uint64_t bar_full[C::STAGES];
    __shared__ __align__(8) uint64_t bar_empty[C::STAGES];
    __shared__ __align__(8) uint64_t bar_tfull[2];
    __shared__ __align__(8) uint64_t bar_tempty[2];
    __shared__ __align__(8) uint64_t bar_drain;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;

    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dsmem) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = base;
    uint8_t* sB = base + C::STAGES * C::A_BYTES;
    uint8_t* sE = sB + C::STAGES * C::B_BYTES;  // epilogue staging, 1024-byte aligned
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int num_tiles = tab.total_tiles;
    // tiles are dealt to CTAs, or in PAIR form to CTA pairs (clusters), round-robin
    const uint32_t rank = PAIR ? cluster_rank() : 0u;
    const bool leader = rank == 0;
    const int first_tile = PAIR ? (int)cluster_id() : (int)blockIdx.x;
    const int tile_step = PAIR ? (int)cluster_count() : (int)gridDim.x;

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; ++s) {
            mbar_init(smem_u32(&bar_full[s]), 1);
            mbar_init(smem_u32(&bar_empty[s]), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(smem_u32(&bar_tfull[a]), 1);
            mbar_init(smem_u32(&bar_tempty[a]), PAIR ? 8 : 4);  // the epilogue warps of the CTA (pair)
        }
        mbar_init(smem_u32(&bar_drain), 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        if constexpr (PAIR)
            tmem_alloc_pair(smem_u32(&s_tmem), (uint32_t)C::TMEM_COLS);
        else
            tmem_alloc(smem_u32(&s_tmem), (uint32_t)C::TMEM_COLS);
    }
    tc_fence_before();
    if constexpr (PAIR)
        cluster_sync();  // the peer's barriers are initialised before any copy or arrive targets them
    else
        __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    if (warp == 0 && lane == 0) {
        // ------------------------------------------------ TMA producer
        int stage = 0;
        uint32_t phase = 0;
        uint32_t issued_mask = 0, issued_phase = 0;
        bool aborted = false;
        for (int tile = first_tile; tile < num_tiles && !aborted; tile += tile_step) {
            const GemmProblem& pr = tab.prob[find_problem(tab, tile)];
            int tm, tn;
            tile_coords(tile - pr.tile_begin, pr.tiles_m, pr.tiles_n, pr.raster, &tm, &tn);
            const int num_kb = problem_kb<BK>(pr);
            for (int kb = 0; kb < num_kb; ++kb) {
                if (!wait_fast(smem_u32(&bar_empty[stage]), phase ^ 1u, &s_abort)) {
                    aborted = true;
                    break;
                }
                const uint32_t fb = smem_u32(&bar_full[stage]);
                if constexpr (PAIR) {
                    // both CTAs' copies complete on the even CTA's barrier, which awaits all 64 KB;
                    // a peer copy may land before that CTA's expect_tx (the phase cannot complete
                    // while its one arrival is pending)
                    const uint32_t fb0 = smem_peer(fb, 0);
                    if (leader) mbar_expect_tx(fb, C::STAGE_TX);
                    tma_load_2d_pair(smem_u32(sA + stage * C::A_BYTES), &pr.mapA, fb0, kb * BK,
                                     tm * C::TILE_M + BM * (int)rank);
                    if (!EK && pr.b_mn) {
                        for (int j = 0; j < C::B_ROWS / 64; ++j)
                            tma_load_2d_pair(smem_u32(sB + stage * C::B_BYTES + j * kMnBoxBytes), &pr.mapB, fb0,
                                             tn * BN + C::B_ROWS * (int)rank + 64 * j, kb * BK);
                    } else {
                        tma_load_2d_pair(smem_u32(sB + stage * C::B_BYTES), &pr.mapB, fb0, kb * BK,
                                         tn * BN + C::B_ROWS * (int)rank);
                    }
                } else {
                    mbar_expect_tx(fb, C::STAGE_TX);
                    tma_load_2d(smem_u32(sA + stage * C::A_BYTES), &pr.mapA, fb, kb * BK, tm * BM);
                    if (!EK && pr.b_mn) {
                        for (int j = 0; j < C::B_ROWS / 64; ++j)
                            tma_load_2d(smem_u32(sB + stage * C::B_BYTES + j * kMnBoxBytes), &pr.mapB, fb,
                                        tn * BN + 64 * j, kb * BK);
                    } else {
                        tma_load_2d(smem_u32(sB + stage * C::B_BYTES), &pr.mapB, fb, kb * BK, tn * BN);
                    }
                }
                issued_mask |= 1u << stage;
                issued_phase = (issued_phase & ~(1u << stage)) | (phase << stage);
                if (++stage == C::STAGES) {
                    stage = 0;
                    phase ^= 1u;
                }
            }
        }
        // let the copies in flight land before the CTA's shared memory goes away (in PAIR form
        // the peer's bytes count on the even CTA's barriers: both CTAs wait out a grace period
        // at the end instead)
        if (aborted && !PAIR) {
            for (int s = 0; s < C::STAGES; ++s)
                if (issued_mask & (1u << s)) mbar_wait(smem_u32(&bar_full[s]), (issued_phase >> s) & 1u, nullptr);
        }
    } else if (warp == 1 && lane == 0 && leader) {
        // ------------------------------------------------ MMA issuer (the even CTA of a pair)
        int stage = 0;
        uint32_t phase = 0;
        int it = 0;
        bool aborted = false;
        for (int tile = first_tile; tile < num_tiles && !aborted; tile += tile_step, ++it) {
            const GemmProblem& pr = tab.prob[find_problem(tab, tile)];
            const int num_kb = problem_kb<BK>(pr);
            const bool bmn = !EK && pr.b_mn;  // B MN-major (BF16 only)
            const int acc = C::ACCS == 2 ? (it & 1) : 0;
            const uint32_t aph = C::ACCS == 2 ? (uint32_t)((it >> 1) & 1) : (uint32_t)(it & 1);
            if (!wait_fast(smem_u32(&bar_tempty[acc]), aph ^ 1u, &s_abort)) {
                aborted = true;
                break;
            }
            tc_fence_after();
            const uint32_t d = tmem + (uint32_t)(acc * BN);
            for (int kb = 0; kb < num_kb; ++kb) {
                if (!wait_fast(smem_u32(&bar_full[stage]), phase, &s_abort)) {
                    aborted = true;
                    break;
                }
                tc_fence_after();
                const uint64_t ad = sw128_desc(smem_u32(sA + stage * C::A_BYTES));
                const uint32_t baddr = smem_u32(sB + stage * C::B_BYTES);
                // one branch per stage; each form issues with compile-time descriptor steps
                if (bmn)
                    mma_stage<C, EK, PAIR, true>(d, ad, sw128_mn_desc(baddr, kMnBoxBytes), kb > 0);
                else
                    mma_stage<C, EK, PAIR, false>(d, ad, sw128_desc(baddr), kb > 0);
                if constexpr (PAIR)
                    tc_commit_pair_mc(smem_u32(&bar_empty[stage]), (uint16_t)3);
                else
                    tc_commit(smem_u32(&bar_empty[stage]));
                if (++stage == C::STAGES) {
                    stage = 0;
                    phase ^= 1u;
                }
            }
            if (aborted) break;
            if constexpr (PAIR)
                tc_commit_pair_mc(smem_u32(&bar_tfull[acc]), (uint16_t)3);
            else
                tc_commit(smem_u32(&bar_tfull[acc]));
        }
        if (aborted) {  // wait for the MMAs already issued before TMEM is freed
            if constexpr (PAIR)
                tc_commit_pair_mc(smem_u32(&bar_drain), (uint16_t)1);
            else
                tc_commit(smem_u32(&bar_drain));
            mbar_wait(smem_u32(&bar_drain), 0u, nullptr);
        }
    } else if (warp >= 2) {
        // ------------------------------------------------ epilogue
        const int q = warp & 3;
        int it = 0;
        int nchunk = 0;  // staged chunks so far: selects the buffer
        for (int tile = first_tile; tile < num_tiles; tile += tile_step, ++it) {
            const GemmProblem& pr = tab.prob[find_problem(tab, tile)];
            const int num_kb = problem_kb<BK>(pr);
            const int acc = C::ACCS == 2 ? (it & 1) : 0;
            const uint32_t aph = C::ACCS == 2 ? (uint32_t)((it >> 1) & 1) : (uint32_t)(it & 1);
            if (!mbar_wait(smem_u32(&bar_tfull[acc]), aph, &s_abort)) break;
            tc_fence_after();
            int tm, tn;
            tile_coords(tile - pr.tile_begin, pr.tiles_m, pr.tiles_n, pr.raster, &tm, &tn);
            const int row = tm * C::TILE_M + BM * (int)rank + q * 32 + lane;
            const int M = pr.M, N = pr.N;
            const float sc = pr.scale != nullptr ? *pr.scale : 1.0f;
#pragma unroll 1
            for (int cc = 0; cc < BN / 32; ++cc) {
                uint32_t r[32];
                const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * BN + cc * 32);
                TMEM_LD_32X32B_X32(taddr, r);
                tmem_ld_wait();
                if (num_kb == 0) {
#pragma unroll
                    for (int e = 0; e < 32; ++e) r[e] = 0u;
                }
                if (EK) {
#pragma unroll
                    for (int e = 0; e < 32; ++e) r[e] = __float_as_uint(__uint_as_float(r[e]) * sc);
                }
                // accumulator column c: MMA h = c / 256; its columns w = c mod 256 below 128 are the
                // even CTA's B rows 128 h + w, the others the odd CTA's, which holds tile columns
                // B_ROWS .. 2 B_ROWS - 1
                int tcol = cc * 32;
                if constexpr (PAIR) {
                    const int h = tcol / 256, w = tcol % 256;
                    tcol = w < 128 ? 128 * h + w : C::B_ROWS + 128 * h + (w - 128);
                }
                const int col0 = tn * BN + tcol;
                if (pr.tma_out) {
                    // this warp's 32 rows x 32 columns: row = lane, 16-byte chunk c of the row at
                    // chunk c ^ (row mod 8) of its 128 bytes (the 128-byte swizzle the map expects).
                    // A block wholly past the matrix is neither staged nor stored, so that every
                    // staged block is one bulk group and the wait below covers the store that last
                    // read this buffer (the map clips rows >= M and columns >= N of the others).
                    const int row0 = row - lane;
                    if (row0 < M && col0 < N) {  // the same for every lane of the warp
                        uint8_t* buf = sE + (q * 2 + (nchunk & 1)) * 4096;
                        if (lane == 0) bulk_wait_read<1>();  // the store issued from this buffer before has read it
                        __syncwarp();
#pragma unroll
                        for (int c = 0; c < 8; ++c)
                            *reinterpret_cast<float4*>(buf + lane * 128 + ((c ^ (lane & 7)) << 4)) =
                                make_float4(__uint_as_float(r[4 * c]), __uint_as_float(r[4 * c + 1]),
                                            __uint_as_float(r[4 * c + 2]), __uint_as_float(r[4 * c + 3]));
                        fence_async_smem();
                        __syncwarp();
                        if (lane == 0) {
                            if (pr.accumulate)
                                tma_reduce_add_2d(&pr.mapO, smem_u32(buf), col0, row0);
                            else
                                tma_store_2d(&pr.mapO, smem_u32(buf), col0, row0);
                            bulk_commit();
                        }
                        ++nchunk;
                    }
                } else if (row < M && col0 < N) {
                    float* o = pr.out + (long long)row * pr.ldo + col0;
                    if (pr.vec_ok && col0 + 32 <= N) {
#pragma unroll
                        for (int v = 0; v < 8; ++v) {
                            float4 val = make_float4(__uint_as_float(r[4 * v]), __uint_as_float(r[4 * v + 1]),
                                                     __uint_as_float(r[4 * v + 2]), __uint_as_float(r[4 * v + 3]));
                            if (pr.accumulate) {
                                const float4 old = *reinterpret_cast<const float4*>(o + 4 * v);
                                val.x += old.x; val.y += old.y; val.z += old.z; val.w += old.w;
                            }
                            *reinterpret_cast<float4*>(o + 4 * v) = val;
                        }
                    } else {
                        const int ne = min(32, N - col0);
#pragma unroll
                        for (int e = 0; e < 32; ++e)  // unrolled: r[] stays in registers
                            if (e < ne) o[e] = (pr.accumulate ? o[e] : 0.0f) + __uint_as_float(r[e]);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                if constexpr (PAIR)
                    mbar_arrive_cluster(smem_peer(smem_u32(&bar_tempty[acc]), 0));
                else
                    mbar_arrive(smem_u32(&bar_tempty[acc]));
            }
        }
        if (lane == 0) bulk_wait<0>();  // the output is written and the staging buffers are read
    }

    tc_fence_before();
    if constexpr (PAIR) {
        // all roles of both CTAs are done (every wait above is bounded); if either CTA gave up,
        // copies it or its peer issued may still be landing: wait 1 ms before shared memory goes away
        cluster_sync();
        const int any_abort = s_abort | ld_cluster_s32(smem_peer(smem_u32((const void*)&s_abort), rank ^ 1u));
        cluster_sync();
        if (any_abort) {
            const uint64_t t0 = globaltimer();
            while (globaltimer() - t0 < 1000000ull) {
            }
        }
    } else {
        __syncthreads();
    }
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        if constexpr (PAIR)
            tmem_dealloc_pair(tmem, (uint32_t)C::TMEM_COLS);
        else
            tmem_dealloc(tmem, (uint32_t)C::TMEM_COLS);
    }
    if (threadIdx.x == 0 && s_abort) set_status(st, BMM_ERR_TIMEOUT, 1);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    // looked up once; a function-local static is initialised once even under concurrent callers
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        return nullptr;
    }();
    return fn;
}

// esize: bytes per element (2 = BF16, 1 = e4m3 bytes); a box is 128 bytes of K by box_rows rows
bool make_map(CUtensorMap* m, const void* ptr, int64_t rows, int64_t kdim, int64_t ld, int box_rows, int esize) {
    auto fn = encode_fn();
    if (fn == nullptr) return false;
    cuuint64_t dims[2] = {(cuuint64_t)kdim, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * esize)};
    cuuint32_t box[2] = {(cuuint32_t)(ROW_BYTES / esize), (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(m, esize == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 2,
                    const_cast<void*>(ptr), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// FP32 output of M rows and N columns (row stride ldo elements): 32 x 32 boxes (128 bytes by 32 rows),
// 128-byte swizzle, for the epilogue's TMA stores
bool make_out_map(CUtensorMap* m, float* out, int64_t M, int64_t N, int64_t ldo) {
    auto fn = encode_fn();
    if (fn == nullptr) return false;
    cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)M};
    cuuint64_t strides[1] = {(cuuint64_t)(ldo * 4)};
    cuuint32_t box[2] = {32, 32};
    cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, out, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// MN-major BF16 B: a row-major K x N matrix (row stride ld elements), boxes of 64 N (128 bytes) by
// 64 K rows, 128-byte swizzle (the canonical MN-major layout: 8-row atoms of 1024 bytes)
bool make_map_mn(CUtensorMap* m, const void* ptr, int64_t N, int64_t kdim, int64_t ld) {
    auto fn = encode_fn();
    if (fn == nullptr) return false;
    cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)kdim};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
    cuuint32_t box[2] = {64, 64};
    cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int num_sms() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

// Fill one table entry for tile choice bn (128 or 256: one CTA, 128 x bn tiles; kPairTile: a CTA
// pair, 256 x 256 tiles with 128-row boxes of A and B per CTA); returns false when a tensor map
// cannot be made.
bool fill_problem(GemmProblem* pr, int bn, int raster, const void* A, int64_t lda, const void* B, int64_t ldb,
                  int64_t M, int64_t N, int64_t kdim, int64_t k_host, const int64_t* k_dev, int k_mult, float* out,
                  int64_t ldo, int accumulate, int elem, const float* scale, bool b_mn = false) {
    const int esize = elem == GEMM_ELEM_E4M3 ? 1 : 2;
    const bool pair = bn == kPairTile || bn == kPairTileWide;
    const int tile_m = pair ? 2 * BM : BM, tile_n = bn == kPairTileWide ? 512 : (pair ? 256 : bn);
    const int b_rows = pair ? tile_n / 2 : bn;
    if (b_mn && elem != GEMM_ELEM_BF16) return false;
    if (!make_map(&pr->mapA, A, M, kdim, lda, BM, esize) ||
        !(b_mn ? make_map_mn(&pr->mapB, B, N, kdim, ldb) : make_map(&pr->mapB, B, N, kdim, ldb, b_rows, esize)))
        return false;
    pr->b_mn = b_mn ? 1 : 0;
    pr->scale = scale;
    pr->out = out;
    pr->ldo = ldo;
    pr->k_dev = reinterpret_cast<const long long*>(k_dev);
    pr->k_host = k_host;
    pr->M = (int)M;
    pr->N = (int)N;
    pr->tiles_m = (int)ceil_div(M, tile_m);
    pr->tiles_n = (int)ceil_div(N, tile_n);
    pr->k_mult = k_mult;
    pr->accumulate = accumulate;
    pr->vec_ok = ((reinterpret_cast<uintptr_t>(out) & 15) == 0) && (ldo % 4 == 0);
    pr->tma_out = pr->vec_ok && make_out_map(&pr->mapO, out, M, N, ldo) ? 1 : 0;
    pr->raster = raster;
    return true;
}

template <int BN, int G, int EK, bool PAIR>
cudaError_t launch_table(const GemmTable<G>& tab, DevStatus* st, cudaStream_t s) {
    using C = Cfg<BN, EK, PAIR>;
    auto kern = gemm_bf16_tc_kernel<BN, G, EK, PAIR>;
    static std::atomic<int> units{0};  // CTAs, or CTA pairs, that are resident at once (set once)
    if (units.load() == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
        if (e != cudaSuccess) return e;
        int n = num_sms();
        if (PAIR) {
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = 2;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.gridDim = dim3((unsigned)(n & ~1));
            cfg.blockDim = dim3(192);
            cfg.dynamicSmemBytes = C::SMEM;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int clusters = 0;
            e = cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg);
            if (e != cudaSuccess) return e;
            n = clusters > 0 ? clusters : 1;
        }
        units.store(n);
    }
    if (tab.total_tiles == 0) return cudaSuccess;
    const int grid = (int)imin(tab.total_tiles, (int64_t)units.load());
    count_launch();
    if constexpr (PAIR) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)(2 * grid));
        cfg.blockDim = dim3(192);
        cfg.dynamicSmemBytes = C::SMEM;
        cfg.stream = s;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, kern, tab, st);
    } else {
        kern<<<grid, 192, C::SMEM, s>>>(tab, st);
        return cudaGetLastError();
    }
}

template <int G>
cudaError_t launch_any(int bn, int elem, const GemmTable<G>& tab, DevStatus* st, cudaStream_t s) {
    if (elem == GEMM_ELEM_E4M3) {
        if (bn == kPairTileWide) return launch_table<512, G, 1, true>(tab, st, s);
        if (bn == kPairTile) return launch_table<256, G, 1, true>(tab, st, s);
        return bn == 128 ? launch_table<128, G, 1, false>(tab, st, s) : launch_table<256, G, 1, false>(tab, st, s);
    }
    if (bn == kPairTileWide) return launch_table<512, G, 0, true>(tab, st, s);
    if (bn == kPairTile) return launch_table<256, G, 0, true>(tab, st, s);
    return bn == 128 ? launch_table<128, G, 0, false>(tab, st, s) : launch_table<256, G, 0, false>(tab, st, s);
}

// strides multiples of 16 bytes, K padded to the 128-byte stage with a host extent
bool gemm_args_ok(const void* A, int64_t lda, const void* B, int64_t ldb, int64_t M, int64_t N, int64_t kdim,
                  int64_t k_host, const int64_t* k_dev, int elem, bool b_mn = false) {
    const int64_t per16 = elem == GEMM_ELEM_E4M3 ? 16 : 8, bk = elem == GEMM_ELEM_E4M3 ? 128 : 64;
    if (M > 0x7fffffff || N > 0x7fffffff || (lda % per16) != 0 || (ldb % per16) != 0 || kdim <= 0 || kdim > lda ||
        (b_mn ? (N > ldb || elem != GEMM_ELEM_BF16) : kdim > ldb) || (k_dev == nullptr && (k_host % bk) != 0))
        return false;
    return !((reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15));
}

// ---------------------------------------------------------------- tile choices
// The tile width (BN) and raster group of each product come from a process-wide table filled by
// the autotuner (bmm_autotune_gemm), keyed by element kind and the rounded-up base-2 logarithms of
// M, N and K; shapes never tuned take BN = 128 for N <= 128, else 256 for M <= 128 (a CTA pair's
// second 128 rows would be empty), else the CTA-pair tile, and raster group 8.  Neither choice
// changes a result: every output element is the same dot product in the same K order.
std::mutex& tune_mutex() {
    static std::mutex mu;
    return mu;
}
std::map<uint64_t, TileChoice>& tune_table() {
    static std::map<uint64_t, TileChoice> t;
    return t;
}
uint64_t tune_key(int elem, int64_t M, int64_t N, int64_t K) {
    auto lg = [](int64_t v) {
        uint64_t b = 0;
        while (b < 62 && (int64_t(1) << b) < v) ++b;
        return b;
    };
    return ((uint64_t)elem << 24) | (lg(M) << 16) | (lg(N) << 8) | lg(K);
}

}  // namespace

TileChoice gemm_tile_choice(int elem, int64_t M, int64_t N, int64_t K) {
    std::lock_guard<std::mutex> lock(tune_mutex());
    const auto it = tune_table().find(tune_key(elem, M, N, K));
    if (it != tune_table().end()) return it->second;
    return TileChoice{N <= 128 ? 128 : (M <= 128 ? 256 : kPairTile), 8};
}

bool gemm_tile_valid(const TileChoice& c) {
    return (c.bn == 128 || c.bn == 256 || c.bn == kPairTile || c.bn == kPairTileWide) &&
           (c.raster == 4 || c.raster == 8 || c.raster == 16);
}

void gemm_tile_set(int elem, int64_t M, int64_t N, int64_t K, const TileChoice& c) {
    std::lock_guard<std::mutex> lock(tune_mutex());
    tune_table()[tune_key(elem, M, N, K)] = c;
}

void gemm_tile_clear() {
    std::lock_guard<std::mutex> lock(tune_mutex());
    tune_table().clear();
}

bool tc_gemm_supported() {
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    return major == 10 && minor == 3 && encode_fn() != nullptr;
}

cudaError_t launch_gemm_bf16_tc(const void* A, int64_t lda, const void* B, int64_t ldb, int64_t M, int64_t N,
                                int64_t kdim, int64_t k_host, const int64_t* k_dev, int k_mult, float* out, int64_t ldo,
                                int accumulate, DevStatus* st, cudaStream_t s, int elem, const float* scale,
                                int64_t tune_k, bool b_mn) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (!gemm_args_ok(A, lda, B, ldb, M, N, kdim, k_host, k_dev, elem, b_mn)) return cudaErrorInvalidValue;
    const TileChoice tc = gemm_tile_choice(elem, M, N, tune_k > 0 ? tune_k : kdim);
    const int BN = tc.bn;
    GemmTable<1> tab;
    tab.count = 1;
    if (!fill_problem(&tab.prob[0], BN, tc.raster, A, lda, B, ldb, M, N, kdim, k_host, k_dev, k_mult, out, ldo,
                      accumulate, elem, scale, b_mn))
        return cudaErrorInvalidValue;
    tab.prob[0].tile_begin = 0;
    tab.total_tiles = tab.prob[0].tiles_m * tab.prob[0].tiles_n;
    return launch_any<1>(BN, elem, tab, st, s);
}

cudaError_t launch_gemm_bf16_tc_grouped(const GemmArgs* args, int64_t count, DevStatus* st, cudaStream_t s) {
    // products are grouped by tile width and element kind; each launch takes up to kMaxGroup of them
    std::vector<TileChoice> choice((size_t)count);
    for (int64_t i = 0; i < count; ++i) choice[i] = gemm_tile_choice(args[i].elem, args[i].M, args[i].N, args[i].kdim);
    for (int pass = 0; pass < 8; ++pass) {
        const int BN = pass % 4 == 0 ? 128 : (pass % 4 == 1 ? 256 : (pass % 4 == 2 ? kPairTile : kPairTileWide));
        const int elem = pass / 4;
        static thread_local GemmTable<kMaxGroup> tab;  // host-side staging of the kernel parameter, one per host thread (30 KB)
        tab.count = 0;
        tab.total_tiles = 0;
        for (int64_t i = 0; i <= count; ++i) {
            const bool flush = (i == count) || tab.count == kMaxGroup;
            if (flush && tab.count > 0) {
                cudaError_t e = launch_any<kMaxGroup>(BN, elem, tab, st, s);
                if (e != cudaSuccess) return e;
                tab.count = 0;
                tab.total_tiles = 0;
            }
            if (i == count) break;
            const GemmArgs& g = args[i];
            if (g.M <= 0 || g.N <= 0) continue;
            if (choice[i].bn != BN || g.elem != elem) continue;
            if (!gemm_args_ok(g.A, g.lda, g.B, g.ldb, g.M, g.N, g.kdim, g.k_host, g.k_dev, g.elem))
                return cudaErrorInvalidValue;
            GemmProblem& pr = tab.prob[tab.count];
            if (!fill_problem(&pr, BN, choice[i].raster, g.A, g.lda, g.B, g.ldb, g.M, g.N, g.kdim, g.k_host, g.k_dev,
                              g.k_mult, g.out, g.ldo, g.accumulate, g.elem, g.scale))
                return cudaErrorInvalidValue;
            pr.tile_begin = tab.total_tiles;
            tab.total_tiles += pr.tiles_m * pr.tiles_n;
            ++tab.count;
        }
    }
    return cudaSuccess;
}

// ---------------------------------------------------------------- autotuner
static int64_t align256(int64_t b) { return round_up(b, 256); }

int64_t gemm_autotune_bytes(int64_t M, int64_t N, int64_t K, int elem) {
    if (M <= 0 || N <= 0 || K <= 0) return 0;
    const int64_t es = elem == GEMM_ELEM_E4M3 ? 1 : 2, bk = elem == GEMM_ELEM_E4M3 ? 128 : 64;
    const int64_t Kp = round_up(K, bk);
    return align256(M * Kp * es) + align256(N * Kp * es) + align256(M * N * 4);
}

// Times every (BN, raster group) candidate on scratch operands of shape M x K and N x K (the
// contents do not affect the result's timing in a way that matters: constant operands), one
// warm-up launch and three timed launches each on stream s, and records the fastest in the table.
// Synchronises s.  scratch: gemm_autotune_bytes(M, N, K, elem) bytes, 256-byte aligned.
cudaError_t gemm_autotune(int64_t M, int64_t N, int64_t K, int elem, void* scratch, size_t bytes, DevStatus* st,
                          cudaStream_t s, TileChoice* best_out, float* best_ms) {
    if (M <= 0 || N <= 0 || K <= 0 || M > 0x7fffffff || N > 0x7fffffff) return cudaErrorInvalidValue;
    if ((int64_t)bytes < gemm_autotune_bytes(M, N, K, elem) || (reinterpret_cast<uintptr_t>(scratch) & 255))
        return cudaErrorInvalidValue;
    const int64_t es = elem == GEMM_ELEM_E4M3 ? 1 : 2, bk = elem == GEMM_ELEM_E4M3 ? 128 : 64;
    const int64_t Kp = round_up(K, bk);
    char* base = static_cast<char*>(scratch);
    void* A = base;
    void* B = base + align256(M * Kp * es);
    float* out = reinterpret_cast<float*>(base + align256(M * Kp * es) + align256(N * Kp * es));
    cudaError_t e;
    if ((e = cudaMemsetAsync(A, 0x3c, (size_t)(M * Kp * es), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(B, 0x3c, (size_t)(N * Kp * es), s)) != cudaSuccess) return e;
    cudaEvent_t e0, e1;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) { cudaEventDestroy(e0); return e; }
    TileChoice best{0, 0};
    float best_t = 0.f;
    for (int bn : {128, 256, kPairTile, kPairTileWide}) {
        for (int raster : {4, 8, 16}) {
            GemmTable<1> tab;
            tab.count = 1;
            if (!fill_problem(&tab.prob[0], bn, raster, A, Kp, B, Kp, M, N, Kp, Kp, nullptr, 1, out, N, 0, elem, nullptr)) {
                e = cudaErrorInvalidValue;
                break;
            }
            tab.prob[0].tile_begin = 0;
            tab.total_tiles = tab.prob[0].tiles_m * tab.prob[0].tiles_n;
            float t_min = 0.f;
            for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
                cudaEventRecord(e0, s);
                e = launch_any<1>(bn, elem, tab, st, s);
                cudaEventRecord(e1, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float t = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
                if (rep == 1 || (rep > 1 && t < t_min)) t_min = t;  // launch 0 is the warm-up
            }
            if (e != cudaSuccess) break;
            if (best.bn == 0 || t_min < best_t) {
                best = TileChoice{bn, raster};
                best_t = t_min;
            }
        }
        if (e != cudaSuccess) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    gemm_tile_set(elem, M, N, Kp, best);
    if (best_out) *best_out = best;
    if (best_ms) *best_ms = best_t;
    return cudaSuccess;
}

}  // namespace bmm
