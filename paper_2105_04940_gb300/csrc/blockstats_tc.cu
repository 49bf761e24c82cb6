// blockstats_tc.cu -- the statistics pass and ||M^k N_k||_F^2 in one read of M and N.
//
// f_k = ||M^k N_k||_F^2 = <G_M, G_N>_F with G_M = M^kT M^k and G_N = N_k N_kT (n_k x n_k Grams;
// eq. 1.2, eq. 3.9).  Its diagonal is s_k = sum_i x_i y_i, which this kernel accumulates exactly
// (float-float folded into FP64) together with x_i = ||M^(i)||^2 and y_i = ||N_(i)||^2; the
// off-diagonal part sum_{i != j} G_M[i,j] G_N[i,j] comes from tensor-core Grams in TMEM: TF32 for
// FP32 inputs, BF16 (exact products) for BF16 inputs, FP32 accumulation.
//
// One CTA per SM pulls blocks from a global counter that runs over the blocks of every product of
// the launch (a table of products in the kernel parameters: one product for bmm_probs, up to
// kMaxProducts of them for bmm_probs_batched).  For block k it streams the vectors of the
// block -- columns of M (length m), then rows of N (length p) -- in sub-tiles of E coordinates
// (E = 128 bytes / element size: 32 FP32 or 64 BF16), several sub-tiles (up to 40 KB) per stage:
//   warp 0      one lane: TMA loads into a 5-stage ring of 40 KB and a record per stage and per
//               block.  A strided operand stage is nb boxes of E columns x 64 rows (128-byte
//               swizzle; in 32-byte atoms for FP32); a contiguous operand stage is one box of E
//               coordinates x 32 nb vectors per sub-tile (128-byte swizzle).  Few large copies keep
//               the TMA unit, which takes about as long for a small box as for a large one, from
//               limiting the pass;
//   warp 1      one lane: tcgen05.mma (M = 128, 32 bytes of K per instruction) with the same operand
//               tile as A and B.  A tile whose vectors are its rows (contiguous storage) is a K-major
//               operand, one whose vectors are its columns (strided storage: row-major M,
//               column-major N) an MN-major operand; both are read where TMA put them.  G_M and G_N
//               of a block take two of three 160-column TMEM slots used in turn, so the Grams of the
//               next block build up while the epilogue of the previous one reads its slots;
//   warps 2-17  (statistics pass) sum the squares of each stage's elements, every warp a
//               sixteenth of each sub-tile for all vectors, float-float sums per lane and vector; at
//               the end of a block they fold the norms into a_k, s_k, ||M^k||_F^2, ||N_k||_F^2, and
//               (both passes) reduce the off-diagonal Gram products from TMEM.
// Positions.  A strided operand's first box starts at the 16-byte boundary at or below the block's
// first column (TMA needs a 16-byte-aligned inner coordinate), so its vectors are operand rows
// d .. d + n_k - 1 with d = off_k mod (16 bytes / element size); the contiguous operand of the same
// block is loaded d rows early to match.  The MMA takes operand rows 0..127 as its M side and rows
// 0..npad-1 (npad <= 144) as its N side.  When d + n_k exceeds 128 (a "wide" block) the missing
// Gram rows are the transposes of columns >= 128 of the rows below 128, which the epilogue counts
// twice, except for the products among the <= 7 vectors at rows >= 128: a second MMA (A = rows
// R0..R0+127 with R0 = 32 for FP32, 64 for BF16, B = rows 128..143, N = 16) computes those into the
// last 16 columns of the slot.
// Operand rows outside the block hold neighbouring data or zeros and are masked out of every sum.
// All waits are bounded; on expiry the CTA records BMM_ERR_TIMEOUT, lets its copies and MMAs in
// flight land, frees TMEM and returns.
#include <type_traits>

#include "internal.h"
#include "tc_ptx.cuh"

namespace bmm {
namespace {

using namespace ptx;

constexpr int kRowBytes = 128;                // one swizzled row: E elements
constexpr int kRowsPerGroup = 32;             // K-major boxes come in multiples of 32 vector rows
constexpr int kGroupBytes = kRowsPerGroup * kRowBytes;  // 4 KB
constexpr int kMnRows = 64;                   // rows per strided box
constexpr int kMnBoxBytes = kMnRows * kRowBytes;        // 8 KB (wide blocks; narrower ones use taller boxes)
constexpr int kStageBytes = 40 * 1024;        // 40 KB per pipeline stage
constexpr int kStages = 5;
constexpr int kBlockSlots = 4;                // block records in flight
constexpr int kConvWarps = 16;
constexpr int kConvThreads = 32 * kConvWarps;
constexpr int kThreads = 64 + kConvThreads;
constexpr int kSmem = kStages * kStageBytes + 1024;
constexpr uint32_t kTmemCols = 512;
constexpr int kSlotCols = 160;                // TMEM columns per Gram slot (3 slots)
constexpr int kCornerCol = 144;               // wide blocks: rows >= 128 x rows >= 128, N = 16
constexpr int kMaxBlock = 128;
constexpr int kFoldStages = 4;                // stages between folds into the second-level sums
constexpr int kMaxKMaps = 6;                  // K-major box heights 32 .. 192 rows
// Element-type traits.  E elements fill a 128-byte row; one MMA consumes 32 bytes of K.
template <typename T> struct Tr;
template <> struct Tr<float> {
    static constexpr int E = 32;
    static constexpr int kAlign = 4;            // elements per 16 bytes
    static constexpr int kMnSubRows = 32;       // rows of a strided sub-tile (4 MMAs of K = 8)
    static constexpr uint32_t kMnKstep = 64;    // 8 rows x 128 bytes, in descriptor units
    static constexpr int kCornerRow0 = 32;      // first operand row of the corner MMA's A
    static constexpr uint32_t kFmt = 2;         // TF32
    static constexpr CUtensorMapDataType kTmaType = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    static constexpr CUtensorMapSwizzle kMnSwizzle = CU_TENSOR_MAP_SWIZZLE_128B_ATOM_32B;
    static __device__ __forceinline__ uint64_t mn_desc(uint32_t addr, uint32_t box_bytes) {
        return sw128_atom32_mn_desc(addr, box_bytes);
    }
    static __device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
        tc_mma_tf32(d, a, b, idesc, acc);
    }
    // byte offset of (row h, column cc) in a strided box: 32-byte chunk cc / 8 at chunk (cc / 8) ^ (h mod 4)
    static __device__ __forceinline__ int mn_offset(int h, int cc) {
        return h * kRowBytes + ((((cc >> 3) ^ (h & 3)) << 5) | ((cc & 7) << 2));
    }
    // byte offset of 16-byte chunk c16 (columns 4 c16 .. 4 c16 + 3) of row h in a strided box
    static __device__ __forceinline__ int mn_chunk_offset(int h, int c16) {
        return h * kRowBytes + ((((c16 >> 1) ^ (h & 3)) << 5) | ((c16 & 1) << 4));
    }
    static __device__ __forceinline__ float to_f(float v) { return v; }
    static __device__ __forceinline__ void add_sq(FF2& acc, float2 v) { acc.add_sq(v); }
};
template <> struct Tr<__nv_bfloat16> {
    static constexpr int E = 64;
    static constexpr int kAlign = 8;
    static constexpr int kMnSubRows = 64;       // 4 MMAs of K = 16
    static constexpr uint32_t kMnKstep = 128;   // 16 rows x 128 bytes
    static constexpr int kCornerRow0 = 64;      // an MN atom is 64 rows wide
    static constexpr uint32_t kFmt = 1;         // BF16 (kind::f16)
    static constexpr CUtensorMapDataType kTmaType = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    static constexpr CUtensorMapSwizzle kMnSwizzle = CU_TENSOR_MAP_SWIZZLE_128B;
    static __device__ __forceinline__ uint64_t mn_desc(uint32_t addr, uint32_t box_bytes) {
        return sw128_mn_desc(addr, box_bytes);
    }
    static __device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
        tc_mma_bf16(d, a, b, idesc, acc);
    }
    // 16-byte chunk (2 cc) / 16 of row h at chunk ^ (h mod 8)
    static __device__ __forceinline__ int mn_offset(int h, int cc) {
        return h * kRowBytes + ((((cc >> 3) ^ (h & 7)) << 4) | ((cc & 7) << 1));
    }
    // 16-byte chunk c16 (columns 8 c16 .. 8 c16 + 7) of row h
    static __device__ __forceinline__ int mn_chunk_offset(int h, int c16) {
        return h * kRowBytes + ((c16 ^ (h & 7)) << 4);
    }
    static __device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
    // a BF16 value has 8 significant bits, so its square is exact in FP32
    static __device__ __forceinline__ void add_sq(FF2& acc, float2 v) { acc.add_sq_exact(v); }
};

// Sub-tiles per stage of a contiguous operand whose sub-tiles are nb groups of 32 vector rows.
// The MMA reads 128 operand rows (16 KB) from the start of every sub-tile and a wide block's
// corner MMA reads up to R0 + 128 rows; rows past the block belong to the next sub-tile (masked)
// but must stay inside the 40 KB stage: (per - 1) * nb * 4 KB + 16 KB <= 40 KB for nb <= 4; wide
// FP32 blocks (nb = 5, corner to 20 KB) take 2 and wide BF16 blocks (nb = 6, corner to 24 KB) 1.
// A strided operand stage is nb boxes of E columns x mn_rows rows.  The MMA's M side always spans
// 128 vectors, i.e. 128 / E boxes at the box stride, whatever nb is, and these reads must stay
// inside the stage: FP32 (four boxes) keeps 64-row boxes (8 KB, 32 KB read); BF16 (two boxes) takes
// 128-row boxes (16 KB, 32 KB read) for blocks of one or two boxes and 64-row boxes for wide
// blocks.  A stage holds at most 40 KB (a wide FP32 block's five boxes).
__host__ __device__ __forceinline__ int subtiles_per_stage(int nb) { return nb >= 6 ? 1 : (nb == 5 ? 2 : 1 + 6 / nb); }
template <typename T> __host__ __device__ __forceinline__ int mn_map_index(int nb) {
    return (sizeof(T) == 2 && nb <= 2) ? 1 : 0;
}
template <typename T> __host__ __device__ __forceinline__ int mn_rows(int nb) { return kMnRows << mn_map_index<T>(nb); }

enum StageFlags : int {
    ST_PHASE = 1,   // 0: columns of M, 1: rows of N
    ST_FIRST = 2,   // first stage of the phase
    ST_LAST = 4,    // last stage of the phase
    ST_MN = 8,      // vectors are tile columns: MN-major operand
    ST_WIDE = 16,   // d + n_k > 128: corner MMA
};

struct __align__(16) StageInfo {
    int block;      // -1: no more work
    int flags;      // StageFlags
    int nk;         // block size
    int d;          // tile row (K-major) or column (MN-major) of the block's first vector
    int dpos;       // operand row of the block's first vector, the same in both phases
    int nb;         // groups per sub-tile: 32-row groups (K-major) or E-column boxes (MN-major)
    int nsub;       // sub-tiles in this stage
    int sub_bytes;  // distance between sub-tiles in the stage
    int box_bytes;  // MN-major: bytes of one box (E columns x mn_rows rows)
};

// One window of consecutive blocks: the unit of work of a CTA (see stats_windows_kernel).
struct __align__(16) BlockInfo {
    long long lo;  // first column of the window
    long long kb;  // first block of the window within its product, -1: no more work
    int q;         // product
    int nk;        // vectors in the window (the sum of its block sizes)
    int dpos;      // operand row of the window's first vector
    int nblk;      // blocks in the window
};

// Tensor maps of one operand: strided storage uses map[mn_map_index(nb)] (E x 64 or 128 boxes);
// contiguous storage uses map[nb - 1] (E coordinates x 32 nb vectors).
struct OperandMaps {
    CUtensorMap map[kMaxKMaps];
};

// One product of a launch.  Outputs x, y [n] and a, s, mf, nf [K] are written in the statistics
// pass (STATS) and read (s) in the Gram-only pass; f [K] is written by both.  wins
// [stats_windows_ints(K)] is workspace: the window starts (wins[0 .. W], wins[W] = K), wins[K + 1] = W,
// wins[K + 2] = T and wins[K + 3 .. K + 3 + T) the order in which the last T windows are handed out.
struct StatsProblem {
    OperandMaps mM, mN;
    const int64_t* off;
    long long K, n, m, p;
    int* wins;
    double *x, *y, *a, *s, *mf, *nf, *f;
    DevStatus* st;
    int M_strided, N_strided;
};
template <int G> struct StatsTable {
    int count;
    long long total_blocks;  // an upper bound of the launch's windows
    StatsProblem prob[G];
};
constexpr int kMaxProducts = (32760 - 64) / (int)sizeof(StatsProblem);  // kernel-parameter limit
static_assert(sizeof(StatsTable<kMaxProducts>) <= 32764, "statistics table exceeds the kernel-parameter limit");

template <typename T>
__device__ __forceinline__ uint32_t idesc_of(int npad, bool mn_major) {
    // D = F32 (bits 4-5), A and B format (bits 7-9, 10-12), A and B MN-major (bits 15, 16) or
    // K-major, N>>3 at 17, M>>4 at 24
    const uint32_t major = mn_major ? (3u << 15) : 0u;
    return (1u << 4) | (Tr<T>::kFmt << 7) | (Tr<T>::kFmt << 10) | major | ((uint32_t)(npad >> 3) << 17) |
           ((uint32_t)(128 >> 4) << 24);
}

// Four K steps (128 bytes of K) of one sub-tile, A = B = the operand at descriptor (lo, hi): the
// start address is in the low word, so a K step is a 32-bit add (32 bytes K-major, 8 or 16 rows
// MN-major).  The first MMA overwrites the accumulator when `fresh`.
template <typename T, bool MN>
__device__ __forceinline__ void mma_sub(uint32_t d, uint32_t lo_a, uint32_t lo_b, uint32_t hi, uint32_t idesc, bool fresh) {
    constexpr uint32_t ks = MN ? Tr<T>::kMnKstep : 2u;
    const uint64_t h = (uint64_t)hi << 32;
    Tr<T>::mma(d, h | lo_a, h | lo_b, idesc, fresh ? 0u : 1u);
    Tr<T>::mma(d, h | (lo_a + ks), h | (lo_b + ks), idesc, 1u);
    Tr<T>::mma(d, h | (lo_a + 2 * ks), h | (lo_b + 2 * ks), idesc, 1u);
    Tr<T>::mma(d, h | (lo_a + 3 * ks), h | (lo_b + 3 * ks), idesc, 1u);
}

template <typename T, bool MN>
__device__ __forceinline__ void mma_stage(uint32_t d_main, uint32_t d_corner, uint32_t addr, uint32_t sub_bytes,
                                          uint32_t box_bytes, int nsub, uint32_t idesc, uint32_t idesc16, bool first,
                                          bool wide) {
    // corner operands, in descriptor units: A from operand row R0, B from operand row 128.
    // MN-major: an E-row block of operand rows is one box (8 KB for wide blocks); K-major: a row is
    // 128 bytes.
    constexpr uint32_t ca = MN ? (uint32_t)(Tr<T>::kCornerRow0 / Tr<T>::E) * (kMnBoxBytes >> 4)
                               : (uint32_t)(Tr<T>::kCornerRow0 * kRowBytes) >> 4;
    constexpr uint32_t cb = MN ? (uint32_t)(128 / Tr<T>::E) * (kMnBoxBytes >> 4) : (uint32_t)(128 * kRowBytes) >> 4;
    const uint64_t d0 = MN ? Tr<T>::mn_desc(addr, box_bytes) : sw128_desc(addr);
    const uint32_t hi = (uint32_t)(d0 >> 32);
    uint32_t lo = (uint32_t)d0;
    const uint32_t step = sub_bytes >> 4;
    for (int s = 0; s < nsub; ++s, lo += step) {
        const bool fresh = first && s == 0;
        mma_sub<T, MN>(d_main, lo, lo, hi, idesc, fresh);
        if (wide) mma_sub<T, MN>(d_corner, lo + ca, lo + cb, hi, idesc16, fresh);
    }
}

__device__ __forceinline__ bool wait_fast(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
    return mbar_try_wait_sleep(bar, parity) || mbar_wait<true>(bar, parity, abort_flag);
}

// Barrier over the converter warps built on an mbarrier, so that its wait is bounded like every
// other wait (a bar.sync could not give up if a warp left the loop after a timeout).
__device__ __forceinline__ bool conv_sync(uint32_t bar, int& uses, volatile int* abort_flag) {
    __threadfence_block();
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(bar);
    const bool ok = wait_fast(bar, (uint32_t)(uses & 1), abort_flag);
    ++uses;
    return ok;
}

// Sums of squares of one phase of a block with d + n_k <= 128, every vector inside the first 128
// tile columns (strided) or rows (contiguous).  Each lane reads whole 16-byte chunks and keeps
// float-float sums per element position of its chunk, so no lane idles on a vector outside the
// block except at the block's edges.  Return false when a wait expired.
//
// Strided (MN) stages: nb boxes of E columns x 64 rows, the block's columns in the first 8 nb
// 16-byte chunks of each row.  A row is read by lpr = 8 nb lanes (rounded up to 8, 16 or 32), so
// one warp reads 32 / lpr rows per step: lane chunk cg covers columns kCpc cg .. kCpc cg + kCpc - 1
// and rows hp + rps (cw + 16 r) (hp = lane / lpr, rps = 32 / lpr).  The swizzle of a chunk depends on
// the row mod 4 (FP32) or mod 8 (BF16) only, which is fixed per lane.  Partial sums go to
// part[warp][vector], summed over the warps by the caller.
template <typename T>
__device__ __forceinline__ bool squares_strided(const uint8_t* base, const StageInfo* info, uint64_t* bar_full,
                                                uint64_t* bar_empty, int& stage, uint32_t& ph, volatile int* abort_flag,
                                                int cw, int lane, int nk, int d, float2 (*part)[kMaxBlock]) {
    using TR = Tr<T>;
    constexpr int kCpc = 16 / (int)sizeof(T);
    const int nb = info[stage].nb, box_bytes = info[stage].box_bytes;  // the same in every stage of the phase
    const int lpr = nb == 1 ? 8 : (nb == 2 ? 16 : 32);
    const int rps = 32 / lpr;
    const int steps = mn_rows<T>(nb) / (16 * rps);  // <= 4
    const int step_bytes = 16 * rps * kRowBytes;
    const int cg = lane & (lpr - 1), hp = lane / lpr;
    const int box = cg >> 3;
    const int h0 = hp + rps * cw;
    const int lane_off = box * box_bytes + TR::mn_chunk_offset(h0, cg & 7);
    // element u of the chunk goes to half u & 1 of pair u / 2 (two vectors per paired sum)
    FF2 acc[kCpc / 2], tot[kCpc / 2];
#pragma unroll
    for (int u = 0; u < kCpc / 2; ++u) { acc[u].zero(); tot[u].zero(); }
    int since_fold = 0;
    while (true) {
        if (!wait_fast(smem_u32(&bar_full[stage]), ph, abort_flag)) return false;
        const int rows = info[stage].nsub * TR::kMnSubRows;
        const bool last = info[stage].flags & ST_LAST;
        if (box < nb) {
            const uint8_t* src = base + stage * kStageBytes + lane_off;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                if (r < steps && h0 + 16 * rps * r < rows) {
                    const uint4 w4 = *reinterpret_cast<const uint4*>(src + r * step_bytes);
                    const T* e = reinterpret_cast<const T*>(&w4);
#pragma unroll
                    for (int u = 0; u < kCpc / 2; ++u)
                        TR::add_sq(acc[u], make_float2(TR::to_f(e[2 * u]), TR::to_f(e[2 * u + 1])));
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bar_empty[stage]));
        if (++stage == kStages) { stage = 0; ph ^= 1u; }
#pragma unroll
        for (int u = 0; u < kCpc / 2; ++u) acc[u].renorm();
        if (++since_fold == kFoldStages || last) {
#pragma unroll
            for (int u = 0; u < kCpc / 2; ++u) {
                tot[u].add(acc[u]);
                tot[u].renorm();
                acc[u].zero();
            }
            since_fold = 0;
        }
        if (last) break;
    }
    // the rps lanes of a chunk combine their rows
    for (int o = lpr; o < 32; o <<= 1) {
#pragma unroll
        for (int u = 0; u < kCpc / 2; ++u) {
            FF2 other;
            other.hi.x = __shfl_xor_sync(0xffffffffu, tot[u].hi.x, o);
            other.hi.y = __shfl_xor_sync(0xffffffffu, tot[u].hi.y, o);
            other.lo.x = __shfl_xor_sync(0xffffffffu, tot[u].lo.x, o);
            other.lo.y = __shfl_xor_sync(0xffffffffu, tot[u].lo.y, o);
            tot[u].add(other);
            tot[u].renorm();
        }
    }
    if (hp == 0) {
#pragma unroll
        for (int u = 0; u < kCpc; ++u) {
            const int i = kCpc * cg + u - d;
            const FF h = tot[u >> 1].half(u & 1);
            if (i >= 0 && i < nk) part[cw][i] = make_float2(h.hi, h.lo);
        }
    }
    return true;
}

// Contiguous (K-major) stages: sub-tiles of 32 nb vector rows x 128 bytes.  Lane t = 32 cw + lane
// reads chunk t mod 8 of rows t / 8 and t / 8 + 64, every element of a chunk belonging to the same
// vector; the eight lanes of a row combine their sums and write x_i or y_i to xy[i].
template <typename T>
__device__ __forceinline__ bool squares_contig(const uint8_t* base, const StageInfo* info, uint64_t* bar_full,
                                               uint64_t* bar_empty, int& stage, uint32_t& ph, volatile int* abort_flag,
                                               int cw, int lane, int nk, int d, float2* xy) {
    using TR = Tr<T>;
    constexpr int kCpc = 16 / (int)sizeof(T);
    const int t = 32 * cw + lane;
    const int q = t & 7, r0 = t >> 3;
    const int sw = (q ^ (r0 & 7)) << 4;  // (r0 + 64) mod 8 == r0 mod 8
    const bool in0 = r0 >= d && r0 < d + nk, in1 = r0 + 64 >= d && r0 + 64 < d + nk;
    // acc[j]: row r0 + 64 j, elements 2u and 2u + 1 of the chunk in the two halves (added at the end)
    FF2 acc[2], tot[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) { acc[u].zero(); tot[u].zero(); }
    int since_fold = 0;
    while (true) {
        if (!wait_fast(smem_u32(&bar_full[stage]), ph, abort_flag)) return false;
        const int nsub = info[stage].nsub, sub_bytes = info[stage].sub_bytes;
        const bool last = info[stage].flags & ST_LAST;
        const uint8_t* tile = base + stage * kStageBytes + r0 * kRowBytes + sw;
        for (int s = 0; s < nsub; ++s) {
            const uint8_t* sub = tile + s * sub_bytes;
            if (in0) {
                const uint4 w4 = *reinterpret_cast<const uint4*>(sub);
                const T* e = reinterpret_cast<const T*>(&w4);
#pragma unroll
                for (int u = 0; u < kCpc / 2; ++u)
                    TR::add_sq(acc[0], make_float2(TR::to_f(e[2 * u]), TR::to_f(e[2 * u + 1])));
            }
            if (in1) {
                const uint4 w4 = *reinterpret_cast<const uint4*>(sub + 64 * kRowBytes);
                const T* e = reinterpret_cast<const T*>(&w4);
#pragma unroll
                for (int u = 0; u < kCpc / 2; ++u)
                    TR::add_sq(acc[1], make_float2(TR::to_f(e[2 * u]), TR::to_f(e[2 * u + 1])));
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bar_empty[stage]));
        if (++stage == kStages) { stage = 0; ph ^= 1u; }
#pragma unroll
        for (int u = 0; u < 2; ++u) acc[u].renorm();
        if (++since_fold == kFoldStages || last) {
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                tot[u].add(acc[u]);
                tot[u].renorm();
                acc[u].zero();
            }
            since_fold = 0;
        }
        if (last) break;
    }
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            FF2 other;
            other.hi.x = __shfl_xor_sync(0xffffffffu, tot[u].hi.x, o);
            other.hi.y = __shfl_xor_sync(0xffffffffu, tot[u].hi.y, o);
            other.lo.x = __shfl_xor_sync(0xffffffffu, tot[u].lo.x, o);
            other.lo.y = __shfl_xor_sync(0xffffffffu, tot[u].lo.y, o);
            tot[u].add(other);
            tot[u].renorm();
        }
    if (q == 0) {
        if (in0) {
            const FF f = tot[0].both();
            xy[r0 - d] = make_float2(f.hi, f.lo);
        }
        if (in1) {
            const FF f = tot[1].both();
            xy[r0 + 64 - d] = make_float2(f.hi, f.lo);
        }
    }
    return true;
}

// Sums of squares of one phase of a wide block (d + n_k > 128): lane handles vectors lane + 32 v,
// every element by itself.  Rare, so kept out of line to spare the kernel's registers.  Returns
// the next (stage, phase bit) as stage | phase << 8, or -1 when a wait expired.
template <typename T>
__device__ __noinline__ int squares_wide(const uint8_t* base, const StageInfo* info, uint64_t* bar_full,
                                         uint64_t* bar_empty, int stage, uint32_t ph, volatile int* abort_flag,
                                         int cw, int lane, float2 (*part)[kMaxBlock]) {
    using TR = Tr<T>;
    bool aborted = false;
    // two levels of float-float sums: acc over at most kFoldStages stages, folded
    // into tot (FP32 operations only: the FP64 pipe is slow on this part); FP64 once
    // per phase
    FF acc[4], tot[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) { acc[v].zero(); tot[v].zero(); }
    int since_fold = 0;
    bool mn_phase = false;
    while (true) {
        if (!wait_fast(smem_u32(&bar_full[stage]), ph, abort_flag)) { aborted = true; break; }
        const StageInfo si = info[stage];
        mn_phase = si.flags & ST_MN;
        const uint8_t* tile = base + stage * kStageBytes;
        const int sub_bytes = si.sub_bytes;
        if (mn_phase) {
            // rows h = cw + 16 r of every sub-tile; vector i is tile column d + i
            for (int s = 0; s < si.nsub; ++s) {
                const uint8_t* sub = tile + s * sub_bytes;
#pragma unroll
                for (int r = 0; r < TR::kMnSubRows / 16; ++r) {
                    const int h = cw + 16 * r;
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const int i = lane + 32 * v;
                        if (i < si.nk) {
                            const int j = i + si.d;
                            const float e = TR::to_f(*reinterpret_cast<const T*>(
                                sub + (j / TR::E) * kMnBoxBytes + TR::mn_offset(h, j % TR::E)));
                            acc[v].add_prod(e, e);
                        }
                    }
                }
            }
        } else {
            // 16-byte chunk cw / 2 of every sub-tile row, vectors i = lane + 32 v for
            // v = cw mod 2 and cw mod 2 + 2; vector i is tile row d + i
            const int q = cw >> 1;
            for (int s = 0; s < si.nsub; ++s) {
                const uint8_t* sub = tile + s * sub_bytes;
#pragma unroll
                for (int vv = 0; vv < 2; ++vv) {
                    // acc[vv] holds vector group (cw mod 2) + 2 vv in this layout
                    const int i = lane + 32 * ((cw & 1) + 2 * vv);
                    if (i < si.nk) {
                        const int r = i + si.d;
                        const uint4 w4 =
                            *reinterpret_cast<const uint4*>(sub + r * kRowBytes + ((q ^ (r & 7)) << 4));
                        const T* e = reinterpret_cast<const T*>(&w4);
#pragma unroll
                        for (int u = 0; u < 16 / (int)sizeof(T); ++u) {
                            const float ev = TR::to_f(e[u]);
                            acc[vv].add_prod(ev, ev);
                        }
                    }
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bar_empty[stage]));
        if (++stage == kStages) { stage = 0; ph ^= 1u; }
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[v].renorm();
        const bool last = si.flags & ST_LAST;
        if (++since_fold == kFoldStages || last) {
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                tot[v].add(acc[v]);
                tot[v].renorm();
                acc[v].zero();
            }
            since_fold = 0;
        }
        if (last) break;
    }
    if (mn_phase) {
#pragma unroll
        for (int v = 0; v < 4; ++v) part[cw][lane + 32 * v] = make_float2(tot[v].hi, tot[v].lo);
    } else {
        part[cw][lane + 32 * (cw & 1)] = make_float2(tot[0].hi, tot[0].lo);
        part[cw][lane + 32 * ((cw & 1) + 2)] = make_float2(tot[1].hi, tot[1].lo);
        part[cw][lane + 32 * ((cw & 1) ^ 1)] = make_float2(0.f, 0.f);
        part[cw][lane + 32 * (((cw & 1) ^ 1) + 2)] = make_float2(0.f, 0.f);
    }
    return aborted ? -1 : (stage | (int)(ph << 8));
}

constexpr int kWinThreads = 1024;
constexpr int kWinChunk = 2 * kWinThreads;  // blocks per pass through shared memory

// Windows: runs of consecutive blocks of a product whose vectors, counted from the 16-byte
// boundary at or below the run's first column (for strided operands), fit the 128 operand rows of
// one MMA tile.  They are taken greedily from block 0: a window ends before the first block that
// would overflow it, and a block that fills the tile by itself (a wide block) is a window alone.
// Packing small blocks this way gives the MMA, the TMA and the norm warps fuller tiles.  One CTA
// per product, in passes of kWinChunk blocks (no window crosses a pass).  With next[k] = the end
// of the window that starts at block k, the windows are the orbit of the pass's first block under
// next, found by pointer doubling: after the round with jump J = next^(2^r), every next^i(0) with
// i < 2^(r+1) is marked.  Writes wins[0 .. W] (window starts, wins[W] = K) and wins[K + 1] = W;
// CTA 0 also zeroes the work counter of the statistics launch that follows.
// The statistics kernel's CTAs claim windows in order, which lets neighbouring windows share their
// edge boxes through L2, but leaves a tail: with about 4.5 windows of 1 to 4 boxes per CTA, the last
// CTA to finish carries about 17% more than the mean.  So the launch's last product also gets a
// hand-out order for its last T = min(W, tail) windows, largest first (by vector span, ties in block
// order): wins[K + 2] = T and wins[K + 3 + r] = the window handed out r-th among them (T = 0 for
// the other products).  Tail lengths of 3/4 of the CTAs cut the simulated excess to about 6%.
template <typename T, int G>
__global__ void __launch_bounds__(kWinThreads)
    stats_windows_kernel(const __grid_constant__ StatsTable<G> tab, int* __restrict__ counter, int tail) {
    __shared__ long long s_off[kWinChunk + 1];
    __shared__ int s_next[kWinChunk + 1];
    __shared__ unsigned char s_mark[kWinChunk];
    __shared__ int s_scan[kWinThreads / 32];
    if (blockIdx.x == 0 && threadIdx.x == 0) *counter = 0;
    if ((int)blockIdx.x >= tab.count) return;
    const StatsProblem& pr = tab.prob[blockIdx.x];
    const long long K = pr.K;
    const long long align_mask = (pr.M_strided || pr.N_strided) ? Tr<T>::kAlign - 1 : 0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int base = 0;
    for (long long c0 = 0; c0 < K; c0 += kWinChunk) {
        const int L = (int)imin(kWinChunk, K - c0);
        __syncthreads();  // the previous pass is done with shared memory
        for (int i = threadIdx.x; i <= L; i += kWinThreads) s_off[i] = pr.off[c0 + i];
        __syncthreads();
        for (int k = threadIdx.x; k < L; k += kWinThreads) {
            // largest e in [k + 1, min(L, k + 128)] with off[e] - (off[k] rounded down to 16 bytes) <= 128
            const long long lim = s_off[k] - (s_off[k] & align_mask) + 128;
            int lo = k + 1, hi = (int)imin(L, k + 128);
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_off[mid] <= lim) lo = mid;
                else hi = mid - 1;
            }
            s_next[k] = lo;
            s_mark[k] = k == 0;
        }
        if (threadIdx.x == 0) s_next[L] = L;
        __syncthreads();
        for (int jump = 1; jump < L; jump <<= 1) {
            for (int k = threadIdx.x; k < L; k += kWinThreads)
                if (s_mark[k] && s_next[k] < L) s_mark[s_next[k]] = 1;
            __syncthreads();
            int jn[kWinChunk / kWinThreads];
#pragma unroll
            for (int u = 0; u < kWinChunk / kWinThreads; ++u) {
                const int k = threadIdx.x + u * kWinThreads;
                jn[u] = k < L ? s_next[s_next[k]] : L;
            }
            __syncthreads();
#pragma unroll
            for (int u = 0; u < kWinChunk / kWinThreads; ++u) {
                const int k = threadIdx.x + u * kWinThreads;
                if (k < L) s_next[k] = jn[u];
            }
            __syncthreads();
        }
        // compaction in block order: thread t owns blocks 2t and 2t + 1
        const int k0 = 2 * threadIdx.x;
        const int m0 = k0 < L ? s_mark[k0] : 0, m1 = k0 + 1 < L ? s_mark[k0 + 1] : 0;
        int v = m0 + m1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int x = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += x;
        }
        if (lane == 31) s_scan[warp] = v;
        __syncthreads();
        if (warp == 0) {
            int w = s_scan[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int x = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += x;
            }
            s_scan[lane] = w;
        }
        __syncthreads();
        const int excl = base + (warp ? s_scan[warp - 1] : 0) + v - m0 - m1;
        if (m0) pr.wins[excl] = (int)(c0 + k0);
        if (m1) pr.wins[excl + m0] = (int)(c0 + k0 + 1);
        base += s_scan[kWinThreads / 32 - 1];
    }
    if (threadIdx.x == 0) {
        pr.wins[base] = (int)K;
        pr.wins[K + 1] = base;
    }
    const int W = base;
    const int nt = (int)blockIdx.x == tab.count - 1 ? (int)imin(imin(W, tail), kWinTailMax) : 0;
    __syncthreads();  // every window start written above is visible to the block
    for (int i = threadIdx.x; i < nt; i += kWinThreads) {
        const int w = W - nt + i;
        const long long lo = pr.off[pr.wins[w]], hi = pr.off[pr.wins[w + 1]];
        s_off[i] = hi - lo + (lo & 31);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nt; i += kWinThreads) {
        int rank = 0;
        for (int j = 0; j < nt; ++j) rank += (s_off[j] > s_off[i]) || (s_off[j] == s_off[i] && j < i);
        pr.wins[K + 3 + rank] = W - nt + i;
    }
    if (threadIdx.x == 0) pr.wins[K + 2] = nt;
}

template <typename T, bool STATS, int G>
__global__ void __launch_bounds__(kThreads, 1)
    blockstats_tc_kernel(const __grid_constant__ StatsTable<G> tab, int* __restrict__ counter) {
    using TR = Tr<T>;
    extern __shared__ uint8_t dsmem[];
    __shared__ __align__(8) uint64_t bar_full[kStages], bar_empty[kStages];
    __shared__ __align__(8) uint64_t bar_bfull[kBlockSlots], bar_bempty[kBlockSlots];
    __shared__ __align__(8) uint64_t bar_slot_free[3], bar_tfull[2], bar_drain, bar_cs;
    __shared__ StageInfo info[kStages];
    __shared__ BlockInfo binfo[kBlockSlots];
    __shared__ long long s_wb[G + 1];                               // first window of each product
    __shared__ int s_seg[kMaxBlock + 1];                            // block starts in the window
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;
    __shared__ float2 part[STATS ? kConvWarps : 1][kMaxBlock];   // [warp][vector] float-float, one phase
    __shared__ float2 xy_ff[STATS ? 2 : 1][kMaxBlock];            // [phase][vector]: x_i, y_i (float-float)
    __shared__ float2 rowpart[4][kMaxBlock];                      // off-diagonal sums per [quarter][row]

    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dsmem) + 1023) & ~uintptr_t(1023));
    auto stage_ptr = [&](int s) { return base + s * kStageBytes; };
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(smem_u32(&bar_full[s]), 1);
            // released by the MMA's commit once its reads are done, and in the statistics pass by
            // the 16 converter warps once they have read the stage
            mbar_init(smem_u32(&bar_empty[s]), STATS ? kConvWarps + 1 : 1);
        }
        for (int b = 0; b < kBlockSlots; ++b) {
            mbar_init(smem_u32(&bar_bfull[b]), 1);
            mbar_init(smem_u32(&bar_bempty[b]), kConvWarps);
        }
        for (int q = 0; q < 3; ++q) mbar_init(smem_u32(&bar_slot_free[q]), kConvWarps);
        for (int q = 0; q < 2; ++q) mbar_init(smem_u32(&bar_tfull[q]), 1);
        mbar_init(smem_u32(&bar_drain), 1);
        mbar_init(smem_u32(&bar_cs), kConvWarps);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // operand tiles start as zeros, so rows no copy ever wrote are finite
    for (int e = threadIdx.x; e < kStages * kStageBytes / 16; e += kThreads)
        reinterpret_cast<uint4*>(base)[e] = make_uint4(0, 0, 0, 0);
    fence_async_smem();
    if (warp == 1) tmem_alloc(smem_u32(&s_tmem), kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    if (warp == 0) {
        if (lane == 0) {
            // ------------------------------------------------ producer
            int stage = 0, bslot = 0, q = 0;
            uint32_t ph = 0, bph = 0;
            uint32_t issued_mask = 0, issued_phase = 0;
            bool aborted = false;
            // the launch numbers the windows of its products one after another
            long long total = 0;
            for (int u = 0; u < tab.count; ++u) {
                s_wb[u] = total;
                total += tab.prob[u].wins[tab.prob[u].K + 1];
            }
            s_wb[tab.count] = total;
            while (!aborted) {
                const long long kg = atomicAdd(counter, 1);
                if (kg >= total) {
                    if (!wait_fast(smem_u32(&bar_bempty[bslot]), bph ^ 1u, &s_abort)) { aborted = true; break; }
                    binfo[bslot].kb = -1;
                    mbar_arrive(smem_u32(&bar_bfull[bslot]));
                    if (!wait_fast(smem_u32(&bar_empty[stage]), ph ^ 1u, &s_abort)) { aborted = true; break; }
                    info[stage].block = -1;
                    mbar_arrive(smem_u32(&bar_full[stage]));
                    break;
                }
                // windows are claimed in increasing order, so this CTA's product index only grows
                while (q + 1 < tab.count && kg >= s_wb[q + 1]) ++q;
                const StatsProblem& pr = tab.prob[q];
                long long w = kg - s_wb[q];
                {  // the last windows of the launch's last product go out in the precomputed order
                    const long long W = s_wb[q + 1] - s_wb[q];
                    const int nt = pr.wins[pr.K + 2];
                    if (nt > 0 && nt <= kWinTailMax && nt <= W && w >= W - nt) {
                        const long long wt = pr.wins[pr.K + 3 + (w - (W - nt))];
                        if (wt >= W - nt && wt < W) w = wt;
                    }
                }
                const long long k = pr.wins[w], ke = pr.wins[w + 1];  // blocks k .. ke - 1
                const bool range_ok = k >= 0 && ke > k && ke <= pr.K && ke - k <= kMaxBlock;
                const long long lo = range_ok ? pr.off[k] : 0, hi = range_ok ? pr.off[ke] : 0;
                const long long nk = hi - lo;
                const int M_strided = pr.M_strided, N_strided = pr.N_strided;
                const int dlo = (int)(lo & (TR::kAlign - 1));
                const int dpos = (M_strided || N_strided) ? dlo : 0;
                if (!range_ok || lo < 0 || hi > pr.n || nk <= 0 || (ke - k == 1 ? nk > kMaxBlock : dpos + nk > 128)) {
                    set_status(pr.st, BMM_ERR_SHAPE, (int)k);
                    if (range_ok)
                        for (long long kk = k; kk < ke; ++kk) {
                            if (STATS) { pr.a[kk] = 0.0; pr.s[kk] = 0.0; pr.mf[kk] = 0.0; pr.nf[kk] = 0.0; }
                            pr.f[kk] = 0.0;
                        }
                    continue;
                }
                const bool wide = dpos + nk > 128;  // a window of one block only
                if (!wait_fast(smem_u32(&bar_bempty[bslot]), bph ^ 1u, &s_abort)) { aborted = true; break; }
                binfo[bslot].lo = lo;
                binfo[bslot].kb = k;
                binfo[bslot].q = q;
                binfo[bslot].nk = (int)nk;
                binfo[bslot].dpos = dpos;
                binfo[bslot].nblk = (int)(ke - k);
                mbar_arrive(smem_u32(&bar_bfull[bslot]));
                if (++bslot == kBlockSlots) { bslot = 0; bph ^= 1u; }
                for (int phase = 0; phase < 2 && !aborted; ++phase) {
                    const int strided = phase == 0 ? M_strided : N_strided;
                    const long long len = phase == 0 ? pr.m : pr.p;
                    const int d = strided ? dlo : dpos;
                    // strided: boxes of E columns; contiguous: groups of 32 vector rows (a wide
                    // BF16 block takes 6 so that the corner's rows 64..191 are loaded)
                    int nb = strided ? (int)((d + nk + TR::E - 1) / TR::E) : (int)((d + nk + 31) / 32);
                    if (!strided && wide && TR::kCornerRow0 + 128 > 32 * nb) nb = (TR::kCornerRow0 + 128) / 32;
                    const int box_bytes = strided ? mn_rows<T>(nb) * kRowBytes : 0;
                    const int per = strided ? mn_rows<T>(nb) / TR::kMnSubRows : subtiles_per_stage(nb);
                    const long long nsub_total = (len + TR::E - 1) / TR::E;
                    const OperandMaps& maps = phase == 0 ? pr.mM : pr.mN;
                    const CUtensorMap* map = &maps.map[strided ? mn_map_index<T>(nb) : nb - 1];
                    for (long long c0 = 0; c0 < nsub_total; c0 += per) {
                        const int nsub = (int)imin(per, nsub_total - c0);
                        if (!wait_fast(smem_u32(&bar_empty[stage]), ph ^ 1u, &s_abort)) { aborted = true; break; }
                        StageInfo& si = info[stage];
                        si.block = (int)k;
                        si.flags = phase | (c0 == 0 ? ST_FIRST : 0) | (c0 + per >= nsub_total ? ST_LAST : 0) |
                                   (strided ? ST_MN : 0) | (wide ? ST_WIDE : 0);
                        si.nk = (int)nk;
                        si.d = d;
                        si.dpos = dpos;
                        si.nb = nb;
                        si.nsub = nsub;
                        si.sub_bytes = strided ? TR::kMnSubRows * kRowBytes : nb * kGroupBytes;
                        si.box_bytes = box_bytes;
                        const uint32_t fb = smem_u32(&bar_full[stage]);
                        uint8_t* dst = stage_ptr(stage);
                        if (strided) {
                            // nb boxes of E columns x mn_rows rows (rows past the operand read as zeros)
                            mbar_expect_tx(fb, (uint32_t)(nb * box_bytes));
                            for (int b = 0; b < nb; ++b)
                                tma_load_2d(smem_u32(dst + b * box_bytes), map, fb, (int32_t)(lo - d + TR::E * b),
                                            (int32_t)(TR::kMnSubRows * c0));
                        } else {
                            // one box of E coordinates x 32 nb vectors per sub-tile
                            mbar_expect_tx(fb, (uint32_t)(nsub * nb * kGroupBytes));
                            for (int s = 0; s < nsub; ++s)
                                tma_load_2d(smem_u32(dst + s * nb * kGroupBytes), map, fb, (int32_t)(TR::E * (c0 + s)),
                                            (int32_t)(lo - d));
                        }
                        issued_mask |= 1u << stage;
                        issued_phase = (issued_phase & ~(1u << stage)) | (ph << stage);
                        if (++stage == kStages) { stage = 0; ph ^= 1u; }
                    }
                }
            }
            if (aborted)
                for (int s = 0; s < kStages; ++s)
                    if (issued_mask & (1u << s)) mbar_wait(smem_u32(&bar_full[s]), (issued_phase >> s) & 1u, nullptr);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ------------------------------------------------ MMA issuer
            int stage = 0;
            uint32_t ph = 0;
            int it = 0;
            uint32_t slot_col = 0;
            bool aborted = false;
            while (true) {
                if (!wait_fast(smem_u32(&bar_full[stage]), ph, &s_abort)) { aborted = true; break; }
                const StageInfo si = info[stage];
                if (si.block < 0) break;
                const int phase = si.flags & ST_PHASE;
                const bool first = si.flags & ST_FIRST;
                if (first) {
                    // slot of this Gram: the (2 it + phase)-th use of the 3-slot ring
                    const int u = 2 * it + phase;
                    const int q = u % 3;
                    const uint32_t par = ((uint32_t)(u / 3) & 1u) ^ 1u;
                    if (!wait_fast(smem_u32(&bar_slot_free[q]), par, &s_abort)) {
                        aborted = true;
                        break;
                    }
                    slot_col = (uint32_t)(q * kSlotCols);
                }
                tc_fence_after();
                const bool mn = si.flags & ST_MN;
                const bool wide = si.flags & ST_WIDE;
                const int npad = (si.dpos + si.nk + 15) & ~15;  // <= 144
                const uint32_t d_main = tmem + slot_col, d_corner = tmem + slot_col + kCornerCol;
                const uint32_t addr = smem_u32(stage_ptr(stage));
                const uint32_t sub_bytes = (uint32_t)si.sub_bytes;
                if (mn) {
                    mma_stage<T, true>(d_main, d_corner, addr, sub_bytes, (uint32_t)si.box_bytes, si.nsub,
                                       idesc_of<T>(npad, true), idesc_of<T>(16, true), first, wide);
                } else {
                    mma_stage<T, false>(d_main, d_corner, addr, sub_bytes, 0u, si.nsub, idesc_of<T>(npad, false),
                                        idesc_of<T>(16, false), first, wide);
                }
                tc_commit(smem_u32(&bar_empty[stage]));
                if ((si.flags & ST_LAST) && phase == 1) {
                    tc_commit(smem_u32(&bar_tfull[it & 1]));
                    ++it;
                }
                if (++stage == kStages) { stage = 0; ph ^= 1u; }
            }
            if (aborted) {
                tc_commit(smem_u32(&bar_drain));
                mbar_wait(smem_u32(&bar_drain), 0u, nullptr);
            }
        }
    } else {
        // ------------------------------------------------ norms, block epilogue
        const int t = threadIdx.x - 64;
        const int cw = warp - 2;  // converter warp 0..15
        int stage = 0, bslot = 0;
        uint32_t ph = 0, bph = 0;
        int it = 0;
        int cs_uses = 0;
        const uint32_t cs_bar = smem_u32(&bar_cs);
        bool aborted = false;
        while (!aborted) {
            if (!wait_fast(smem_u32(&bar_bfull[bslot]), bph, &s_abort)) break;
            const BlockInfo bi = binfo[bslot];
            if (bi.kb < 0) break;
            const int nk = bi.nk, dpos = bi.dpos;
            // block starts relative to the window (read in the epilogue, after the converter syncs)
            if (t <= bi.nblk) s_seg[t] = (int)(tab.prob[bi.q].off[bi.kb + t] - bi.lo);

            if constexpr (STATS) {
                // ---- squares of every element, per vector
                for (int phase = 0; phase < 2 && !aborted; ++phase) {
                    bool reduce_parts = true;
                    if (dpos + nk <= 128) {
                        // every lane on whole 16-byte chunks (strided: partial sums per warp in
                        // part[]; contiguous: x_i or y_i written directly)
                        if (!wait_fast(smem_u32(&bar_full[stage]), ph, &s_abort)) { aborted = true; break; }
                        const bool mn = info[stage].flags & ST_MN;
                        const bool ok =
                            mn ? squares_strided<T>(base, info, bar_full, bar_empty, stage, ph, &s_abort, cw, lane, nk,
                                                    dpos, part)
                               : squares_contig<T>(base, info, bar_full, bar_empty, stage, ph, &s_abort, cw, lane, nk,
                                                   dpos, xy_ff[phase]);
                        if (!ok) { aborted = true; break; }
                        reduce_parts = mn;
                    } else {
                        const int r = squares_wide<T>(base, info, bar_full, bar_empty, stage, ph, &s_abort, cw, lane,
                                                      part);
                        if (r < 0) { aborted = true; break; }
                        stage = r & 0xff;
                        ph = (uint32_t)(r >> 8);
                    }
                    // x_i (phase 0) or y_i (phase 1): the float-float sum of the warps' shares, one
                    // FP64 conversion per vector
                    conv_sync(cs_bar, cs_uses, &s_abort);
                    if (reduce_parts && t < kMaxBlock) {
                        FF sum;
                        sum.zero();
#pragma unroll
                        for (int w = 0; w < kConvWarps; ++w) {
                            const float2 v2 = part[STATS ? w : 0][t];
                            FF o;
                            o.hi = v2.x;
                            o.lo = v2.y;
                            sum.add(o);
                            sum.renorm();
                        }
                        xy_ff[STATS ? phase : 0][t] = make_float2(sum.hi, sum.lo);
                    }
                    conv_sync(cs_bar, cs_uses, &s_abort);  // part[] is reused by the next phase
                }
                if (aborted) break;
            }

            // ---- window epilogue
            const long long kb = bi.kb;
            const long long lo = bi.lo;
            const int nblk = bi.nblk;
            const StatsProblem& pr = tab.prob[bi.q];
            if constexpr (!STATS) conv_sync(cs_bar, cs_uses, &s_abort);  // s_seg[] is visible
            if (STATS && t < nk) {
                const float2 xf = xy_ff[0][t], yf = xy_ff[STATS ? 1 : 0][t];
                pr.x[lo + t] = (double)xf.x + (double)xf.y;
                pr.y[lo + t] = (double)yf.x + (double)yf.y;
            }
            // off-diagonal Gram products from TMEM: rows = lanes of this warp's quadrant (operand
            // rows 0..127), the ten 16-column chunks of a slot split between the quadrant's four
            // warps; a product counts when both vectors belong to the same block of the window
            FF offf;
            offf.zero();
            FF2 offp;  // main-Gram products, two columns at a time
            offp.zero();
            const int u0 = 2 * it;
            const int q0 = u0 % 3, q1 = (u0 + 1) % 3;
            const int q4 = warp & 3, quarter = cw >> 2;
            const int r = 32 * q4 + lane;  // operand row
            if (wait_fast(smem_u32(&bar_tfull[it & 1]), (uint32_t)(it >> 1) & 1u, &s_abort)) {
                tc_fence_after();
                const int end = dpos + nk;
                const bool wide = end > 128;  // a window of one block
                // the block of operand row r spans operand rows blo .. bhi - 1
                int blo = 0, bhi = 0;
                const int v = r - dpos;
                if (v >= 0 && v < nk) {
                    int ja = 0, jb = nblk - 1;  // the last block starting at or before v
                    while (ja < jb) {
                        const int mid = (ja + jb + 1) >> 1;
                        if (s_seg[mid] <= v) ja = mid;
                        else jb = mid - 1;
                    }
                    blo = dpos + s_seg[ja];
                    bhi = dpos + s_seg[ja + 1];
                }
                // chunks holding no column of any of the warp's rows' blocks are skipped (the TMEM
                // loads are warp-wide, so the test is too)
                const int w_hi = __reduce_max_sync(0xffffffffu, bhi);
                const int w_lo = __reduce_min_sync(0xffffffffu, bhi > blo ? blo : 1 << 20);
                const uint32_t lane_base = tmem + ((uint32_t)(32 * q4) << 16);
#pragma unroll 1
                for (int cchunk = quarter; cchunk < kSlotCols / 16; cchunk += 4) {
                    const int c0 = 16 * cchunk;
                    if ((c0 >= w_hi || c0 + 16 <= w_lo) && !(wide && c0 >= kCornerCol)) continue;
                    uint32_t gm[16], gn[16];
                    TMEM_LD_32X32B_X16(lane_base + (uint32_t)(q0 * kSlotCols + c0), gm);
                    TMEM_LD_32X32B_X16(lane_base + (uint32_t)(q1 * kSlotCols + c0), gn);
                    tmem_ld_wait();
                    if (c0 < kCornerCol) {
                        // main Gram: operand rows r (< 128) and col; the missing rows >= 128 of a
                        // wide block are the transposes of these columns.  Two columns per paired
                        // instruction; a column outside the row's block adds an exact zero.
#pragma unroll
                        for (int e = 0; e < 16; e += 2) {
                            float2 a2, b2;
                            {
                                const int col = c0 + e;
                                const bool in = col >= blo && col < bhi && col != r;
                                const float g = __uint_as_float(gm[e]);
                                a2.x = in ? (col >= 128 ? 2.0f * g : g) : 0.f;
                                b2.x = in ? __uint_as_float(gn[e]) : 0.f;
                            }
                            {
                                const int col = c0 + e + 1;
                                const bool in = col >= blo && col < bhi && col != r;
                                const float g = __uint_as_float(gm[e + 1]);
                                a2.y = in ? (col >= 128 ? 2.0f * g : g) : 0.f;
                                b2.y = in ? __uint_as_float(gn[e + 1]) : 0.f;
                            }
                            offp.add_prod(a2, b2);
                        }
                        continue;
                    }
                    // the corner chunk of a wide block: operand rows R0 + r (>= 128 counted) and
                    // 128 + (col - 144)
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const int rr = r + TR::kCornerRow0, cc = 128 + e;
                        if (rr >= 128 && rr < end && cc < end && cc != rr)
                            offf.add_prod(__uint_as_float(gm[e]), __uint_as_float(gn[e]));
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(smem_u32(&bar_slot_free[q0]));
                    mbar_arrive(smem_u32(&bar_slot_free[q1]));
                }
            } else {
                aborted = true;
            }
            ++it;
            offf.add(offp.both());
            offf.renorm();
            rowpart[quarter][r] = make_float2(offf.hi, offf.lo);
            conv_sync(cs_bar, cs_uses, &s_abort);
            // per block of the window: warp cw takes blocks cw, cw + 16, ...; its lanes run over the
            // block's vectors from the block's first, so the sums do not depend on where the block
            // sits in its window.  Every sum is float-float on the FP32 pipe (GB300's FP64 pipe is
            // slow: FP64 square roots and sums took half of this epilogue): w_i = sqrt(x_i y_i) from
            // a float-float product and square root, converted to FP64 once per block.  A warp
            // whose x_i, y_i or x_i y_i leave [2^-100, 2^120] (where float-float loses digits or
            // overflows) takes the FP64 path for its block instead.
            for (int j = cw; j < nblk; j += kConvWarps) {
                const int b0 = s_seg[j], b1 = s_seg[j + 1];
                const long long k = kb + j;
                const bool ok = b0 >= 0 && b1 > b0 && b1 <= nk;
                FF off, fa, fs, fx, fy;
                off.zero();
                fa.zero(); fs.zero(); fx.zero(); fy.zero();
                bool in_range = true;
                if (ok) {
                    for (int i = b0 + lane; i < b1; i += 32) {
                        const int rr = dpos + i;
                        if (rr < 128) {
#pragma unroll
                            for (int qq = 0; qq < 4; ++qq) {
                                FF o;
                                o.hi = rowpart[qq][rr].x;
                                o.lo = rowpart[qq][rr].y;
                                off.add(o);
                                off.renorm();
                            }
                        }
                        if (STATS) {
                            FF xi, yi;
                            xi.hi = xy_ff[0][i].x; xi.lo = xy_ff[0][i].y;
                            yi.hi = xy_ff[STATS ? 1 : 0][i].x; yi.lo = xy_ff[STATS ? 1 : 0][i].y;
                            const FF xy = ff_mul(xi, yi);
                            auto ok_range = [](float v) { return v == 0.f || (v >= 0x1p-100f && v <= 0x1p120f); };
                            in_range = in_range && ok_range(xi.hi) && ok_range(yi.hi) && ok_range(xy.hi);
                            fa.add(ff_sqrt(xy));
                            fa.renorm();
                            fs.add(xy);
                            fs.renorm();
                            fx.add(xi);
                            fx.renorm();
                            fy.add(yi);
                            fy.renorm();
                        }
                    }
                }
                auto warp_ff = [&](FF& v) {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        FF other;
                        other.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
                        other.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
                        v.add(other);
                        v.renorm();
                    }
                };
                warp_ff(off);
                double sa = 0.0, ss = 0.0, sx = 0.0, sy = 0.0;
                if (STATS) {
                    if (__all_sync(0xffffffffu, in_range)) {
                        warp_ff(fa);
                        warp_ff(fs);
                        warp_ff(fx);
                        warp_ff(fy);
                        if (lane == 0) {  // FP64 once per block
                            sa = fa.value();
                            ss = fs.value();
                            sx = fx.value();
                            sy = fy.value();
                        }
                    } else if (ok) {
                        for (int i = b0 + lane; i < b1; i += 32) {
                            const double xi = (double)xy_ff[0][i].x + (double)xy_ff[0][i].y;
                            const double yi = (double)xy_ff[STATS ? 1 : 0][i].x + (double)xy_ff[STATS ? 1 : 0][i].y;
                            const double xy = __dmul_rn(xi, yi);
                            sa += sqrt(xy);
                            ss += xy;
                            sx += xi;
                            sy += yi;
                        }
                        sa = warp_sum(sa);
                        ss = warp_sum(ss);
                        sx = warp_sum(sx);
                        sy = warp_sum(sy);
                    }
                }
                if (lane == 0) {
                    if (!ok) {
                        set_status(pr.st, BMM_ERR_SHAPE, (int)k);
                        if (STATS) { pr.a[k] = 0.0; pr.s[k] = 0.0; pr.mf[k] = 0.0; pr.nf[k] = 0.0; }
                        pr.f[k] = 0.0;
                    } else {
                        const double sk = STATS ? ss : pr.s[k];
                        if (STATS) { pr.a[k] = sa; pr.s[k] = ss; pr.mf[k] = sx; pr.nf[k] = sy; }
                        pr.f[k] = sk + off.value();
                    }
                }
            }
            conv_sync(cs_bar, cs_uses, &s_abort);  // xy_sum[], rowpart[] and s_seg[] are reused by the next window
            if (lane == 0) mbar_arrive(smem_u32(&bar_bempty[bslot]));
            if (++bslot == kBlockSlots) { bslot = 0; bph ^= 1u; }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
    if (threadIdx.x == 0 && s_abort)
        for (int q = 0; q < tab.count; ++q) set_status(tab.prob[q].st, BMM_ERR_TIMEOUT, 2);
}

// Strided operands (vectors along the storage rows' inner dimension) feed the MMA MN-major: FP32
// wants 32-byte swizzle atoms, BF16 the plain 128-byte swizzle; contiguous ones are K-major with the
// plain 128-byte swizzle.  Boxes are 128 bytes wide and box_rows high.
template <typename T>
bool make_map(CUtensorMap* mp, const void* ptr, int64_t rows, int64_t cols, int64_t ld, bool strided, int box_rows) {
    // looked up once; a function-local static is initialised once even under concurrent callers
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
        void* q = nullptr;
        cudaDriverEntryPointQueryResult r;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &q, 12000, cudaEnableDefault, &r) != cudaSuccess ||
            r != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(q);
    }();
    if (fn == nullptr) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * (int64_t)sizeof(T))};
    cuuint32_t box[2] = {(cuuint32_t)Tr<T>::E, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return fn(mp, Tr<T>::kTmaType, 2, const_cast<void*>(ptr), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              strided ? Tr<T>::kMnSwizzle : CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename T>
bool maps_of(OperandMaps& om, const VecSet& v) {
    const bool strided = v.mode == VEC_STRIDED;
    const int64_t rows = strided ? v.len : v.count, cols = strided ? v.count : v.len;
    for (int g = 0; g < (strided ? 2 : kMaxKMaps); ++g)
        if (!make_map<T>(&om.map[g], v.data, rows, cols, v.ld, strided, strided ? kMnRows << g : 32 * (g + 1)))
            return false;
    return true;
}

template <typename T>
bool fill_problem(StatsProblem* pr, const StatsArgs& g) {
    if (!maps_of<T>(pr->mM, g.vM) || !maps_of<T>(pr->mN, g.vN)) return false;
    pr->off = g.off;
    pr->K = g.K;
    pr->n = g.n;
    pr->m = g.vM.len;
    pr->p = g.vN.len;
    pr->x = g.x; pr->y = g.y; pr->a = g.a; pr->s = g.s; pr->mf = g.mf; pr->nf = g.nf; pr->f = g.f;
    pr->st = g.st;
    pr->wins = g.wins;
    pr->M_strided = g.vM.mode == VEC_STRIDED;
    pr->N_strided = g.vN.mode == VEC_STRIDED;
    return true;
}

template <typename T, bool STATS, int G>
cudaError_t launch_table(const StatsTable<G>& tab, int* counter, cudaStream_t s) {
    static std::atomic<bool> attr{false};  // set once; setting the attribute again is harmless
    if (!attr.load()) {
        cudaError_t e = cudaFuncSetAttribute(blockstats_tc_kernel<T, STATS, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
        if (e != cudaSuccess) return e;
        attr.store(true);
    }
    if (tab.total_blocks == 0) return cudaSuccess;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = (int)imin(tab.total_blocks, sms);
    // the windows of every product (and the zeroed work counter), then the pass over them
    (count_launch(), stats_windows_kernel<T, G><<<tab.count, kWinThreads, 0, s>>>(tab, counter, 3 * grid / 4));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    (count_launch(), blockstats_tc_kernel<T, STATS, G><<<grid, kThreads, kSmem, s>>>(tab, counter));
    return cudaGetLastError();
}

template <typename T, bool STATS>
cudaError_t launch_grouped_t(const StatsArgs* args, int64_t count, int* counter, cudaStream_t s) {
    if (count == 1) {  // a single product: a one-entry table keeps the kernel parameter small
        StatsTable<1> one;
        one.count = 1;
        if (!fill_problem<T>(&one.prob[0], args[0])) return cudaErrorInvalidValue;
        one.total_blocks = args[0].K;
        return launch_table<T, STATS, 1>(one, counter, s);
    }
    static thread_local StatsTable<kMaxProducts> tab;  // host-side staging of the kernel parameter, one per host thread (~32 KB)
    tab.count = 0;
    tab.total_blocks = 0;
    for (int64_t i = 0; i <= count; ++i) {
        if ((i == count || tab.count == kMaxProducts) && tab.count > 0) {
            cudaError_t e = launch_table<T, STATS, kMaxProducts>(tab, counter, s);
            if (e != cudaSuccess) return e;
            tab.count = 0;
            tab.total_blocks = 0;
        }
        if (i == count) break;
        StatsProblem& pr = tab.prob[tab.count];
        if (!fill_problem<T>(&pr, args[i])) return cudaErrorInvalidValue;
        tab.total_blocks += args[i].K;
        ++tab.count;
    }
    return cudaSuccess;
}

}  // namespace

bool blockstats_tc_supported(const VecSet& vM, const VecSet& vN, int64_t max_nk) {
    if (vM.dtype != vN.dtype || (vM.dtype != BMM_F32 && vM.dtype != BMM_BF16) || max_nk > kMaxBlock) return false;
    if (vM.len < 1 || vN.len < 1) return false;  // every block needs stages in both phases
    const int align = vM.dtype == BMM_F32 ? 4 : 8;  // elements per 16 bytes
    if ((vM.ld % align) || (vN.ld % align)) return false;
    if ((reinterpret_cast<uintptr_t>(vM.data) & 15) || (reinterpret_cast<uintptr_t>(vN.data) & 15)) return false;
    if (vM.len > 0x7fffffffLL || vN.len > 0x7fffffffLL || vM.count > 0x7fffffffLL) return false;
    return tc_gemm_supported();
}

cudaError_t launch_blockstats_tc(const VecSet& vM, const VecSet& vN, const int64_t* off, int64_t K, int64_t n,
                                 bool stats, int* counter, int* wins, double* x, double* y, double* a, double* ssum,
                                 double* mf, double* nf, double* f, DevStatus* st, cudaStream_t s) {
    const StatsArgs g{vM, vN, off, K, n, x, y, a, ssum, mf, nf, f, st, wins};
    return launch_blockstats_tc_grouped(&g, 1, stats, counter, s);
}

cudaError_t launch_blockstats_tc_grouped(const StatsArgs* args, int64_t count, bool stats, int* counter, cudaStream_t s) {
    // one launch per element type and kMaxProducts products
    for (int pass = 0; pass < 2; ++pass) {
        const int dtype = pass == 0 ? BMM_F32 : BMM_BF16;
        int64_t i = 0;
        while (i < count) {
            // a run of consecutive products of this element type (others are skipped here)
            if (args[i].vM.dtype != dtype) { ++i; continue; }
            int64_t j = i;
            while (j < count && args[j].vM.dtype == dtype) ++j;
            cudaError_t e;
            if (dtype == BMM_F32)
                e = stats ? launch_grouped_t<float, true>(args + i, j - i, counter, s)
                          : launch_grouped_t<float, false>(args + i, j - i, counter, s);
            else
                e = stats ? launch_grouped_t<__nv_bfloat16, true>(args + i, j - i, counter, s)
                          : launch_grouped_t<__nv_bfloat16, false>(args + i, j - i, counter, s);
            if (e != cudaSuccess) return e;
            i = j;
        }
    }
    return cudaSuccess;
}

}  // namespace bmm
