/*
 * bmm.h -- C ABI of the GB300 (sm_103a) randomized block matrix multiplication library.
 *
 * Method: Niu & Li, "Optimal Sampling Algorithms for Block Matrix Multiplication".
 * MN (M m x n, N n x p) is approximated by sampling outer products M^{k(i)} N_{k(i)}
 * inside each of K contraction blocks (Alg. 2, eq. 3.3), or whole blocks (the
 * baselines of eq. 1.2 and eq. 1.4).  A product runs as
 *
 *     bmm_probs -> bmm_blocksizes -> bmm_sample -> bmm_apply   (+ bmm_backward)
 *
 * Conventions shared by every call
 *   - Every pointer inside the descriptors and every array argument is DEVICE memory
 *     owned by the caller, unless marked "host".  The library allocates nothing, creates no
 *     stream and keeps no state between calls beyond a diagnostic launch counter, the cached
 *     driver entry point of the tensor-map encoder, the GEMM tile table (bmm_autotune_*) and the
 *     device address of bmm_probs_static's array; all work is enqueued on the caller's stream and
 *     the calls return without synchronising (except bmm_read_device_status and
 *     bmm_autotune_gemm, which times with two events it creates and destroys itself).
 *   - Argument, shape and feasibility errors are returned before anything is launched.
 *     Conditions only the GPU can see (non-finite data, bad offsets, a probability
 *     segment with zero mass, a bounded wait that expired) are recorded in a sticky
 *     status word at the start of the workspace; read it with bmm_read_device_status.
 *     Nothing traps.
 *   - Workspace: ws must be 256-byte aligned and hold bmm_workspace_size(...) bytes.
 *     Its first 256 bytes are the status block; bmm_clear_device_status zeroes it.
 *     The rest is scratch that no call preserves.
 *   - Calls that share a workspace must be ordered (same stream or events).
 */
#ifndef BMM_H_
#define BMM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st* bmm_stream_t;

typedef enum {
    BMM_OK = 0,
    BMM_ERR_ARG = 1,         /* null pointer, unknown enum, bad probability vector */
    BMM_ERR_SHAPE = 2,       /* inconsistent dimensions, leading dimensions or block offsets */
    BMM_ERR_DTYPE = 3,       /* element type not supported by this call */
    BMM_ERR_INFEASIBLE = 4,  /* budget outside what Alg. 2 allows (c < K or c > n) */
    BMM_ERR_NONFINITE = 5,   /* NaN or Inf met in the data (device-detected) */
    BMM_ERR_WORKSPACE = 6,   /* workspace too small or misaligned */
    BMM_ERR_CUDA = 7,        /* a CUDA runtime call failed */
    BMM_ERR_TIMEOUT = 8,     /* a bounded device-side wait expired; the kernel returned early */
    BMM_ERR_UNSUPPORTED = 9  /* valid request this library or device does not support */
} bmm_status;

/* Element types. */
enum { BMM_F64 = 0, BMM_F32 = 1, BMM_BF16 = 2 };
/* Storage orders. ROW: element (r, c) at data[r * ld + c]; COL: at data[c * ld + r]. */
enum { BMM_ROW_MAJOR = 0, BMM_COL_MAJOR = 1 };

/* Probabilities (Sec. 1 and Table 2). */
enum {
    BMM_P_COL_OPT = 0,      /* eq. 3.8: p_{k_i} = ||M^{k(i)}|| ||N_{k(i)}|| / a_k, per column, sums to 1 in each block */
    BMM_P_COL_UNIFORM = 1,  /* Table 2 (UU, ONU pilot): p_{k_i} = 1/n_k */
    BMM_P_BLK_PRODNORM = 2, /* eq. 1.2: p_k = ||M^k N_k||_F / sum_j ||M^j N_j||_F, per block */
    BMM_P_BLK_NORMPROD = 3  /* eq. 1.4 (SSM): p_k = ||M^k||_F ||N_k||_F / sum_j (...), per block */
};

/* Block sizes (Thm 2.2, Sec. 3). */
enum {
    BMM_CK_OPT = 0,   /* eq. 3.9: c_k proportional to (a_k^2 - ||M^k N_k||_F^2)^{1/2}; needs st->f */
    BMM_CK_HAT = 1,   /* eq. 4.2: c_k proportional to a_k */
    BMM_CK_TILDE = 2, /* eq. 4.7 / Alg. 3: c_k proportional to |a_k^2 - ||C^{0k} D_{0k}||_F^2|^{1/2} */
    BMM_CK_EQUAL = 3  /* Table 2 (UU): c_k = c/K */
};

/* How ||M^k N_k||_F^2 is computed by bmm_probs. */
enum {
    BMM_F_NONE = 0,  /* not computed (st->f untouched) */
    BMM_F_EXACT = 1, /* trace identity <M^kT M^k, N_k N_kT>_F with FP64-accurate sums on CUDA cores */
    BMM_F_TC = 2     /* s_k (exact) + off-diagonal part of the trace identity from TF32 tcgen05 Grams,
                        fused with the statistics pass (FP32 data, row- or column-major, ld % 4 == 0,
                        blocks of at most 128); other inputs fall back to BMM_F_EXACT */
};
/* Flag or-ed into bmm_probs' fmode: st already holds this M, N's statistics.  The pass
 * over M and N is skipped; f is computed if fmode says so (else st->f is used as given),
 * then p.  COL_UNIFORM never reads st, M or N. */
enum { BMM_REUSE_STATS = 0x100 };

/* Sampling unit. */
enum {
    BMM_UNIT_COLUMN = 0, /* Alg. 2: idx are column indices of M (row indices of N) in [0, n) */
    BMM_UNIT_BLOCK = 1   /* block sampling: idx are block indices in [0, K) */
};

/* Arithmetic of the sampled product. */
enum {
    BMM_GEMM_F64 = 0,        /* FP64 operands and accumulation on CUDA cores; out is FP64 */
    BMM_GEMM_BF16 = 1,       /* BF16 operands on tcgen05 tensor cores, FP32 accumulation; out is FP32 */
    BMM_GEMM_SPLIT_BF16 = 2, /* x = hi + lo (both BF16); hi*hi + hi*lo + lo*hi on tcgen05, FP32 accumulation */
    BMM_GEMM_E4M3 = 3        /* FP8 e4m3 operands on tcgen05 (kind::f8f6f4), FP32 accumulation; out is FP32.
                                Per drawn outer product t, C^(t) is scaled by 2^(e_t) and D_(t) by 2^(-e_t)
                                (balancing their magnitudes; the product is unchanged), and each operand by
                                one power of two that brings its largest value to at most 448, restored in
                                the epilogue.  bmm_apply / bmm_apply_batched only. */
};

/* Purposes folded into a stream id: stream_id = (replicate << 8) | purpose. */
enum { BMM_PURPOSE_MAIN = 0, BMM_PURPOSE_PILOT = 1 };

/* A dense matrix in device memory. */
typedef struct {
    const void* data;  /* device pointer, aligned to its element size */
    int64_t rows;      /* logical rows */
    int64_t cols;      /* logical columns */
    int64_t ld;        /* leading dimension in elements (>= cols for ROW, >= rows for COL) */
    int32_t dtype;     /* BMM_F64 / BMM_F32 / BMM_BF16 */
    int32_t layout;    /* BMM_ROW_MAJOR / BMM_COL_MAJOR */
} bmm_mat;

/* The K contraction blocks of eq. 2.3: block k holds indices [offsets[k], offsets[k+1]). */
typedef struct {
    int64_t K;               /* number of blocks, >= 1 */
    int64_t n;               /* contraction length, = offsets[K] */
    int64_t max_nk;          /* host: largest block size (sizes workspace for block sampling) */
    const int64_t* offsets;  /* device [K+1]: offsets[0] = 0, strictly increasing, offsets[K] = n */
} bmm_blocks;

/* Statistics of Sec. 2-3, all device FP64 arrays owned by the caller. */
typedef struct {
    double* x;   /* [n] ||M^{(i)}||_2^2 */
    double* y;   /* [n] ||N_{(i)}||_2^2 */
    double* a;   /* [K] a_k = sum_{i in k} ||M^{k(i)}|| ||N_{k(i)}||   (eq. 3.8 denominator) */
    double* s;   /* [K] s_k = sum_{i in k} ||M^{k(i)}||^2 ||N_{k(i)}||^2 */
    double* mf;  /* [K] ||M^k||_F^2 */
    double* nf;  /* [K] ||N_k||_F^2 */
    double* f;   /* [K] ||M^k N_k||_F^2 (eq. 1.2, eq. 3.9); may be NULL when not requested */
} bmm_stats;

/*
 * Bytes of workspace that any call below needs for this problem.  unit is the sampling
 * unit that bmm_apply / bmm_backward will see; max_draws the largest draw count (c, and
 * the Alg. 3 pilot's total draws) passed to any call; gemm_mode the largest mode used
 * (SPLIT_BF16 needs the most).  Returns 0 on invalid input.  Host-only, no CUDA calls.
 */
size_t bmm_workspace_size(const bmm_mat* M, const bmm_mat* N, const bmm_blocks* B, int32_t unit,
                          int64_t max_draws, int32_t gemm_mode);

/*
 * bmm_probs -- statistics and sampling probabilities.
 * Sec. 2-3: x_i, y_i, a_k, s_k, ||M^k||_F^2, ||N_k||_F^2 in one read of M and N,
 * optionally f_k = ||M^k N_k||_F^2 (fmode), then p by pkind (eq. 3.8, Table 2,
 * eq. 1.2, eq. 1.4).  M is m x n, N is n x p, either storage order, same dtype.
 *   p_out: [n] for the column kinds, [K] for the block kinds.  May be NULL.
 *   st:    all pointers but f required; f required when fmode != BMM_F_NONE or
 *          pkind == BMM_P_BLK_PRODNORM.  With BMM_REUSE_STATS the pass over M and N is
 *          skipped and only st->f (if computed) is written.
 * A block with a_k = 0 gets uniform column probabilities; all-zero block weights give 1/K.
 */
bmm_status bmm_probs(const bmm_mat* M, const bmm_mat* N, const bmm_blocks* B,
                     int32_t pkind, int32_t fmode, double* p_out, const bmm_stats* st,
                     void* ws, size_t ws_bytes, bmm_stream_t stream);

/*
 * bmm_probs_batched -- bmm_probs for `count` independent products (arrays of descriptors, one
 * workspace per product), in as few launches as the kernel-parameter limit allows.  For each i
 * the results are those of bmm_probs(&Ms[i], &Ns[i], &Bs[i], pkind, fmode, p_outs ? p_outs[i] :
 * NULL, &sts[i], ws[i], ws_bytes[i], stream).  Products that the tensor-core pass supports
 * (fmode BMM_F_TC, FP32 or BF16 inputs with 16-byte aligned leading dimensions, n_k <= 128) share
 * launches of up to ~19 products whose CTAs draw blocks from one work counter (in ws of the first
 * such product); the others are computed one by one.  All work is on `stream`; nothing is
 * synchronised or allocated, so the call can be recorded in a CUDA graph.  Errors: as bmm_probs,
 * the first failing product's status is returned and later products are not started.
 */
bmm_status bmm_probs_batched(int64_t count, const bmm_mat* Ms, const bmm_mat* Ns, const bmm_blocks* Bs,
                             int32_t pkind, int32_t fmode, double* const* p_outs, const bmm_stats* sts,
                             void* const* ws, const size_t* ws_bytes, bmm_stream_t stream);

/*
 * bmm_probs_static -- bmm_probs without a workspace.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory at call time, such as a plugin whose
 * host program owns all GPU memory through a fixed pool, or a latency-critical loop that cannot
 * afford cudaMalloc's implicit synchronisation.  The statistics pass keeps its partial column sums
 * in a 16 MiB array compiled into the library (held on every GPU that loads it until exit);
 * problems needing more are rejected with BMM_ERR_WORKSPACE before any launch.
 *   pkind:      BMM_P_COL_OPT, BMM_P_COL_UNIFORM or BMM_P_BLK_NORMPROD (no ||M^k N_k||_F).
 *   status_out: device int32[2], 4-byte aligned, zeroed by the caller; receives what bmm_probs
 *               records in the workspace status block (first error code, detail).
 *   M, N, B, p_out, st: as for bmm_probs (st->f unused), checked by the same tests in the same order
 *               with the same codes; a null or misaligned status_out is BMM_ERR_ARG.
 * The first call on each device looks up the array's address with that device current; make it
 * before any stream capture starts.  The address is kept for the life of the process, so resetting
 * a device after its first call (cudaDeviceReset) is not supported.  Calls share the array: calls
 * that overlap on the GPU race.
 */
bmm_status bmm_probs_static(const bmm_mat* M, const bmm_mat* N, const bmm_blocks* B, int32_t pkind,
                            double* p_out, const bmm_stats* st, int32_t* status_out, bmm_stream_t stream);

/*
 * bmm_blocksizes -- integer block sizes c_k for Alg. 2 (Thm 2.2 eq. 3.9, eq. 4.2,
 * eq. 4.7 with Alg. 3 step 1, Table 2 c/K).  c is the total number of outer products
 * (the paper's c); K <= c <= n is required (each block gets 1 <= c_k <= n_k).
 * Weights g_k (all zero falls back to a_k, then to n_k) are turned into integers by the
 * largest FP64 lam with sum_k clamp(floor(lam g_k), 1, n_k) <= c, the remainder going one
 * each, in increasing k, to the blocks that grow at the next representable lam.
 *   st:          a (and f for BMM_CK_OPT) used; may be NULL for BMM_CK_EQUAL.
 *   pilot_idx, pilot_scale, pilot_per_block: BMM_CK_TILDE only -- the Alg. 3 step-1
 *                sample (draws of block k at positions [k*per_block, (k+1)*per_block),
 *                scale 1/(c0' p0) each), from which ||C^{0k} D_{0k}||_F^2 is computed.
 *   ck_out:      device int64 [K].   g_out, fhat_out: optional device FP64 [K].
 */
bmm_status bmm_blocksizes(const bmm_mat* M, const bmm_mat* N, const bmm_blocks* B,
                          const bmm_stats* st, int32_t ckind, int64_t c,
                          const int32_t* pilot_idx, const double* pilot_scale, int64_t pilot_per_block,
                          int64_t* ck_out, double* g_out, double* fhat_out,
                          void* ws, size_t ws_bytes, bmm_stream_t stream);

/*
 * bmm_blocksizes_batched -- bmm_blocksizes for `count` independent products in one launch (one CTA
 * per product, up to 400 per launch), for ckind BMM_CK_OPT, BMM_CK_HAT or BMM_CK_EQUAL (the Alg. 3
 * pilot form takes bmm_blocksizes).  For each i the results are those of
 * bmm_blocksizes(NULL, NULL, &Bs[i], &sts[i], ckind, cs[i], NULL, NULL, 0, ck_outs[i],
 * g_outs ? g_outs[i] : NULL, NULL, ws[i], ws_bytes[i], stream), bit for bit.  sts may be NULL for
 * BMM_CK_EQUAL.  Host-side checks of every product come before any launch; nothing is synchronised
 * or allocated (graph-capturable).
 */
bmm_status bmm_blocksizes_batched(int64_t count, const bmm_blocks* Bs, const bmm_stats* sts, int32_t ckind,
                                  const int64_t* cs, int64_t* const* ck_outs, double* const* g_outs,
                                  void* const* ws, const size_t* ws_bytes, bmm_stream_t stream);

/*
 * bmm_sample -- i.i.d. draws with replacement (Alg. 1 step 1(a), Alg. 2 step 1).
 * Philox4x32-10 with key (seed_lo, seed_hi) and counter (t_lo, t_hi, sid_lo, sid_hi) for
 * global draw number t gives r = (x1 << 32) | x0; W_j = floor(p_j 2^62); the draw is the
 * smallest j of its segment with prefix S_j > floor(r T / 2^64).
 *   BMM_UNIT_COLUMN: p is [n]; block k gets ck[k] draws (device int64 [K], sum = c),
 *                    numbered consecutively block after block; scale = 1/(c_k p_i) (eq. 3.2).
 *   BMM_UNIT_BLOCK:  p is [K]; c draws over the blocks; scale = 1/(c p_k); ck ignored.
 *   idx_out: device int32 [c] global indices; scale_out: device FP64 [c].
 * p must be finite in [0, 1] with non-zero mass in every segment (device-checked).
 */
bmm_status bmm_sample(const double* p, int32_t unit, const bmm_blocks* B, const int64_t* ck,
                      int64_t c, uint64_t seed, uint64_t stream_id,
                      int32_t* idx_out, double* scale_out,
                      void* ws, size_t ws_bytes, bmm_stream_t stream);

/*
 * bmm_sample_batched -- bmm_sample for `count` independent products (host arrays of length count:
 * p[i], Bs[i], ck[i] (column unit), cs[i] draws, seeds[i], stream_ids[i], idx_out[i], scale_out[i],
 * ws[i] / ws_bytes[i]) in three launches per up to 200 products.  For each i the draws are those of
 * bmm_sample(p[i], unit, &Bs[i], ck[i], cs[i], seeds[i], stream_ids[i], idx_out[i], scale_out[i], ws[i],
 * ws_bytes[i], stream), bit for bit (the same exact integer prefix sums).  Every product is checked on
 * the host before anything is launched; device-detected errors go to each product's status block.
 * Nothing is synchronised or allocated (graph-capturable).
 */
bmm_status bmm_sample_batched(int64_t count, const double* const* p, int32_t unit, const bmm_blocks* Bs,
                              const int64_t* const* ck, const int64_t* cs, const uint64_t* seeds,
                              const uint64_t* stream_ids, int32_t* const* idx_out, double* const* scale_out,
                              void* const* ws, const size_t* ws_bytes, bmm_stream_t stream);

/*
 * bmm_apply -- the sampled product CD = sum_t scale_t M^{(i_t)} N_{(i_t)} (eq. 3.3,
 * Alg. 2 step 4), or sum_t scale_t M^{k_t} N_{k_t} for BMM_UNIT_BLOCK.
 * Draws of the same index are one term: the draws are first reduced to their distinct indices,
 * ascending, each weighted by its multiplicity times its scale (the same sum; draws with
 * replacement repeat heavy columns, and one product's GEMM runs over the distinct ones).  Every draw
 * of an index must carry the same scale, as every draw of bmm_sample does (1/(c_k p_i), 1/(c p_k));
 * another scale is BMM_ERR_ARG on the device.  The distinct columns/rows are gathered, multiplied
 * by the square root of their weight (Alg. 1 step 1(b)), converted to the mode's operand type and
 * multiplied on the tensor cores.
 *   out: m x p, row-major (layout must be ROW), FP32 for the BF16 modes, FP64 for F64.
 *   accumulate: 0 -> out = CD, 1 -> out += CD.   count = number of draws (>= 0).
 */
bmm_status bmm_apply(const bmm_mat* M, const bmm_mat* N, const bmm_blocks* B, int32_t unit,
                     const int32_t* idx, const double* scale, int64_t count, int32_t gemm_mode,
                     const bmm_mat* out, int32_t accumulate,
                     void* ws, size_t ws_bytes, bmm_stream_t stream);

/* Parts of a column-sampled BF16 product for bmm_apply_part. */
enum {
    BMM_APPLY_GATHER_B = 0, /* gather N's drawn rows (rows row0, row1 ignored) */
    BMM_APPLY_GATHER_A = 1, /* gather M's drawn columns for output rows [row0, row1) */
    BMM_APPLY_GEMM = 2,     /* the GEMM of output rows [row0, row1) */
    BMM_APPLY_REDUCE = 3    /* repeated draws to distinct indices with summed scales (rows ignored) */
};

/*
 * bmm_apply_part -- one part of bmm_apply(M, N, B, BMM_UNIT_COLUMN, idx, scale, count, BMM_GEMM_BF16,
 * out, accumulate, ws, ws_bytes, stream), so that the caller can overlap the memory-bound gathers with
 * the tensor-core GEMM on streams of its own (eq. 3.3, Alg. 1 step 1(b)); the library creates no
 * stream or event.  The operands live in ws, laid out as bmm_apply lays them out, so all parts of one
 * product take the same ws and arguments.  REDUCE comes first: it reduces the draws to their
 * distinct indices with summed scales in ws (five small launches).  GATHER_B and every GATHER_A need
 * it complete and may then run in either order; the GEMM of rows [row0, row1) needs GATHER_B and the
 * GATHER_A of those rows complete (same stream, or ordered by the caller's events).  Every output
 * element is the full-depth dot product of a single bmm_apply, so any split of the rows gives the
 * same bits.  row0 and row1: multiples of 128 (row1 may be m), 0 <= row0 <= row1 <= m;
 * count >= 1.  Errors as bmm_apply; a bad part is BMM_ERR_ARG, a bad row range BMM_ERR_SHAPE.
 */
bmm_status bmm_apply_part(const bmm_mat* M, const bmm_mat* N, const bmm_blocks* B, const int32_t* idx,
                          const double* scale, int64_t count, const bmm_mat* out, int32_t accumulate, int32_t part,
                          int64_t row0, int64_t row1, void* ws, size_t ws_bytes, bmm_stream_t stream);

/*
 * bmm_apply_batched -- bmm_apply for `count` independent products of any shapes (the batched
 * configuration of many uneven products).  Host arrays of length count describe product i:
 * Ms[i], Ns[i], Bs[i], idx[i], scale[i], draws[i] (its draw count), outs[i], and ws[i] / ws_bytes[i],
 * a workspace of its own sized by bmm_workspace_size.  Each product's operands are gathered as in
 * bmm_apply; the BF16 / split-BF16 products then share persistent tcgen05 launches whose tile
 * scheduler walks the tiles of up to 80 products at a time (the FP64 mode runs per product).
 * Device-detected errors of the gathers go to each product's status block, those of the shared
 * GEMM launches to ws[0]'s.  Nothing is synchronised or allocated; the sequence can be recorded
 * into a CUDA graph together with the calls that produce idx and scale.
 */
bmm_status bmm_apply_batched(int64_t count, const bmm_mat* Ms, const bmm_mat* Ns, const bmm_blocks* Bs,
                             int32_t unit, const int32_t* const* idx, const double* const* scale,
                             const int64_t* draws, int32_t gemm_mode, const bmm_mat* outs, int32_t accumulate,
                             void* const* ws, const size_t* ws_bytes, bmm_stream_t stream);

/*
 * bmm_backward -- adjoint of bmm_apply for a loss l(CD) with G = dl/d(CD) (m x p).
 * The sample is not stored: it is redrawn from (p, ck, c, seed, stream_id) exactly as
 * bmm_sample draws it, and p is held constant (stop-gradient).  For every distinct index i
 * drawn with total weight w_i = sum_{t: i_t = i} scale_t:
 *     dM^{(i)} += w_i G N_{(i)}^T,   dN_{(i)} += w_i M^{(i)T} G
 * (whole blocks for BMM_UNIT_BLOCK).  Columns/rows never drawn are left unchanged
 * (accumulate = 1) or set to zero (accumulate = 0).  Either of dM, dN may be NULL.
 *   G: row-major, FP32 for the BF16 mode, FP64 for BMM_GEMM_F64.  dM, dN: either storage order,
 *   the dtype of G, or BF16 for the BF16 mode (each touched element is its FP32 value rounded to
 *   BF16 once, after adding the stored value when accumulate = 1).
 */
bmm_status bmm_backward(const bmm_mat* G, const bmm_mat* M, const bmm_mat* N, const bmm_blocks* B,
                        int32_t unit, const double* p, const int64_t* ck, int64_t c,
                        uint64_t seed, uint64_t stream_id, int32_t gemm_mode,
                        const bmm_mat* dM, const bmm_mat* dN, int32_t accumulate,
                        void* ws, size_t ws_bytes, bmm_stream_t stream);

/* ---- Error bars of the sampled product (Lemma 3.1, Thm 3.1, Remark 2.2, Thm 3.3, Thm 4.2, Thm 4.4).
 * Reports beside the product, not part of it; FP64 throughout; all arrays are device memory and
 * every call only enqueues work on the stream. */

/* Fields of the bmm_error_report output (FP64 [BMM_REPORT_LEN]); NaN where an input is missing. */
enum {
    BMM_REPORT_EXPECTED_SQ_ERROR = 0, /* E||MN - CD||_F^2 = sum_k (1/c_k)(sum_{i in k} x_i y_i / p_i - f_k)
                                         (Remark 2.2: eq. 3.7 summed over all entries); needs f */
    BMM_REPORT_EQ310 = 1,             /* (1/c) [sum_k (a_k^2 - f_k)^{1/2}]^2 (eq. 3.10); needs f */
    BMM_REPORT_THETA1 = 2,            /* min_k 1 - v_k^2, v_k^2 = f_k / a_k^2 (Thm 3.3), a_k > 0; needs f */
    BMM_REPORT_THETA2 = 3,            /* max_k 1 - v_k^2; needs f */
    BMM_REPORT_BETA = 4,              /* min(1, min_i p_i / p*_i), p* the eq. 3.8 probabilities */
    BMM_REPORT_M_FRO2 = 5,            /* ||M||_F^2 = sum_k mf_k */
    BMM_REPORT_N_FRO2 = 6,            /* ||N||_F^2 = sum_k nf_k */
    BMM_REPORT_PHI = 7,               /* phi of Thm 3.3 */
    BMM_REPORT_EQ311 = 8,             /* phi^2 / (beta c) ||M||_F^2 ||N||_F^2 (eq. 3.11) */
    BMM_REPORT_ETA312 = 9,            /* eta = phi + (theta2/theta1)^{1/2} (8/beta log(1/delta))^{1/2} */
    BMM_REPORT_EQ312 = 10,            /* eta^2 / (beta c) ||M||_F^2 ||N||_F^2: eq. 3.12, probability >= 1 - delta */
    BMM_REPORT_PHIHAT = 11,           /* (1 - beta (1 - theta2))^{1/2} (Thm 4.2) */
    BMM_REPORT_EQ43 = 12,             /* eq. 4.3 */
    BMM_REPORT_ETA44 = 13,            /* phihat + (8/beta log(1/delta))^{1/2} */
    BMM_REPORT_EQ44 = 14,             /* eq. 4.4 */
    BMM_REPORT_THETA1HAT = 15,        /* min_k |1 - fhat_k / a_k^2| (Thm 4.3); needs f and fhat */
    BMM_REPORT_THETA2HAT = 16,        /* max_k |1 - fhat_k / a_k^2| */
    BMM_REPORT_PHITILDE = 17,         /* phi-tilde of Thm 4.4 */
    BMM_REPORT_EQ48 = 18,             /* eq. 4.8 */
    BMM_REPORT_ETA49 = 19,
    BMM_REPORT_EQ49 = 20,             /* eq. 4.9, probability >= 1 - delta */
    BMM_REPORT_LEN = 21
};

/*
 * bmm_error_report -- the whole-matrix error quantities of Alg. 2 (fields above) from the
 * statistics (st->x, y, a, mf, nf required; st->f optional), the probabilities p [n], the block
 * sizes ck [K] (device int64; the expected error is exact for these integers, while the bounds of
 * Thm 3.3 / 4.2 are stated for the real-valued eq. 3.9 / 4.2 sizes) and their total c.  fhat
 * (optional, device FP64 [K]): the Alg. 3 pilot estimates of ||M^k N_k||_F^2.  delta in (0, 1).
 * report_out: device FP64 [BMM_REPORT_LEN].  One CTA; no workspace.
 */
bmm_status bmm_error_report(const bmm_blocks* B, const bmm_stats* st, const double* p, const int64_t* ck, int64_t c,
                            const double* fhat, double delta, double* report_out, bmm_stream_t stream);

/*
 * bmm_entry_variance -- Var[(CD)_hf] for each listed entry (Lemma 3.1, eq. 3.7: the sigma^2 of
 * Thm 3.1) for the design (p, ck) before any draw:
 *   BMM_UNIT_COLUMN: sum_k (1/c_k) [sum_{i in k, p_i > 0} M_hi^2 N_if^2 / p_i - (sum_{i in k, p_i > 0} M_hi N_if)^2],
 *                    p [n], ck [K];
 *   BMM_UNIT_BLOCK:  (1/c) [sum_{k: p_k > 0} ((M^k N_k)_hf)^2 / p_k - (sum_{k: p_k > 0} (M^k N_k)_hf)^2],
 *                    p [K], ck ignored, c draws.
 * Terms with zero probability are never drawn and are left out (the variance of the estimator as
 * run).  entries: device int64 [count][2] = (h, f); an entry outside the m x p product gets NaN.
 * sigma2_out: device FP64 [count].  Reads O(n) elements of M and N per entry; no workspace.
 */
bmm_status bmm_entry_variance(const bmm_mat* M, const bmm_mat* N, const bmm_blocks* B, int32_t unit,
                              const double* p, const int64_t* ck, int64_t c, const int64_t* entries, int64_t count,
                              double* sigma2_out, bmm_stream_t stream);

/*
 * bmm_entry_estimate -- from one sample (the idx, scale of bmm_sample, `draws` of them): each listed
 * entry's value (CD)_hf = sum_t Z_t, Z_t = scale_t M_{h,i_t} N_{i_t,f} in FP64, and the one-sample
 * estimate of its variance:
 *   BMM_UNIT_COLUMN: sum over blocks with c_k >= 2 of c_k/(c_k - 1) sum_{t in k} (Z_t - Zbar_k)^2
 *                    (the draws of block k are consecutive, c_k of them; blocks with c_k = 1 add their
 *                    value but no variance -- one draw carries no spread);
 *   BMM_UNIT_BLOCK:  c/(c - 1) sum_t (Z_t - Zbar)^2 with Z_t = scale_t (M^{k_t} N_{k_t})_hf.
 * Unbiased for the variance of the blocks it covers, so (CD)_hf +- z sqrt(s2) is the normal interval
 * of Thm 3.1.  ck: device int64 [K] (column unit; sum must equal draws, else BMM_ERR_SHAPE in the
 * workspace status).  cd_out, s2_out: device FP64 [count]; NaN for an entry outside the product.
 * ws: 256-byte aligned, at least 256 + 8 (K + 1) bytes rounded up to a multiple of 256 (any
 * bmm_workspace_size of the problem holds them); its status word records a draw-count mismatch.
 */
bmm_status bmm_entry_estimate(const bmm_mat* M, const bmm_mat* N, const bmm_blocks* B, int32_t unit,
                              const int64_t* ck, const int32_t* idx, const double* scale, int64_t draws,
                              const int64_t* entries, int64_t count, double* cd_out, double* s2_out, void* ws,
                              size_t ws_bytes, bmm_stream_t stream);

/*
 * bmm_f_tc_supported -- whether bmm_probs with BMM_F_TC computes ||M^k N_k||_F^2 of this problem on the
 * tensor cores (*uses_tc = 1: FP32 or BF16 data, 16-byte aligned base pointers and leading dimensions,
 * blocks of at most 128, an sm_103 device) or falls back to BMM_F_EXACT (*uses_tc = 0).  Host only,
 * no launch.  No counterpart in the paper (the path is this library's choice, eq. 1.2 / eq. 3.9 only
 * fix the value).  Errors: as the descriptor checks of bmm_probs; uses_tc NULL is BMM_ERR_ARG.
 */
bmm_status bmm_f_tc_supported(const bmm_mat* M, const bmm_mat* N, const bmm_blocks* B, int32_t* uses_tc);

/*
 * bmm_wait_selftest -- diagnostic, no counterpart in the paper.  Every pipelined kernel of the library
 * waits on barriers with a bound: past it the kernel gives up, records BMM_ERR_TIMEOUT in the status
 * word and returns, instead of hanging.  This call exercises that path on purpose: one CTA waits, with
 * the library's wait routine, on barriers that nothing completes (nothing else is in flight), gives up
 * after the bound (2 s) and records BMM_ERR_TIMEOUT with detail = the number of waits that gave up (2:
 * one on the time bound, one through the CTA's abort flag).  ws: 256-byte aligned, >= 256 bytes, its
 * status block zeroed by the caller; read it with bmm_read_device_status.
 */
bmm_status bmm_wait_selftest(void* ws, size_t ws_bytes, bmm_stream_t stream);

/* Synchronises the stream, then returns the first device-recorded error (BMM_OK if none). */
bmm_status bmm_read_device_status(const void* ws, bmm_stream_t stream);
/* Enqueues a reset of the device status word. */
bmm_status bmm_clear_device_status(void* ws, bmm_stream_t stream);
/* Static, NUL-terminated description of a status code. */
const char* bmm_status_string(bmm_status s);
/* Diagnostics (no counterpart in the paper): number of CUDA kernels this library has
 * enqueued since it was loaded, summed over all threads and calls. */
uint64_t bmm_launch_count(void);

/* ---- GEMM tile autotuner (no counterpart in the paper: a tuning aid for the batched
 * configuration, whose products have uneven m, p and L).
 * The sampled product of an m x n by n x p problem with L drawn outer products is, on the tensor
 * cores, a GEMM of M = m rows, N = p columns and depth K = L rounded up to 64 (BF16), 128 (e4m3)
 * or three times 64-rounded L (split BF16).  Its tile width and raster group (4, 8 or 16 row tiles
 * walked together for L2 reuse) come from a process-wide table keyed by the element kind and the
 * base-2 logarithms (rounded up) of M, N and K.  Tile widths: BN = 128 or 256 (one SM per 128 x BN
 * output tile), BMM_TILE_PAIR (two SMs of a thread-block cluster per 256 x 256 tile, cta_group::2
 * MMAs, each SM loading half of the tile's A and B rows) or BMM_TILE_PAIR_WIDE (the same per
 * 256 x 512 tile: fewer operand bytes per MMA, one accumulator, so its epilogue does not overlap
 * the next tile's MMAs).  Shapes not in the table use BN = 128
 * when N <= 128, else 256 when M <= 128, else BMM_TILE_PAIR, and a raster group of 8.  No choice changes any result bit: each output
 * element is the same dot product in the same order.
 * gemm_mode: BMM_GEMM_BF16, BMM_GEMM_SPLIT_BF16 or BMM_GEMM_E4M3 (else BMM_ERR_ARG). */

/* Workspace bytes bmm_autotune_gemm needs for this shape (0 for an invalid one). */
size_t bmm_autotune_workspace_size(int64_t m, int64_t p, int64_t L, int32_t gemm_mode);
/* Times every (BN, raster group) candidate on constant scratch operands carved from ws (device,
 * 256-byte aligned, caller-owned; contents overwritten) on the stream: one warm-up and three timed
 * launches each, CUDA events.  Records the fastest for the shape's bucket and returns it in
 * *bn_out, *raster_out and *ms_out (any may be NULL).  Synchronises the stream: call it before
 * timing or graph capture.  Errors: BMM_ERR_ARG, BMM_ERR_WORKSPACE, BMM_ERR_UNSUPPORTED (no
 * sm_103 device), BMM_ERR_CUDA. */
bmm_status bmm_autotune_gemm(int64_t m, int64_t p, int64_t L, int32_t gemm_mode, void* ws, size_t ws_bytes,
                             bmm_stream_t stream, int32_t* bn_out, int32_t* raster_out, float* ms_out);
/* The choice the next launch of this shape will use (host only, no device access). */
bmm_status bmm_autotune_get(int64_t m, int64_t p, int64_t L, int32_t gemm_mode, int32_t* bn_out,
                            int32_t* raster_out);
#define BMM_TILE_PAIR 512
#define BMM_TILE_PAIR_WIDE 1024
/* Records a choice for the shape's bucket (bn 128, 256, BMM_TILE_PAIR or BMM_TILE_PAIR_WIDE, raster
 * 4, 8 or 16; else BMM_ERR_ARG). */
bmm_status bmm_autotune_set(int64_t m, int64_t p, int64_t L, int32_t gemm_mode, int32_t bn, int32_t raster);
/* Forgets every recorded choice. */
void bmm_autotune_clear(void);

#ifdef __cplusplus
}
#endif
#endif /* BMM_H_ */
