// internal.h -- host-side launchers shared between the translation units of the library.
// Nothing here is exported; the ABI is include/bmm.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace bmm {

// A matrix seen through its storage: `rows_s` storage rows of `cols_s` elements, stride ld.
struct View {
    const void* data;
    int64_t rows_s, cols_s, ld;
    int dtype;
};

// Vectors of the contraction index i: column i of M (length m) or row i of N (length p).
// CONTIG: vector i is storage row i (element h at data[i*ld + h]).
// STRIDED: vector i is storage column i (element h at data[h*ld + i]).
enum VecMode { VEC_CONTIG = 0, VEC_STRIDED = 1 };
struct VecSet {
    const void* data;
    int64_t len;   // vector length (m for M, p for N)
    int64_t count; // number of vectors (n)
    int64_t ld;
    int dtype;
    int mode;      // VecMode
};

VecSet vecset_of_M(const bmm_mat* M);  // columns of M
VecSet vecset_of_N(const bmm_mat* N);  // rows of N

// ---- api.cu: host-side argument checks, identical for every entry point that takes them
size_t esize(int dtype);  // bytes per element of BMM_F64 / BMM_F32 / BMM_BF16
// null data, unknown dtype (BMM_ERR_DTYPE) or layout, negative sizes or short ld (BMM_ERR_SHAPE),
// data not aligned to its element size (BMM_ERR_ARG)
bmm_status check_mat(const bmm_mat* A);
// null offsets, K < 1, n < K, max_nk outside [1, n] (BMM_ERR_SHAPE), n above INT32_MAX (BMM_ERR_UNSUPPORTED)
bmm_status check_blocks(const bmm_blocks* B);
// both matrices and the blocks, then n = cols(M) = rows(N) (BMM_ERR_SHAPE) and one dtype (BMM_ERR_DTYPE)
bmm_status check_problem(const bmm_mat* M, const bmm_mat* N, const bmm_blocks* B);

// ---- norms.cu
// out[i] = ||vector i||^2 for i < count (FP64-accurate)
cudaError_t launch_vec_sqnorms(const VecSet& v, double* out, double* partial, int64_t partial_cap,
                               cudaStream_t s);
int64_t vec_sqnorms_partial_elems(const VecSet& v);
cudaError_t launch_block_stats(const double* x, const double* y, const int64_t* off, int64_t K, int64_t n,
                               double* a, double* ssum, double* mf, double* nf, DevStatus* st, cudaStream_t s);
// The same for many vector sets / products in one launch per kernel kind (FP32 and BF16 sets).
struct NormJobArgs {
    VecSet v;
    double* out;
    double* partial;      // strided sets: row-slice sums, vec_sqnorms_partial_elems(v) doubles (or null)
    int64_t partial_cap;
};
cudaError_t launch_vec_sqnorms_grouped(const NormJobArgs* jobs, int64_t count, cudaStream_t s);
struct BlockStatsArgs {
    const double *x, *y;
    const int64_t* off;
    int64_t K, n;
    double *a, *s, *mf, *nf;
    DevStatus* st;
    double* p;  // optional [n]: eq. 3.8 probabilities, written with a_k (nullptr: none)
};
cudaError_t launch_block_stats_grouped(const BlockStatsArgs* args, int64_t count, cudaStream_t s);

// ---- errors.cu
// A matrix for element access by (row, column): either storage order, F64 / F32 / BF16.
struct MatView {
    const void* data;
    int64_t rows, cols, ld;
    int dtype;
    int row_major;
};
cudaError_t launch_entry_variance(const MatView& M, const MatView& N, const int64_t* off, int64_t K, int unit,
                                  const double* p, const int64_t* ck, int64_t c, const int64_t* entries, int64_t count,
                                  double* out, cudaStream_t s);
cudaError_t launch_entry_estimate(const MatView& M, const MatView& N, const int64_t* off, int64_t K, int unit,
                                  const int64_t* ck, const int32_t* idx, const double* scale, int64_t draws,
                                  const int64_t* entries, int64_t count, double* cd, double* s2, int64_t* start,
                                  DevStatus* st, cudaStream_t s);
cudaError_t launch_error_report(const double* x, const double* y, const double* p, const int64_t* off, int64_t K,
                                int64_t n, const int64_t* ck, const double* a, const double* f, const double* mf,
                                const double* nf, const double* fhat, int64_t c, double delta, double* out,
                                cudaStream_t s);

// ---- frob.cu
// Per segment k: f[k] = || sum_t w_t u_t v_t^T ||_F^2 over the listed vectors of the segment,
// computed as sum_{t,t'} w_t w_t' <u_t,u_t'> <v_t,v_t'> with FP64-accurate dot products.
// cols == nullptr: segment k lists its own contraction indices off[k]..off[k+1]-1 with w = 1.
// cols != nullptr: segment k lists cols[k*per + j], j < per, with weights wts[...].
cudaError_t launch_gram_frob(const VecSet& U, const VecSet& V, const int64_t* off, int64_t K, int64_t max_len,
                             const int32_t* cols, const double* wts, int64_t per,
                             double* f, double* partial, int64_t partial_cap, DevStatus* st, cudaStream_t s);
int64_t gram_frob_partial_elems(int64_t K, int64_t max_len);
// Partial-buffer elements launch_gram_frob needs for K blocks (or pilots) of len vectors of
// lengths m and p: the direct form's slices of the m x p product when m p is the smaller cost
// (frob_use_direct), else the Gram form's pair tiles.
bool frob_use_direct(int64_t m, int64_t p, int64_t len);
int64_t frob_partial_elems(int64_t K, int64_t len, int64_t m, int64_t p);

// ---- blockstats_tc.cu
bool blockstats_tc_supported(const VecSet& vM, const VecSet& vN, int64_t max_nk);
// One product of a grouped statistics launch (outputs as for launch_blockstats_tc).
struct StatsArgs {
    VecSet vM, vN;
    const int64_t* off;
    int64_t K, n;
    double *x, *y, *a, *s, *mf, *nf, *f;
    DevStatus* st;
    int* wins;  // workspace, stats_windows_ints(K) ints
};
// window starts [K + 1], the window count, and the hand-out order of up to kWinTailMax last windows
constexpr int kWinTailMax = 256;
inline int64_t stats_windows_ints(int64_t K) { return K + 3 + kWinTailMax; }
// Many products (each supported by blockstats_tc_supported) in launches of up to ~19 products of
// one element type, every launch's CTAs sharing one work counter over all its blocks.
cudaError_t launch_blockstats_tc_grouped(const StatsArgs* args, int64_t count, bool stats, int* counter, cudaStream_t s);
// stats = true: writes x, y, a, ssum, mf, nf and f; stats = false: reads ssum, writes f only
cudaError_t launch_blockstats_tc(const VecSet& vM, const VecSet& vN, const int64_t* off, int64_t K, int64_t n,
                                 bool stats, int* counter, int* wins, double* x, double* y, double* a, double* ssum,
                                 double* mf, double* nf, double* f, DevStatus* st, cudaStream_t s);

// ---- design.cu
cudaError_t launch_probs(int kind, const double* x, const double* y, const double* a, const double* mf,
                         const double* nf, const double* f, const int64_t* off, int64_t K, int64_t n,
                         double* p, DevStatus* st, cudaStream_t s);
cudaError_t launch_blocksizes(int kind, const double* a, const double* f, const int64_t* off, int64_t K, int64_t n,
                              int64_t c, int64_t* ck, double* g, DevStatus* st, cudaStream_t s);
// One product's block-size job (bmm_blocksizes without the pilot), for the grouped launch.
struct SizesJob {
    int kind;
    const double *a, *f;
    const int64_t* off;
    int64_t K, n, c;
    int64_t* ck;
    double* g;
    DevStatus* st;
};
constexpr int kMaxSizesJobs = 400;  // 80-byte jobs under the kernel-parameter limit
cudaError_t launch_blocksizes_grouped(const SizesJob* jobs, int64_t count, cudaStream_t s);

// ---- sampler.cu
int64_t sampler_scratch_bytes(int64_t len, int64_t K);
// One product of a grouped sampler launch: the arguments of launch_sample.
struct SampleArgs {
    const double* p;
    int unit;
    const int64_t* off;
    int64_t K, n;
    const int64_t* ck;
    int64_t c;
    uint64_t seed, sid;
    int32_t* idx;
    double* scale;
    void* scratch;
    DevStatus* st;
};
// Many products' draws in three launches per up to 200 products, identical to launch_sample's.
cudaError_t launch_sample_grouped(const SampleArgs* args, int64_t count, cudaStream_t s);
cudaError_t launch_sample(const double* p, int unit, const int64_t* off, int64_t K, int64_t n, const int64_t* ck,
                          int64_t c, uint64_t seed, uint64_t sid, int32_t* idx, double* scale,
                          void* scratch, DevStatus* st, cudaStream_t s);

// ---- gather.cu
// Column list of the product: col[j], w[j] for j < ext, ext on the device (*ext_dev).
// count_dev (optional): the number of valid draws on the device (<= count).
cudaError_t launch_expand_blocks(const int32_t* kidx, const double* kscale, int64_t count, const int64_t* count_dev,
                                 const int64_t* off, int64_t K, int64_t n, int64_t max_nk, int32_t* col, double* w,
                                 int64_t* ext_dev, int64_t* prefix_scratch, DevStatus* st, cudaStream_t s);
// Operand rows: out[r][j] = cvt(f_j * vec_{col_j}[r]) for r < v.len, j < ext, zero up to the padded
// extent (a multiple of 64, of 128 for e4m3), with f_j = sqrt(w_j), or colscale[j] when given.
// mode: BMM_GEMM_BF16 (bf16), BMM_GEMM_SPLIT_BF16 (bf16 segments; `split_role` 0 = [hi|hi|lo], 1 = [hi|lo|hi]),
//       BMM_GEMM_E4M3 (fp8 e4m3 bytes, saturating), BMM_GEMM_F64 (double).  ldo = storage row stride of
//       out in elements.
cudaError_t launch_gather_operand(const VecSet& v, const int32_t* col, const double* w, const int64_t* ext_dev,
                                  int64_t ext_max, int mode, int split_role, bool apply_weight, void* out,
                                  int64_t ldo, DevStatus* st, cudaStream_t s, const float* colscale = nullptr);
// One operand gather of a grouped launch (bmm_apply_batched): the extent is a host value and
// the weight's square root scales every gathered vector (BF16, split-BF16 or e4m3 operands).
struct GatherJob {
    VecSet v;
    const int32_t* col;
    const double* w;
    int64_t ext;  // draws (host), or their upper bound when ext_dev is given
    int mode, role;
    void* out;
    int64_t ldo;
    DevStatus* st;
    const int64_t* ext_dev = nullptr;  // device count of draws (distinct draws), read in the kernel
};
cudaError_t launch_gather_grouped(const GatherJob* jobs, int64_t count, cudaStream_t s);
// FP8 operand scales.  amax[j] = sqrt(w_j) * max_r |vec_{col_j}[r]| (amax must start at zero);
// then per drawn index j an exponent e_j balancing the two operands and one exponent per operand,
// gA and gB, that bring each operand's largest value to at most 448 (the e4m3 maximum):
// sa[j] = sqrt(w_j) 2^(e_j + gA), sb[j] = sqrt(w_j) 2^(gB - e_j), out_scale = 2^-(gA + gB).
cudaError_t launch_vec_absmax(const VecSet& v, const int32_t* col, const double* w, const int64_t* ext_dev,
                              int64_t ext_max, float* amax, cudaStream_t s);
cudaError_t launch_fp8_scales(const float* amaxA, const float* amaxB, const double* w, const int64_t* ext_dev,
                              float* sa, float* sb, float* out_scale, cudaStream_t s);

// ---- gemm_tc.cu / gemm_f64.cu
// Element kinds of the tensor-core GEMM.
enum GemmElem { GEMM_ELEM_BF16 = 0, GEMM_ELEM_E4M3 = 1 };
// out[M x N] (+)= scale * A[M x K] * B[N x K]^T, A and B K-major, BF16 or e4m3 bytes, with row strides
// lda/ldb (elements, 16-byte multiples).  Columns >= kdim of A and B read as zero.  The K loop runs
// to k_mult * round_up(*k_dev, BK) if k_dev, else to k_host (a multiple of BK); BK = 64 (BF16) or
// 128 (e4m3).  scale (device, e4m3 only) may be null.  tune_k: the depth whose tile choice to use
// (a K-chunk of a longer product takes the whole product's), kdim if 0.  b_mn (BF16 only): B is
// given MN-major instead, as a row-major K x N matrix with row stride ldb >= N (rows >= kdim read as
// zero); every output element is the same dot product in the same K order as with a K-major B.
cudaError_t launch_gemm_bf16_tc(const void* A, int64_t lda, const void* B, int64_t ldb, int64_t M, int64_t N,
                                int64_t kdim, int64_t k_host, const int64_t* k_dev, int k_mult, float* out,
                                int64_t ldo, int accumulate, DevStatus* st, cudaStream_t s,
                                int elem = GEMM_ELEM_BF16, const float* scale = nullptr, int64_t tune_k = 0,
                                bool b_mn = false);
// K is k_host, or *k_dev rounded up to 64; k_max bounds it for the choice of K splits, whose
// partial tiles go to part (gemm_f64_split_elems(M, N, k_max) doubles; without it, no split).
cudaError_t launch_gemm_f64(const double* A, int64_t lda, const double* B, int64_t ldb, int64_t M, int64_t N,
                            int64_t k_host, const int64_t* k_dev, double* out, int64_t ldo, int accumulate,
                            cudaStream_t s, int64_t k_max = 0, double* part = nullptr, int64_t part_cap = 0);
int64_t gemm_f64_split_elems(int64_t M, int64_t N, int64_t K);
bool tc_gemm_supported();
// Many independent products in as few persistent launches as the kernel-parameter limit allows.
struct GemmArgs {
    const void* A;
    int64_t lda;
    const void* B;
    int64_t ldb;
    int64_t M, N, kdim, k_host;
    const int64_t* k_dev;
    int k_mult;
    float* out;
    int64_t ldo;
    int accumulate;
    int elem = GEMM_ELEM_BF16;
    const float* scale = nullptr;
};
cudaError_t launch_gemm_bf16_tc_grouped(const GemmArgs* args, int64_t count, DevStatus* st, cudaStream_t s);
// Tile width (BN, 128 or 256: one CTA per 128 x BN tile; kPairTile: a CTA pair per 256 x 256 tile)
// and raster group (4, 8 or 16 M-tiles) of a tensor-core GEMM: from the autotuner's table when the
// shape's bucket was tuned, else BN = 128 for N <= 128, 256 for M <= 128, else kPairTile; group 8.
constexpr int kPairTile = 512;       // a CTA pair per 256 x 256 tile
constexpr int kPairTileWide = 1024;  // a CTA pair per 256 x 512 tile
struct TileChoice {
    int bn, raster;
};
TileChoice gemm_tile_choice(int elem, int64_t M, int64_t N, int64_t K);
bool gemm_tile_valid(const TileChoice& c);
void gemm_tile_set(int elem, int64_t M, int64_t N, int64_t K, const TileChoice& c);
void gemm_tile_clear();
int64_t gemm_autotune_bytes(int64_t M, int64_t N, int64_t K, int elem);
cudaError_t gemm_autotune(int64_t M, int64_t N, int64_t K, int elem, void* scratch, size_t bytes, DevStatus* st,
                          cudaStream_t s, TileChoice* best_out, float* best_ms);

// ---- backward.cu
int64_t unique_scratch_bytes(int64_t space, int64_t count);
// Distinct indices of idx[0..count) (values in [0, space)), ascending, each with its multiplicity
// times its scale (the draws of one index share one scale; another scale records BMM_ERR_ARG).
cudaError_t launch_unique(const int32_t* idx, const double* scale, int64_t count, int64_t space,
                          int32_t* uidx, double* uw, int64_t* ucount_dev, void* scratch, DevStatus* st,
                          cudaStream_t s);
// The same for many products at once (five launches per up to 256 products; scratch of
// unique_scratch_bytes(space, count) bytes per product).
struct UniqueJob {
    const int32_t* idx;
    const double* scale;
    int64_t count, space;
    void* scratch;
    int32_t* uidx;
    double* uw;
    int64_t* ucount;
    DevStatus* st;
};
cudaError_t launch_unique_grouped(const UniqueJob* jobs, int64_t n, cudaStream_t s);
cudaError_t launch_convert_f32_to_bf16(const float* G, int64_t rows, int64_t cols, int64_t ldg,
                                       __nv_bfloat16* out, int64_t ldo, cudaStream_t s);
cudaError_t launch_convert_to_f64(const void* G, int dtype, int64_t rows, int64_t cols, int64_t ldg, bool transpose,
                                  double* out, int64_t ldo, cudaStream_t s);
// dst vector col_j (of a VecSet-shaped gradient) += w_j * src[j] (src: GEMM result, one row or column per j)
cudaError_t launch_scatter_grad(void* dst, int dst_dtype, int64_t dst_ld, int dst_mode, int64_t len,
                                const void* src, int src_dtype, int64_t src_ld, bool src_rows,
                                const int32_t* col, const double* w, const int64_t* ext_dev, int64_t ext_max,
                                cudaStream_t s);
// out[j][r] = vec_{col_j}[r] for j < *ext_dev, zero rows up to jmax (bf16, or double if f64)
cudaError_t launch_gather_rows(const VecSet& v, const int32_t* col, const int64_t* ext_dev, int64_t jmax, void* out,
                               int64_t ldo, bool f64, cudaStream_t s);
cudaError_t launch_zero_matrix(void* dst, int dtype, int64_t rows, int64_t cols, int64_t ld, cudaStream_t s);

}  // namespace bmm
