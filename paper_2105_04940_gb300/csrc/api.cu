// api.cu -- the exported C ABI (include/bmm.h): argument checks, workspace carving, launch order.
#include <string.h>

#include <vector>

#include "internal.h"

#define BMM_API extern "C" __attribute__((visibility("default")))

namespace bmm {

VecSet vecset_of_M(const bmm_mat* M) {
    VecSet v;
    v.data = M->data;
    v.len = M->rows;
    v.count = M->cols;
    v.ld = M->ld;
    v.dtype = M->dtype;
    v.mode = (M->layout == BMM_ROW_MAJOR) ? VEC_STRIDED : VEC_CONTIG;
    return v;
}

VecSet vecset_of_N(const bmm_mat* N) {
    VecSet v;
    v.data = N->data;
    v.len = N->cols;
    v.count = N->rows;
    v.ld = N->ld;
    v.dtype = N->dtype;
    v.mode = (N->layout == BMM_ROW_MAJOR) ? VEC_CONTIG : VEC_STRIDED;
    return v;
}

size_t esize(int dtype) { return dtype == BMM_F64 ? 8 : (dtype == BMM_F32 ? 4 : 2); }

// ---- argument checks shared by the entry points (bmm_probs_static included)
bmm_status check_mat(const bmm_mat* A) {
    if (A == nullptr || A->data == nullptr) return BMM_ERR_ARG;
    if (A->dtype != BMM_F64 && A->dtype != BMM_F32 && A->dtype != BMM_BF16) return BMM_ERR_DTYPE;
    if (A->layout != BMM_ROW_MAJOR && A->layout != BMM_COL_MAJOR) return BMM_ERR_ARG;
    if (A->rows < 0 || A->cols < 0) return BMM_ERR_SHAPE;
    const int64_t inner = (A->layout == BMM_ROW_MAJOR) ? A->cols : A->rows;
    if (A->ld < imax(inner, 1)) return BMM_ERR_SHAPE;
    if (reinterpret_cast<uintptr_t>(A->data) % esize(A->dtype)) return BMM_ERR_ARG;
    return BMM_OK;
}

bmm_status check_blocks(const bmm_blocks* B) {
    if (B == nullptr || B->offsets == nullptr) return BMM_ERR_ARG;
    if (B->K < 1 || B->n < B->K || B->max_nk < 1 || B->max_nk > B->n) return BMM_ERR_SHAPE;
    if (B->n > 0x7fffffffLL) return BMM_ERR_UNSUPPORTED;  // indices are int32
    return BMM_OK;
}

bmm_status check_problem(const bmm_mat* M, const bmm_mat* N, const bmm_blocks* B) {
    bmm_status s;
    if ((s = check_mat(M)) != BMM_OK) return s;
    if ((s = check_mat(N)) != BMM_OK) return s;
    if ((s = check_blocks(B)) != BMM_OK) return s;
    if (M->cols != N->rows || M->cols != B->n) return BMM_ERR_SHAPE;
    if (M->dtype != N->dtype) return BMM_ERR_DTYPE;
    return BMM_OK;
}

namespace {

constexpr size_t kStatusBytes = 256;

// bump allocator over the workspace scratch; with base == nullptr it only counts
struct Carver {
    char* base;
    size_t off = 0;
    template <typename T> T* take(int64_t n) {
        const size_t b = (size_t)round_up(imax(n, 1) * (int64_t)sizeof(T), 256);
        T* r = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += b;
        return r;
    }
};

bmm_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return BMM_OK;
    if (e == cudaErrorInvalidValue) return BMM_ERR_UNSUPPORTED;
    return BMM_ERR_CUDA;
}

#define BMM_TRY(expr)                                   \
    do {                                                \
        const bmm_status _s = from_cuda(expr);          \
        if (_s != BMM_OK) return _s;                    \
    } while (0)

bmm_status check_ws(const void* ws, size_t ws_bytes, size_t need) {
    if (ws == nullptr || (reinterpret_cast<uintptr_t>(ws) & 255)) return BMM_ERR_WORKSPACE;
    if (ws_bytes < need + kStatusBytes) return BMM_ERR_WORKSPACE;
    return BMM_OK;
}

DevStatus* status_of(void* ws) { return static_cast<DevStatus*>(ws); }

// ------------------------------------------------------------------ per-call workspace plans
struct ProbsPlan {
    double* partial;
    int64_t partial_cap;
    double* gpart;
    int64_t gpart_cap;
    int* counter;
    int* wins;
};
void plan_probs(Carver& cv, const bmm_mat* M, const bmm_mat* N, const bmm_blocks* B, bool need_f, ProbsPlan* p) {
    p->partial_cap = imax(vec_sqnorms_partial_elems(vecset_of_M(M)), vec_sqnorms_partial_elems(vecset_of_N(N)));
    p->partial = cv.take<double>(p->partial_cap);
    p->gpart_cap = need_f ? frob_partial_elems(B->K, B->max_nk, vecset_of_M(M).len, vecset_of_N(N).len) : 0;
    p->gpart = need_f ? cv.take<double>(p->gpart_cap) : nullptr;
    p->counter = cv.take<int>(1);
    p->wins = need_f ? cv.take<int>(stats_windows_ints(B->K)) : nullptr;
}

struct SizesPlan {
    double* g;
    double* fhat;
    double* gpart;
    int64_t gpart_cap;
};
// m, pp: lengths of M's columns and N's rows (the pilot's vectors); used only by BMM_CK_TILDE
void plan_sizes(Carver& cv, const bmm_blocks* B, int ckind, int64_t per, double* g_out, double* fhat_out,
                SizesPlan* p, int64_t m = 0, int64_t pp = 0) {
    p->g = g_out ? g_out : cv.take<double>(B->K);
    p->fhat = nullptr;
    p->gpart = nullptr;
    p->gpart_cap = 0;
    if (ckind == BMM_CK_TILDE) {
        p->fhat = fhat_out ? fhat_out : cv.take<double>(B->K);
        p->gpart_cap = frob_partial_elems(B->K, per, m, pp);
        p->gpart = cv.take<double>(p->gpart_cap);
    }
}

void* plan_sample(Carver& cv, int unit, const bmm_blocks* B) {
    const int64_t len = unit == BMM_UNIT_COLUMN ? B->n : B->K;
    return cv.take<char>(sampler_scratch_bytes(len, B->K));
}

struct ApplyPlan {
    void* uscr;        // distinct draws: scratch of the reduction,
    int32_t* uidx;     // the distinct indices (columns, or blocks for the block unit), ascending,
    double* uw;        // their multiplicity times their scale,
    int64_t* ucount;   // and their count (device)
    int64_t nuniq;     // an upper bound of that count
    int32_t* col;
    double* w;
    int64_t* prefix;
    int64_t* ext;
    void* A;
    void* Bop;
    int64_t lmax, kseg_max, ktot;
    float *amaxA, *amaxB, *sa, *sb, *oscale;  // e4m3 operand scales
    double* kpart;                            // FP64: partial products of the K splits
    int64_t kpart_cap;
};
void plan_apply(Carver& cv, const bmm_mat* M, const bmm_mat* N, const bmm_blocks* B, int unit, int64_t count,
                int mode, ApplyPlan* p) {
    const int64_t space = unit == BMM_UNIT_COLUMN ? B->n : B->K;
    p->nuniq = imax(1, imin(count, space));
    p->uscr = cv.take<char>(unique_scratch_bytes(space, count));
    p->uidx = cv.take<int32_t>(p->nuniq);
    p->uw = cv.take<double>(p->nuniq);
    p->ucount = cv.take<int64_t>(1);
    p->lmax = unit == BMM_UNIT_COLUMN ? p->nuniq : p->nuniq * B->max_nk;
    p->col = nullptr;
    p->w = nullptr;
    p->prefix = nullptr;
    if (unit == BMM_UNIT_BLOCK) {
        p->col = cv.take<int32_t>(p->lmax);
        p->w = cv.take<double>(p->lmax);
        p->prefix = cv.take<int64_t>(p->nuniq);
    }
    p->ext = cv.take<int64_t>(1);
    p->kseg_max = round_up(imax(p->lmax, 1), mode == BMM_GEMM_E4M3 ? 128 : 64);
    p->ktot = p->kseg_max * (mode == BMM_GEMM_SPLIT_BF16 ? 3 : 1);
    const size_t es = mode == BMM_GEMM_F64 ? 8 : (mode == BMM_GEMM_E4M3 ? 1 : 2);
    p->amaxA = p->amaxB = p->sa = p->sb = p->oscale = nullptr;
    if (mode == BMM_GEMM_E4M3) {
        p->amaxA = cv.take<float>(p->lmax);
        p->amaxB = cv.take<float>(p->lmax);
        p->sa = cv.take<float>(p->lmax);
        p->sb = cv.take<float>(p->lmax);
        p->oscale = cv.take<float>(4);
    }
    p->A = cv.take<char>(M->rows * p->ktot * (int64_t)es);
    p->Bop = cv.take<char>(N->cols * p->ktot * (int64_t)es);
    p->kpart_cap = mode == BMM_GEMM_F64 ? gemm_f64_split_elems(M->rows, N->cols, p->ktot) : 0;
    p->kpart = p->kpart_cap > 0 ? cv.take<double>(p->kpart_cap) : nullptr;
}

struct BackPlan {
    int32_t* idx;
    double* scale;
    void* sscr;
    void* uscr;
    int32_t* uidx;
    double* uw;
    int64_t* ucount;
    int32_t* col;
    double* w;
    int64_t* prefix;
    int64_t* ext;
    int64_t lmax, ldG, ldGT, ldOM, ldON;
    void *Gop, *Nu, *outM, *GT, *MuT, *outN;
};
void plan_backward(Carver& cv, const bmm_mat* M, const bmm_mat* N, const bmm_blocks* B, int unit, int64_t c, int mode,
                   bool want_dM, bool want_dN, BackPlan* p) {
    const int64_t space = unit == BMM_UNIT_COLUMN ? B->n : B->K;
    const int64_t m = M->rows, pp = N->cols;
    const int64_t nuniq = imax(1, imin(c, space));
    p->idx = cv.take<int32_t>(c);
    p->scale = cv.take<double>(c);
    p->sscr = plan_sample(cv, unit, B);
    p->uscr = cv.take<char>(unique_scratch_bytes(space, c));
    p->uidx = cv.take<int32_t>(nuniq);
    p->uw = cv.take<double>(nuniq);
    p->ucount = cv.take<int64_t>(1);
    if (unit == BMM_UNIT_BLOCK) {
        p->lmax = nuniq * B->max_nk;
        p->col = cv.take<int32_t>(p->lmax);
        p->w = cv.take<double>(p->lmax);
        p->prefix = cv.take<int64_t>(nuniq);
        p->ext = cv.take<int64_t>(1);
    } else {
        p->lmax = nuniq;
        p->col = p->uidx;
        p->w = p->uw;
        p->prefix = nullptr;
        p->ext = p->ucount;
    }
    const bool f64 = mode == BMM_GEMM_F64;
    const int64_t es = f64 ? 8 : 2;
    p->ldG = f64 ? pp : round_up(pp, 8);
    p->ldGT = f64 ? m : round_up(m, 8);
    p->ldOM = round_up(p->lmax, 4);
    p->ldON = round_up(pp, 4);
    p->Gop = p->Nu = p->outM = p->GT = p->MuT = p->outN = nullptr;
    // BF16: both GEMMs read G in BF16 as it is stored (K-major A of the first, MN-major B of the
    // second); FP64 keeps a transposed copy for the second
    if (want_dM || (want_dN && !f64)) p->Gop = cv.take<char>(m * p->ldG * es);
    if (want_dM) {
        p->Nu = cv.take<char>(p->lmax * p->ldG * es);
        p->outM = cv.take<char>(m * p->ldOM * (f64 ? 8 : 4));
    }
    if (want_dN) {
        if (f64) p->GT = cv.take<char>(pp * p->ldGT * es);
        p->MuT = cv.take<char>(p->lmax * p->ldGT * es);
        p->outN = cv.take<char>(p->lmax * p->ldON * (f64 ? 8 : 4));
    }
}

bool valid_gemm_mode(int mode) {
    return mode == BMM_GEMM_F64 || mode == BMM_GEMM_BF16 || mode == BMM_GEMM_SPLIT_BF16 || mode == BMM_GEMM_E4M3;
}

}  // namespace
}  // namespace bmm

using namespace bmm;

BMM_API size_t bmm_workspace_size(const bmm_mat* M, const bmm_mat* N, const bmm_blocks* B, int32_t unit,
                                  int64_t max_draws, int32_t gemm_mode) {
    if (check_problem(M, N, B) != BMM_OK || max_draws < 0 || !valid_gemm_mode(gemm_mode)) return 0;
    if (unit != BMM_UNIT_COLUMN && unit != BMM_UNIT_BLOCK) return 0;
    size_t need = 0;
    {
        Carver cv{nullptr};
        ProbsPlan p;
        plan_probs(cv, M, N, B, true, &p);
        need = cv.off > need ? cv.off : need;
    }
    {
        Carver cv{nullptr};
        SizesPlan p;
        plan_sizes(cv, B, BMM_CK_TILDE, ceil_div(imax(max_draws, 1), B->K), nullptr, nullptr, &p, vecset_of_M(M).len,
                   vecset_of_N(N).len);
        need = cv.off > need ? cv.off : need;
    }
    {
        Carver cv{nullptr};
        plan_sample(cv, BMM_UNIT_COLUMN, B);
        plan_sample(cv, BMM_UNIT_BLOCK, B);
        need = cv.off > need ? cv.off : need;
    }
    {
        Carver cv{nullptr};
        ApplyPlan p;
        plan_apply(cv, M, N, B, unit, max_draws, gemm_mode, &p);
        need = cv.off > need ? cv.off : need;
    }
    {
        Carver cv{nullptr};
        BackPlan p;
        plan_backward(cv, M, N, B, unit, max_draws, gemm_mode, true, true, &p);
        need = cv.off > need ? cv.off : need;
    }
    return need + kStatusBytes;
}

BMM_API bmm_status bmm_probs(const bmm_mat* M, const bmm_mat* N, const bmm_blocks* B, int32_t pkind, int32_t fmode,
                             double* p_out, const bmm_stats* st, void* ws, size_t ws_bytes, bmm_stream_t stream) {
    const bool reuse = (fmode & BMM_REUSE_STATS) != 0;
    fmode &= ~BMM_REUSE_STATS;
    if (pkind < BMM_P_COL_OPT || pkind > BMM_P_BLK_NORMPROD) return BMM_ERR_ARG;
    if (fmode != BMM_F_NONE && fmode != BMM_F_EXACT && fmode != BMM_F_TC) return BMM_ERR_ARG;
    bmm_status s;
    if (pkind == BMM_P_COL_UNIFORM && (reuse || st == nullptr)) {  // needs the blocks only
        if ((s = check_blocks(B)) != BMM_OK) return s;
        if (p_out == nullptr) return BMM_OK;
        if (ws == nullptr || (reinterpret_cast<uintptr_t>(ws) & 255) || ws_bytes < kStatusBytes) return BMM_ERR_WORKSPACE;
        BMM_TRY(launch_probs(pkind, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, B->offsets, B->K, B->n, p_out,
                             status_of(ws), reinterpret_cast<cudaStream_t>(stream)));
        return BMM_OK;
    }
    s = check_problem(M, N, B);
    if (s != BMM_OK) return s;
    if (st == nullptr || !st->x || !st->y || !st->a || !st->s || !st->mf || !st->nf) return BMM_ERR_ARG;
    const bool need_f = fmode != BMM_F_NONE || pkind == BMM_P_BLK_PRODNORM;
    if (need_f && st->f == nullptr) return BMM_ERR_ARG;
    if (reuse) {  // statistics given; compute f (fmode EXACT) and p only
        Carver cnt{nullptr};
        ProbsPlan plan;
        plan_probs(cnt, M, N, B, fmode != BMM_F_NONE, &plan);
        if ((s = check_ws(ws, ws_bytes, cnt.off)) != BMM_OK) return s;
        Carver cv{static_cast<char*>(ws) + kStatusBytes};
        plan_probs(cv, M, N, B, fmode != BMM_F_NONE, &plan);
        cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
        const VecSet vM = vecset_of_M(M), vN = vecset_of_N(N);
        if (fmode == BMM_F_TC && blockstats_tc_supported(vM, vN, B->max_nk))
            BMM_TRY(launch_blockstats_tc(vM, vN, B->offsets, B->K, B->n, false, plan.counter, plan.wins, st->x, st->y, st->a,
                                         st->s, st->mf, st->nf, st->f, status_of(ws), cs));
        else if (fmode != BMM_F_NONE)
            BMM_TRY(launch_gram_frob(vM, vN, B->offsets, B->K, B->max_nk, nullptr, nullptr, 0, st->f, plan.gpart,
                                     plan.gpart_cap, status_of(ws), cs));
        if (p_out)
            BMM_TRY(launch_probs(pkind, st->x, st->y, st->a, st->mf, st->nf, st->f, B->offsets, B->K, B->n, p_out,
                                 status_of(ws), cs));
        return BMM_OK;
    }
    Carver cnt{nullptr};
    ProbsPlan plan;
    plan_probs(cnt, M, N, B, need_f, &plan);
    if ((s = check_ws(ws, ws_bytes, cnt.off)) != BMM_OK) return s;
    Carver cv{static_cast<char*>(ws) + kStatusBytes};
    plan_probs(cv, M, N, B, need_f, &plan);
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    DevStatus* dst = status_of(ws);
    const VecSet vM = vecset_of_M(M), vN = vecset_of_N(N);
    if (fmode == BMM_F_TC && blockstats_tc_supported(vM, vN, B->max_nk)) {
        // one fused pass: statistics and f_k
        BMM_TRY(launch_blockstats_tc(vM, vN, B->offsets, B->K, B->n, true, plan.counter, plan.wins, st->x, st->y, st->a, st->s,
                                     st->mf, st->nf, st->f, dst, cs));
    } else {
        BMM_TRY(launch_vec_sqnorms(vM, st->x, plan.partial, plan.partial_cap, cs));
        BMM_TRY(launch_vec_sqnorms(vN, st->y, plan.partial, plan.partial_cap, cs));
        BMM_TRY(launch_block_stats(st->x, st->y, B->offsets, B->K, B->n, st->a, st->s, st->mf, st->nf, dst, cs));
        if (need_f)
            BMM_TRY(launch_gram_frob(vM, vN, B->offsets, B->K, B->max_nk, nullptr, nullptr, 0, st->f, plan.gpart,
                                     plan.gpart_cap, dst, cs));
    }
    if (p_out)
        BMM_TRY(launch_probs(pkind, st->x, st->y, st->a, st->mf, st->nf, st->f, B->offsets, B->K, B->n, p_out, dst,
                             cs));
    return BMM_OK;
}

namespace bmm {
namespace {
// bmm_probs_batched without f_k: the norm pass of every FP32 / BF16 product in grouped launches
// (x_i, y_i of all products, then a_k, s_k, ||M^k||_F^2, ||N_k||_F^2), then each product's
// probabilities; other products take bmm_probs's path on their own.
bmm_status probs_batched_norms(int64_t count, const bmm_mat* Ms, const bmm_mat* Ns, const bmm_blocks* Bs,
                               int32_t pkind, double* const* p_outs, const bmm_stats* sts, void* const* ws,
                               const size_t* ws_bytes, bmm_stream_t stream) {
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    std::vector<NormJobArgs> norms;
    std::vector<BlockStatsArgs> blocks;
    std::vector<int64_t> which;
    for (int64_t i = 0; i < count; ++i) {
        const bmm_mat* M = &Ms[i];
        const bmm_mat* N = &Ns[i];
        const bmm_blocks* B = &Bs[i];
        const bmm_stats* st = &sts[i];
        const bool eligible = check_problem(M, N, B) == BMM_OK && st->x && st->y && st->a && st->s && st->mf &&
                              st->nf && (M->dtype == BMM_F32 || M->dtype == BMM_BF16) && N->dtype == M->dtype &&
                              ws[i] != nullptr && (reinterpret_cast<uintptr_t>(ws[i]) & 255) == 0 &&
                              ws_bytes[i] >= kStatusBytes;
        if (!eligible) {
            bmm_status s = bmm_probs(M, N, B, pkind, BMM_F_NONE, p_outs ? p_outs[i] : nullptr, st, ws[i], ws_bytes[i],
                                     stream);
            if (s != BMM_OK) return s;
            continue;
        }
        // the row-slice buffer of the product's workspace serves its first strided set (M's columns
        // when M is row-major); a second strided set in the same launch goes without slices
        Carver cnt{nullptr};
        ProbsPlan plan;
        plan_probs(cnt, M, N, B, false, &plan);
        if (check_ws(ws[i], ws_bytes[i], cnt.off) != BMM_OK) return BMM_ERR_WORKSPACE;
        Carver cv{static_cast<char*>(ws[i]) + kStatusBytes};
        plan_probs(cv, M, N, B, false, &plan);
        const VecSet vM = vecset_of_M(M), vN = vecset_of_N(N);
        const bool m_slices = vM.mode == VEC_STRIDED;
        norms.push_back(NormJobArgs{vM, st->x, m_slices ? plan.partial : nullptr, m_slices ? plan.partial_cap : 0});
        norms.push_back(NormJobArgs{vN, st->y, m_slices ? nullptr : plan.partial, m_slices ? 0 : plan.partial_cap});
        // eq. 3.8 probabilities come out of the grouped block-statistics kernel; the block kind
        // (eq. 1.4) needs all K block sums first and keeps its own launch below
        double* p_col = (p_outs && pkind == BMM_P_COL_OPT) ? p_outs[i] : nullptr;
        blocks.push_back(BlockStatsArgs{st->x, st->y, B->offsets, B->K, B->n, st->a, st->s, st->mf, st->nf,
                                        status_of(ws[i]), p_col});
        which.push_back(i);
    }
    if (!norms.empty()) BMM_TRY(launch_vec_sqnorms_grouped(norms.data(), (int64_t)norms.size(), cs));
    if (!blocks.empty()) BMM_TRY(launch_block_stats_grouped(blocks.data(), (int64_t)blocks.size(), cs));
    for (const int64_t i : which) {
        double* p_out = p_outs ? p_outs[i] : nullptr;
        if (p_out == nullptr || pkind == BMM_P_COL_OPT) continue;
        const bmm_stats* st = &sts[i];
        BMM_TRY(launch_probs(pkind, st->x, st->y, st->a, st->mf, st->nf, st->f, Bs[i].offsets, Bs[i].K, Bs[i].n, p_out,
                             status_of(ws[i]), cs));
    }
    return BMM_OK;
}
}  // namespace
}  // namespace bmm

BMM_API bmm_status bmm_probs_batched(int64_t count, const bmm_mat* Ms, const bmm_mat* Ns, const bmm_blocks* Bs,
                                     int32_t pkind, int32_t fmode, double* const* p_outs, const bmm_stats* sts,
                                     void* const* ws, const size_t* ws_bytes, bmm_stream_t stream) {
    if (count < 0 || (count > 0 && (Ms == nullptr || Ns == nullptr || Bs == nullptr || sts == nullptr || ws == nullptr ||
                                    ws_bytes == nullptr)))
        return BMM_ERR_ARG;
    const bool reuse = (fmode & BMM_REUSE_STATS) != 0;
    const int32_t fbase = fmode & ~BMM_REUSE_STATS;
    if (pkind < BMM_P_COL_OPT || pkind > BMM_P_BLK_NORMPROD) return BMM_ERR_ARG;
    if (fbase != BMM_F_NONE && fbase != BMM_F_EXACT && fbase != BMM_F_TC) return BMM_ERR_ARG;
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    if (fbase == BMM_F_NONE && !reuse && pkind != BMM_P_COL_UNIFORM && pkind != BMM_P_BLK_PRODNORM)
        return probs_batched_norms(count, Ms, Ns, Bs, pkind, p_outs, sts, ws, ws_bytes, stream);
    std::vector<StatsArgs> grouped;
    std::vector<int64_t> which;
    int* counter = nullptr;
    for (int64_t i = 0; i < count; ++i) {
        const bmm_mat* M = &Ms[i];
        const bmm_mat* N = &Ns[i];
        const bmm_blocks* B = &Bs[i];
        const bmm_stats* st = &sts[i];
        double* p_out = p_outs ? p_outs[i] : nullptr;
        bool eligible = fbase == BMM_F_TC && pkind != BMM_P_COL_UNIFORM && check_problem(M, N, B) == BMM_OK &&
                        st->x && st->y && st->a && st->s && st->mf && st->nf && st->f;
        if (eligible) eligible = blockstats_tc_supported(vecset_of_M(M), vecset_of_N(N), B->max_nk);
        if (!eligible) {  // the product on its own, with bmm_probs's rules
            bmm_status s = bmm_probs(M, N, B, pkind, fmode, p_out, st, ws[i], ws_bytes[i], stream);
            if (s != BMM_OK) return s;
            continue;
        }
        Carver cnt{nullptr};
        ProbsPlan plan;
        plan_probs(cnt, M, N, B, true, &plan);
        bmm_status s = check_ws(ws[i], ws_bytes[i], cnt.off);
        if (s != BMM_OK) return s;
        Carver cv{static_cast<char*>(ws[i]) + kStatusBytes};
        plan_probs(cv, M, N, B, true, &plan);
        if (counter == nullptr) counter = plan.counter;
        grouped.push_back(StatsArgs{vecset_of_M(M), vecset_of_N(N), B->offsets, B->K, B->n, st->x, st->y, st->a, st->s,
                                    st->mf, st->nf, st->f, status_of(ws[i]), plan.wins});
        which.push_back(i);
    }
    if (!grouped.empty())
        BMM_TRY(launch_blockstats_tc_grouped(grouped.data(), (int64_t)grouped.size(), !reuse, counter, cs));
    for (size_t u = 0; u < which.size(); ++u) {
        const int64_t i = which[u];
        double* p_out = p_outs ? p_outs[i] : nullptr;
        if (p_out == nullptr) continue;
        const bmm_stats* st = &sts[i];
        BMM_TRY(launch_probs(pkind, st->x, st->y, st->a, st->mf, st->nf, st->f, Bs[i].offsets, Bs[i].K, Bs[i].n, p_out,
                             status_of(ws[i]), cs));
    }
    return BMM_OK;
}

BMM_API bmm_status bmm_blocksizes(const bmm_mat* M, const bmm_mat* N, const bmm_blocks* B, const bmm_stats* st,
                                  int32_t ckind, int64_t c, const int32_t* pilot_idx, const double* pilot_scale,
                                  int64_t pilot_per_block, int64_t* ck_out, double* g_out, double* fhat_out, void* ws,
                                  size_t ws_bytes, bmm_stream_t stream) {
    bmm_status s = check_blocks(B);
    if (s != BMM_OK) return s;
    if (ckind < BMM_CK_OPT || ckind > BMM_CK_EQUAL || ck_out == nullptr) return BMM_ERR_ARG;
    if (ckind != BMM_CK_EQUAL && (st == nullptr || st->a == nullptr)) return BMM_ERR_ARG;
    if (ckind == BMM_CK_OPT && st->f == nullptr) return BMM_ERR_ARG;
    if (ckind == BMM_CK_TILDE) {
        if ((s = check_problem(M, N, B)) != BMM_OK) return s;
        if (pilot_idx == nullptr || pilot_scale == nullptr || pilot_per_block < 1) return BMM_ERR_ARG;
    }
    if (c < B->K || c > B->n) return BMM_ERR_INFEASIBLE;
    const int64_t per = ckind == BMM_CK_TILDE ? pilot_per_block : 0;
    const int64_t vm = ckind == BMM_CK_TILDE ? vecset_of_M(M).len : 0, vp = ckind == BMM_CK_TILDE ? vecset_of_N(N).len : 0;
    Carver cnt{nullptr};
    SizesPlan plan;
    plan_sizes(cnt, B, ckind, per, g_out, fhat_out, &plan, vm, vp);
    if ((s = check_ws(ws, ws_bytes, cnt.off)) != BMM_OK) return s;
    Carver cv{static_cast<char*>(ws) + kStatusBytes};
    plan_sizes(cv, B, ckind, per, g_out, fhat_out, &plan, vm, vp);
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    DevStatus* dst = status_of(ws);
    const double* fvec = nullptr;
    if (ckind == BMM_CK_OPT) fvec = st->f;
    if (ckind == BMM_CK_TILDE) {
        BMM_TRY(launch_gram_frob(vecset_of_M(M), vecset_of_N(N), B->offsets, B->K, per, pilot_idx, pilot_scale, per,
                                 plan.fhat, plan.gpart, plan.gpart_cap, dst, cs));
        fvec = plan.fhat;
    }
    BMM_TRY(launch_blocksizes(ckind, ckind == BMM_CK_EQUAL ? nullptr : st->a, fvec, B->offsets, B->K, B->n, c, ck_out, plan.g,
                              dst, cs));
    return BMM_OK;
}

BMM_API bmm_status bmm_blocksizes_batched(int64_t count, const bmm_blocks* Bs, const bmm_stats* sts, int32_t ckind,
                                          const int64_t* cs, int64_t* const* ck_outs, double* const* g_outs,
                                          void* const* ws, const size_t* ws_bytes, bmm_stream_t stream) {
    if (count < 0 || (count > 0 && (Bs == nullptr || cs == nullptr || ck_outs == nullptr || ws == nullptr ||
                                    ws_bytes == nullptr)))
        return BMM_ERR_ARG;
    if (ckind != BMM_CK_OPT && ckind != BMM_CK_HAT && ckind != BMM_CK_EQUAL) return BMM_ERR_ARG;
    if (count == 0) return BMM_OK;
    if (ckind != BMM_CK_EQUAL && sts == nullptr) return BMM_ERR_ARG;
    std::vector<SizesJob> jobs;
    jobs.reserve((size_t)count);
    for (int64_t i = 0; i < count; ++i) {
        const bmm_blocks* B = &Bs[i];
        bmm_status s = check_blocks(B);
        if (s != BMM_OK) return s;
        if (ck_outs[i] == nullptr) return BMM_ERR_ARG;
        const bmm_stats* st = ckind == BMM_CK_EQUAL ? nullptr : &sts[i];
        if (st != nullptr && (st->a == nullptr || (ckind == BMM_CK_OPT && st->f == nullptr))) return BMM_ERR_ARG;
        if (cs[i] < B->K || cs[i] > B->n) return BMM_ERR_INFEASIBLE;
        double* g_out = g_outs ? g_outs[i] : nullptr;
        Carver cnt{nullptr};
        SizesPlan plan;
        plan_sizes(cnt, B, ckind, 0, g_out, nullptr, &plan);
        if ((s = check_ws(ws[i], ws_bytes[i], cnt.off)) != BMM_OK) return s;
        Carver cv{static_cast<char*>(ws[i]) + kStatusBytes};
        plan_sizes(cv, B, ckind, 0, g_out, nullptr, &plan);
        jobs.push_back(SizesJob{ckind, st ? st->a : nullptr, ckind == BMM_CK_OPT ? st->f : nullptr, B->offsets, B->K,
                                B->n, cs[i], ck_outs[i], plan.g, status_of(ws[i])});
    }
    if (!jobs.empty())
        BMM_TRY(launch_blocksizes_grouped(jobs.data(), (int64_t)jobs.size(), reinterpret_cast<cudaStream_t>(stream)));
    return BMM_OK;
}

BMM_API bmm_status bmm_sample(const double* p, int32_t unit, const bmm_blocks* B, const int64_t* ck, int64_t c,
                              uint64_t seed, uint64_t stream_id, int32_t* idx_out, double* scale_out, void* ws,
                              size_t ws_bytes, bmm_stream_t stream) {
    bmm_status s = check_blocks(B);
    if (s != BMM_OK) return s;
    if (p == nullptr || idx_out == nullptr || scale_out == nullptr || c < 0) return BMM_ERR_ARG;
    if (unit != BMM_UNIT_COLUMN && unit != BMM_UNIT_BLOCK) return BMM_ERR_ARG;
    if (unit == BMM_UNIT_COLUMN && ck == nullptr) return BMM_ERR_ARG;
    if (c > 0x7fffffffLL) return BMM_ERR_UNSUPPORTED;
    Carver cnt{nullptr};
    plan_sample(cnt, unit, B);
    if ((s = check_ws(ws, ws_bytes, cnt.off)) != BMM_OK) return s;
    Carver cv{static_cast<char*>(ws) + kStatusBytes};
    void* scr = plan_sample(cv, unit, B);
    BMM_TRY(launch_sample(p, unit, B->offsets, B->K, B->n, ck, c, seed, stream_id, idx_out, scale_out, scr,
                          status_of(ws), reinterpret_cast<cudaStream_t>(stream)));
    return BMM_OK;
}

BMM_API bmm_status bmm_sample_batched(int64_t count, const double* const* p, int32_t unit, const bmm_blocks* Bs,
                                      const int64_t* const* ck, const int64_t* cs, const uint64_t* seeds,
                                      const uint64_t* stream_ids, int32_t* const* idx_out, double* const* scale_out,
                                      void* const* ws, const size_t* ws_bytes, bmm_stream_t stream) {
    if (count < 0) return BMM_ERR_ARG;
    if (count == 0) return BMM_OK;
    if (!p || !Bs || !cs || !seeds || !stream_ids || !idx_out || !scale_out || !ws || !ws_bytes) return BMM_ERR_ARG;
    if (unit != BMM_UNIT_COLUMN && unit != BMM_UNIT_BLOCK) return BMM_ERR_ARG;
    if (unit == BMM_UNIT_COLUMN && ck == nullptr) return BMM_ERR_ARG;
    std::vector<SampleArgs> jobs;
    jobs.reserve((size_t)count);
    for (int64_t i = 0; i < count; ++i) {  // every product checked as bmm_sample checks it, before any launch
        const bmm_blocks* B = &Bs[i];
        bmm_status s = check_blocks(B);
        if (s != BMM_OK) return s;
        if (p[i] == nullptr || idx_out[i] == nullptr || scale_out[i] == nullptr || cs[i] < 0) return BMM_ERR_ARG;
        if (unit == BMM_UNIT_COLUMN && ck[i] == nullptr) return BMM_ERR_ARG;
        if (cs[i] > 0x7fffffffLL) return BMM_ERR_UNSUPPORTED;
        Carver cnt{nullptr};
        plan_sample(cnt, unit, B);
        if ((s = check_ws(ws[i], ws_bytes[i], cnt.off)) != BMM_OK) return s;
        Carver cv{static_cast<char*>(ws[i]) + kStatusBytes};
        void* scr = plan_sample(cv, unit, B);
        jobs.push_back(SampleArgs{p[i], unit, B->offsets, B->K, B->n, unit == BMM_UNIT_COLUMN ? ck[i] : nullptr, cs[i],
                                  seeds[i], stream_ids[i], idx_out[i], scale_out[i], scr, status_of(ws[i])});
    }
    BMM_TRY(launch_sample_grouped(jobs.data(), (int64_t)jobs.size(), reinterpret_cast<cudaStream_t>(stream)));
    return BMM_OK;
}

namespace bmm {
namespace {
// Checks and gathers of one product of bmm_apply / bmm_apply_batched.  On BMM_OK either *done
// (nothing left to compute) or *g describes the product's GEMM (BF16 modes; FP64 is launched here).
// With `defer` (bmm_apply_batched, bmm_apply_part), a column-unit BF16 or split-BF16 product launches
// no gather: its two gathers are appended to *defer for one grouped launch, and its reduction of the
// draws to *udefer when given (else it is launched here); the gathers and the GEMM read the number of
// distinct draws on the device, capped by the host capacity.  Checks the arguments, lays out the workspace and reduces the draws to their distinct indices (each
// with its multiplicity times its scale: the same sum of outer products, one term per index), then
// queues the gathers (or runs them) and describes the GEMM.  reduce = false reuses the distinct draws
// a previous call with the same arguments left in the workspace (the later parts of bmm_apply_part).
bmm_status apply_prepare(const bmm_mat* M, const bmm_mat* N, const bmm_blocks* B, int32_t unit, const int32_t* idx,
                         const double* scale, int64_t count, int32_t gemm_mode, const bmm_mat* out,
                         int32_t accumulate, void* ws, size_t ws_bytes, cudaStream_t cs, GemmArgs* g, bool* done,
                         std::vector<GatherJob>* defer = nullptr, bool reduce = true,
                         std::vector<UniqueJob>* udefer = nullptr) {
    *done = true;
    bmm_status s = check_problem(M, N, B);
    if (s != BMM_OK) return s;
    if (unit != BMM_UNIT_COLUMN && unit != BMM_UNIT_BLOCK) return BMM_ERR_ARG;
    if (!valid_gemm_mode(gemm_mode) || count < 0 || (count > 0 && (idx == nullptr || scale == nullptr)))
        return BMM_ERR_ARG;
    if ((s = check_mat(out)) != BMM_OK) return s;
    if (out->layout != BMM_ROW_MAJOR || out->rows != M->rows || out->cols != N->cols) return BMM_ERR_SHAPE;
    if (out->dtype != (gemm_mode == BMM_GEMM_F64 ? BMM_F64 : BMM_F32)) return BMM_ERR_DTYPE;
    if (gemm_mode != BMM_GEMM_F64 && !tc_gemm_supported()) return BMM_ERR_UNSUPPORTED;
    if (count > 0x7fffffffLL) return BMM_ERR_UNSUPPORTED;
    void* odata = const_cast<void*>(out->data);
    if (count == 0 || M->rows == 0 || N->cols == 0) {
        if (!accumulate) BMM_TRY(launch_zero_matrix(odata, out->dtype, out->rows, out->cols, out->ld, cs));
        return BMM_OK;
    }
    Carver cnt{nullptr};
    ApplyPlan plan;
    plan_apply(cnt, M, N, B, unit, count, gemm_mode, &plan);
    if ((s = check_ws(ws, ws_bytes, cnt.off)) != BMM_OK) return s;
    Carver cv{static_cast<char*>(ws) + kStatusBytes};
    plan_apply(cv, M, N, B, unit, count, gemm_mode, &plan);
    DevStatus* dst = status_of(ws);
    const int64_t space = unit == BMM_UNIT_COLUMN ? B->n : B->K;
    const bool deferred = defer != nullptr && unit == BMM_UNIT_COLUMN &&
                          (gemm_mode == BMM_GEMM_BF16 || gemm_mode == BMM_GEMM_SPLIT_BF16);
    if (reduce) {
        const UniqueJob uj{idx, scale, count, space, plan.uscr, plan.uidx, plan.uw, plan.ucount, dst};
        if (deferred && udefer != nullptr) udefer->push_back(uj);  // launched with the other products'
        else BMM_TRY(launch_unique_grouped(&uj, 1, cs));
    }
    const int32_t* col = plan.uidx;
    const double* w = plan.uw;
    const int64_t* ext = plan.ucount;
    const VecSet vM = vecset_of_M(M), vN = vecset_of_N(N);
    if (deferred) {
        GatherJob jA{vM, col, w, plan.nuniq, gemm_mode, 0, plan.A, plan.ktot, dst};
        GatherJob jB{vN, col, w, plan.nuniq, gemm_mode, 1, plan.Bop, plan.ktot, dst};
        jA.ext_dev = jB.ext_dev = ext;
        defer->push_back(jA);
        defer->push_back(jB);
        const int k_mult = gemm_mode == BMM_GEMM_SPLIT_BF16 ? 3 : 1;
        *g = GemmArgs{plan.A, plan.ktot, plan.Bop, plan.ktot, M->rows, N->cols, plan.ktot, plan.ktot, ext, k_mult,
                      static_cast<float*>(odata), out->ld, accumulate, GEMM_ELEM_BF16, nullptr};
        *done = false;
        return BMM_OK;
    }
    if (unit == BMM_UNIT_BLOCK) {
        if (reduce)
            BMM_TRY(launch_expand_blocks(plan.uidx, plan.uw, plan.nuniq, plan.ucount, B->offsets, B->K, B->n,
                                         B->max_nk, plan.col, plan.w, plan.ext, plan.prefix, dst, cs));
        col = plan.col;
        w = plan.w;
        ext = plan.ext;
    }
    if (gemm_mode == BMM_GEMM_E4M3) {
        // column maxima of C and row maxima of D, then their power-of-two scales
        BMM_TRY(cudaMemsetAsync(plan.amaxA, 0, sizeof(float) * plan.lmax, cs));
        BMM_TRY(cudaMemsetAsync(plan.amaxB, 0, sizeof(float) * plan.lmax, cs));
        BMM_TRY(launch_vec_absmax(vM, col, w, ext, plan.lmax, plan.amaxA, cs));
        BMM_TRY(launch_vec_absmax(vN, col, w, ext, plan.lmax, plan.amaxB, cs));
        BMM_TRY(launch_fp8_scales(plan.amaxA, plan.amaxB, w, ext, plan.sa, plan.sb, plan.oscale, cs));
    }
    BMM_TRY(launch_gather_operand(vM, col, w, ext, plan.lmax, gemm_mode, 0, true, plan.A, plan.ktot, dst, cs,
                                  plan.sa));
    BMM_TRY(launch_gather_operand(vN, col, w, ext, plan.lmax, gemm_mode, 1, true, plan.Bop, plan.ktot, dst, cs,
                                  plan.sb));
    if (gemm_mode == BMM_GEMM_F64) {
        BMM_TRY(launch_gemm_f64(static_cast<const double*>(plan.A), plan.ktot, static_cast<const double*>(plan.Bop),
                                plan.ktot, M->rows, N->cols, 0, ext, static_cast<double*>(odata), out->ld,
                                accumulate, cs, plan.ktot, plan.kpart, plan.kpart_cap));
        return BMM_OK;
    }
    *g = GemmArgs{plan.A, plan.ktot, plan.Bop, plan.ktot, M->rows, N->cols, plan.ktot, plan.ktot, ext,
                  gemm_mode == BMM_GEMM_SPLIT_BF16 ? 3 : 1, static_cast<float*>(odata), out->ld, accumulate,
                  gemm_mode == BMM_GEMM_E4M3 ? GEMM_ELEM_E4M3 : GEMM_ELEM_BF16, plan.oscale};
    *done = false;
    return BMM_OK;
}
}  // namespace
}  // namespace bmm

BMM_API bmm_status bmm_apply(const bmm_mat* M, const bmm_mat* N, const bmm_blocks* B, int32_t unit,
                             const int32_t* idx, const double* scale, int64_t count, int32_t gemm_mode,
                             const bmm_mat* out, int32_t accumulate, void* ws, size_t ws_bytes, bmm_stream_t stream) {
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    GemmArgs g;
    bool done = true;
    bmm_status s = apply_prepare(M, N, B, unit, idx, scale, count, gemm_mode, out, accumulate, ws, ws_bytes, cs, &g, &done);
    if (s != BMM_OK || done) return s;
    BMM_TRY(launch_gemm_bf16_tc(g.A, g.lda, g.B, g.ldb, g.M, g.N, g.kdim, g.k_host, g.k_dev, g.k_mult, g.out, g.ldo,
                                g.accumulate, status_of(ws), cs, g.elem, g.scale));
    return BMM_OK;
}

// One part of a column-sampled BF16 bmm_apply, so that a caller can overlap the parts on streams of
// its own: the reduction of the draws to distinct indices, the gather of N's drawn rows (operand B),
// the gather of M's drawn columns for a range of output rows (operand A), and the GEMM of a range of
// output rows.  The operands live in the
// workspace, as bmm_apply lays them out; every output element is the full-depth dot product of a
// single bmm_apply, so any split gives the same bits.
BMM_API bmm_status bmm_apply_part(const bmm_mat* M, const bmm_mat* N, const bmm_blocks* B, const int32_t* idx,
                                  const double* scale, int64_t count, const bmm_mat* out, int32_t accumulate,
                                  int32_t part, int64_t row0, int64_t row1, void* ws, size_t ws_bytes,
                                  bmm_stream_t stream) {
    if (part != BMM_APPLY_GATHER_B && part != BMM_APPLY_GATHER_A && part != BMM_APPLY_GEMM &&
        part != BMM_APPLY_REDUCE)
        return BMM_ERR_ARG;
    if (count < 1 || M == nullptr || N == nullptr || M->rows < 1 || N->cols < 1) return BMM_ERR_ARG;
    if ((part == BMM_APPLY_GATHER_A || part == BMM_APPLY_GEMM) &&
        (row0 < 0 || row1 < row0 || row1 > M->rows || row0 % 128 || (row1 % 128 && row1 != M->rows)))
        return BMM_ERR_SHAPE;
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    GemmArgs g;
    bool done = true;
    std::vector<GatherJob> jobs;
    // the REDUCE part reduces the draws to their distinct indices in the workspace; the other parts,
    // issued after it, use that reduction
    bmm_status s = apply_prepare(M, N, B, BMM_UNIT_COLUMN, idx, scale, count, BMM_GEMM_BF16, out, accumulate, ws,
                                 ws_bytes, cs, &g, &done, &jobs, part == BMM_APPLY_REDUCE);
    if (s != BMM_OK || done || part == BMM_APPLY_REDUCE) return s;
    if (part == BMM_APPLY_GATHER_B) {
        BMM_TRY(launch_gather_grouped(&jobs[1], 1, cs));
        return BMM_OK;
    }
    if (row1 == row0) return BMM_OK;
    if (part == BMM_APPLY_GATHER_A) {
        const GatherJob& jM = jobs[0];
        GatherJob sub = jM;
        // element r of a column of M: at data[r * ld + i] (strided) or data[i * ld + r] (contiguous)
        sub.v.data = static_cast<const char*>(jM.v.data) + (jM.v.mode == VEC_STRIDED ? row0 * jM.v.ld : row0) *
                                                             (int64_t)esize(jM.v.dtype);
        sub.v.len = row1 - row0;
        sub.out = static_cast<__nv_bfloat16*>(jM.out) + row0 * jM.ldo;
        BMM_TRY(launch_gather_grouped(&sub, 1, cs));
        return BMM_OK;
    }
    BMM_TRY(launch_gemm_bf16_tc(static_cast<const __nv_bfloat16*>(g.A) + row0 * g.lda, g.lda, g.B, g.ldb, row1 - row0,
                                g.N, g.kdim, g.k_host, g.k_dev, g.k_mult, g.out + row0 * g.ldo, g.ldo, g.accumulate,
                                status_of(ws), cs, GEMM_ELEM_BF16, nullptr, g.kdim));
    return BMM_OK;
}

BMM_API bmm_status bmm_apply_batched(int64_t count, const bmm_mat* Ms, const bmm_mat* Ns, const bmm_blocks* Bs,
                                     int32_t unit, const int32_t* const* idx, const double* const* scale,
                                     const int64_t* draws, int32_t gemm_mode, const bmm_mat* outs,
                                     int32_t accumulate, void* const* ws, const size_t* ws_bytes,
                                     bmm_stream_t stream) {
    if (count < 0) return BMM_ERR_ARG;
    if (count == 0) return BMM_OK;
    if (!Ms || !Ns || !Bs || !idx || !scale || !draws || !outs || !ws || !ws_bytes) return BMM_ERR_ARG;
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    std::vector<GemmArgs> gemms;
    std::vector<GatherJob> gathers;
    std::vector<UniqueJob> uniq;
    gemms.reserve((size_t)count);
    gathers.reserve(2 * (size_t)count);
    uniq.reserve((size_t)count);
    for (int64_t i = 0; i < count; ++i) {
        GemmArgs g;
        bool done = true;
        const bmm_status s = apply_prepare(&Ms[i], &Ns[i], &Bs[i], unit, idx[i], scale[i], draws[i], gemm_mode, &outs[i],
                                           accumulate, ws[i], ws_bytes[i], cs, &g, &done, &gathers, true, &uniq);
        if (s != BMM_OK) return s;
        if (!done) gemms.push_back(g);
    }
    if (!uniq.empty()) BMM_TRY(launch_unique_grouped(uniq.data(), (int64_t)uniq.size(), cs));
    if (!gathers.empty()) BMM_TRY(launch_gather_grouped(gathers.data(), (int64_t)gathers.size(), cs));
    if (!gemms.empty())
        BMM_TRY(launch_gemm_bf16_tc_grouped(gemms.data(), (int64_t)gemms.size(), status_of(ws[0]), cs));
    return BMM_OK;
}

BMM_API bmm_status bmm_backward(const bmm_mat* G, const bmm_mat* M, const bmm_mat* N, const bmm_blocks* B,
                                int32_t unit, const double* p, const int64_t* ck, int64_t c, uint64_t seed,
                                uint64_t stream_id, int32_t gemm_mode, const bmm_mat* dM, const bmm_mat* dN,
                                int32_t accumulate, void* ws, size_t ws_bytes, bmm_stream_t stream) {
    bmm_status s = check_problem(M, N, B);
    if (s != BMM_OK) return s;
    if (unit != BMM_UNIT_COLUMN && unit != BMM_UNIT_BLOCK) return BMM_ERR_ARG;
    if (!valid_gemm_mode(gemm_mode) || p == nullptr || c < 0 || (unit == BMM_UNIT_COLUMN && ck == nullptr))
        return BMM_ERR_ARG;
    if (gemm_mode == BMM_GEMM_SPLIT_BF16 || gemm_mode == BMM_GEMM_E4M3) return BMM_ERR_UNSUPPORTED;
    const int gd = gemm_mode == BMM_GEMM_F64 ? BMM_F64 : BMM_F32;
    if ((s = check_mat(G)) != BMM_OK) return s;
    if (G->layout != BMM_ROW_MAJOR || G->rows != M->rows || G->cols != N->cols) return BMM_ERR_SHAPE;
    if (G->dtype != gd) return BMM_ERR_DTYPE;
    // gradients in the product's precision (FP64 / FP32), or BF16 for the BF16 mode
    auto grad_dtype_ok = [&](int dt) { return dt == gd || (gd == BMM_F32 && dt == BMM_BF16); };
    if (dM) {
        if ((s = check_mat(dM)) != BMM_OK) return s;
        if (dM->rows != M->rows || dM->cols != M->cols) return BMM_ERR_SHAPE;
        if (!grad_dtype_ok(dM->dtype)) return BMM_ERR_DTYPE;
    }
    if (dN) {
        if ((s = check_mat(dN)) != BMM_OK) return s;
        if (dN->rows != N->rows || dN->cols != N->cols) return BMM_ERR_SHAPE;
        if (!grad_dtype_ok(dN->dtype)) return BMM_ERR_DTYPE;
    }
    if (gemm_mode != BMM_GEMM_F64 && !tc_gemm_supported()) return BMM_ERR_UNSUPPORTED;
    if (c > 0x7fffffffLL) return BMM_ERR_UNSUPPORTED;
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    if (!accumulate) {
        if (dM) BMM_TRY(launch_zero_matrix(const_cast<void*>(dM->data), dM->dtype, dM->layout == BMM_ROW_MAJOR ? dM->rows : dM->cols,
                                           dM->layout == BMM_ROW_MAJOR ? dM->cols : dM->rows, dM->ld, cs));
        if (dN) BMM_TRY(launch_zero_matrix(const_cast<void*>(dN->data), dN->dtype, dN->layout == BMM_ROW_MAJOR ? dN->rows : dN->cols,
                                           dN->layout == BMM_ROW_MAJOR ? dN->cols : dN->rows, dN->ld, cs));
    }
    if (c == 0 || (!dM && !dN)) return BMM_OK;
    Carver cnt{nullptr};
    BackPlan plan;
    plan_backward(cnt, M, N, B, unit, c, gemm_mode, dM != nullptr, dN != nullptr, &plan);
    if ((s = check_ws(ws, ws_bytes, cnt.off)) != BMM_OK) return s;
    Carver cv{static_cast<char*>(ws) + kStatusBytes};
    plan_backward(cv, M, N, B, unit, c, gemm_mode, dM != nullptr, dN != nullptr, &plan);
    DevStatus* dst = status_of(ws);
    const int64_t space = unit == BMM_UNIT_COLUMN ? B->n : B->K;
    const int64_t m = M->rows, pp = N->cols;
    const bool f64 = gemm_mode == BMM_GEMM_F64;
    BMM_TRY(launch_sample(p, unit, B->offsets, B->K, B->n, ck, c, seed, stream_id, plan.idx, plan.scale, plan.sscr,
                          dst, cs));
    BMM_TRY(launch_unique(plan.idx, plan.scale, c, space, plan.uidx, plan.uw, plan.ucount, plan.uscr, dst, cs));
    if (unit == BMM_UNIT_BLOCK)
        BMM_TRY(launch_expand_blocks(plan.uidx, plan.uw, imin(c, space), plan.ucount, B->offsets, B->K, B->n,
                                     B->max_nk, plan.col, plan.w, plan.ext, plan.prefix, dst, cs));
    const VecSet vM = vecset_of_M(M), vN = vecset_of_N(N);
    if (!f64)  // G in BF16, row-major, for both GEMMs
        BMM_TRY(launch_convert_f32_to_bf16(static_cast<const float*>(G->data), m, pp, G->ld,
                                           static_cast<__nv_bfloat16*>(plan.Gop), plan.ldG, cs));
    if (dM) {
        // outM[h][j] = sum_f G[h,f] N[col_j, f]
        if (f64) BMM_TRY(launch_convert_to_f64(G->data, G->dtype, m, pp, G->ld, false, static_cast<double*>(plan.Gop), plan.ldG, cs));
        BMM_TRY(launch_gather_rows(vN, plan.col, plan.ext, plan.lmax, plan.Nu, plan.ldG, f64, cs));
        if (f64)
            BMM_TRY(launch_gemm_f64(static_cast<const double*>(plan.Gop), plan.ldG, static_cast<const double*>(plan.Nu),
                                    plan.ldG, m, plan.lmax, pp, nullptr, static_cast<double*>(plan.outM), plan.ldOM, 0, cs));
        else
            BMM_TRY(launch_gemm_bf16_tc(static_cast<const __nv_bfloat16*>(plan.Gop), plan.ldG,
                                        static_cast<const __nv_bfloat16*>(plan.Nu), plan.ldG, m, plan.lmax, pp,
                                        round_up(pp, 64), nullptr, 1, static_cast<float*>(plan.outM), plan.ldOM, 0,
                                        dst, cs));
        const int mode = dM->layout == BMM_ROW_MAJOR ? VEC_STRIDED : VEC_CONTIG;
        BMM_TRY(launch_scatter_grad(const_cast<void*>(dM->data), dM->dtype, dM->ld, mode, m, plan.outM, gd, plan.ldOM, false,
                                    plan.col, plan.w, plan.ext, plan.lmax, cs));
    }
    if (dN) {
        // outN[j][f] = sum_h M[h, col_j] G[h, f]; BF16: G is the GEMM's MN-major B as converted above
        if (f64) BMM_TRY(launch_convert_to_f64(G->data, G->dtype, m, pp, G->ld, true, static_cast<double*>(plan.GT), plan.ldGT, cs));
        BMM_TRY(launch_gather_rows(vM, plan.col, plan.ext, plan.lmax, plan.MuT, plan.ldGT, f64, cs));
        if (f64)
            BMM_TRY(launch_gemm_f64(static_cast<const double*>(plan.MuT), plan.ldGT, static_cast<const double*>(plan.GT),
                                    plan.ldGT, plan.lmax, pp, m, nullptr, static_cast<double*>(plan.outN), plan.ldON, 0, cs));
        else
            BMM_TRY(launch_gemm_bf16_tc(static_cast<const __nv_bfloat16*>(plan.MuT), plan.ldGT,
                                        static_cast<const __nv_bfloat16*>(plan.Gop), plan.ldG, plan.lmax, pp, m,
                                        round_up(m, 64), nullptr, 1, static_cast<float*>(plan.outN), plan.ldON, 0,
                                        dst, cs, GEMM_ELEM_BF16, nullptr, 0, true));
        const int mode = dN->layout == BMM_ROW_MAJOR ? VEC_CONTIG : VEC_STRIDED;
        BMM_TRY(launch_scatter_grad(const_cast<void*>(dN->data), dN->dtype, dN->ld, mode, pp, plan.outN, gd, plan.ldON, true,
                                    plan.col, plan.w, plan.ext, plan.lmax, cs));
    }
    return BMM_OK;
}

BMM_API bmm_status bmm_read_device_status(const void* ws, bmm_stream_t stream) {
    if (ws == nullptr) return BMM_ERR_ARG;
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(cs) != cudaSuccess) return BMM_ERR_CUDA;
    DevStatus h{0, 0};
    if (cudaMemcpy(&h, ws, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return BMM_ERR_CUDA;
    return static_cast<bmm_status>(h.code);
}

BMM_API bmm_status bmm_clear_device_status(void* ws, bmm_stream_t stream) {
    if (ws == nullptr) return BMM_ERR_ARG;
    return cudaMemsetAsync(ws, 0, kStatusBytes, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess ? BMM_OK
                                                                                                       : BMM_ERR_CUDA;
}

BMM_API const char* bmm_status_string(bmm_status s) {
    switch (s) {
        case BMM_OK: return "ok";
        case BMM_ERR_ARG: return "invalid argument";
        case BMM_ERR_SHAPE: return "inconsistent shape or block offsets";
        case BMM_ERR_DTYPE: return "unsupported element type";
        case BMM_ERR_INFEASIBLE: return "infeasible budget (need K <= c <= n)";
        case BMM_ERR_NONFINITE: return "non-finite value in the data";
        case BMM_ERR_WORKSPACE: return "workspace too small or misaligned";
        case BMM_ERR_CUDA: return "CUDA runtime error";
        case BMM_ERR_TIMEOUT: return "bounded device wait expired";
        case BMM_ERR_UNSUPPORTED: return "not supported by this library or device";
    }
    return "unknown status";
}

BMM_API uint64_t bmm_launch_count(void) { return launch_counter().load(std::memory_order_relaxed); }

// ---- GEMM tile autotuner
namespace {
// element kind and GEMM depth of a sampled product with L outer products in gemm_mode
bool tune_shape(int64_t m, int64_t p, int64_t L, int32_t mode, int* elem, int64_t* K) {
    if (m < 1 || p < 1 || L < 1 || m > 0x7fffffff || p > 0x7fffffff || L > (int64_t(1) << 40)) return false;
    if (mode != BMM_GEMM_BF16 && mode != BMM_GEMM_SPLIT_BF16 && mode != BMM_GEMM_E4M3) return false;
    *elem = mode == BMM_GEMM_E4M3 ? bmm::GEMM_ELEM_E4M3 : bmm::GEMM_ELEM_BF16;
    *K = bmm::round_up(L, mode == BMM_GEMM_E4M3 ? 128 : 64) * (mode == BMM_GEMM_SPLIT_BF16 ? 3 : 1);
    return true;
}
}  // namespace

BMM_API size_t bmm_autotune_workspace_size(int64_t m, int64_t p, int64_t L, int32_t gemm_mode) {
    int elem;
    int64_t K;
    if (!tune_shape(m, p, L, gemm_mode, &elem, &K)) return 0;
    return (size_t)(kStatusBytes + gemm_autotune_bytes(m, p, K, elem));
}

BMM_API bmm_status bmm_autotune_gemm(int64_t m, int64_t p, int64_t L, int32_t gemm_mode, void* ws, size_t ws_bytes,
                                     bmm_stream_t stream, int32_t* bn_out, int32_t* raster_out, float* ms_out) {
    int elem;
    int64_t K;
    if (!tune_shape(m, p, L, gemm_mode, &elem, &K)) return BMM_ERR_ARG;
    if (ws == nullptr || (reinterpret_cast<uintptr_t>(ws) & 255) ||
        ws_bytes < (size_t)(kStatusBytes + gemm_autotune_bytes(m, p, K, elem)))
        return BMM_ERR_WORKSPACE;
    if (!tc_gemm_supported()) return BMM_ERR_UNSUPPORTED;
    TileChoice best{0, 0};
    float ms = 0.f;
    BMM_TRY(gemm_autotune(m, p, K, elem, static_cast<char*>(ws) + kStatusBytes, ws_bytes - kStatusBytes, status_of(ws),
                          reinterpret_cast<cudaStream_t>(stream), &best, &ms));
    if (bn_out) *bn_out = best.bn;
    if (raster_out) *raster_out = best.raster;
    if (ms_out) *ms_out = ms;
    return BMM_OK;
}

BMM_API bmm_status bmm_autotune_get(int64_t m, int64_t p, int64_t L, int32_t gemm_mode, int32_t* bn_out,
                                    int32_t* raster_out) {
    int elem;
    int64_t K;
    if (!tune_shape(m, p, L, gemm_mode, &elem, &K)) return BMM_ERR_ARG;
    const TileChoice c = gemm_tile_choice(elem, m, p, K);
    if (bn_out) *bn_out = c.bn;
    if (raster_out) *raster_out = c.raster;
    return BMM_OK;
}

BMM_API bmm_status bmm_autotune_set(int64_t m, int64_t p, int64_t L, int32_t gemm_mode, int32_t bn, int32_t raster) {
    int elem;
    int64_t K;
    const TileChoice c{bn, raster};
    if (!tune_shape(m, p, L, gemm_mode, &elem, &K) || !gemm_tile_valid(c)) return BMM_ERR_ARG;
    gemm_tile_set(elem, m, p, K, c);
    return BMM_OK;
}

BMM_API void bmm_autotune_clear(void) { gemm_tile_clear(); }

// ------------------------------------------------------------------ error bars
namespace bmm {
namespace {
MatView view_of(const bmm_mat* A) {
    return MatView{A->data, A->rows, A->cols, A->ld, A->dtype, A->layout == BMM_ROW_MAJOR ? 1 : 0};
}
}  // namespace
}  // namespace bmm

BMM_API bmm_status bmm_error_report(const bmm_blocks* B, const bmm_stats* st, const double* p, const int64_t* ck,
                                    int64_t c, const double* fhat, double delta, double* report_out,
                                    bmm_stream_t stream) {
    bmm_status s = check_blocks(B);
    if (s != BMM_OK) return s;
    if (st == nullptr || st->x == nullptr || st->y == nullptr || st->a == nullptr || st->mf == nullptr ||
        st->nf == nullptr || p == nullptr || ck == nullptr || report_out == nullptr)
        return BMM_ERR_ARG;
    if (!(delta > 0.0 && delta < 1.0) || c < 1) return BMM_ERR_ARG;
    BMM_TRY(launch_error_report(st->x, st->y, p, B->offsets, B->K, B->n, ck, st->a, st->f, st->mf, st->nf,
                                st->f != nullptr ? fhat : nullptr, c, delta, report_out,
                                reinterpret_cast<cudaStream_t>(stream)));
    return BMM_OK;
}

BMM_API bmm_status bmm_entry_variance(const bmm_mat* M, const bmm_mat* N, const bmm_blocks* B, int32_t unit,
                                      const double* p, const int64_t* ck, int64_t c, const int64_t* entries,
                                      int64_t count, double* sigma2_out, bmm_stream_t stream) {
    bmm_status s = check_problem(M, N, B);
    if (s != BMM_OK) return s;
    if (unit != BMM_UNIT_COLUMN && unit != BMM_UNIT_BLOCK) return BMM_ERR_ARG;
    if (count < 0 || p == nullptr || (count > 0 && (entries == nullptr || sigma2_out == nullptr))) return BMM_ERR_ARG;
    if (unit == BMM_UNIT_COLUMN && ck == nullptr) return BMM_ERR_ARG;
    if (unit == BMM_UNIT_BLOCK && c < 1) return BMM_ERR_ARG;
    BMM_TRY(launch_entry_variance(view_of(M), view_of(N), B->offsets, B->K, unit, p, ck, c, entries, count, sigma2_out,
                                  reinterpret_cast<cudaStream_t>(stream)));
    return BMM_OK;
}

BMM_API bmm_status bmm_entry_estimate(const bmm_mat* M, const bmm_mat* N, const bmm_blocks* B, int32_t unit,
                                      const int64_t* ck, const int32_t* idx, const double* scale, int64_t draws,
                                      const int64_t* entries, int64_t count, double* cd_out, double* s2_out, void* ws,
                                      size_t ws_bytes, bmm_stream_t stream) {
    bmm_status s = check_problem(M, N, B);
    if (s != BMM_OK) return s;
    if (unit != BMM_UNIT_COLUMN && unit != BMM_UNIT_BLOCK) return BMM_ERR_ARG;
    if (count < 0 || draws < 0 || (draws > 0 && (idx == nullptr || scale == nullptr))) return BMM_ERR_ARG;
    if (count > 0 && (entries == nullptr || cd_out == nullptr || s2_out == nullptr)) return BMM_ERR_ARG;
    if (unit == BMM_UNIT_COLUMN && ck == nullptr) return BMM_ERR_ARG;
    Carver cnt{nullptr};
    cnt.take<int64_t>(B->K + 1);
    if ((s = check_ws(ws, ws_bytes, cnt.off)) != BMM_OK) return s;
    Carver cv{static_cast<char*>(ws) + kStatusBytes};
    int64_t* start = cv.take<int64_t>(B->K + 1);
    BMM_TRY(launch_entry_estimate(view_of(M), view_of(N), B->offsets, B->K, unit, ck, idx, scale, draws, entries, count,
                                  cd_out, s2_out, start, status_of(ws), reinterpret_cast<cudaStream_t>(stream)));
    return BMM_OK;
}
