// design.cu -- sampling probabilities (eq. 3.8, Table 2, eq. 1.2, eq. 1.4) and integer
// block sizes (eq. 3.9, eq. 4.2, eq. 4.7, c/K) for Alg. 2.
//
// The block-size search is exact and order-free: F(lam) = sum_k clamp(floor(lam g_k), 1, n_k)
// is an integer sum of element-wise IEEE operations, so the largest FP64 lam with F(lam) <= c
// is one number whatever the reduction order.  One CTA finds it by a 32-way search over
// the IEEE bit patterns of the non-negative doubles (13 rounds instead of 63 bisections).
#include "internal.h"

namespace bmm {

__device__ __forceinline__ bool seg_ok(const int64_t* off, int64_t k, int64_t K, int64_t n, int64_t* lo, int64_t* hi) {
    *lo = off[k];
    *hi = off[k + 1];
    return *lo >= 0 && *hi > *lo && *hi <= n && (k != 0 || *lo == 0) && (k != K - 1 || *hi == n);
}

// ---------------------------------------------------------------- column probabilities
__global__ void probs_col_kernel(int kind, const double* __restrict__ x, const double* __restrict__ y,
                                 const double* __restrict__ a, const int64_t* __restrict__ off, int64_t K,
                                 int64_t n, double* __restrict__ p, DevStatus* st) {
    const int lane = threadIdx.x & 31;
    const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (k >= K) return;
    int64_t lo, hi;
    if (!seg_ok(off, k, K, n, &lo, &hi)) {
        if (lane == 0) set_status(st, BMM_ERR_SHAPE, (int)k);
        return;
    }
    const double uni = __ddiv_rn(1.0, (double)(hi - lo));
    const double ak = (kind == BMM_P_COL_OPT) ? a[k] : 0.0;
    for (int64_t i = lo + lane; i < hi; i += 32) {
        double v = uni;
        if (kind == BMM_P_COL_OPT && ak > 0.0) v = __ddiv_rn(sqrt(__dmul_rn(x[i], y[i])), ak);
        p[i] = v;
    }
}

// ---------------------------------------------------------------- block probabilities (one CTA)
__device__ double block_sum_1024(double v, double* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
        t = warp_sum(t);
        if (lane == 0) red[32] = t;
    }
    __syncthreads();
    t = red[32];
    __syncthreads();
    return t;
}

__global__ void __launch_bounds__(1024) probs_blk_kernel(int kind, const double* __restrict__ mf,
                                                         const double* __restrict__ nf,
                                                         const double* __restrict__ f, int64_t K,
                                                         double* __restrict__ p, DevStatus* st) {
    __shared__ double red[33];
    double part = 0.0;
    for (int64_t k = threadIdx.x; k < K; k += blockDim.x) {
        const double v = (kind == BMM_P_BLK_PRODNORM) ? sqrt(f[k]) : sqrt(__dmul_rn(mf[k], nf[k]));
        if (!isfinite(v)) set_status(st, BMM_ERR_NONFINITE, (int)k);
        part += v;
    }
    const double total = block_sum_1024(part, red);
    const double uni = __ddiv_rn(1.0, (double)K);
    for (int64_t k = threadIdx.x; k < K; k += blockDim.x) {
        const double v = (kind == BMM_P_BLK_PRODNORM) ? sqrt(f[k]) : sqrt(__dmul_rn(mf[k], nf[k]));
        p[k] = total > 0.0 ? __ddiv_rn(v, total) : uni;
    }
}

cudaError_t launch_probs(int kind, const double* x, const double* y, const double* a, const double* mf,
                         const double* nf, const double* f, const int64_t* off, int64_t K, int64_t n, double* p,
                         DevStatus* st, cudaStream_t s) {
    if (kind == BMM_P_COL_OPT || kind == BMM_P_COL_UNIFORM) {
        (count_launch(), probs_col_kernel<<<(unsigned)ceil_div(K * 32, 256), 256, 0, s>>>(kind, x, y, a, off, K, n, p, st));
    } else {
        (count_launch(), probs_blk_kernel<<<1, 1024, 0, s>>>(kind, mf, nf, f, K, p, st));
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- block sizes (one CTA)
constexpr unsigned long long kInfBits = 0x7FF0000000000000ull;
constexpr int kActiveCap = 2048;  // blocks tracked in shared memory (K above: no pruning, FP64 counts)

__device__ __forceinline__ long long count_at(double lam, double g, long long nk) {
    if (!(g > 0.0)) return 1;
    // trunc == floor for lam * g >= 0; the conversion saturates, so +inf and huge values clamp to nk
    long long v = __double2ll_rz(__dmul_rn(lam, g));
    return v < 1 ? 1 : (v > nk ? nk : v);
}

// count_at(lam, g, nk), decided in FP32 when that is certain.  lamf = RN32(lam), gf = RN32(g): with
// all three in the normal range, t = RN32(lamf * gf) is within 3 * 2^-24 of lam * g, and the FP64
// product RN64(lam * g) within 2^-53 of it, so RN64(lam * g) lies in [t - 4e-7 t, t + 4e-7 t].
// When that interval holds one integer floor (or lies below 1, or at or above nk), the FP64 count
// is known without an FP64 instruction (GB300's FP64 pipe is ~1/64 of FP32); otherwise it is
// computed exactly.  The result is always count_at's.
__device__ __forceinline__ long long count_fast(double lam, float lamf, float gf, int nk, double g) {
    const float t = __fmul_rn(lamf, gf);
    if (lamf >= 1.17549435e-38f && gf >= 1.17549435e-38f && t >= 1.17549435e-38f && t <= 1.0e30f) {
        const float mg = __fmul_rn(t, 4.0e-7f);
        const float th = __fadd_rn(t, mg);
        if (th < 1.0f) return 1;
        const float tl = __fsub_rn(t, mg);
        if (nk < (1 << 24) && tl >= (float)nk) return nk;
        const float fl = floorf(tl);
        if (fl == floorf(th)) {
            const long long v = (long long)fl;
            return v < 1 ? 1 : (v > nk ? nk : v);
        }
    }
    return count_at(lam, g, nk);
}

__device__ __forceinline__ double bits_to_lam(unsigned long long u) { return __longlong_as_double((long long)u); }

// exclusive scan of one value per thread over a 1024-thread block (exact)
__device__ long long block_exclusive_scan(long long v, long long* sm, long long* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) sm[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        long long w = sm[lane];
        long long wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        sm[lane] = wi - w;   // exclusive prefix of warp totals
        if (lane == 31) sm[32] = wi;
    }
    __syncthreads();
    const long long res = sm[warp] + inc - v;
    *total = sm[32];
    __syncthreads();
    return res;
}

__device__ long long block_sum_ll(long long v, long long* sm) {
    long long t;
    block_exclusive_scan(v, sm, &t);
    return t;
}

// F(u) = sum_k count(u, k) over all blocks, by the whole CTA (exact)
__device__ long long block_F(unsigned long long u, const double* g, const int64_t* off, int64_t K, long long* sm) {
    const double lam = bits_to_lam(u);
    long long acc = 0;
    for (int64_t k = threadIdx.x; k < K; k += 1024) acc += count_at(lam, g[k], off[k + 1] - off[k]);
    return block_sum_ll(acc, sm);
}

__global__ void __launch_bounds__(1024) blocksizes_kernel(int kind, const double* __restrict__ a,
                                                          const double* __restrict__ f,
                                                          const int64_t* __restrict__ off, int64_t K, int64_t n,
                                                          int64_t c, int64_t* __restrict__ ck, double* __restrict__ g,
                                                          DevStatus* st) {
    __shared__ long long sF[32];
    __shared__ unsigned long long sLoHi[2];
    __shared__ long long sScan[33];
    __shared__ int sAct[2][kActiveCap];
    __shared__ float sGf[kActiveCap];  // RN32(g_k), for count_fast
    __shared__ int sNk[kActiveCap];
    __shared__ int sNact[2];
    __shared__ double sRed[33];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // 1. weights g_k
    int bad = 0, bad_off = 0, any_pos = 0, any_a = 0;
    for (int64_t k = tid; k < K; k += 1024) {
        const int64_t lo = off[k], hi = off[k + 1];
        if (hi <= lo || lo < 0 || hi > n) bad_off = 1;
        double gk = 1.0;
        if (kind != BMM_CK_EQUAL) {
            const double ak = a[k];
            if (!isfinite(ak) || ak < 0.0) bad = 1;
            any_a |= ak > 0.0;
            if (kind == BMM_CK_OPT || kind == BMM_CK_TILDE) {
                const double fk = f[k];
                if (!isfinite(fk)) bad = 1;
                const double d = __dsub_rn(__dmul_rn(ak, ak), fk);
                gk = (kind == BMM_CK_OPT) ? sqrt(fmax(d, 0.0)) : sqrt(fabs(d));
            } else {
                gk = ak;
            }
        }
        if (!isfinite(gk)) bad = 1;
        any_pos |= gk > 0.0;
        g[k] = gk;
    }
    bad = __syncthreads_or(bad);
    bad_off = __syncthreads_or(bad_off);
    any_pos = __syncthreads_or(any_pos);
    any_a = __syncthreads_or(any_a);
    if (bad || bad_off) {
        if (tid == 0) set_status(st, bad_off ? BMM_ERR_SHAPE : BMM_ERR_NONFINITE);
        for (int64_t k = tid; k < K; k += 1024) ck[k] = 1;
        return;
    }
    if (!any_pos) {  // every weight zero: fall back to a_k, then to n_k
        for (int64_t k = tid; k < K; k += 1024) g[k] = any_a ? a[k] : (double)(off[k + 1] - off[k]);
    }
    __syncthreads();

    // 2. lam* = the largest FP64 lam with F(lam) <= c.  F is monotone, so any bracket
    //    lo < hi with F(lo) <= c < F(hi) leads to the same lam*.
    const long long Finf = block_F(kInfBits, g, off, K, sScan);
    const bool inf_case = Finf <= c;
    unsigned long long lo = 0ull, hi = kInfBits;
    if (!inf_case) {
        // a guess lam0 = c / sum g narrows the bracket when it verifies
        double gs = 0.0;
        for (int64_t k = tid; k < K; k += 1024) gs += g[k];
        gs = warp_sum(gs);
        if (lane == 0) sRed[warp] = gs;
        __syncthreads();
        if (warp == 0) {
            double t = warp_sum(sRed[lane]);
            if (lane == 0) sRed[32] = t;
        }
        __syncthreads();
        const double lam0 = (double)c / sRed[32];
        if (isfinite(lam0) && lam0 > 0.0) {
            const unsigned long long ulo = (unsigned long long)__double_as_longlong(lam0 * 0.25);
            const unsigned long long uhi = (unsigned long long)__double_as_longlong(lam0 * 4.0);
            if (uhi < kInfBits && block_F(ulo, g, off, K, sScan) <= c) lo = ulo;
            if (uhi < kInfBits && block_F(uhi, g, off, K, sScan) > c) hi = uhi;
        }
        // active list: blocks whose count may still change inside (lo, hi)
        const bool track = K <= kActiveCap;
        if (tid == 0) { sNact[0] = 0; sLoHi[0] = lo; sLoHi[1] = hi; }
        if (track)
            for (int64_t k = tid; k < K; k += 1024) {
                sGf[k] = __double2float_rn(g[k]);
                sNk[k] = (int)(off[k + 1] - off[k]);
            }
        __syncthreads();
        int cur = 0;
        long long base = 0;
        if (track) {
            long long mine = 0;
            const double llo = bits_to_lam(lo), lhi = bits_to_lam(hi);
            const float flo = __double2float_rn(llo), fhi = __double2float_rn(lhi);
            for (int64_t k = tid; k < K; k += 1024) {
                const int nk = sNk[k];
                const long long clo = count_fast(llo, flo, sGf[k], nk, g[k]), chi = count_fast(lhi, fhi, sGf[k], nk, g[k]);
                if (clo == chi) mine += clo;
                else sAct[0][atomicAdd(&sNact[0], 1)] = (int)k;
            }
            base = block_sum_ll(mine, sScan);
        }
        while (hi - lo > 1ull) {
            const unsigned long long d = hi - lo;
            const int nact = track ? sNact[cur] : 0;
            if (warp >= 1) {
                const unsigned long long w = (unsigned long long)warp;
                const unsigned long long u = lo + (d >> 5) * w + (((d & 31ull) * w) >> 5);
                const double lam = bits_to_lam(u);
                const float lamf = __double2float_rn(lam);
                long long acc = 0;
                if (track) {
                    for (int i = lane; i < nact; i += 32) {
                        const int k = sAct[cur][i];
                        acc += count_fast(lam, lamf, sGf[k], sNk[k], g[k]);
                    }
                } else {
                    for (int64_t k = lane; k < K; k += 32) acc += count_at(lam, g[k], off[k + 1] - off[k]);
                }
                acc = warp_sum_ll(acc);
                if (lane == 0) sF[warp] = base + acc;
            }
            __syncthreads();
            if (tid == 0) {
                unsigned long long nlo = lo, nhi = hi;
                for (int w = 1; w < 32; ++w) {
                    const unsigned long long u =
                        lo + (d >> 5) * (unsigned long long)w + (((d & 31ull) * (unsigned long long)w) >> 5);
                    if (sF[w] <= c) {
                        if (u > nlo) nlo = u;
                    } else if (u < nhi) {
                        nhi = u;
                    }
                }
                sLoHi[0] = nlo;
                sLoHi[1] = nhi;
                sNact[cur ^ 1] = 0;
            }
            __syncthreads();
            lo = sLoHi[0];
            hi = sLoHi[1];
            if (track) {  // drop the blocks whose count is now constant on [lo, hi]
                long long mine = 0;
                const double llo = bits_to_lam(lo), lhi = bits_to_lam(hi);
                const float flo = __double2float_rn(llo), fhi = __double2float_rn(lhi);
                for (int i = tid; i < nact; i += 1024) {
                    const int k = sAct[cur][i];
                    const int nk = sNk[k];
                    const long long clo = count_fast(llo, flo, sGf[k], nk, g[k]);
                    const long long chi = count_fast(lhi, fhi, sGf[k], nk, g[k]);
                    if (clo == chi) mine += clo;
                    else sAct[cur ^ 1][atomicAdd(&sNact[cur ^ 1], 1)] = k;
                }
                base += block_sum_ll(mine, sScan);
                cur ^= 1;
            }
            __syncthreads();
        }
    }
    const unsigned long long ustar = inf_case ? kInfBits : lo;
    const double lam = bits_to_lam(ustar);

    // 3. counts at lam*, each thread owning a contiguous run of k
    const int64_t chunk = ceil_div(K, 1024);
    const int64_t k0 = imin(K, tid * chunk), k1 = imin(K, k0 + chunk);
    long long mine = 0;
    for (int64_t k = k0; k < k1; ++k) {
        const long long v = count_at(lam, g[k], off[k + 1] - off[k]);
        ck[k] = v;
        mine += v;
    }
    long long total;
    block_exclusive_scan(mine, sScan, &total);
    const long long r = c - total;
    if (r > 0) {
        if (!inf_case) {
            const double lam2 = bits_to_lam(ustar + 1ull);
            long long gcount = 0;
            for (int64_t k = k0; k < k1; ++k) gcount += count_at(lam2, g[k], off[k + 1] - off[k]) > ck[k];
            long long gt;
            long long rank = block_exclusive_scan(gcount, sScan, &gt);
            for (int64_t k = k0; k < k1; ++k) {
                if (count_at(lam2, g[k], off[k + 1] - off[k]) > ck[k]) {
                    if (rank < r) ck[k] += 1;
                    ++rank;
                }
            }
            if (tid == 0 && gt <= r) set_status(st, BMM_ERR_INFEASIBLE, 1);
        } else {
            long long cap = 0;
            for (int64_t k = k0; k < k1; ++k) cap += (off[k + 1] - off[k]) - ck[k];
            long long ct;
            long long before = block_exclusive_scan(cap, sScan, &ct);
            for (int64_t k = k0; k < k1; ++k) {
                const long long capk = (off[k + 1] - off[k]) - ck[k];
                long long add = r - before;
                add = add < 0 ? 0 : (add > capk ? capk : add);
                ck[k] += add;
                before += capk;
            }
            if (tid == 0 && ct < r) set_status(st, BMM_ERR_INFEASIBLE, 2);
        }
    }
}

cudaError_t launch_blocksizes(int kind, const double* a, const double* f, const int64_t* off, int64_t K, int64_t n,
                              int64_t c, int64_t* ck, double* g, DevStatus* st, cudaStream_t s) {
    (count_launch(), blocksizes_kernel<<<1, 1024, 0, s>>>(kind, a, f, off, K, n, c, ck, g, st));
    return cudaGetLastError();
}

}  // namespace bmm
