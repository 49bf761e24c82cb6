// design.cu -- sampling probabilities (eq. 3.8, Table 2, eq. 1.2, eq. 1.4) and integer
// block sizes (eq. 3.9, eq. 4.2, eq. 4.7, c/K) for Alg. 2.
//
// The block-size search is exact and order-free: F(lam) = sum_k clamp(floor(lam g_k), 1, n_k)
// is an integer sum of element-wise IEEE operations, so the largest FP64 lam with F(lam) <= c
// is one number whatever the reduction order.  One CTA finds it: 32 candidates lam0 2^j around
// lam0 = c / sum g give a bracket one binade wide, 32-way rounds over the IEEE bit patterns in the
// bracket narrow it (blocks whose count is constant on it leave an active list), and once at most
// 256 steps of F are left each step is located exactly and lam* read off by rank.
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
// computed exactly.  The result is always count_at's.  Floors are taken by adding 2^23 rounding
// down (exact for 0 <= x < 2^23, and >= 2^23 for larger x, which only the clamp at nk < 2^23
// sees), so that no conversion instruction is needed.
__device__ __forceinline__ long long count_fast(double lam, float lamf, float gf, int nk, const double* g) {
    const float t = __fmul_rn(lamf, gf);
    if (lamf >= 1.17549435e-38f && gf >= 1.17549435e-38f && t >= 1.17549435e-38f && t <= 1.0e30f &&
        nk < (1 << 23)) {
        const float mg = __fmul_rn(t, 4.0e-7f);
        const float th = __fadd_rn(t, mg);
        if (th < 1.0f) return 1;
        const float tl = __fsub_rn(t, mg);
        const int il = __float_as_int(__fadd_rd(tl, 8388608.0f)) - 0x4B000000;  // floor(tl)
        if (il >= nk) return nk;
        const int ih = __float_as_int(__fadd_rd(th, 8388608.0f)) - 0x4B000000;  // floor(th)
        if (il == ih) return il < 1 ? 1 : il;
    }
    return count_at(lam, *g, nk);
}

__device__ __forceinline__ double bits_to_lam(unsigned long long u) { return __longlong_as_double((long long)u); }

// The smallest lam (as a bit pattern) with count_at(lam, g, nk) >= j, for 2 <= j <= nk and g > 0:
// there trunc(RN(lam g)) >= j iff RN(lam g) >= j, which is monotone in lam.  RN(j / g) puts
// RN(lam g) within a few units in the last place of j, so single bit-pattern steps from it end
// within two; more than eight (or an overflow) report failure and the caller keeps bisecting.
__device__ __forceinline__ bool breakpoint_of(double g, long long j, unsigned long long* out) {
    const double jd = (double)j;
    unsigned long long u = (unsigned long long)__double_as_longlong(__ddiv_rn(jd, g));
    if (u >= kInfBits) return false;
    int steps = 0;
    if (__dmul_rn(bits_to_lam(u), g) >= jd) {
        while (u > 0ull && __dmul_rn(bits_to_lam(u - 1ull), g) >= jd) {
            --u;
            if (++steps > 8) return false;
        }
    } else {
        do {
            ++u;
            if (++steps > 8 || u >= kInfBits) return false;
        } while (!(__dmul_rn(bits_to_lam(u), g) >= jd));
    }
    *out = u;
    return true;
}

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

// two block-wide sums at once (exact), returned in place to every thread; sm holds 64 values
__device__ void block_sum2_ll(long long* a, long long* b, long long* sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
    long long x = *a, y = *b;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, o);
        y += __shfl_xor_sync(0xffffffffu, y, o);
    }
    if (lane == 0) {
        sm[warp] = x;
        sm[32 + warp] = y;
    }
    __syncthreads();
    x = lane < nw ? sm[lane] : 0;
    y = lane < nw ? sm[32 + lane] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, o);
        y += __shfl_xor_sync(0xffffffffu, y, o);
    }
    __syncthreads();  // every read done before sm is written again
    *a = x;
    *b = y;
}

// F(u) = sum_k count(u, k) over all blocks, by the whole CTA (exact)
__device__ long long block_F(unsigned long long u, const double* g, const int64_t* off, int64_t K, long long* sm) {
    const double lam = bits_to_lam(u);
    long long acc = 0;
    for (int64_t k = threadIdx.x; k < K; k += 1024) acc += count_at(lam, g[k], off[k + 1] - off[k]);
    return block_sum_ll(acc, sm);
}

// candidate w of n = 32 or 1024 evenly spaced bit patterns in [lo, lo + d): lo + floor(w d / n)
__device__ __forceinline__ unsigned long long cand_32(unsigned long long lo, unsigned long long d, unsigned long long w) {
    return lo + (d >> 5) * w + (((d & 31ull) * w) >> 5);
}
__device__ __forceinline__ unsigned long long cand_1024(unsigned long long lo, unsigned long long d, unsigned long long w) {
    return lo + (d >> 10) * w + (((d & 1023ull) * w) >> 10);
}

// appends k to an active list for the lanes with keep set: one shared atomic per warp
__device__ __forceinline__ void push_active(bool keep, int k, int* list, int* count, int lane) {
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    int pos = 0;
    if (lane == 0 && m != 0u) pos = atomicAdd(count, __popc(m));
    pos = __shfl_sync(0xffffffffu, pos, 0);
    if (keep) list[pos + __popc(m & ((1u << lane) - 1u))] = k;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

constexpr int kEndgameSteps = 256;  // steps of F left in (lo, hi] at or below which they are found directly

// The block sizes of one product by the whole (1024-thread) CTA.
__device__ __forceinline__ void blocksizes_body(int kind, const double* __restrict__ a, const double* __restrict__ f,
                                                const int64_t* __restrict__ off, int64_t K, int64_t n, int64_t c,
                                                int64_t* __restrict__ ck, double* __restrict__ g, DevStatus* st) {
    __shared__ long long sF[32];
    __shared__ unsigned long long sLoHi[2];
    __shared__ long long sScan[33];
    __shared__ long long sSum2[64];
    __shared__ int sAct[2][kActiveCap];
    __shared__ float sGf[kActiveCap];  // RN32(g_k), for count_fast
    __shared__ int sNk[kActiveCap];
    __shared__ int sNact[2];
    __shared__ float sRedF[32];
    __shared__ double sLam0;
    __shared__ int sEgLo[kEndgameSteps], sEgPre[kEndgameSteps];
    __shared__ unsigned long long sEgStep[kEndgameSteps];
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
        // a guess lam0 = c / sum g (an FP32 sum is enough: it only places the candidates below)
        float gs = 0.f;
        for (int64_t k = tid; k < K; k += 1024) gs += __double2float_rn(g[k]);
        gs = warp_sum_f(gs);
        if (lane == 0) sRedF[warp] = gs;
        const bool track = K <= kActiveCap;
        if (tid == 0) sNact[0] = 0;
        if (track)
            for (int64_t k = tid; k < K; k += 1024) {
                sGf[k] = __double2float_rn(g[k]);
                sNk[k] = (int)(off[k + 1] - off[k]);
            }
        __syncthreads();
        if (warp == 0) {
            const float t = warp_sum_f(sRedF[lane]);
            if (lane == 0) sLam0 = (double)c / (double)t;
        }
        __syncthreads();
        // 32 candidates lam0 2^(w - 8), w = 0..31, one per warp, its lanes splitting the blocks; F is
        // monotone, so the candidates with F <= c form a prefix and the bracket becomes the pair
        // around its end (an exponent step: exact).  Candidates past the largest double are +inf
        // (F(inf) > c), those below the normal range 0 (F(0) = K <= c).  Without a usable lam0
        // the bracket stays [0, inf).
        const double lam0 = sLam0;
        const unsigned long long b0 = (unsigned long long)__double_as_longlong(lam0);
        const long long e0 = (long long)((b0 >> 52) & 0x7FFull);
        const bool usable = isfinite(lam0) && lam0 > 0.0 && e0 >= 1;
        auto geo = [&](int w) -> unsigned long long {
            const long long e = e0 + (w - 8);
            return e >= 2047 ? kInfBits : (e <= 0 ? 0ull : b0 + ((unsigned long long)(long long)(w - 8) << 52));
        };
        if (usable) {
            const unsigned long long u = geo(warp);
            const double lam = bits_to_lam(u);
            const float lamf = __double2float_rn(lam);
            long long acc = 0;
            if (track) {
                for (int k = lane; k < (int)K; k += 32) acc += count_fast(lam, lamf, sGf[k], sNk[k], g + k);
            } else {
                for (int64_t k = lane; k < K; k += 32) acc += count_at(lam, g[k], off[k + 1] - off[k]);
            }
            acc = warp_sum_ll(acc);
            if (lane == 0) sF[warp] = acc;
        }
        __syncthreads();
        if (usable) {
            if (warp == 0) {
                const int t = __popc(__ballot_sync(0xffffffffu, sF[lane] <= c)) - 1;
                if (lane == 0) {
                    sLoHi[0] = t >= 0 ? geo(t) : 0ull;
                    sLoHi[1] = t < 31 ? geo(t + 1) : kInfBits;
                }
            }
            __syncthreads();
            lo = sLoHi[0];
            hi = sLoHi[1];
        }
        // active list: blocks whose count may still change inside (lo, hi); counts of the others
        // are summed into base, and nbrk = F(hi) - F(lo) counts the steps of F inside (lo, hi]
        int cur = 0;
        long long base = 0, nbrk = 0;
        if (track) {
            long long mine = 0, steps = 0;
            const double llo = bits_to_lam(lo), lhi = bits_to_lam(hi);
            const float flo = __double2float_rn(llo), fhi = __double2float_rn(lhi);
            for (int k0 = warp * 32; k0 < (int)K; k0 += 1024) {  // warp-uniform trips
                const int k = k0 + lane;
                bool keep = false;
                if (k < (int)K) {
                    const long long clo = count_fast(llo, flo, sGf[k], sNk[k], g + k);
                    const long long chi = count_fast(lhi, fhi, sGf[k], sNk[k], g + k);
                    if (clo == chi) mine += clo;
                    else keep = true;
                    steps += chi - clo;
                }
                push_active(keep, k, sAct[0], &sNact[0], lane);
            }
            block_sum2_ll(&mine, &steps, sSum2);
            base = mine;
            nbrk = steps;
        }
        bool endgame = true;
        while (hi - lo > 1ull) {
            const unsigned long long d = hi - lo;
            const int nact = track ? sNact[cur] : 0;
            if (track && endgame && nbrk <= kEndgameSteps && nbrk > 0 && nact <= kEndgameSteps) {
                // Few steps of F are left in (lo, hi]: find each one exactly (the bit pattern where an
                // active block's count reaches j), then lam* sits just below the (c - F(lo) + 1)-th
                // smallest of them.  F(lam) = F(lo) + #{steps <= lam} on [lo, hi].
                long long clo = 0, dlt = 0;
                if (tid < nact) {
                    const int k = sAct[cur][tid];
                    clo = count_at(bits_to_lam(lo), g[k], sNk[k]);
                    dlt = count_at(bits_to_lam(hi), g[k], sNk[k]) - clo;
                    sEgLo[tid] = (int)clo;
                }
                long long total_lo = clo, total_dlt = dlt;
                block_sum2_ll(&total_lo, &total_dlt, sSum2);
                long long nsteps;
                const long long pre = block_exclusive_scan(tid < nact ? dlt : 0, sScan, &nsteps);
                if (tid < nact) sEgPre[tid] = (int)pre;
                __syncthreads();
                bool fail = nsteps != nbrk || nsteps > kEndgameSteps;
                if (!fail && tid < nsteps) {
                    int a = 0, b = nact - 1;  // the active block whose steps hold step number tid
                    while (a < b) {
                        const int mid = (a + b + 1) >> 1;
                        if (sEgPre[mid] <= tid) a = mid;
                        else b = mid - 1;
                    }
                    const int k = sAct[cur][a];
                    const long long jj = (long long)sEgLo[a] + 1 + (tid - sEgPre[a]);
                    unsigned long long u = 0ull;
                    fail = !breakpoint_of(g[k], jj, &u);
                    sEgStep[tid] = u;
                }
                fail = __syncthreads_or(fail);
                if (!fail) {
                    const long long r = c - (base + total_lo);  // 0 <= r < nsteps
                    if (tid < nsteps) {
                        const unsigned long long v = sEgStep[tid];
                        int less = 0, eq = 0;
                        for (int q = 0; q < (int)nsteps; ++q) {
                            const unsigned long long w = sEgStep[q];
                            less += w < v;
                            eq += w == v;
                        }
                        if (less <= r && r < less + eq) sLoHi[0] = v - 1ull;
                    }
                    __syncthreads();
                    lo = sLoHi[0];
                    hi = lo + 1ull;
                    break;
                }
                endgame = false;  // not expected; bisection below stays exact
            }
            if (tid == 0) sNact[cur ^ 1] = 0;
            // 32 candidates u_w = lo + floor(w d / 32), warp w >= 1 evaluating u_w with its lanes
            // splitting the blocks; warp 0 picks the last candidate with F <= c by a ballot
            if (warp >= 1) {
                const unsigned long long u = cand_32(lo, d, (unsigned long long)warp);
                const double lam = bits_to_lam(u);
                const float lamf = __double2float_rn(lam);
                long long acc = 0;
                if (track) {
                    for (int i = lane; i < nact; i += 32) {
                        const int k = sAct[cur][i];
                        acc += count_fast(lam, lamf, sGf[k], sNk[k], g + k);
                    }
                } else {
                    for (int64_t k = lane; k < K; k += 32) acc += count_at(lam, g[k], off[k + 1] - off[k]);
                }
                acc = warp_sum_ll(acc);
                if (lane == 0) sF[warp] = base + acc;
            }
            __syncthreads();
            if (warp == 0) {
                const bool ok = lane == 0 || sF[lane] <= c;
                const int t = __popc(__ballot_sync(0xffffffffu, ok)) - 1;  // a prefix: F is monotone
                if (lane == 0) {
                    sLoHi[0] = cand_32(lo, d, (unsigned long long)t);
                    sLoHi[1] = t < 31 ? cand_32(lo, d, (unsigned long long)(t + 1)) : hi;
                }
            }
            __syncthreads();
            lo = sLoHi[0];
            hi = sLoHi[1];
            if (track) {  // drop the blocks whose count is now constant on [lo, hi]
                long long mine = 0, steps = 0;
                if (warp * 32 < nact) {
                    const double llo = bits_to_lam(lo), lhi = bits_to_lam(hi);
                    const float flo = __double2float_rn(llo), fhi = __double2float_rn(lhi);
                    for (int i0 = warp * 32; i0 < nact; i0 += 1024) {  // warp-uniform trips
                        const int i = i0 + lane;
                        bool keep = false;
                        int k = 0;
                        if (i < nact) {
                            k = sAct[cur][i];
                            const long long clo = count_fast(llo, flo, sGf[k], sNk[k], g + k);
                            const long long chi = count_fast(lhi, fhi, sGf[k], sNk[k], g + k);
                            if (clo == chi) mine += clo;
                            else keep = true;
                            steps += chi - clo;
                        }
                        push_active(keep, k, sAct[cur ^ 1], &sNact[cur ^ 1], lane);
                    }
                }
                block_sum2_ll(&mine, &steps, sSum2);
                base += mine;
                nbrk = steps;
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

__global__ void __launch_bounds__(1024) blocksizes_kernel(int kind, const double* __restrict__ a,
                                                          const double* __restrict__ f,
                                                          const int64_t* __restrict__ off, int64_t K, int64_t n,
                                                          int64_t c, int64_t* __restrict__ ck, double* __restrict__ g,
                                                          DevStatus* st) {
    blocksizes_body(kind, a, f, off, K, n, c, ck, g, st);
}

cudaError_t launch_blocksizes(int kind, const double* a, const double* f, const int64_t* off, int64_t K, int64_t n,
                              int64_t c, int64_t* ck, double* g, DevStatus* st, cudaStream_t s) {
    (count_launch(), blocksizes_kernel<<<1, 1024, 0, s>>>(kind, a, f, off, K, n, c, ck, g, st));
    return cudaGetLastError();
}

// Many products' block sizes in one launch: CTA i computes job i (the same body, so every c_k is
// the one bmm_blocksizes gives for that product alone).
struct SizesTable {
    int count;
    SizesJob job[kMaxSizesJobs];
};
static_assert(sizeof(SizesTable) <= 32764, "block-size table exceeds the kernel-parameter limit");

__global__ void __launch_bounds__(1024) blocksizes_grouped_kernel(const __grid_constant__ SizesTable tab) {
    const SizesJob& j = tab.job[blockIdx.x];
    blocksizes_body(j.kind, j.a, j.f, j.off, j.K, j.n, j.c, j.ck, j.g, j.st);
}

cudaError_t launch_blocksizes_grouped(const SizesJob* jobs, int64_t count, cudaStream_t s) {
    static thread_local SizesTable tab;  // host-side staging of the kernel parameter, one per host thread
    for (int64_t i0 = 0; i0 < count; i0 += kMaxSizesJobs) {
        tab.count = (int)imin(count - i0, kMaxSizesJobs);
        for (int q = 0; q < tab.count; ++q) tab.job[q] = jobs[i0 + q];
        (count_launch(), blocksizes_grouped_kernel<<<(unsigned)tab.count, 1024, 0, s>>>(tab));
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace bmm
