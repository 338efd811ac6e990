// Input affinities of each chunk: per-row precision search (Eq. 1, Eq. 2) and
// the symmetric joint P (Eq. 3, with n := z, the chunk size).
//
// Row search: a group of 128 threads per row holds the row in registers as
// t_j = d_ij - m_i (m_i = min_{j!=i} d_ij; the shift cancels in Eq. 1).  The
// entropy H(beta) = ln S + beta T1 / S with S = sum e_j, T1 = sum t_j e_j,
// e_j = exp(-beta t_j), is non-increasing in beta, so the root of
// H(beta) = ln(perplexity) is bracketed and found by bisection on beta,
// accelerated by Newton steps in ln(beta) (dH/dln(beta) = -beta^2 Var_p(t))
// whenever the Newton point falls inside the bracket.  Sums are FP32 per
// thread (compensated once the root is near) and combined across the group
// with error-free two-sums; warp 0 combines them, takes the step and
// publishes the next beta through shared memory.  A row whose FP32 search
// stalls (bracket collapsed, or 64 evaluations) is redone in FP64 by the same
// group.
#include <float.h>

#include "ptsne_internal.cuh"

namespace ptsne {

namespace {
constexpr int kGroup = 128;            // threads per row
constexpr float kBig = 1e37f;          // stands for "excluded" (diagonal, tail padding)
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kTolFine = 1e-6f;      // |H - ln perp| (nats) accepted from the FP32 search
constexpr float kTolCoarse = 1e-3f;    // switch to compensated sums below this
// The entropy error f maps to a relative beta error f / (beta^2 Var(t))
// (dH / d ln beta = -beta^2 Var(t)), and a relative beta error e moves an
// entry p ~ exp(-beta t) by e beta t relative: entries down to 1e-6 of the
// row's largest (beta t ~ 14) stay within ~4e-5 when e <= 3e-6.  So a row is
// accepted when |f| <= min(kTolFine, kTolBeta beta^2 Var(t)).
constexpr float kTolBeta = 3e-6f;
constexpr double kTol64 = 1e-9;        // FP64 fallback tolerance
constexpr int kMaxEval32 = 64;
constexpr int kMaxEval64 = 200;
// FP64 redo: an entry with b t > 40 weighs e^-40 < 2^-57 of the row's largest
// (t = 0), so the sums cannot see it; the entries with b0 t <= 60 at the
// redo's starting beta b0 are compacted once and stand for the row while
// b >= (2/3) b0 (then every entry with b t <= 40 is among them).
constexpr double kNear64 = 60.0;
constexpr double kNearKeep = 2.0 / 3.0;
constexpr int kNearMax = 1024;
}  // namespace

// Mixed-precision bookkeeping of a search (all NULL: none): the chunks
// computed in FP32 whole, the window tiles of the dense rows, and the window
// pairs and (z - 1) summed per chunk-size bin.
struct FormArgs {
    const uint8_t* chunk_fp32 = nullptr;
    uint8_t* tflag = nullptr;
    const int64_t* tflag_off = nullptr;
    unsigned long long* form_acc = nullptr;
    int zmin = 0, zmax = 0;
    bool fp32_warm = false;   // beta_init of the FP32 chunks' rows is a warm start (else unset)
};

// packed FP32 pairs (f32x2 arithmetic, round to nearest like the scalar ops)
typedef unsigned long long f2;
__device__ __forceinline__ f2 pk(float a, float b) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk(f2 v, float& a, float& b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v)); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// s + v with the rounding error carried in c (error-free two-sum)
__device__ __forceinline__ void two_sum_add(float& s, float& c, float v, float cv) {
    const float t = s + v;
    const float bb = t - s;
    const float e = (s - (t - bb)) + (v - bb);
    s = t;
    c = c + cv + e;
}

__device__ __forceinline__ float group_sum(float v, float* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float a = red[0];
#pragma unroll
    for (int w = 1; w < kGroup / 32; ++w) a += red[w];
    __syncthreads();
    return a;
}
__device__ __forceinline__ float group_min(float v, float* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_min(v);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float a = red[0];
#pragma unroll
    for (int w = 1; w < kGroup / 32; ++w) a = fminf(a, red[w]);
    __syncthreads();
    return a;
}

struct RowSums {
    float S, T1, T2;
};

// S, T1 and T2 summed over the 128-thread group: each warp reduces its sums
// with shuffles and lane 0 publishes them (with comp, S and T1 carry their
// rounding errors, combined by error-free two-sums); after a barrier,
// combine_sums3 adds the 4 warps' partials in a fixed order.
__device__ __forceinline__ void publish_sums3(float S, float cS, float T1, float cT, float T2, bool comp,
                                              float (*red)[5]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (comp) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float s1 = __shfl_xor_sync(0xffffffffu, S, o), c1 = __shfl_xor_sync(0xffffffffu, cS, o);
            const float s2 = __shfl_xor_sync(0xffffffffu, T1, o), c2 = __shfl_xor_sync(0xffffffffu, cT, o);
            T2 += __shfl_xor_sync(0xffffffffu, T2, o);
            two_sum_add(S, cS, s1, c1);
            two_sum_add(T1, cT, s2, c2);
        }
    } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            S += __shfl_xor_sync(0xffffffffu, S, o);
            T1 += __shfl_xor_sync(0xffffffffu, T1, o);
            T2 += __shfl_xor_sync(0xffffffffu, T2, o);
        }
    }
    if (lane == 0) {
        red[warp][0] = S; red[warp][1] = cS; red[warp][2] = T1; red[warp][3] = cT; red[warp][4] = T2;
    }
}
__device__ __forceinline__ RowSums combine_sums3(bool comp, const float (*red)[5]) {
    float a = red[0][0], ac = red[0][1], b = red[0][2], bc = red[0][3], c = red[0][4];
#pragma unroll
    for (int w = 1; w < kGroup / 32; ++w) {
        if (comp) {
            two_sum_add(a, ac, red[w][0], red[w][1]);
            two_sum_add(b, bc, red[w][2], red[w][3]);
        } else {
            a += red[w][0];
            b += red[w][2];
        }
        c += red[w][4];
    }
    RowSums out;
    out.S = a + ac;
    out.T1 = b + bc;
    out.T2 = c;
    return out;
}

// S, T1, T2 of the row held in registers (excluded entries are kBig: e = 0),
// two entries per packed f32x2 instruction (two partial sums per thread),
// published per warp (see publish_sums3).
// Segment q (entries 512 q .. 512 q + 511 of the row) is skipped by the whole
// group when it lies beyond the chunk (z <= 512 q), so rows of small chunks do
// not pay for the register width of the largest one.
template <int VPT>
__device__ __forceinline__ void row_sums(const float (&t)[VPT], float beta, bool fine, float (*red5)[5], int z) {
    const float b2 = beta * kLog2e;
    const f2 NB = pk(-b2, -b2);
    float lo, hi;
    if (!fine) {
        f2 S = 0, T1 = 0, T2 = 0;
#pragma unroll
        for (int k = 0; k < VPT; k += 2) {
            if (4 * kGroup * (k / 4) >= z) break;
            const f2 T = pk(t[k], t[k + 1]);
            float x0, x1;
            upk(mul2(NB, T), x0, x1);
            const f2 E = pk(hw_ex2(x0), hw_ex2(x1));
            const f2 TE = mul2(T, E);
            S = add2(S, E);
            T1 = add2(T1, TE);
            T2 = fma2(TE, T, T2);
        }
        float s, t1, t2;
        upk(S, lo, hi); s = lo + hi;
        upk(T1, lo, hi); t1 = lo + hi;
        upk(T2, lo, hi); t2 = lo + hi;
        publish_sums3(s, 0.f, t1, 0.f, t2, false, red5);
        return;
    }
    // Kahan per half: true sum = S - cS
    f2 S = 0, cS = 0, T1 = 0, cT = 0, T2 = 0;
#pragma unroll
    for (int k = 0; k < VPT; k += 2) {
        if (4 * kGroup * (k / 4) >= z) break;
        const f2 T = pk(t[k], t[k + 1]);
        float x0, x1;
        upk(mul2(NB, T), x0, x1);
        const f2 E = pk(hw_ex2(x0), hw_ex2(x1));
        const f2 TE = mul2(T, E);
        f2 y = sub2(E, cS), s2 = add2(S, y);
        cS = sub2(sub2(s2, S), y);
        S = s2;
        y = sub2(TE, cT);
        s2 = add2(T1, y);
        cT = sub2(sub2(s2, T1), y);
        T1 = s2;
        T2 = fma2(TE, T, T2);
    }
    // the two halves' (sum, error) pairs combined error-free
    float s, cs, t1, ct, chi, t2;
    upk(S, s, hi);
    upk(cS, cs, chi);
    cs = -cs;
    two_sum_add(s, cs, hi, -chi);
    upk(T1, t1, hi);
    upk(cT, ct, chi);
    ct = -ct;
    two_sum_add(t1, ct, hi, -chi);
    upk(T2, lo, hi);
    t2 = lo + hi;
    publish_sums3(s, cs, t1, ct, t2, true, red5);
}

// One row per 128-thread block; thread `tid` holds entries j = 4 tid + 512 q + e.
// The search is bound by each row's chain of evaluations, so the more rows in
// flight the better: up to 40 entries per thread the kernel fits 8 blocks per
// SM (64 registers; measured 8% faster than 4 blocks at 121 registers).
template <int VPT>
__global__ void __launch_bounds__(kGroup, VPT >= 48 ? 3 : (VPT >= 16 ? 8 : 6))
bisect_group_kernel(const float* __restrict__ D, Layout L, int64_t r0, int64_t r1, double ln_perp_d,
                    float* __restrict__ beta_out, float* __restrict__ m_out, float* __restrict__ S_out,
                    DeviceStats* st, const float* beta_init, int coarse, const unsigned int* maxnorm,
                    uint8_t* __restrict__ row_dense, FormArgs fa) {
    __shared__ float red[kGroup / 32];
    __shared__ unsigned long long s_form[kFormBins][2];   // this block's window pairs and (z - 1) per size bin
    __shared__ float red5[kGroup / 32][5];
    __shared__ float s_bc[4];    // warp 0's decision: next beta, S, f, state
    __shared__ double redd3[kGroup / 32][3];
    __shared__ double s_bd[4];   // the same for the FP64 search
    __shared__ float s_near[kNearMax];   // FP64 redo: the row's entries that can matter
    __shared__ int s_wcnt[kGroup / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float ln_perp = (float)ln_perp_d;
    if (tid < 2 * kFormBins) s_form[tid >> 1][tid & 1] = 0ull;
    __syncthreads();
    for (int64_t r = r0 + blockIdx.x; r < r1; r += gridDim.x) {
        const int c = L.chunk_of_row[r];
        const int64_t off = L.off[c];
        const int z = (int)(L.off[c + 1] - off);
        const int i = (int)(r - off);
        const int ld = L.ld[c];
        const float* src = D + L.moff[c] + (int64_t)i * ld;
        const bool fp32_chunk = fa.chunk_fp32 && fa.chunk_fp32[c];
        if (coarse && fp32_chunk) {
            // computed in FP32 whole (the fine search alone): on to this
            // block's first row past the chunk (block-uniform)
            const int64_t end = L.off[c + 1];
            r += (end - r - 1) / gridDim.x * gridDim.x;
            continue;
        }

        float t[VPT];
        float mn = FLT_MAX;
#pragma unroll
        for (int q = 0; q < VPT / 4; ++q) {
            const int j0 = 4 * tid + 4 * kGroup * q;
            float4 v = make_float4(kBig, kBig, kBig, kBig);
            if (j0 < z) v = *reinterpret_cast<const float4*>(src + j0);   // j0 + 3 < ld
            const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int j = j0 + e;
                const float x = (j < z && j != i) ? vv[e] : kBig;
                t[4 * q + e] = x;
                if (x < kBig) mn = fminf(mn, x);
            }
        }
        mn = group_min(mn, red);
        float tsum = 0.f;
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
            if (t[k] < kBig) {
                t[k] -= mn;
                tsum += t[k];
            }
        }
        tsum = group_sum(tsum, red);

        float beta, S, herr;
        int evals = 0;
        bool fp64 = false, failed = false;
        if (!(tsum > 0.f)) {
            // every neighbour at the same distance: p_{j|i} = 1/(z-1) for every beta
            beta = 0.f;
            S = (float)(z - 1);
            herr = fabsf(logf((float)(z - 1)) - ln_perp);
            failed = herr > kTolFine;
        } else {
            float lo = 0.f, hi = INFINITY;
            beta = (float)(z - 1) / tsum;
            float f = INFINITY;
            // warm start (a chunk computed in FP32 whole holds no coarse beta:
            // its rows start from the previous epoch's, or from 1 / mean)
            if (beta_init && (!fp32_chunk || fa.fp32_warm)) {   // expected near the root: compensated at once
                const float b0 = beta_init[r];
                if (b0 > 0.f && isfinite(b0)) { beta = b0; f = 0.f; }
            }
            // Every warp evaluates its share of the row; warp 0 combines the sums,
            // keeps the bracket and the best compensated evaluation (H step one
            // ulp of beta makes there), decides, and publishes the next beta:
            // the other warps skip that scalar work.
            bool conv = false;
            float best_f = INFINITY, best_beta = beta, best_S = 0.f, best_ulp_h = 0.f;
            float Scur = 0.f;
            for (int it = 0; it < kMaxEval32; ++it) {
                const bool fine = !coarse && fabsf(f) < kTolCoarse;
                row_sums<VPT>(t, beta, fine, red5, z);
                ++evals;
                __syncthreads();
                if (warp == 0) {
                    const RowSums s = combine_sums3(fine, red5);
                    float nbeta = beta, fo, So = s.S;
                    int state = 0;
                    bool cv = false;
                    // H in nats; logf and the division are correctly rounded to ~1 ulp
                    fo = (logf(s.S) + beta * (s.T1 / s.S)) - ln_perp;
                    const float mean = s.T1 / s.S;
                    const float var = fmaxf(s.T2 / s.S - mean * mean, 0.f);
                    const float denom = beta * beta * var;   // -dH / d ln(beta)
                    if (fine && fabsf(fo) < best_f) {
                        best_f = fabsf(fo); best_beta = beta; best_S = s.S; best_ulp_h = denom * 6e-8f;
                    }
                    // accept only from a compensated evaluation (coarse: from any, to 1e-3 nats)
                    if (coarse ? fabsf(fo) <= kTolCoarse : (fine && fabsf(fo) <= fminf(kTolFine, kTolBeta * denom))) {
                        cv = true;
                        state = 1;
                    } else {
                        if (fo > 0.f) lo = beta; else hi = beta;
                        float step = denom > 0.f ? fo / denom : 0.f;
                        step = fminf(fmaxf(step, -3.f), 3.f);
                        float nb = beta * expf(step);
                        if (!(nb > lo && nb < hi)) nb = isinf(hi) ? 2.f * beta : 0.5f * (lo + hi);
                        if (nb == beta || (hi - lo) <= 4e-7f * beta) {   // FP32 bracket collapsed
                            // sharp rows: when the error is within 4 ulps of beta's effect on H,
                            // beta is resolved as finely as FP32 allows and an FP64 root would
                            // round to it; otherwise the row is redone in FP64
                            if (best_f <= 4.f * best_ulp_h) { nbeta = best_beta; So = best_S; fo = best_f; cv = true; }
                            state = 1;
                        } else {
                            nbeta = nb;
                        }
                    }
                    if (lane == 0) {
                        s_bc[0] = nbeta;
                        s_bc[1] = So;
                        s_bc[2] = fo;
                        s_bc[3] = (float)(state | (cv ? 2 : 0));
                    }
                }
                __syncthreads();
                beta = s_bc[0];
                Scur = s_bc[1];
                f = s_bc[2];
                const int st = (int)s_bc[3];
                conv = (st & 2) != 0;
                if (st & 1) break;
            }
            S = Scur;
            herr = fabsf(f);
            if (coarse) conv = true;   // only brackets the window; never redone in FP64
            if (!conv) {
                // FP64 redo of the same search on the held (FP32) row; as above,
                // warp 0 combines the sums (one reduction of three values) and
                // takes the step
                fp64 = true;
                double b = beta, blo = 0.0, bhi = INFINITY, fd = INFINITY, Sd = 0.0;
                // compact the entries that can matter (in thread order: deterministic)
                const double b0 = b;
                int mine = 0;
#pragma unroll
                for (int k = 0; k < VPT; ++k)
                    mine += (t[k] < kBig && b0 * (double)t[k] <= kNear64) ? 1 : 0;
                int incl = mine;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += v;
                }
                if (lane == 31) s_wcnt[warp] = incl;
                __syncthreads();
                int nnear = 0, wbase = 0;
#pragma unroll
                for (int w = 0; w < kGroup / 32; ++w) {
                    wbase += w < warp ? s_wcnt[w] : 0;
                    nnear += s_wcnt[w];
                }
                const bool compact = nnear <= kNearMax;
                if (compact) {
                    int pos = wbase + incl - mine;
#pragma unroll
                    for (int k = 0; k < VPT; ++k)
                        if (t[k] < kBig && b0 * (double)t[k] <= kNear64) s_near[pos++] = t[k];
                }
                __syncthreads();
                for (int it = 0; it < kMaxEval64; ++it) {
                    double sS = 0.0, sT1 = 0.0, sT2 = 0.0;
                    if (compact && b >= kNearKeep * b0) {   // block-uniform
                        for (int k = tid; k < nnear; k += kGroup) {
                            const double tk = (double)s_near[k];
                            const double e = exp(-b * tk);
                            sS += e; sT1 += tk * e; sT2 += tk * tk * e;
                        }
                    } else {
#pragma unroll
                        for (int k = 0; k < VPT; ++k) {
                            if (4 * kGroup * (k / 4) >= z) break;
                            if (t[k] >= kBig) continue;
                            const double e = exp(-b * (double)t[k]);
                            sS += e; sT1 += (double)t[k] * e; sT2 += (double)t[k] * t[k] * e;
                        }
                    }
                    sS = warp_sum(sS);
                    sT1 = warp_sum(sT1);
                    sT2 = warp_sum(sT2);
                    if (lane == 0) { redd3[warp][0] = sS; redd3[warp][1] = sT1; redd3[warp][2] = sT2; }
                    ++evals;
                    __syncthreads();
                    if (warp == 0) {
                        sS = redd3[0][0];
                        sT1 = redd3[0][1];
                        sT2 = redd3[0][2];
#pragma unroll
                        for (int w = 1; w < kGroup / 32; ++w) {
                            sS += redd3[w][0];
                            sT1 += redd3[w][1];
                            sT2 += redd3[w][2];
                        }
                        double nbd = b;
                        int state = 0;
                        const double fo = log(sS) + b * sT1 / sS - ln_perp_d;
                        if (fabs(fo) <= kTol64) {
                            state = 1;
                        } else {
                            if (fo > 0.0) blo = b; else bhi = b;
                            const double mean = sT1 / sS;
                            const double var = fmax(sT2 / sS - mean * mean, 0.0);
                            double step = var > 0.0 ? fo / (b * b * var) : 0.0;
                            step = fmin(fmax(step, -3.0), 3.0);
                            double nb = b * exp(step);
                            if (!(nb > blo && nb < bhi)) nb = isinf(bhi) ? 2.0 * b : 0.5 * (blo + bhi);
                            if (nb == b) state = 1;
                            else nbd = nb;
                        }
                        if (lane == 0) {
                            s_bd[0] = nbd;
                            s_bd[1] = sS;
                            s_bd[2] = fo;
                            s_bd[3] = (double)state;
                        }
                    }
                    __syncthreads();
                    b = s_bd[0];
                    Sd = s_bd[1];
                    fd = s_bd[2];
                    if (s_bd[3] != 0.0) break;
                }
                beta = (float)b;
                S = (float)Sd;
                herr = (float)fabs(fd);
                failed = herr > kTolFine;
            }
        }
        if (coarse || (fp32_chunk && (i & 7) == 0)) {
            // the row's window (the pairs whose weight can reach e^-T of the
            // largest; Eq. 1 with the BF16 error bound): its size feeds the
            // form choice of the next affinities; in the coarse search, a row
            // whose window covers >= 1/16 of the chunk flags the 64 x 64 tiles
            // holding its window pairs, recomputed whole in FP32 (in a chunk
            // computed in FP32 whole, every eighth row is counted)
            const float dmax = window_dmax(beta, mn, __uint_as_float(*maxnorm), L.dp);
            float ncand = 0.f;
#pragma unroll
            for (int k = 0; k < VPT; ++k) ncand += (t[k] < kBig && t[k] + mn <= dmax) ? 1.f : 0.f;
            ncand = group_sum(ncand, red);
            const bool dense = coarse && ncand * 16.f >= (float)z;
            if (dense) {   // block-uniform
                const int T = (z + kTile - 1) / kTile;
                uint8_t* fl = fa.tflag + fa.tflag_off[c] + (int64_t)(i / kTile) * T;
#pragma unroll
                for (int q = 0; q < VPT / 4; ++q) {
                    if (4 * kGroup * q >= z) break;
                    bool has = false;
#pragma unroll
                    for (int e = 0; e < 4; ++e) has |= t[4 * q + e] < kBig && t[4 * q + e] + mn <= dmax;
                    // lanes 16h .. 16h + 15 hold the 64 entries of column block 2 warp + h + 8 q
                    const unsigned m = __ballot_sync(0xffffffffu, has);
                    if ((lane & 15) == 0 && ((m >> (lane & 16)) & 0xffffu) != 0u)
                        fl[(4 * tid + 4 * kGroup * q) / kTile] = 1;
                }
            }
            if (tid == 0) {
                if (coarse) row_dense[r] = dense ? 1 : 0;
                const int b = min(kFormBins - 1, (int)((int64_t)(z - fa.zmin) * kFormBins / (fa.zmax - fa.zmin + 1)));
                s_form[b][0] += (unsigned long long)ncand;
                s_form[b][1] += (unsigned long long)(z - 1);
            }
        }
        if (tid == 0) {
            beta_out[r] = beta;
            m_out[r] = mn;
            S_out[r] = S;
            if (fp64) atomicAdd(&st->fp64_rows, 1ull);
            if (failed) atomicAdd(&st->failed_rows, 1ull);
            atomicAdd(&st->bisect_evals, (unsigned long long)evals);
            if (!coarse) atomicMax(&st->max_herr_bits, __float_as_uint(herr));
        }
        __syncthreads();
    }
    __syncthreads();
    if (fa.form_acc && tid < 2 * kFormBins) {
        const unsigned long long v = s_form[tid >> 1][tid & 1];
        if (v) atomicAdd(&fa.form_acc[tid], v);
    }
}

// Joint P of Eq. 3 on one 64 x 64 upper tile (I <= J) of the dense layout,
// written to the tile and its transpose; the (J, I) tile of D is staged
// transposed in shared memory so that each conditional uses its own row:
//   p_ij = (exp(-beta_i (d_ij - m_i)) / S_i + exp(-beta_j (d_ji - m_j)) / S_j) / (2z).
// The padded columns [z, ld) of every row are set to 0.
__global__ void __launch_bounds__(256)
psym_kernel(const float* __restrict__ D, float* __restrict__ P, Layout L, const TileDesc* __restrict__ tiles,
            int64_t t0, const float* __restrict__ beta, const float* __restrict__ mrow,
            const float* __restrict__ Srow) {
    __shared__ float pb[2][kTile], pm[2][kTile], ps[2][kTile];
    __shared__ float dT[kTile][kTile + 1];   // dT[jj][ii] = d_{j i}
    const TileDesc td = tiles[t0 + blockIdx.x];
    const int c = td.chunk;
    const int64_t off = L.off[c];
    const int z = (int)(L.off[c + 1] - off);
    const int ld = L.ld[c];
    const int i0 = td.I * kTile, j0 = td.J * kTile;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    if (tid < 2 * kTile) {
        const int side = tid >> 6, k = tid & 63;
        const int g = (side ? j0 : i0) + k;
        if (g < z) {
            pb[side][k] = beta[off + g] * kLog2e;
            pm[side][k] = mrow[off + g];
            ps[side][k] = 1.0f / Srow[off + g];
        } else {
            pb[side][k] = 0.f; pm[side][k] = 0.f; ps[side][k] = 0.f;
        }
    }
    const float* dbase = D + L.moff[c];
    // rows j0.. of D at columns i0..: coalesced float4 reads
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int jj = ty * 4 + r, j = j0 + jj;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (j < z) v = *reinterpret_cast<const float4*>(dbase + (int64_t)j * ld + i0 + tx * 4);
        dT[jj][tx * 4 + 0] = v.x; dT[jj][tx * 4 + 1] = v.y; dT[jj][tx * 4 + 2] = v.z; dT[jj][tx * 4 + 3] = v.w;
    }
    __syncthreads();
    const float inv2z = 1.0f / (2.0f * (float)z);
    float* pbase = P + L.moff[c];
    float out[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int li = ty * 4 + r, i = i0 + li;
        float4 dv = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < z) dv = *reinterpret_cast<const float4*>(dbase + (int64_t)i * ld + j0 + tx * 4);
        const float d4[4] = {dv.x, dv.y, dv.z, dv.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int lj = tx * 4 + q, j = j0 + lj;
            float p = 0.f;
            if (i < z && j < z && i != j) {
                // explicitly rounded products and sum: no FMA contraction, so the two
                // halves of a diagonal tile round identically
                const float cij = __fmul_rn(hw_ex2(-pb[0][li] * (d4[q] - pm[0][li])), ps[0][li]);
                const float cji = __fmul_rn(hw_ex2(-pb[1][lj] * (dT[lj][li] - pm[1][lj])), ps[1][lj]);
                p = __fmul_rn(__fadd_rn(cij, cji), inv2z);
            }
            out[r][q] = p;
        }
        if (i < z)
            *reinterpret_cast<float4*>(pbase + (int64_t)i * ld + j0 + tx * 4) =
                make_float4(out[r][0], out[r][1], out[r][2], out[r][3]);
    }
    if (td.I != td.J) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = j0 + tx * 4 + q;
            if (j < z)
                *reinterpret_cast<float4*>(pbase + (int64_t)j * ld + i0 + ty * 4) =
                    make_float4(out[0][q], out[1][q], out[2][q], out[3][q]);
        }
    }
}

template <int VPT>
static void launch_group(const ptsne_ctx* c, int64_t r0, int64_t r1, cudaStream_t s, const float* beta_init,
                         int coarse, const FormArgs& fa) {
    int64_t blocks = r1 - r0;
    if (blocks > 152 * 32) blocks = 152 * 32;
    bisect_group_kernel<VPT><<<(unsigned)blocks, kGroup, 0, s>>>(c->D, make_layout(c), r0, r1,
                                                                   log(c->p.perplexity), c->beta, c->mrow, c->Srow,
                                                                   c->dstats, beta_init, coarse, c->maxnorm,
                                                                   c->row_dense, fa);
}

cudaError_t launch_bisect(const ptsne_ctx* c, int64_t row_begin, int64_t row_end, cudaStream_t s,
                          const float* beta_init, int coarse, int form) {
    if (row_end <= row_begin) return cudaSuccess;
    // mixed precision: the per-chunk form, the window tiles and the size-bin
    // window fractions (the FP32 and the distance-input searches use none)
    FormArgs fa;
    if (form) {
        if (!c->chunk_fp32 || !c->maxnorm) return cudaErrorInvalidValue;
        fa.chunk_fp32 = c->chunk_fp32;
        fa.tflag = c->tflag;
        fa.tflag_off = c->d_tflag_off;
        fa.form_acc = c->form_acc;
        fa.zmin = (int)c->zmin;
        fa.zmax = (int)c->zmax;
        fa.fp32_warm = form == 2;
    } else if (coarse) {
        return cudaErrorInvalidValue;
    }
    const int64_t per = (c->zmax + 4 * kGroup - 1) / (4 * kGroup) * 4;   // values per thread
    if (per <= 8) launch_group<8>(c, row_begin, row_end, s, beta_init, coarse, fa);
    else if (per <= 16) launch_group<16>(c, row_begin, row_end, s, beta_init, coarse, fa);
    else if (per <= 24) launch_group<24>(c, row_begin, row_end, s, beta_init, coarse, fa);
    else if (per <= 32) launch_group<32>(c, row_begin, row_end, s, beta_init, coarse, fa);
    else if (per <= 40) launch_group<40>(c, row_begin, row_end, s, beta_init, coarse, fa);
    else if (per <= 48) launch_group<48>(c, row_begin, row_end, s, beta_init, coarse, fa);
    else launch_group<64>(c, row_begin, row_end, s, beta_init, coarse, fa);
    return launched(c, 1);
}

cudaError_t launch_psym(const ptsne_ctx* c, int64_t tile_begin, int64_t tile_end, cudaStream_t s) {
    const int64_t nt = tile_end - tile_begin;
    if (nt <= 0) return cudaSuccess;
    psym_kernel<<<(unsigned)nt, 256, 0, s>>>(c->D, c->P, make_layout(c), c->d_tiles, tile_begin, c->beta,
                                             c->mrow, c->Srow);
    return launched(c, 1);
}

}  // namespace ptsne
