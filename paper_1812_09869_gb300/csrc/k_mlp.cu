// Learned out-of-sample mapper: MLP d_in -> 256 -> 256 -> out_dim with exact
// GELU, BF16 weights and activations, FP32 accumulation on the tensor cores.
// No counterpart in the paper (it maps new points by re-running ptSNE); the
// network is trained on ptSNE's own maps and used to place held-out points
// and to warm-start ptsne_run.
//
// Training: one GEMM kernel serves every contraction, C = A B^T with A (M x K) and
// B (N x K) BF16, both K-major, staged by TMA (128-byte swizzle, a ring of
// up to 3 stages, as many as the CTA's K blocks need), one elected thread
// issuing tcgen05.mma (M = 128, N = NT, K = 16) into an FP32 accumulator of
// NT columns in tensor memory, and CG groups of four warps reading it back
// (tcgen05.ld; warp w reads accumulator rows 32 (w mod 4) .. + 31, one row per
// thread, and group w / 4 takes NT / CG of the columns) for a fused epilogue.
// The epilogue (exact GELU per element) is the heavy part: the 256-column
// GELU epilogues carry 16 warps (four column groups, one CTA per SM), the
// others 8 warps with two CTAs per SM (2 x 256 TMEM columns, <= 2 x 96 KB of
// stages), one CTA's loads and MMAs under the other's epilogue.
//
//   FWD        u = acc + b; U = u (FP32), H = g(u) (BF16), H^T (BF16)
//   HEAD_TRAIN h = g(acc + b2); y = W3 h + b3 per row (each column group's
//              partial sums of the row, added in group order); then
//              r = (y - t) / B, loss += |y - t|^2 / (2B),
//              dL/dW3 += r h^T, dL/db3 += r, and, re-reading the accumulator,
//              dA2 = (W3^T r) * g'(u2) (BF16, and transposed), dL/db2 += dA2
//   DGELU      dA1 = acc * g'(U1) (transposed, BF16), dL/db1 += dA1
//   ATOMIC     C += acc (FP32 atomics; split-K weight gradients)
//
// A training step (batch B rows):
//   gather    X[rows] -> Xb (B x 64, BF16, zero-padded), Xb^T; T[rows] -> t
//   FWD       Xb  x W1b^T   -> U1, H1, H1^T                (K = 64)
//   HEAD_TRAIN H1 x W2b^T   -> loss, dW3, db3, dA2, dA2^T, db2  (K = 256)
//   ATOMIC    dA2^T x H1^T  -> dW2 (256 x 256)              (K = B, split)
//   DGELU     dA2 x W2^T    -> dA1^T, db1                   (K = 256)
//   ATOMIC    dA1^T x Xb^T  -> dW1 (256 x d_in)             (K = B, split)
//   AdamW on the FP32 master parameters, rewriting the BF16 copies.
//
// Inference runs in one fused, warp-specialised kernel (mlp_infer_kernel,
// below): FP32 X read in place, both layers and the head per 128-row tile,
// the hidden activations kept in shared memory.
#include <float.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <string>

#include "ptsne_internal.cuh"
#include "ptsne_mlp.h"
#include "tc_common.cuh"

using bf16 = __nv_bfloat16;

namespace ptsne {
namespace mlp {

constexpr int kH = PTSNE_MLP_HIDDEN;   // 256
constexpr int kKin = 64;               // input features padded to one K block
constexpr int kStages = 3;              // at most; a CTA uses min(kStages, its K blocks)
constexpr int kMaxStagesPair = 2;       // stages when K needs more: two CTAs per SM fit

enum Epi { EPI_FWD = 0, EPI_HEAD_TRAIN = 2, EPI_DGELU = 3, EPI_ATOMIC = 4 };

struct GemmArgs {
    int M;               // valid rows of A (rows >= M are computed but not stored)
    int kblocks;         // K / 64
    int kb_per_split;    // K blocks per CTA along gridDim.y
    const float* bias;   // FWD, HEAD_TRAIN, DGELU: [NT]
    float* U;            // FWD: pre-activation [M][NT] (optional)
    bf16* H;             // FWD: activation [M][NT] (optional); HEAD_TRAIN: dA2 [M][NT]
    bf16* HT;            // FWD: activation^T; HEAD_TRAIN: dA2^T; DGELU: dA1^T  ([NT][ldT])
    int64_t ldT;
    const float* Uin;    // DGELU: pre-activation [M][NT]
    float* colsum;       // DGELU: db1; HEAD_TRAIN: db2  ([NT])
    float* C;            // ATOMIC: [M][ldc]
    int ldc, ncols;
    int red_width;       // ATOMIC: floats per vector reduction (4, 2 or 1), from C's and ldc's alignment
    const bf16* W3;      // HEAD_TRAIN: [OD][NT]
    const float* b3;     // HEAD_TRAIN: [OD]
    const float* T;      // HEAD_TRAIN: standardised targets [M][OD]
    float invB;          // HEAD_TRAIN
    int stages;          // ring stages (1 .. kStages)
    double* loss;        // HEAD_TRAIN: accumulates sum |y - t|^2 / (2B)
    float* gW3;          // HEAD_TRAIN: [OD][NT]
    float* gb3;          // HEAD_TRAIN: [OD]
    unsigned int* timeouts;
};

// Exact GELU g(u) = u Phi(u) and g'(u) = Phi(u) + u phi(u), with the normal
// CDF from the rational approximation of Abramowitz & Stegun, Handbook of
// Mathematical Functions, formula 7.1.26:
//   erfc(a) = (a1 t + a2 t^2 + a3 t^3 + a4 t^4 + a5 t^5) exp(-a^2), t = 1 / (1 + p a),
// a >= 0, absolute error <= 1.5e-7 (so |Phi - Phi~| <= 7.5e-8), taken at
// a = |u| / sqrt 2; Phi(u) = 1 - erfc(a) / 2 for u >= 0 and erfc(a) / 2 below.
// No cancellation for negative u (erfc is formed directly), one reciprocal
// and one exponential (both MUFU) shared by g and g'.
struct NormalParts {
    float Phi, e;   // Phi(u) and exp(-u^2 / 2)
};
__device__ __forceinline__ NormalParts normal_parts(float u) {
    constexpr float kP = 0.3275911f, kA1 = 0.254829592f, kA2 = -0.284496736f, kA3 = 1.421413741f,
                    kA4 = -1.453152027f, kA5 = 1.061405429f;
    constexpr float kRsqrt2 = 0.70710678118654752f, kHalfLog2e = 0.72134752044448170f;
    const float a = fabsf(u) * kRsqrt2;
    const float t = hw_rcp(fmaf(kP, a, 1.0f));
    const float e = hw_ex2(-(u * u) * kHalfLog2e);
    const float poly = t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, kA5, kA4), kA3), kA2), kA1);
    const float q = poly * e;   // erfc(|u| / sqrt 2)
    NormalParts r;
    r.Phi = u >= 0.f ? fmaf(-0.5f, q, 1.0f) : 0.5f * q;
    r.e = e;
    return r;
}
// Forward-only GELU of two values at once (packed f32x2), Phi from the
// approximation of Abramowitz & Stegun formula 7.1.28, which needs a single
// reciprocal and no exponential:
//   erfc(a) = (1 + b1 a + b2 a^2 + b3 a^3 + b4 a^4 + b5 a^5 + b6 a^6)^-16,
// a >= 0, absolute error <= 3e-7 (the 16th power, four squarings in FP32,
// adds ~1.6e-6 relative to erfc).  erfc overflows to an exact 0 for large a.
typedef unsigned long long f2m;
__device__ __forceinline__ f2m pkm(float a, float b) {
    f2m r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upkm(f2m v, float& a, float& b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v)); }
__device__ __forceinline__ f2m fma2m(f2m a, f2m b, f2m c) {
    f2m d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2m mul2m(f2m a, f2m b) {
    f2m d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2m gelu2p(f2m u) {
    constexpr float kB1 = 0.0705230784f, kB2 = 0.0422820123f, kB3 = 0.0092705272f, kB4 = 0.0001520143f,
                    kB5 = 0.0002765672f, kB6 = 0.0000430638f, kRsqrt2 = 0.70710678118654752f;
    float x, y;
    upkm(u, x, y);
    const f2m A = pkm(fabsf(x) * kRsqrt2, fabsf(y) * kRsqrt2);
    f2m P = fma2m(A, pkm(kB6, kB6), pkm(kB5, kB5));
    P = fma2m(A, P, pkm(kB4, kB4));
    P = fma2m(A, P, pkm(kB3, kB3));
    P = fma2m(A, P, pkm(kB2, kB2));
    P = fma2m(A, P, pkm(kB1, kB1));
    P = fma2m(A, P, pkm(1.0f, 1.0f));
    P = mul2m(P, P);
    P = mul2m(P, P);
    P = mul2m(P, P);
    P = mul2m(P, P);
    float px, py;
    upkm(P, px, py);
    const float qx = hw_rcp(px), qy = hw_rcp(py);   // erfc(|u| / sqrt 2)
    const float fx = x >= 0.f ? fmaf(-0.5f, qx, 1.0f) : 0.5f * qx;
    const float fy = y >= 0.f ? fmaf(-0.5f, qy, 1.0f) : 0.5f * qy;
    return mul2m(u, pkm(fx, fy));
}
__device__ __forceinline__ void gelu2(float& x, float& y) { upkm(gelu2p(pkm(x, y)), x, y); }
__device__ __forceinline__ float gelu(float u) { return u * normal_parts(u).Phi; }
__device__ __forceinline__ float gelu_grad(float u) {
    const NormalParts n = normal_parts(u);
    return fmaf(u * 0.39894228040143268f, n.e, n.Phi);
}

// v[32] on each lane -> on lane l, the sum over the warp's lanes of v[l]
// (recursive halving: 31 shuffles for 32 columns).  Destroys v.
__device__ __forceinline__ float warp_transpose_sum(float (&v)[32], int lane) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < o; ++i) {
            const float send = upper ? v[i] : v[i + o];
            const float keep = upper ? v[i + o] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return v[0];
}

__device__ __forceinline__ void store_bf16x32(bf16* dst, const float (&v)[32]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint4 pk;
        uint32_t* w = reinterpret_cast<uint32_t*>(&pk);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const __nv_bfloat162 b2 = __floats2bfloat162_rn(v[8 * q + 2 * e], v[8 * q + 2 * e + 1]);
            w[e] = *reinterpret_cast<const uint32_t*>(&b2);
        }
        reinterpret_cast<uint4*>(dst)[q] = pk;
    }
}

__device__ __forceinline__ void store_bf16x16(bf16* dst, const float (&v)[16]) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        uint4 pk;
        uint32_t* w = reinterpret_cast<uint32_t*>(&pk);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const __nv_bfloat162 b2 = __floats2bfloat162_rn(v[8 * q + 2 * e], v[8 * q + 2 * e + 1]);
            w[e] = *reinterpret_cast<const uint32_t*>(&b2);
        }
        reinterpret_cast<uint4*>(dst)[q] = pk;
    }
}

// FP32 vector reductions into global memory (relaxed, GPU scope): 4
// consecutive floats at a 16-byte-aligned address, or 2 at an 8-byte one.
__device__ __forceinline__ void red_add4(float* p, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}
__device__ __forceinline__ void red_add2(float* p, float a, float b) {
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(a), "f"(b) : "memory");
}

template <int NT, int EPI, int OD, int CG>
__global__ void __launch_bounds__(128 * CG, CG >= 4 ? 1 : 2)
mlp_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const GemmArgs a) {
    static_assert((NT / 32) % CG == 0, "column groups must split the accumulator's 32-column chunks");
    constexpr int kBRows = NT < 128 ? 128 : NT;
    constexpr uint32_t kABytes = tc::kTileBytes;
    constexpr uint32_t kBBytes = (uint32_t)kBRows * 128u;
    constexpr uint32_t kStageBytes = kABytes + kBBytes;
    constexpr bool kHead = EPI == EPI_HEAD_TRAIN;
    extern __shared__ unsigned char dsmem[];
    __shared__ uint64_t full_bar[kStages], done_bar[kStages], drain_bar;
    __shared__ uint32_t tmem_base;
    __shared__ float sb[NT];
    __shared__ float sw3[kHead ? OD : 1][NT];
    __shared__ float s_y[kHead ? CG : 1][128][OD];   // HEAD: per column group, partial outputs of each row
    constexpr int kThreads = 128 * CG;
    constexpr int kChunks = NT / 32 / CG;            // 32-column chunks per column group
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int grp = warp >> 2, c0 = grp * kChunks;    // this warp's column group and first chunk
    const int nst = a.stages;
    const uint32_t sbase = (tc::smem_addr(dsmem) + 1023u) & ~1023u;
    const int m0 = blockIdx.x * 128;
    const int kb0 = blockIdx.y * a.kb_per_split;
    const int kb1 = min(kb0 + a.kb_per_split, a.kblocks);
    const int nkb = kb1 - kb0;   // >= 1 (the launcher sizes gridDim.y)

    if (warp == 0) tc::tmem_alloc(tc::smem_addr(&tmem_base), NT < 32 ? 32 : NT);
    if (tid == 0) {
        for (int s = 0; s < nst; ++s) {
            tc::mbar_init(tc::smem_addr(&full_bar[s]), 1);
            tc::mbar_init(tc::smem_addr(&done_bar[s]), 1);
        }
        tc::mbar_init(tc::smem_addr(&drain_bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (EPI == EPI_FWD || kHead)
        for (int n = tid; n < NT; n += kThreads) sb[n] = a.bias[n];
    if (kHead)
        for (int idx = tid; idx < OD * NT; idx += kThreads) sw3[idx / NT][idx % NT] = __bfloat162float(a.W3[idx]);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (tid == 0) {
        const uint32_t idesc = tc::idesc_bf16_f32(128, NT);
        bool ok = true;
        int issued = 0;   // K blocks whose loads were issued
        auto issue = [&](int i) {
            const int s = i % nst;
            const uint32_t fb = tc::smem_addr(&full_bar[s]);
            const uint32_t sa = sbase + (uint32_t)s * kStageBytes, sbb = sa + kABytes;
            tc::mbar_expect_tx(fb, kStageBytes);
            const int col = (kb0 + i) * tc::kTileK;
            tc::tma_load_2d(sa, &tmA, col, m0, fb);
#pragma unroll
            for (int r = 0; r < kBRows / 128; ++r) tc::tma_load_2d(sbb + (uint32_t)r * tc::kTileBytes, &tmB, col, r * 128, fb);
            issued = i + 1;
        };
        for (int i = 0; i < nst && i < nkb; ++i) issue(i);
        for (int i = 0; i < nkb; ++i) {
            const int s = i % nst;
            const uint32_t par = (uint32_t)(i / nst) & 1u;
            if (!(ok = tc::mbar_wait(tc::smem_addr(&full_bar[s]), par))) break;
            tc::tc_fence_after();
            const uint32_t sa = sbase + (uint32_t)s * kStageBytes, sbb = sa + kABytes;
            const uint64_t da = tc::sw128_desc(sa), db = tc::sw128_desc(sbb);
#pragma unroll
            for (int k16 = 0; k16 < tc::kTileK / 16; ++k16)
                tc::mma_bf16(tmem, da + 2 * k16, db + 2 * k16, idesc, (i > 0 || k16 > 0) ? 1u : 0u);
            tc::mma_commit(tc::smem_addr(&done_bar[s]));
            if (i + nst < nkb) {   // stage s is free once these MMAs are done
                if (!(ok = tc::mbar_wait(tc::smem_addr(&done_bar[s]), par))) break;
                issue(i + nst);
            }
        }
        const int last = nkb - 1;
        if (ok) ok = tc::mbar_wait(tc::smem_addr(&done_bar[last % nst]), (uint32_t)(last / nst) & 1u);
        if (!ok) {   // the host reports the count; nothing issued stays in flight
            atomicAdd(a.timeouts, 1u);
            tc::drain_issued(tc::smem_addr(&full_bar[0]), nst, issued, tc::smem_addr(&drain_bar));
        }
    }
    __syncthreads();
    tc::tc_fence_after();

    const int row = (warp & 3) * 32 + lane;
    const int m = m0 + row;
    const bool valid = m < a.M;
    const uint32_t tb = tmem + ((uint32_t)((warp & 3) * 32) << 16);

    if constexpr (EPI == EPI_FWD) {
        // 16 columns at a time (keeps the epilogue within the register budget
        // of two CTAs per SM)
        for (int c = 2 * c0; c < 2 * (c0 + kChunks); ++c) {
            float v[16];
            tc::tmem_ld16(tb + (uint32_t)(c * 16), v);
#pragma unroll
            for (int e = 0; e < 16; ++e) v[e] += sb[c * 16 + e];
            if (valid && a.U) {
                float4* up = reinterpret_cast<float4*>(a.U + (int64_t)m * NT + c * 16);
#pragma unroll
                for (int q = 0; q < 4; ++q) up[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            }
#pragma unroll
            for (int e = 0; e < 16; e += 2) gelu2(v[e], v[e + 1]);
            if (valid && a.H) store_bf16x16(a.H + (int64_t)m * NT + c * 16, v);
            if (valid && a.HT) {
#pragma unroll
                for (int e = 0; e < 16; ++e) a.HT[(int64_t)(c * 16 + e) * a.ldT + m] = __float2bfloat16_rn(v[e]);
            }
        }
    } else if constexpr (kHead) {
        float y[OD];
#pragma unroll
        for (int k = 0; k < OD; ++k) y[k] = 0.f;
        for (int c = c0; c < c0 + kChunks; ++c) {
            float v[32];
            tc::tmem_ld32(tb + (uint32_t)(c * 32), v);
#pragma unroll
            for (int e = 0; e < 32; e += 2) {
                float h0 = v[e] + sb[c * 32 + e], h1 = v[e + 1] + sb[c * 32 + e + 1];
                gelu2(h0, h1);
#pragma unroll
                for (int k = 0; k < OD; ++k) y[k] = fmaf(h1, sw3[k][c * 32 + e + 1], fmaf(h0, sw3[k][c * 32 + e], y[k]));
            }
        }
        // the groups' partial outputs of each row, summed in group order
#pragma unroll
        for (int k = 0; k < OD; ++k) s_y[grp][row][k] = y[k];
        __syncthreads();
#pragma unroll
        for (int k = 0; k < OD; ++k) {
            float t = 0.f;
#pragma unroll
            for (int g = 0; g < CG; ++g) t += s_y[g][row][k];
            y[k] = t + a.b3[k];
        }
        float r[OD];
        float l2 = 0.f;
#pragma unroll
        for (int k = 0; k < OD; ++k) {
            const float diff = valid ? y[k] - a.T[(int64_t)m * OD + k] : 0.f;
            l2 = fmaf(diff, diff, l2);
            r[k] = diff * a.invB;
        }
        if (grp == 0) {   // every group holds the same r; group 0 reports it
            const double lw = warp_sum((double)l2);
            if (lane == 0) atomicAdd(a.loss, lw * 0.5 * (double)a.invB);
#pragma unroll
            for (int k = 0; k < OD; ++k) {
                const float rs = warp_sum(r[k]);
                if (lane == 0) atomicAdd(&a.gb3[k], rs);
            }
        }
        // second pass over the group's accumulator columns: dW3, dA2 and db2
        for (int c = c0; c < c0 + kChunks; ++c) {
            float v[32], g[32], t[32];
            tc::tmem_ld32(tb + (uint32_t)(c * 32), v);
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                const float u = v[e] + sb[c * 32 + e];
                g[e] = gelu(u);
                v[e] = gelu_grad(u);
            }
#pragma unroll
            for (int k = 0; k < OD; ++k) {
#pragma unroll
                for (int e = 0; e < 32; ++e) t[e] = r[k] * g[e];
                const float s = warp_transpose_sum(t, lane);
                atomicAdd(&a.gW3[k * NT + c * 32 + lane], s);
            }
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                float dh = 0.f;
#pragma unroll
                for (int k = 0; k < OD; ++k) dh = fmaf(r[k], sw3[k][c * 32 + e], dh);
                t[e] = dh * v[e];
            }
            if (valid) {
                store_bf16x32(a.H + (int64_t)m * NT + c * 32, t);
#pragma unroll
                for (int e = 0; e < 32; ++e) a.HT[(int64_t)(c * 32 + e) * a.ldT + m] = __float2bfloat16_rn(t[e]);
            }
            const float s = warp_transpose_sum(t, lane);
            atomicAdd(&a.colsum[c * 32 + lane], s);
        }
    } else if constexpr (EPI == EPI_DGELU) {
        for (int c = c0; c < c0 + kChunks; ++c) {
            float v[32];
            tc::tmem_ld32(tb + (uint32_t)(c * 32), v);
            if (valid) {
                const float4* up = reinterpret_cast<const float4*>(a.Uin + (int64_t)m * NT + c * 32);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float4 u = up[q];
                    v[4 * q] *= gelu_grad(u.x);
                    v[4 * q + 1] *= gelu_grad(u.y);
                    v[4 * q + 2] *= gelu_grad(u.z);
                    v[4 * q + 3] *= gelu_grad(u.w);
                }
#pragma unroll
                for (int e = 0; e < 32; ++e) a.HT[(int64_t)(c * 32 + e) * a.ldT + m] = __float2bfloat16_rn(v[e]);
            } else {
#pragma unroll
                for (int e = 0; e < 32; ++e) v[e] = 0.f;
            }
            const float s = warp_transpose_sum(v, lane);
            atomicAdd(&a.colsum[c * 32 + lane], s);
        }
    } else {   // EPI_ATOMIC
        // a thread's row of 32 columns goes out as vector reductions of 4 (or
        // 2) consecutive floats where the row's alignment allows
        const int vw = a.red_width;
        for (int c = c0; c < c0 + kChunks; ++c) {
            float v[32];
            tc::tmem_ld32(tb + (uint32_t)(c * 32), v);
            const int lim = min(32, a.ncols - c * 32);   // columns of this chunk inside C
            if (valid && lim > 0) {
                float* rowp = a.C + (int64_t)m * a.ldc + c * 32;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int e = 4 * q;
                    if (vw == 4 && e + 4 <= lim) {
                        red_add4(rowp + e, v[e], v[e + 1], v[e + 2], v[e + 3]);
                        continue;
                    }
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int f = e + 2 * h;
                        if (vw >= 2 && f + 2 <= lim) {
                            red_add2(rowp + f, v[f], v[f + 1]);
                        } else {
                            if (f < lim) atomicAdd(rowp + f, v[f]);
                            if (f + 1 < lim) atomicAdd(rowp + f + 1, v[f + 1]);
                        }
                    }
                }
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, NT < 32 ? 32 : NT);
}

// ---------------------------------------------------------------- fused inference
// Inference of 128-row tiles in one persistent, warp-specialised kernel.
// Two loader warps read the tile's FP32 rows of X straight from global
// memory (alternate rows; one row per load instruction, lane l taking
// columns 2l and 2l + 1), round them to BF16 and
// write the layer-1 A operand (zero-padded to 64 columns) into shared memory
// in the 128-byte-swizzled K-major layout that TMA writes (row r, 16-byte
// chunk c of a 64-column K block at r * 128 + ((c ^ (r mod 8)) * 16)).
// Layer 1 (X W1^T + b1, GELU) goes from tensor memory into shared memory in
// the same layout as the A operand of layer 2, so the hidden activations
// never leave the SM; layer 2 (+ b2, GELU) ends in the output head
// (y = W3 h + b3, de-standardised).  Warp 0 (one thread) issues the TMA
// loads of the weights and the MMAs; warps 1..16 are the epilogue (warp w
// reads tensor-memory lanes 32 (w mod 4) .. + 31, one row per thread, and
// column group (w - 1) / 4 of four 64-column groups, which is one K block of
// the layer-2 operand); warps 17 and 18 load X.  Two accumulators (2 x 256
// tensor-memory columns, tile j in accumulator j mod 2, layer 2 overwriting
// layer 1 once its activations are in shared memory) let the tensor cores
// run layer 2 of tile j while the epilogue warps take layer 2 of tile j - 1,
// and layer 1 of tile j + 1 as soon as that accumulator has been read.  W1
// stays in shared memory; W2 streams from L2 in 128-row x 64-column boxes,
// four in flight.  Mbarrier waits are bounded; the first that runs out stops
// every role (the epilogue warps still meet at their named barrier), and the
// issuing thread waits for its copies and MMAs before tensor memory is freed.
constexpr int kInferEpiWarps = 16;
constexpr int kInferLoadWarps = 2;
constexpr int kInferThreads = 32 * (1 + kInferEpiWarps + kInferLoadWarps);
constexpr int kW2Stages = 4;
constexpr uint32_t kBox = 16384;                      // one 128-row x 64-column BF16 box
constexpr uint32_t kOffW1 = 0;                        // W1: 2 boxes (256 rows)
constexpr uint32_t kOffX = kOffW1 + 2 * kBox;         // X: 2 stages
constexpr uint32_t kOffH1 = kOffX + 2 * kBox;         // layer-2 A operand: 4 K blocks
constexpr uint32_t kOffW2 = kOffH1 + 4 * kBox;        // W2: kW2Stages boxes
constexpr size_t kInferSmem = kOffW2 + kW2Stages * kBox + 1024;   // + 1024-byte alignment slack

struct InferArgs {
    const float* X;         // the launch's rows of X [M][din], FP32
    int M;                  // rows of the launch
    int mtiles;             // 128-row tiles of the launch
    int din;
    int pairs;              // 1: din even and X 8-byte aligned (two columns per load)
    const float* b1;
    const float* b2;
    const bf16* W3;         // [OD][256]
    const float* b3;
    const double* scaler;   // mean[OD], std[OD]
    float* Y;               // [M][OD]
    unsigned int* timeouts;
};

// bounded wait that fails at once after any role's wait has failed
__device__ __forceinline__ bool iwait(uint32_t bar, uint32_t parity, volatile int* fail) {
    if (tc::mbar_try(bar, parity)) return true;
    const unsigned long long t0 = tc::now_ns();
    while (!tc::mbar_try(bar, parity)) {
        if (*fail || tc::now_ns() - t0 > tc::kWaitNs) {
            *fail = 1;
            return false;
        }
    }
    return true;
}
__device__ __forceinline__ void mbar_arrive1(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, %0;" ::"n"(32 * kInferEpiWarps) : "memory"); }
__device__ __forceinline__ f2m add2m(f2m a, f2m b) {
    f2m d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint32_t bf16x2_bits(float lo, float hi) {
    const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&p);
}

template <int OD>
__global__ void __launch_bounds__(kInferThreads, 1)
mlp_infer_kernel(const __grid_constant__ CUtensorMap tmW1, const __grid_constant__ CUtensorMap tmW2, const InferArgs a) {
    extern __shared__ unsigned char dsmem[];
    // 0: W1 loaded; 1-2: X stage written; 3-6: W2 stage full; 7-10: W2 stage
    // free; 11-12: layer 1 done (per accumulator and X stage); 13-14: layer 2
    // done; 15: H1 written; 16-17: accumulator read by the layer-2 epilogue;
    // 18: every MMA issued (the exit drain)
    __shared__ uint64_t bars[19];
    __shared__ uint32_t tmem_base;
    __shared__ __align__(16) float sb1[kH];
    __shared__ __align__(16) float sb2[kH];
    __shared__ __align__(16) float sw3[OD][kH];
    __shared__ float s_y[2][4][128][OD];
    __shared__ int s_fail;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t sbase = (tc::smem_addr(dsmem) + 1023u) & ~1023u;
    auto B = [&](int i) { return tc::smem_addr(&bars[i]); };
    const int ntl = ((int)blockIdx.x < a.mtiles) ? (a.mtiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
    auto tile_row = [&](int j) { return ((int)blockIdx.x + j * (int)gridDim.x) * 128; };

    if (warp == 0) tc::tmem_alloc(tc::smem_addr(&tmem_base), 512);
    if (tid == 0) {
        s_fail = 0;
        for (int i = 0; i < 19; ++i) {
            const uint32_t count = (i == 1 || i == 2) ? (uint32_t)kInferLoadWarps
                                 : (i >= 15 && i <= 17) ? (uint32_t)kInferEpiWarps : 1u;
            tc::mbar_init(B(i), count);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    for (int n = tid; n < kH; n += kInferThreads) {
        sb1[n] = a.b1[n];
        sb2[n] = a.b2[n];
    }
    for (int idx = tid; idx < OD * kH; idx += kInferThreads) sw3[idx / kH][idx % kH] = __bfloat162float(a.W3[idx]);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = tmem_base;
    volatile int* fail = &s_fail;

    if (warp == 0) {
        if (lane == 0 && ntl > 0) {
            const uint32_t id1 = tc::idesc_bf16_f32(128, 256), id2 = tc::idesc_bf16_f32(128, 128);
            const int nuse = 8 * ntl;   // W2 boxes: 2 halves x 4 K blocks per tile
            int w2_issued = 0;
            auto load_w2 = [&](int u) {
                const int s = u % kW2Stages, h = (u >> 2) & 1, kb = u & 3;
                const uint32_t bar = B(3 + s);
                tc::mbar_expect_tx(bar, kBox);
                tc::tma_load_2d(sbase + kOffW2 + (uint32_t)s * kBox, &tmW2, kb * 64, h * 128, bar);
                w2_issued = u + 1;
            };
            tc::mbar_expect_tx(B(0), 2 * kBox);
            tc::tma_load_2d(sbase + kOffW1, &tmW1, 0, 0, B(0));
            tc::tma_load_2d(sbase + kOffW1 + kBox, &tmW1, 0, 128, B(0));
            for (int u = 0; u < kW2Stages && u < nuse; ++u) load_w2(u);
            for (int j = 0; j < ntl; ++j) {
                const int b = j & 1;
                const uint32_t acc = tmem + (uint32_t)(b * 256);
                if (!iwait(B(1 + b), (uint32_t)(j >> 1) & 1u, fail)) break;                  // X of tile j written
                if (!iwait(B(16 + b), ((uint32_t)(j >> 1) & 1u) ^ 1u, fail)) break;   // layer 2 of tile j - 2 read
                if (j == 0 && !iwait(B(0), 0u, fail)) break;
                tc::tc_fence_after();
                const uint64_t dx = tc::sw128_desc(sbase + kOffX + (uint32_t)b * kBox), dw1 = tc::sw128_desc(sbase + kOffW1);
#pragma unroll
                for (int k16 = 0; k16 < 4; ++k16) tc::mma_bf16(acc, dx + 2 * k16, dw1 + 2 * k16, id1, k16 > 0 ? 1u : 0u);
                tc::mma_commit(B(11 + b));
                if (!iwait(B(15), (uint32_t)j & 1u, fail)) break;   // layer-1 activations of tile j written
                tc::tc_fence_after();
                bool ok = true;
                for (int h = 0; h < 2 && ok; ++h)
                    for (int kb = 0; kb < 4; ++kb) {
                        const int u = 8 * j + 4 * h + kb, s = u % kW2Stages;
                        if (!iwait(B(3 + s), (uint32_t)(u / kW2Stages) & 1u, fail)) { ok = false; break; }
                        tc::tc_fence_after();
                        const uint64_t dh = tc::sw128_desc(sbase + kOffH1 + (uint32_t)kb * kBox),
                                       dw = tc::sw128_desc(sbase + kOffW2 + (uint32_t)s * kBox);
#pragma unroll
                        for (int k16 = 0; k16 < 4; ++k16)
                            tc::mma_bf16(acc + (uint32_t)(128 * h), dh + 2 * k16, dw + 2 * k16, id2,
                                         (kb > 0 || k16 > 0) ? 1u : 0u);
                        tc::mma_commit(B(7 + s));
                        // the stage of the previous box (its MMAs queued ahead of these) takes box u + 3
                        if (u >= 1 && u + kW2Stages - 1 < nuse) {
                            const int v = u - 1, sv = v % kW2Stages;
                            if (!iwait(B(7 + sv), (uint32_t)(v / kW2Stages) & 1u, fail)) { ok = false; break; }
                            load_w2(u + kW2Stages - 1);
                        }
                    }
                if (!ok) break;
                tc::mma_commit(B(13 + b));
            }
            // Whether or not a wait ran out (in this role or another, also
            // after this thread's last tile): wait (bounded) for W1, the W2
            // loads and every MMA this thread issued, so that none is in
            // flight when the CTA frees tensor memory and exits.  Without a
            // timeout all of them are done by now.
            tc::mbar_wait(B(0), 0u);
            tc::drain_issued(B(3), kW2Stages, w2_issued, B(18));
        }
    } else if (warp > kInferEpiWarps) {
        // X loaders: warp lw takes rows lw, lw + 2, ... of the tile; lane l
        // columns 2l and 2l + 1 (one 4-byte word of 16-byte chunk l / 4).
        constexpr int kRows = 128 / kInferLoadWarps, kU = 16;
        const int lw = warp - 1 - kInferEpiWarps, c0 = 2 * lane;
        const bool in0 = c0 < a.din, in1 = c0 + 1 < a.din;
        for (int j = 0; j < ntl; ++j) {
            const int b = j & 1;
            if (j >= 2 && !iwait(B(11 + b), ((uint32_t)(j >> 1) & 1u) ^ 1u, fail)) break;   // layer 1 of tile j - 2 read it
            const uint32_t stage = sbase + kOffX + (uint32_t)b * kBox + (uint32_t)(lane & 3) * 4u;
            const int m0 = tile_row(j);
            for (int r0 = 0; r0 < kRows; r0 += kU) {
                float2 v[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int m = m0 + lw + kInferLoadWarps * (r0 + u);
                    v[u] = make_float2(0.f, 0.f);
                    if (m < a.M) {
                        const float* src = a.X + (int64_t)m * a.din + c0;
                        if (a.pairs) {
                            if (in0) v[u] = __ldcs(reinterpret_cast<const float2*>(src));
                        } else {
                            if (in0) v[u].x = __ldcs(src);
                            if (in1) v[u].y = __ldcs(src + 1);
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const uint32_t r = (uint32_t)(lw + kInferLoadWarps * (r0 + u));
                    const uint32_t dst = stage + r * 128u + ((((uint32_t)lane >> 2) ^ (r & 7u)) << 4);
                    asm volatile("st.shared.b32 [%0], %1;" ::"r"(dst), "r"(bf16x2_bits(v[u].x, v[u].y)) : "memory");
                }
            }
            // the writes are seen by the tensor cores' (async-proxy) reads
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive1(B(1 + b));
        }
    } else {
        const int q = warp & 3, cg = (warp - 1) >> 2;
        const int row = 32 * q + lane;
        const uint32_t lanes = (uint32_t)(32 * q) << 16;
        const uint32_t h1row = sbase + kOffH1 + (uint32_t)cg * kBox + (uint32_t)row * 128u;
        float b3r[OD];
        double mean[OD], sd[OD];
#pragma unroll
        for (int k = 0; k < OD; ++k) {
            b3r[k] = a.b3[k];
            mean[k] = a.scaler[k];
            sd[k] = a.scaler[OD + k];
        }
        for (int j = 0; j <= ntl; ++j) {
            if (j < ntl) {   // layer 1 of tile j -> the layer-2 operand
                const int b = j & 1;
                bool ok = iwait(B(11 + b), (uint32_t)(j >> 1) & 1u, fail);
                if (ok && j >= 1) ok = iwait(B(13 + ((j - 1) & 1)), (uint32_t)((j - 1) >> 1) & 1u, fail);   // H1 read
                tc::tc_fence_after();
                if (ok) {
                    const uint32_t tb = tmem + (uint32_t)(b * 256 + 64 * cg) + lanes;
                    uint32_t ra[16], rb[16];
                    tc::tmem_ld16_issue(tb, ra);
                    tc::tmem_wait_ld16(ra);
#pragma unroll
                    for (int c16 = 0; c16 < 4; ++c16) {
                        uint32_t(&cur)[16] = (c16 & 1) ? rb : ra;
                        uint32_t(&nxt)[16] = (c16 & 1) ? ra : rb;
                        if (c16 < 3) tc::tmem_ld16_issue(tb + (uint32_t)(16 * (c16 + 1)), nxt);   // in flight during this block
                        const float4* bp = reinterpret_cast<const float4*>(&sb1[64 * cg + 16 * c16]);
                        uint32_t w[8];
#pragma unroll
                        for (int q4 = 0; q4 < 4; ++q4) {
                            const float4 bb = bp[q4];
                            const f2m g0 = gelu2p(add2m(pkm(__uint_as_float(cur[4 * q4]), __uint_as_float(cur[4 * q4 + 1])), pkm(bb.x, bb.y)));
                            const f2m g1 = gelu2p(add2m(pkm(__uint_as_float(cur[4 * q4 + 2]), __uint_as_float(cur[4 * q4 + 3])), pkm(bb.z, bb.w)));
                            float x0, x1, x2, x3;
                            upkm(g0, x0, x1);
                            upkm(g1, x2, x3);
                            w[2 * q4] = bf16x2_bits(x0, x1);
                            w[2 * q4 + 1] = bf16x2_bits(x2, x3);
                        }
#pragma unroll
                        for (int half = 0; half < 2; ++half) {
                            const uint32_t ch = (uint32_t)(2 * c16 + half);
                            const uint32_t dst = h1row + ((ch ^ (uint32_t)(row & 7)) << 4);
                            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(dst), "r"(w[4 * half]),
                                         "r"(w[4 * half + 1]), "r"(w[4 * half + 2]), "r"(w[4 * half + 3])
                                         : "memory");
                        }
                        if (c16 < 3) tc::tmem_wait_ld16(nxt);
                    }
                }
                // the writes are seen by the tensor cores' (async-proxy) reads
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                tc::tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive1(B(15));
            }
            if (j >= 1) {   // layer 2 of tile j - 1 and the head
                const int t = j - 1, b = t & 1;
                const bool ok = iwait(B(13 + b), (uint32_t)(t >> 1) & 1u, fail);
                tc::tc_fence_after();
                f2m y2[OD];
#pragma unroll
                for (int k = 0; k < OD; ++k) y2[k] = pkm(0.f, 0.f);
                if (ok) {
                    const uint32_t tb = tmem + (uint32_t)(b * 256 + 64 * cg) + lanes;
                    uint32_t ra[16], rb[16];
                    tc::tmem_ld16_issue(tb, ra);
                    tc::tmem_wait_ld16(ra);
#pragma unroll
                    for (int c16 = 0; c16 < 4; ++c16) {
                        uint32_t(&cur)[16] = (c16 & 1) ? rb : ra;
                        uint32_t(&nxt)[16] = (c16 & 1) ? ra : rb;
                        if (c16 < 3) tc::tmem_ld16_issue(tb + (uint32_t)(16 * (c16 + 1)), nxt);
                        const int col = 64 * cg + 16 * c16;
                        const float4* bp = reinterpret_cast<const float4*>(&sb2[col]);
#pragma unroll
                        for (int q4 = 0; q4 < 4; ++q4) {
                            const float4 bb = bp[q4];
                            const f2m g0 = gelu2p(add2m(pkm(__uint_as_float(cur[4 * q4]), __uint_as_float(cur[4 * q4 + 1])), pkm(bb.x, bb.y)));
                            const f2m g1 = gelu2p(add2m(pkm(__uint_as_float(cur[4 * q4 + 2]), __uint_as_float(cur[4 * q4 + 3])), pkm(bb.z, bb.w)));
#pragma unroll
                            for (int k = 0; k < OD; ++k) {
                                const float4 ww = reinterpret_cast<const float4*>(&sw3[k][col])[q4];
                                y2[k] = fma2m(g0, pkm(ww.x, ww.y), y2[k]);
                                y2[k] = fma2m(g1, pkm(ww.z, ww.w), y2[k]);
                            }
                        }
                        if (c16 < 3) tc::tmem_wait_ld16(nxt);
                        if (c16 == 2) {
                            // the last block's columns are in registers: the
                            // accumulator is free for layer 1 of tile t + 2
                            // while this warp finishes the arithmetic
                            tc::tc_fence_before();
                            __syncwarp();
                            if (lane == 0) mbar_arrive1(B(16 + b));
                        }
                    }
                } else {
                    tc::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive1(B(16 + b));
                }
#pragma unroll
                for (int k = 0; k < OD; ++k) {
                    float lo, hi;
                    upkm(y2[k], lo, hi);
                    s_y[t & 1][cg][row][k] = lo + hi;
                }
                epi_bar();
                if (ok && cg == 0) {
                    const int m = tile_row(t) + row;
                    if (m < a.M) {
#pragma unroll
                        for (int k = 0; k < OD; ++k) {
                            float s = b3r[k];
#pragma unroll
                            for (int g = 0; g < 4; ++g) s += s_y[t & 1][g][row][k];
                            a.Y[(int64_t)m * OD + k] = (float)((double)s * sd[k] + mean[k]);
                        }
                    }
                }
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (tid == 0 && *fail) atomicAdd(a.timeouts, 1u);   // the host reports PTSNE_ETIMEOUT
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// Batch gather: rows of X (FP32, n x din) -> Xb (B x 64 BF16, zero-padded) and
// Xb^T (64 x B), targets -> standardised t (B x OD).  64 rows per block; a
// thread has all 16 of its (random-row) loads in flight before it uses any.
__global__ void __launch_bounds__(256)
gather_batch_kernel(const float* __restrict__ X, const float* __restrict__ T, int64_t n, int din, int od,
                    const int32_t* __restrict__ rows, int B, const double* __restrict__ scaler, bf16* __restrict__ Xb,
                    bf16* __restrict__ XbT, float* __restrict__ t, unsigned int* bad) {
    constexpr int kPer = 64 * kKin / 256;   // elements per thread
    __shared__ bf16 tile[64][kKin + 8];
    __shared__ int32_t s_rows[64];
    const int b0 = blockIdx.x * 64;
    if (threadIdx.x < 64) s_rows[threadIdx.x] = rows[b0 + threadIdx.x];
    __syncthreads();
    float v[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        const int idx = threadIdx.x + 256 * q, s = idx / kKin, k = idx % kKin;
        const int32_t r = s_rows[s];
        v[q] = (r >= 0 && r < n && k < din) ? X[(int64_t)r * din + k] : 0.f;
    }
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        const int idx = threadIdx.x + 256 * q, s = idx / kKin, k = idx % kKin;
        if (k == 0 && !(s_rows[s] >= 0 && s_rows[s] < n)) atomicAdd(bad, 1u);
        const bf16 bv = __float2bfloat16_rn(v[q]);
        Xb[(int64_t)(b0 + s) * kKin + k] = bv;
        tile[s][k] = bv;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < 64 * kKin; idx += 256) {
        const int k = idx / 64, s = idx % 64;
        XbT[(int64_t)k * B + b0 + s] = tile[s][k];
    }
    for (int idx = threadIdx.x; idx < 64 * od; idx += 256) {
        const int s = idx / od, k = idx % od;
        const int32_t r = s_rows[s];
        const double tv = (r >= 0 && r < n) ? (double)T[(int64_t)r * od + k] : scaler[k];
        t[(int64_t)(b0 + s) * od + k] = (float)((tv - scaler[k]) / scaler[od + k]);
    }
}

struct Offsets {
    int64_t W1, b1, W2, b2, W3, b3, n;
};

__host__ __device__ inline Offsets param_offsets(int din, int od) {
    Offsets o;
    o.W1 = 0;
    o.b1 = o.W1 + (int64_t)kH * din;
    o.W2 = o.b1 + kH;
    o.b2 = o.W2 + (int64_t)kH * kH;
    o.W3 = o.b2 + kH;
    o.b3 = o.W3 + (int64_t)od * kH;
    o.n = o.b3 + od;
    return o;
}

struct Bf16Copies {
    bf16 *W1b, *W2b, *W2Tb, *W3b;
};

__device__ __forceinline__ void write_copy(int64_t idx, float w, const Offsets& o, int din, const Bf16Copies& cp) {
    const bf16 b = __float2bfloat16_rn(w);
    if (idx < o.b1) {
        const int64_t h = idx / din, k = idx % din;
        cp.W1b[h * kKin + k] = b;
    } else if (idx >= o.W2 && idx < o.b2) {
        const int64_t q = idx - o.W2, oo = q / kH, i = q % kH;
        cp.W2b[oo * kH + i] = b;
        cp.W2Tb[i * kH + oo] = b;
    } else if (idx >= o.W3 && idx < o.b3) {
        cp.W3b[idx - o.W3] = b;
    }
}

__global__ void sync_copies_kernel(const float* __restrict__ W, Offsets o, int din, Bf16Copies cp) {
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < o.n; idx += (int64_t)gridDim.x * blockDim.x)
        write_copy(idx, W[idx], o, din, cp);
}

// AdamW (decoupled decay on W1, W2, W3) on the FP32 master parameters; the
// BF16 working copies are rewritten from the updated values.
__global__ void adamw_kernel(float* __restrict__ W, float* __restrict__ m1, float* __restrict__ m2,
                             const float* __restrict__ g, Offsets o, int din, Bf16Copies cp, float lr, float b1,
                             float b2, float eps, float wd, float bc1, float bc2) {
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < o.n; idx += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[idx];
        const float mi = b1 * m1[idx] + (1.0f - b1) * gi;
        const float vi = b2 * m2[idx] + (1.0f - b2) * gi * gi;
        m1[idx] = mi;
        m2[idx] = vi;
        const bool is_w = idx < o.b1 || (idx >= o.W2 && idx < o.b2) || (idx >= o.W3 && idx < o.b3);
        float w = W[idx];
        const float upd = (mi * bc1) / (sqrtf(vi * bc2) + eps) + (is_w ? wd * w : 0.f);
        w -= lr * upd;
        W[idx] = w;
        write_copy(idx, w, o, din, cp);
    }
}

// Scaler: mean (pass 1) and population standard deviation (pass 2) of each
// output coordinate, FP64.  acc holds [sum[od], ssq[od]].
__global__ void scaler_sum_kernel(const float* __restrict__ T, int64_t n, int od, const double* __restrict__ acc,
                                  double* __restrict__ out, int pass) {
    double s[3] = {0.0, 0.0, 0.0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        for (int k = 0; k < od; ++k) {
            const double v = T[i * od + k];
            if (pass == 0) s[k] += v;
            else {
                const double d = v - acc[k] / (double)n;
                s[k] += d * d;
            }
        }
    }
    for (int k = 0; k < od; ++k) {
        const double w = warp_sum(s[k]);
        if ((threadIdx.x & 31) == 0) atomicAdd(&out[k], w);
    }
}
__global__ void scaler_final_kernel(const double* __restrict__ acc, int64_t n, int od, double* __restrict__ scaler) {
    const int k = threadIdx.x;
    if (k < od) {
        scaler[k] = acc[k] / (double)n;
        const double sd = sqrt(acc[od + k] / (double)n);
        scaler[od + k] = sd > 0.0 ? sd : 1.0;
    }
}

}  // namespace mlp
}  // namespace ptsne

using namespace ptsne;
using namespace ptsne::mlp;

struct ptsne_mlp {
    ptsne_mlp_params p{};
    int din = 0, od = 0, B = 0;
    int64_t slab = 0;
    Offsets off{};
    float *W = nullptr, *m1 = nullptr, *m2 = nullptr, *grad = nullptr;
    int64_t step = 0;
    Bf16Copies cp{};
    double* scaler = nullptr;     // mean[od], std[od]
    double* sacc = nullptr;       // sum[od], ssq[od]
    bf16 *Xb = nullptr, *XbT = nullptr, *H1 = nullptr, *H1T = nullptr, *dA2 = nullptr, *dA2T = nullptr,
         *dA1T = nullptr;
    float *U1 = nullptr, *tb = nullptr;
    double* loss = nullptr;       // [1 + max epochs tracked per train call]
    int loss_cap = 0;
    unsigned int* dflags = nullptr;   // [0] timeouts, [1] bad rows
    int split = 0;                    // CTAs along K of the weight-gradient GEMMs (0: heuristic)
    CUtensorMap tmXb, tmW1b, tmH1, tmW2b, tmdA2T, tmH1T, tmdA2, tmW2Tb, tmdA1T, tmXbT;
    std::string err;
};

namespace {

thread_local std::string g_mlp_create_err;

int mfail(ptsne_mlp* m, int code, const char* msg) {
    if (m) m->err = msg;
    return code;
}

#define MCK(call)                                                          \
    do {                                                                   \
        cudaError_t e_ = (call);                                           \
        if (e_ != cudaSuccess) return mfail(m, PTSNE_ECUDA, cudaGetErrorString(e_)); \
    } while (0)

template <class T>
cudaError_t malloc_zero(T** p, size_t count) {
    cudaError_t e = cudaMalloc((void**)p, sizeof(T) * (count ? count : 1));
    if (e != cudaSuccess) {
        *p = nullptr;
        return e;
    }
    return cudaMemset(*p, 0, sizeof(T) * (count ? count : 1));
}

void free_mlp(ptsne_mlp* m) {
    void* ptrs[] = {m->W,   m->m1,  m->m2,   m->grad, m->cp.W1b, m->cp.W2b, m->cp.W2Tb, m->cp.W3b,
                    m->scaler, m->sacc, m->Xb, m->XbT, m->H1, m->H1T, m->dA2, m->dA2T, m->dA1T,
                    m->U1,  m->tb,  m->loss, m->dflags};
    for (void* q : ptrs)
        if (q) cudaFree(q);
}

// Ring stages of a CTA with nkb K blocks: all of them up to two (a single
// block needs one stage), else two, so that two CTAs share an SM.
int gemm_stages(int nkb) { return nkb <= kMaxStagesPair ? (nkb < 1 ? 1 : nkb) : kMaxStagesPair; }

size_t gemm_smem(int nt, int stages) {
    const size_t brows = nt < 128 ? 128 : nt;
    return (size_t)stages * (tc::kTileBytes + brows * 128) + 1024;
}

// Column groups of the epilogue: 4 (16 warps, one CTA per SM) for the
// 256-column GELU epilogues (forward, head, GELU backward), whose 32 row
// tiles per batch leave most SMs idle, so that each thread takes 64 columns;
// else 2 (8 warps) where the accumulator has 64 or more columns.
template <int NT, int EPI>
constexpr int gemm_groups() {
    return (NT == 256 && (EPI == EPI_FWD || EPI == EPI_HEAD_TRAIN || EPI == EPI_DGELU)) ? 4 : (NT >= 64 ? 2 : 1);
}

template <int NT, int EPI, int OD>
cudaError_t launch_gemm(const CUtensorMap& A, const CUtensorMap& B, GemmArgs a, int mtiles, int splits,
                        cudaStream_t s) {
    constexpr int CG = gemm_groups<NT, EPI>();
    auto kern = mlp_gemm_kernel<NT, EPI, OD, CG>;
    a.stages = gemm_stages(a.kb_per_split);
    const size_t smem = gemm_smem(NT, a.stages);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<dim3((unsigned)mtiles, (unsigned)splits), 128 * CG, smem, s>>>(A, B, a);
    return cudaGetLastError();
}

// floats per vector reduction of the split-K epilogue into C (row stride ldc)
int red_width(const float* C, int ldc) {
    const uintptr_t p = (uintptr_t)C;
    if (p % 16 == 0 && ldc % 4 == 0) return 4;
    if (p % 8 == 0 && ldc % 2 == 0) return 2;
    return 1;
}

GemmArgs base_args(ptsne_mlp* m) {
    GemmArgs a{};
    a.timeouts = m->dflags;
    return a;
}

// split-K shape of a K = B contraction: (K blocks per CTA, CTAs along K);
// `want` CTAs along K (0: at most 16)
void split_k(int kblocks, int want, int* per, int* splits) {
    int sp = want > 0 ? want : 16;
    if (sp > kblocks) sp = kblocks;
    *per = (kblocks + sp - 1) / sp;
    *splits = (kblocks + *per - 1) / *per;
}

template <int OD>
cudaError_t run_grad_od(ptsne_mlp* m, const float* X, const float* T, int64_t n, const int32_t* rows, double* loss,
                        cudaStream_t s) {
    const int B = m->B;
    cudaError_t e = cudaMemsetAsync(m->grad, 0, sizeof(float) * m->off.n, s);
    if (e != cudaSuccess) return e;
    gather_batch_kernel<<<B / 64, 256, 0, s>>>(X, T, n, m->din, OD, rows, B, m->scaler, m->Xb, m->XbT, m->tb,
                                               m->dflags + 1);
    // layer 1
    GemmArgs a = base_args(m);
    a.M = B;
    a.kblocks = 1;
    a.kb_per_split = 1;
    a.bias = m->W + m->off.b1;
    a.U = m->U1;
    a.H = m->H1;
    a.HT = m->H1T;
    a.ldT = B;
    if ((e = launch_gemm<kH, EPI_FWD, OD>(m->tmXb, m->tmW1b, a, B / 128, 1, s)) != cudaSuccess) return e;
    // layer 2 + head + loss + dW3 + dA2
    a = base_args(m);
    a.M = B;
    a.kblocks = kH / 64;
    a.kb_per_split = a.kblocks;
    a.bias = m->W + m->off.b2;
    a.H = m->dA2;
    a.HT = m->dA2T;
    a.ldT = B;
    a.colsum = m->grad + m->off.b2;
    a.W3 = m->cp.W3b;
    a.b3 = m->W + m->off.b3;
    a.T = m->tb;
    a.invB = 1.0f / (float)B;
    a.loss = loss;
    a.gW3 = m->grad + m->off.W3;
    a.gb3 = m->grad + m->off.b3;
    if ((e = launch_gemm<kH, EPI_HEAD_TRAIN, OD>(m->tmH1, m->tmW2b, a, B / 128, 1, s)) != cudaSuccess) return e;
    // dW2 = dA2^T H1
    int per, sp;
    split_k(B / 64, m->split, &per, &sp);
    a = base_args(m);
    a.M = kH;
    a.kblocks = B / 64;
    a.kb_per_split = per;
    a.C = m->grad + m->off.W2;
    a.ldc = kH;
    a.ncols = kH;
    a.red_width = red_width(a.C, a.ldc);
    if ((e = launch_gemm<kH, EPI_ATOMIC, OD>(m->tmdA2T, m->tmH1T, a, kH / 128, sp, s)) != cudaSuccess) return e;
    // dA1 = (dA2 W2) * g'(U1)
    a = base_args(m);
    a.M = B;
    a.kblocks = kH / 64;
    a.kb_per_split = a.kblocks;
    a.HT = m->dA1T;
    a.ldT = B;
    a.Uin = m->U1;
    a.colsum = m->grad + m->off.b1;
    if ((e = launch_gemm<kH, EPI_DGELU, OD>(m->tmdA2, m->tmW2Tb, a, B / 128, 1, s)) != cudaSuccess) return e;
    // dW1 = dA1^T Xb
    a = base_args(m);
    a.M = kH;
    a.kblocks = B / 64;
    a.kb_per_split = per;
    a.C = m->grad + m->off.W1;
    a.ldc = m->din;
    a.ncols = m->din;
    a.red_width = red_width(a.C, a.ldc);
    if ((e = launch_gemm<64, EPI_ATOMIC, OD>(m->tmdA1T, m->tmXbT, a, kH / 128, sp, s)) != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t run_grad(ptsne_mlp* m, const float* X, const float* T, int64_t n, const int32_t* rows, double* loss,
                     cudaStream_t s) {
    return m->od == 2 ? run_grad_od<2>(m, X, T, n, rows, loss, s) : run_grad_od<3>(m, X, T, n, rows, loss, s);
}

cudaError_t run_adamw(ptsne_mlp* m, cudaStream_t s) {
    m->step += 1;
    const ptsne_mlp_params& p = m->p;
    const float bc1 = (float)(1.0 / (1.0 - pow((double)p.beta1, (double)m->step)));
    const float bc2 = (float)(1.0 / (1.0 - pow((double)p.beta2, (double)m->step)));
    adamw_kernel<<<152 * 4, 256, 0, s>>>(m->W, m->m1, m->m2, m->grad, m->off, m->din, m->cp, p.lr, p.beta1, p.beta2,
                                         p.eps, p.weight_decay, bc1, bc2);
    return cudaGetLastError();
}

// Rows [0, M) of X through the fused kernel (persistent: one CTA per SM,
// each taking every gridDim.x-th row tile).
template <int OD>
cudaError_t launch_infer(ptsne_mlp* m, const float* X, int M, float* Y, cudaStream_t s) {
    auto kern = mlp_infer_kernel<OD>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kInferSmem);
    if (e != cudaSuccess) return e;
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
    }
    InferArgs a;
    a.X = X;
    a.M = M;
    a.mtiles = (M + 127) / 128;
    a.din = m->din;
    a.pairs = (m->din % 2 == 0 && ((uintptr_t)X & 7u) == 0) ? 1 : 0;
    a.b1 = m->W + m->off.b1;
    a.b2 = m->W + m->off.b2;
    a.W3 = m->cp.W3b;
    a.b3 = m->W + m->off.b3;
    a.scaler = m->scaler;
    a.Y = Y;
    a.timeouts = m->dflags;
    const int grid = a.mtiles < sms ? a.mtiles : sms;
    kern<<<(unsigned)grid, kInferThreads, kInferSmem, s>>>(m->tmW1b, m->tmW2b, a);
    return cudaGetLastError();
}

template <int OD>
cudaError_t run_infer_od(ptsne_mlp* m, const float* X, int64_t n, float* Y, cudaStream_t s) {
    for (int64_t r0 = 0; r0 < n; r0 += m->slab) {
        const int M = (int)((n - r0) < m->slab ? (n - r0) : m->slab);
        const cudaError_t e = launch_infer<OD>(m, X + r0 * m->din, M, Y + r0 * OD, s);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

bool valid_params(const ptsne_mlp_params* p, const char** why) {
    if (p->d_in < 1 || p->d_in > 64) return *why = "d_in must be in [1, 64]", false;
    if (p->out_dim != 2 && p->out_dim != 3) return *why = "out_dim must be 2 or 3", false;
    if (p->batch < 128 || p->batch > 65536 || p->batch % 128) return *why = "batch must be a multiple of 128 in [128, 65536]", false;
    if (p->infer_rows < 128 || p->infer_rows % 128 || p->infer_rows > (1 << 24))
        return *why = "infer_rows must be a multiple of 128 in [128, 2^24]", false;
    if (!(p->lr > 0.f) || !(p->beta1 >= 0.f && p->beta1 < 1.f) || !(p->beta2 >= 0.f && p->beta2 < 1.f) ||
        !(p->eps > 0.f) || !(p->weight_decay >= 0.f))
        return *why = "AdamW settings out of range (lr > 0, 0 <= beta < 1, eps > 0, weight_decay >= 0)", false;
    return true;
}

}  // namespace

extern "C" {

const char* ptsne_mlp_last_error(const ptsne_mlp* m) { return m ? m->err.c_str() : g_mlp_create_err.c_str(); }

int ptsne_mlp_create(ptsne_mlp** out, const ptsne_mlp_params* prm, const float* init_host) {
    if (!out || !prm || !init_host) {
        g_mlp_create_err = "out, params and init_host must be non-NULL";
        return PTSNE_EINVAL;
    }
    *out = nullptr;
    const char* why = nullptr;
    if (!valid_params(prm, &why)) {
        g_mlp_create_err = std::string("invalid parameter: ") + why;
        return PTSNE_EINVAL;
    }
    ptsne_mlp* m = new (std::nothrow) ptsne_mlp();
    if (!m) return PTSNE_ENOMEM;
    m->p = *prm;
    m->din = prm->d_in;
    m->od = prm->out_dim;
    m->B = prm->batch;
    m->slab = prm->infer_rows;
    m->off = param_offsets(m->din, m->od);
    const int64_t B = m->B;
    cudaError_t e = cudaSuccess;
    auto A = [&](cudaError_t r) {
        if (e == cudaSuccess) e = r;
    };
    A(malloc_zero(&m->W, m->off.n));
    A(malloc_zero(&m->m1, m->off.n));
    A(malloc_zero(&m->m2, m->off.n));
    A(malloc_zero(&m->grad, m->off.n));
    A(malloc_zero(&m->cp.W1b, (size_t)kH * kKin));
    A(malloc_zero(&m->cp.W2b, (size_t)kH * kH));
    A(malloc_zero(&m->cp.W2Tb, (size_t)kH * kH));
    A(malloc_zero(&m->cp.W3b, (size_t)m->od * kH));
    A(malloc_zero(&m->scaler, 2 * (size_t)m->od));
    A(malloc_zero(&m->sacc, 2 * (size_t)m->od));
    A(malloc_zero(&m->Xb, (size_t)B * kKin));
    A(malloc_zero(&m->XbT, (size_t)128 * B));   // rows 64..127 stay zero (the 128-row TMA box)
    A(malloc_zero(&m->H1, (size_t)B * kH));
    A(malloc_zero(&m->H1T, (size_t)kH * B));
    A(malloc_zero(&m->dA2, (size_t)B * kH));
    A(malloc_zero(&m->dA2T, (size_t)kH * B));
    A(malloc_zero(&m->dA1T, (size_t)kH * B));
    A(malloc_zero(&m->U1, (size_t)B * kH));
    A(malloc_zero(&m->tb, (size_t)B * m->od));
    m->loss_cap = 1024;
    A(malloc_zero(&m->loss, (size_t)m->loss_cap + 1));
    A(malloc_zero(&m->dflags, 2));
    if (e == cudaSuccess) e = cudaMemcpy(m->W, init_host, sizeof(float) * m->off.n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        std::vector<double> sc(2 * m->od, 0.0);
        for (int k = 0; k < m->od; ++k) sc[m->od + k] = 1.0;
        e = cudaMemcpy(m->scaler, sc.data(), sizeof(double) * sc.size(), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) {
        sync_copies_kernel<<<152, 256>>>(m->W, m->off, m->din, m->cp);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        g_mlp_create_err = std::string("device setup failed: ") + cudaGetErrorString(e);
        free_mlp(m);
        delete m;
        return e == cudaErrorMemoryAllocation ? PTSNE_ENOMEM : PTSNE_ECUDA;
    }
    bool ok = tc::make_bf16_tmap(&m->tmXb, m->Xb, B, kKin) && tc::make_bf16_tmap(&m->tmW1b, m->cp.W1b, kH, kKin) &&
              tc::make_bf16_tmap(&m->tmH1, m->H1, B, kH) && tc::make_bf16_tmap(&m->tmW2b, m->cp.W2b, kH, kH) &&
              tc::make_bf16_tmap(&m->tmdA2T, m->dA2T, kH, B) && tc::make_bf16_tmap(&m->tmH1T, m->H1T, kH, B) &&
              tc::make_bf16_tmap(&m->tmdA2, m->dA2, B, kH) && tc::make_bf16_tmap(&m->tmW2Tb, m->cp.W2Tb, kH, kH) &&
              tc::make_bf16_tmap(&m->tmdA1T, m->dA1T, kH, B) && tc::make_bf16_tmap(&m->tmXbT, m->XbT, 128, B);
    if (!ok) {
        g_mlp_create_err = "the driver refused a TMA tensor map";
        free_mlp(m);
        delete m;
        return PTSNE_ECUDA;
    }
    *out = m;
    return PTSNE_OK;
}

void ptsne_mlp_destroy(ptsne_mlp* m) {
    if (!m) return;
    cudaDeviceSynchronize();
    free_mlp(m);
    delete m;
}

int ptsne_mlp_get_params(ptsne_mlp* m, float* out_host, void* stream) {
    if (!m) return PTSNE_EINVAL;
    if (!out_host) return mfail(m, PTSNE_EINVAL, "out_host must be non-NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    MCK(cudaMemcpyAsync(out_host, m->W, sizeof(float) * m->off.n, cudaMemcpyDeviceToHost, s));
    MCK(cudaStreamSynchronize(s));
    return PTSNE_OK;
}

int ptsne_mlp_fit_scaler(ptsne_mlp* m, const float* T, int64_t n, void* stream) {
    if (!m) return PTSNE_EINVAL;
    if (!T || n < 1) return mfail(m, PTSNE_EINVAL, "T must be a device pointer and n >= 1");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    MCK(cudaMemsetAsync(m->sacc, 0, sizeof(double) * 2 * m->od, s));
    int64_t g = (n + 255) / 256;
    if (g > 152 * 8) g = 152 * 8;
    scaler_sum_kernel<<<(unsigned)g, 256, 0, s>>>(T, n, m->od, m->sacc, m->sacc, 0);
    scaler_sum_kernel<<<(unsigned)g, 256, 0, s>>>(T, n, m->od, m->sacc, m->sacc + m->od, 1);
    scaler_final_kernel<<<1, 32, 0, s>>>(m->sacc, n, m->od, m->scaler);
    MCK(cudaGetLastError());
    return PTSNE_OK;
}

int ptsne_mlp_grad(ptsne_mlp* m, const float* X, const float* T, int64_t n, const int32_t* rows, float* grad_out,
                   double* loss_out, void* stream) {
    if (!m) return PTSNE_EINVAL;
    if (!X || !T || !rows || n < 1) return mfail(m, PTSNE_EINVAL, "X, T and rows must be device pointers, n >= 1");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    MCK(cudaMemsetAsync(m->loss, 0, sizeof(double), s));
    MCK(run_grad(m, X, T, n, rows, m->loss, s));
    if (grad_out) MCK(cudaMemcpyAsync(grad_out, m->grad, sizeof(float) * m->off.n, cudaMemcpyDeviceToDevice, s));
    if (loss_out) MCK(cudaMemcpyAsync(loss_out, m->loss, sizeof(double), cudaMemcpyDeviceToDevice, s));
    return PTSNE_OK;
}

int ptsne_mlp_train_step(ptsne_mlp* m, const float* X, const float* T, int64_t n, const int32_t* rows,
                         double* loss_out, void* stream) {
    if (!m) return PTSNE_EINVAL;
    if (!X || !T || !rows || n < 1) return mfail(m, PTSNE_EINVAL, "X, T and rows must be device pointers, n >= 1");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    MCK(cudaMemsetAsync(m->loss, 0, sizeof(double), s));
    MCK(run_grad(m, X, T, n, rows, m->loss, s));
    MCK(run_adamw(m, s));
    if (loss_out) MCK(cudaMemcpyAsync(loss_out, m->loss, sizeof(double), cudaMemcpyDeviceToDevice, s));
    return PTSNE_OK;
}

int ptsne_mlp_train(ptsne_mlp* m, const float* X, const float* T, int64_t n, const int32_t* orders, int32_t epochs,
                    double* loss_out_host, void* stream) {
    if (!m) return PTSNE_EINVAL;
    if (!X || !T || !orders) return mfail(m, PTSNE_EINVAL, "X, T and orders must be device pointers");
    if (epochs < 0) return mfail(m, PTSNE_EINVAL, "epochs must be >= 0");
    if (n < m->B) return mfail(m, PTSNE_EINVAL, "n must be at least one batch");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int64_t steps = n / m->B;
    MCK(cudaMemsetAsync(m->dflags + 1, 0, sizeof(unsigned int), s));
    std::vector<double> host;
    for (int32_t e0 = 0; e0 < epochs; e0 += m->loss_cap) {
        const int ne = (epochs - e0) < m->loss_cap ? (epochs - e0) : m->loss_cap;
        MCK(cudaMemsetAsync(m->loss + 1, 0, sizeof(double) * ne, s));
        for (int e = 0; e < ne; ++e) {
            const int32_t* ord = orders + (int64_t)(e0 + e) * n;
            for (int64_t b = 0; b < steps; ++b) {
                MCK(run_grad(m, X, T, n, ord + b * m->B, m->loss + 1 + e, s));
                MCK(run_adamw(m, s));
            }
        }
        host.resize(ne);
        MCK(cudaMemcpyAsync(host.data(), m->loss + 1, sizeof(double) * ne, cudaMemcpyDeviceToHost, s));
        MCK(cudaStreamSynchronize(s));
        if (loss_out_host)
            for (int e = 0; e < ne; ++e) loss_out_host[e0 + e] = host[e] / (double)steps;
    }
    unsigned int flags[2];
    MCK(cudaMemcpyAsync(flags, m->dflags, sizeof flags, cudaMemcpyDeviceToHost, s));
    MCK(cudaStreamSynchronize(s));
    if (flags[0]) return mfail(m, PTSNE_ETIMEOUT, "a bounded wait inside a GEMM ran out");
    if (flags[1]) return mfail(m, PTSNE_EINVAL, "orders holds entries outside [0, n)");
    return PTSNE_OK;
}

int ptsne_mlp_autotune(ptsne_mlp* m, const float* X, const float* T, int64_t n, const int32_t* rows,
                       const char* cache_path, int32_t* split_out, void* stream) {
    if (!m) return PTSNE_EINVAL;
    if (!X || !T || !rows || n < 1) return mfail(m, PTSNE_EINVAL, "X, T and rows must be device pointers, n >= 1");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    MCK(cudaGetDevice(&dev));
    MCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaDeviceProp prop;
    MCK(cudaGetDeviceProperties(&prop, dev));
    std::string name(prop.name);
    for (char& ch : name)
        if (ch == ' ' || ch == '|') ch = '_';
    char key[512];
    snprintf(key, sizeof key, "mlp|%s|sm%d|din%d|od%d|batch%d", name.c_str(), sms, m->din, m->od, m->B);
    if (cache_path) {   // the last matching record wins
        if (FILE* f = fopen(cache_path, "r")) {
            char line[1024], k[600];
            int sp = 0;
            bool found = false;
            while (fgets(line, sizeof line, f))
                if (sscanf(line, "%599s %d", k, &sp) == 2 && strcmp(k, key) == 0 && sp > 0) {
                    m->split = sp;
                    found = true;
                }
            fclose(f);
            if (found) {
                if (split_out) *split_out = m->split;
                return PTSNE_OK;
            }
        }
    }
    // time the forward + backward pass (parameters untouched) for each split
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    MCK(cudaEventCreate(&e0));
    MCK(cudaEventCreate(&e1));
    const int kblocks = m->B / 64;
    int best = 0;
    float best_ms = 0.f;
    cudaError_t e = cudaSuccess;
    for (int sp = 1; sp <= 64 && e == cudaSuccess; sp *= 2) {
        if (sp > kblocks) break;
        m->split = sp;
        e = run_grad(m, X, T, n, rows, m->loss, s);   // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        for (int r = 0; r < 5 && e == cudaSuccess; ++r) e = run_grad(m, X, T, n, rows, m->loss, s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && (best == 0 || ms < best_ms)) { best = sp; best_ms = ms; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        m->split = 0;
        return mfail(m, PTSNE_ECUDA, cudaGetErrorString(e));
    }
    m->split = best;
    if (cache_path)
        if (FILE* f = fopen(cache_path, "a")) {
            fprintf(f, "%s %d %.6f\n", key, best, best_ms / 5.0);
            fclose(f);
        }
    if (split_out) *split_out = best;
    return PTSNE_OK;
}

int ptsne_mlp_infer(ptsne_mlp* m, const float* X, int64_t n, float* Y, void* stream) {
    if (!m) return PTSNE_EINVAL;
    if (!X || !Y || n < 1) return mfail(m, PTSNE_EINVAL, "X and Y must be device pointers, n >= 1");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    MCK(m->od == 2 ? run_infer_od<2>(m, X, n, Y, s) : run_infer_od<3>(m, X, n, Y, s));
    return PTSNE_OK;
}

int ptsne_mlp_warm_start(ptsne_mlp* m, ptsne_ctx* ctx, const float* X, const int32_t* perm, const float* Yrand,
                         float* Y, double* kl_out, int32_t* used_out, void* stream) {
    if (!m) return PTSNE_EINVAL;
    if (!ctx || !X || !perm || !Yrand || !Y) return mfail(m, PTSNE_EINVAL, "ctx, X, perm, Y_random and Y are required");
    if (ctx->layers != 1 || ctx->p.d != m->din || ctx->p.out_dim != m->od)
        return mfail(m, PTSNE_EINVAL, "the context needs layers = 1, d = d_in and the mapper's out_dim");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int64_t n = ctx->npts, od = m->od;
    if (!ctx->ycold) {
        MCK(cudaMalloc((void**)&ctx->ycold, sizeof(float) * (size_t)(n * od)));
        ctx->ws_bytes += sizeof(float) * (size_t)(n * od);
    }
    int rc = ptsne_mlp_infer(m, X, n, Y, stream);
    if (rc != PTSNE_OK) return rc;
    MCK(cudaMemcpyAsync(ctx->ycold, Yrand, sizeof(float) * (size_t)(n * od), cudaMemcpyDeviceToDevice, s));
    double warm[3] = {0, 0, 0}, cold[3] = {0, 0, 0};
    rc = ptsne_run(ctx, X, perm, 1, Y, warm, stream);
    if (rc < 0) return mfail(m, rc, ptsne_last_error(ctx));
    rc = ptsne_run(ctx, X, perm, 1, ctx->ycold, cold, stream);
    if (rc < 0) return mfail(m, rc, ptsne_last_error(ctx));
    const bool keep = !(warm[0] > cold[0]);
    if (!keep) {
        MCK(cudaMemcpyAsync(Y, ctx->ycold, sizeof(float) * (size_t)(n * od), cudaMemcpyDeviceToDevice, s));
        MCK(cudaStreamSynchronize(s));
    }
    if (kl_out) {
        kl_out[0] = warm[0];
        kl_out[1] = cold[0];
    }
    if (used_out) *used_out = keep ? 1 : 0;
    return PTSNE_OK;
}

}  // extern "C"
