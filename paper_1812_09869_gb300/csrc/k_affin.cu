// Input affinities of each chunk: per-row precision search (Eq. 1, Eq. 2) and
// the symmetric joint P (Eq. 3, with n := z, the chunk size).
//
// Row search: one warp per row, the row staged once in shared memory as
// t_j = d_ij - m_i (m_i = min_{j!=i} d_ij; the shift cancels in Eq. 1).  The
// entropy H(beta) = ln S + beta T1 / S with S = sum e_j, T1 = sum t_j e_j,
// e_j = exp(-beta t_j), is non-increasing in beta, so the root of
// H(beta) = ln(perplexity) is bracketed and found by bisection on beta,
// accelerated by Newton steps in ln(beta) (dH/dln(beta) = -beta^2 Var_p(t))
// whenever the Newton point falls inside the bracket.  Sums are FP32 per lane
// (compensated once the root is near) and reduced across the warp in FP64.  A
// row whose FP32 search stalls (bracket collapsed, or 64 evaluations) is
// redone in FP64 by the same warp.
#include <float.h>

#include "ptsne_internal.cuh"

namespace ptsne {

namespace {
constexpr int kBisectWarpsMax = 8;
constexpr float kBig = 1e37f;          // stands for "excluded" (diagonal, tail padding)
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kTolFine = 1e-6f;      // |H - ln perp| (nats) accepted from the FP32 search
constexpr float kTolCoarse = 1e-3f;    // switch to compensated sums below this
constexpr double kTol64 = 1e-9;        // FP64 fallback tolerance
constexpr int kMaxEval32 = 64;
constexpr int kMaxEval64 = 200;
}  // namespace

struct RowSums {
    float S, T1, T2;
};

// Warp sum of per-lane values s + c (c a compensation term), combining lanes
// with an error-free two-sum at every level, so the result keeps FP32
// accuracy independently of the tree.
__device__ __forceinline__ float warp_sum_comp(float s, float c) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float so = __shfl_xor_sync(0xffffffffu, s, o);
        const float co = __shfl_xor_sync(0xffffffffu, c, o);
        const float t = s + so;
        const float bb = t - s;
        const float e = (s - (t - bb)) + (so - bb);
        s = t;
        c = c + co + e;
    }
    return s + c;
}

// S, T1, T2 of the staged row at precision beta.  `fine` selects compensated
// (Kahan) per-lane sums and a compensated cross-lane reduction of S and T1.
__device__ __forceinline__ RowSums row_sums(const float* __restrict__ row, int zr, float beta, bool fine) {
    const int lane = threadIdx.x & 31;
    const float b2 = beta * kLog2e;
    const float4* r4 = reinterpret_cast<const float4*>(row);
    const int nq = zr >> 2;  // zr is a multiple of 4 (tail padded with kBig)
    float S = 0.f, T1 = 0.f, T2 = 0.f;
    RowSums out;
    if (!fine) {
        float S2 = 0.f, T12 = 0.f, T22 = 0.f;
        int q = lane;
        for (; q + 32 < nq; q += 64) {
            const float4 a = r4[q], b = r4[q + 32];
            const float ta[4] = {a.x, a.y, a.z, a.w}, tb[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float ea = hw_ex2(-b2 * ta[e]), eb = hw_ex2(-b2 * tb[e]);
                const float tea = ta[e] * ea, teb = tb[e] * eb;
                S += ea; T1 += tea; T2 = fmaf(tea, ta[e], T2);
                S2 += eb; T12 += teb; T22 = fmaf(teb, tb[e], T22);
            }
        }
        for (; q < nq; q += 32) {
            const float4 a = r4[q];
            const float ta[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float ea = hw_ex2(-b2 * ta[e]);
                const float tea = ta[e] * ea;
                S += ea; T1 += tea; T2 = fmaf(tea, ta[e], T2);
            }
        }
        out.S = warp_sum(S + S2);
        out.T1 = warp_sum(T1 + T12);
        out.T2 = warp_sum(T2 + T22);
        return out;
    }
    float cS = 0.f, cT = 0.f;  // Kahan compensations (true sum = S - cS)
    for (int q = lane; q < nq; q += 32) {
        const float4 a = r4[q];
        const float ta[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float ea = hw_ex2(-b2 * ta[e]);
            const float tea = ta[e] * ea;
            float y = ea - cS, t = S + y;
            cS = (t - S) - y; S = t;
            y = tea - cT; t = T1 + y;
            cT = (t - T1) - y; T1 = t;
            T2 = fmaf(tea, ta[e], T2);
        }
    }
    out.S = warp_sum_comp(S, -cS);
    out.T1 = warp_sum_comp(T1, -cT);
    out.T2 = warp_sum(T2);
    return out;
}

__global__ void __launch_bounds__(kBisectWarpsMax * 32)
bisect_kernel(const float* __restrict__ D, Layout L, int64_t r0, int64_t r1, int ldmax, double ln_perp_d,
              float* __restrict__ beta_out, float* __restrict__ m_out, float* __restrict__ S_out,
              DeviceStats* st) {
    extern __shared__ __align__(16) float smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float* row = smem + (size_t)warp * ldmax;
    const float ln_perp = (float)ln_perp_d;
    for (int64_t r = r0 + (int64_t)blockIdx.x * nw + warp; r < r1; r += (int64_t)gridDim.x * nw) {
        const int c = L.chunk_of_row[r];
        const int64_t off = L.off[c];
        const int z = (int)(L.off[c + 1] - off);
        const int i = (int)(r - off);
        const int ld = L.ld[c];
        const int zr = (z + 3) & ~3;
        const float* src = D + L.moff[c] + (int64_t)i * ld;

        // stage the row, excluding the diagonal and the padded tail
        float mn = FLT_MAX;
        for (int j = lane * 4; j < zr; j += 128) {
            float4 v = *reinterpret_cast<const float4*>(src + j);
            float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (j + e >= z || j + e == i) vv[e] = kBig;
                else mn = fminf(mn, vv[e]);
            }
            *reinterpret_cast<float4*>(row + j) = make_float4(vv[0], vv[1], vv[2], vv[3]);
        }
        mn = warp_min(mn);
        __syncwarp();
        float tsum = 0.f;
        for (int j = lane; j < zr; j += 32) {
            const float v = row[j];
            const float t = v >= kBig ? kBig : v - mn;
            row[j] = t;
            if (t < kBig) tsum += t;
        }
        tsum = warp_sum(tsum);
        __syncwarp();

        float beta, S, herr;
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
            bool conv = false;
            RowSums s{};
            for (int it = 0; it < kMaxEval32; ++it) {
                const bool fine = fabsf(f) < kTolCoarse;
                s = row_sums(row, zr, beta, fine);
                // H in nats; logf and the division are correctly rounded to ~1 ulp
                f = (logf(s.S) + beta * (s.T1 / s.S)) - ln_perp;
                // accept only from a compensated evaluation
                if (fine && fabsf(f) <= kTolFine) { conv = true; break; }
                if (f > 0.f) lo = beta; else hi = beta;
                const float mean = s.T1 / s.S;
                const float var = fmaxf(s.T2 / s.S - mean * mean, 0.f);
                const float denom = beta * beta * var;
                float step = denom > 0.f ? f / denom : 0.f;
                step = fminf(fmaxf(step, -3.f), 3.f);
                float nb = beta * expf(step);
                if (!(nb > lo && nb < hi)) nb = isinf(hi) ? 2.f * beta : 0.5f * (lo + hi);
                if (nb == beta || (hi - lo) <= 4e-7f * beta) break;  // FP32 stall
                beta = nb;
            }
            S = s.S;
            herr = fabsf(f);
            if (!conv) {
                // FP64 redo of the same search on the staged (FP32) row
                fp64 = true;
                double b = beta, blo = 0.0, bhi = INFINITY, fd = INFINITY, Sd = 0.0;
                for (int it = 0; it < kMaxEval64; ++it) {
                    double sS = 0.0, sT1 = 0.0, sT2 = 0.0;
                    for (int j = lane; j < zr; j += 32) {
                        const float t = row[j];
                        if (t >= kBig) continue;
                        const double e = exp(-b * (double)t);
                        sS += e; sT1 += (double)t * e; sT2 += (double)t * t * e;
                    }
                    sS = warp_sum(sS); sT1 = warp_sum(sT1); sT2 = warp_sum(sT2);
                    Sd = sS;
                    fd = log(sS) + b * sT1 / sS - ln_perp_d;
                    if (fabs(fd) <= kTol64) break;
                    if (fd > 0.0) blo = b; else bhi = b;
                    const double mean = sT1 / sS;
                    const double var = fmax(sT2 / sS - mean * mean, 0.0);
                    double step = var > 0.0 ? fd / (b * b * var) : 0.0;
                    step = fmin(fmax(step, -3.0), 3.0);
                    double nb = b * exp(step);
                    if (!(nb > blo && nb < bhi)) nb = isinf(bhi) ? 2.0 * b : 0.5 * (blo + bhi);
                    if (nb == b) break;
                    b = nb;
                }
                beta = (float)b;
                S = (float)Sd;
                herr = (float)fabs(fd);
                failed = herr > kTolFine;
            }
        }
        if (lane == 0) {
            beta_out[r] = beta;
            m_out[r] = mn;
            S_out[r] = S;
            if (fp64) atomicAdd(&st->fp64_rows, 1ull);
            if (failed) atomicAdd(&st->failed_rows, 1ull);
            atomicMax(&st->max_herr_bits, __float_as_uint(herr));
        }
        __syncwarp();
    }
}

// Joint P of Eq. 3 on one 64 x 64 upper tile (I <= J), written to the tile and
// its transpose.  D is symmetric, so d_ji is read from the same tile:
//   p_ij = (exp(-beta_i (d_ij - m_i)) / S_i + exp(-beta_j (d_ij - m_j)) / S_j) / (2z).
// The padded columns [z, ld) of every row are set to 0.
__global__ void __launch_bounds__(256)
psym_kernel(const float* __restrict__ D, float* __restrict__ P, Layout L, const TileDesc* __restrict__ tiles,
            int64_t t0, const float* __restrict__ beta, const float* __restrict__ mrow,
            const float* __restrict__ Srow) {
    __shared__ float pb[2][kTile], pm[2][kTile], ps[2][kTile];
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
    __syncthreads();
    const float inv2z = 1.0f / (2.0f * (float)z);
    const float* dbase = D + L.moff[c];
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
                // explicitly rounded products and sum: no FMA contraction, so the
                // (i, j) and (j, i) threads of a diagonal tile round identically
                const float cij = __fmul_rn(hw_ex2(-pb[0][li] * (d4[q] - pm[0][li])), ps[0][li]);
                const float cji = __fmul_rn(hw_ex2(-pb[1][lj] * (d4[q] - pm[1][lj])), ps[1][lj]);
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

cudaError_t launch_bisect(const ptsne_ctx* c, int64_t row_begin, int64_t row_end, cudaStream_t s) {
    const int64_t rows = row_end - row_begin;
    if (rows <= 0) return cudaSuccess;
    const int ldmax = (int)((c->zmax + kTile - 1) / kTile * kTile);
    // one staged row per warp: as many warps as 227 KB of shared memory holds (<= 8)
    int warps = (int)((227 * 1024) / ((size_t)ldmax * sizeof(float)));
    warps = warps > kBisectWarpsMax ? kBisectWarpsMax : (warps < 1 ? 1 : warps);
    const size_t smem = (size_t)warps * ldmax * sizeof(float);
    cudaFuncSetAttribute(bisect_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int64_t blocks = (rows + warps - 1) / warps;
    if (blocks > 152 * 16) blocks = 152 * 16;
    bisect_kernel<<<(unsigned)blocks, warps * 32, smem, s>>>(
        c->D, make_layout(c), row_begin, row_end, ldmax, log(c->p.perplexity), c->beta, c->mrow,
        c->Srow, c->dstats);
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
