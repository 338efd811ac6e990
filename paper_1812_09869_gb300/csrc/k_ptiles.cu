// Packed symmetric P: the joint P of Eq. 3 written into the stored 32 x 32
// tiles the iteration kernel streams (one tile per unordered pair of 32-row
// blocks, values in the order of the warp that evaluates them, see
// packed_index), and the export of those tiles to dense per-chunk matrices.
#include "ptsne_internal.cuh"

namespace ptsne {

// Joint P (Eq. 3) of one stored 32 x 32 tile, written in the packed order:
//   p_ij = (exp(-beta_i (d_ij - m_i)) / S_i + exp(-beta_j (d_ji - m_j)) / S_j) / (2z),
// zero on the diagonal and outside the chunk.  D need not be symmetric: after
// the window recompute each row holds its own exact entries.  128 threads per
// tile (thread: rows r and r + 16, four columns), so that 16 tiles' chains of
// dependent loads are in flight per SM.
constexpr int kPsymThreads = 128;
__global__ void __launch_bounds__(kPsymThreads, 16)
psym_packed_kernel(const float* __restrict__ D, float* __restrict__ P2, Layout L, const int64_t* __restrict__ ptile_off,
                   const TileDesc2* __restrict__ tiles, int64_t t0, const float* __restrict__ beta,
                   const float* __restrict__ mrow, const float* __restrict__ Srow, uint8_t* __restrict__ nz_out) {
    constexpr float kLog2e = 1.4426950408889634f;
    const TileDesc2 td = tiles[t0 + blockIdx.x];
    const int c = td.chunk;
    const int64_t off = L.off[c];
    const int z = (int)(L.off[c + 1] - off);
    const int ld = L.ld[c];
    const int tid = threadIdx.x, r0 = tid >> 3, c4 = tid & 7;
    const int j0 = td.b * kPT + c4 * 4;
    // the (b, a) block of D, transposed: dT[jj][ii] = d_{j i}, so that each
    // conditional of Eq. 3 is taken from its own row of D
    __shared__ float dT[kPT][kPT + 1];
    // beta log2(e), m and 1 / S of the tile's rows (side 0) and columns (side 1)
    __shared__ float pb[2][kPT], pm[2][kPT], ps[2][kPT];
    if (tid < 2 * kPT) {
        const int side = tid >> 5, k = tid & (kPT - 1);
        const int g = (side ? td.b : td.a) * kPT + k;
        float b = 0.f, m = 0.f, si = 0.f;
        if (g < z) {
            b = beta[off + g] * kLog2e;
            m = mrow[off + g];
            si = 1.0f / Srow[off + g];
        }
        pb[side][k] = b;
        pm[side][k] = m;
        ps[side][k] = si;
    }
    // all four 16-byte loads of D are issued before the barrier
    const float* Dc = D + L.moff[c];
    float4 dv[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int i = td.a * kPT + r0 + 16 * h;
        dv[h] = i < z ? *reinterpret_cast<const float4*>(Dc + (int64_t)i * ld + j0) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int rr = r0 + 16 * h, jr = td.b * kPT + rr;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (jr < z) v = *reinterpret_cast<const float4*>(Dc + (int64_t)jr * ld + td.a * kPT + c4 * 4);
        dT[rr][c4 * 4 + 0] = v.x; dT[rr][c4 * 4 + 1] = v.y; dT[rr][c4 * 4 + 2] = v.z; dT[rr][c4 * 4 + 3] = v.w;
    }
    __syncthreads();
    __shared__ __align__(16) float ot[kPTileFloats];
    const float inv2z = 1.0f / (2.0f * (float)z);
    bool any = false;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int r = r0 + 16 * h, i = td.a * kPT + r;
        float out[4] = {0.f, 0.f, 0.f, 0.f};
        if (i < z) {
            const float d4[4] = {dv[h].x, dv[h].y, dv[h].z, dv[h].w};
            const float bi = pb[0][r], mi = pm[0][r], si = ps[0][r];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int j = j0 + e;
                if (j < z && j != i) {
                    const int jj = c4 * 4 + e;
                    const float bj = pb[1][jj], mj = pm[1][jj], sj = ps[1][jj];
                    // explicitly rounded: the two halves of a diagonal tile round identically
                    const float cij = __fmul_rn(hw_ex2(-bi * (d4[e] - mi)), si);
                    const float cji = __fmul_rn(hw_ex2(-bj * (dT[jj][r] - mj)), sj);
                    out[e] = __fmul_rn(__fadd_rn(cij, cji), inv2z);
                }
            }
        }
        // reorder through shared memory into the stored order (float4 F of
        // the tile staged at F ^ ((F >> 5) & 7): few bank conflicts on
        // these writes, none on the contiguous reads below)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int pi = packed_index(r, c4 * 4 + e, L.od);
            ot[(((pi >> 2) ^ ((pi >> 7) & 7)) << 2) | (pi & 3)] = out[e];
        }
        any = any || out[0] != 0.f || out[1] != 0.f || out[2] != 0.f || out[3] != 0.f;
    }
    // a tile whose every entry is exactly zero (far pairs: the FP32
    // exponentials underflow) is flagged (counted by ptsne_get_stats)
    const int nz = __syncthreads_or(any);
    const int64_t gt = ptile_off[c] + td.pos;
    float* dst = P2 + gt * kPTileStride;
#pragma unroll
    for (int h = 0; h < 2; ++h) {   // coalesced 16-byte stores of the tile
        const int F = tid + kPsymThreads * h;
        reinterpret_cast<float4*>(dst)[F] = reinterpret_cast<const float4*>(ot)[F ^ ((F >> 5) & 7)];
    }
    if (tid == 0) {   // trailer: the tile's row and column blocks and its flag
        *reinterpret_cast<int4*>(dst + kPTileFloats) = make_int4(td.a, td.b, nz, 0);
        nz_out[gt] = (uint8_t)nz;
    }
}

// Packed tiles -> dense z x z per chunk (chunks concatenated), both halves.
// src_row (optional): the rows are in locality order; row i of the chunk is
// row src_row[off + i] - off of the caller's partition, where it goes.
__global__ void __launch_bounds__(256)
export_packed_kernel(const float* __restrict__ P2, Layout L, const int64_t* __restrict__ ptile_off,
                     const TileDesc2* __restrict__ tiles, const int64_t* __restrict__ dense_off,
                     const int32_t* __restrict__ src_row, float* __restrict__ out) {
    const TileDesc2 td = tiles[blockIdx.x];
    const int c = td.chunk;
    const int64_t off = L.off[c];
    const int z = (int)(L.off[c + 1] - off);
    const float* src = P2 + (ptile_off[c] + td.pos) * kPTileStride;
    float* dst = out + dense_off[c];
    for (int e = threadIdx.x; e < kPTileFloats; e += blockDim.x) {
        const int r = e >> 5, cc = e & 31;
        int i = td.a * kPT + r, j = td.b * kPT + cc;
        if (i < z && j < z) {
            const float v = src[packed_index(r, cc, L.od)];
            if (src_row) {   // locality order: back to the caller's rows
                i = (int)(src_row[off + i] - off);
                j = (int)(src_row[off + j] - off);
            }
            dst[(int64_t)i * z + j] = v;
            dst[(int64_t)j * z + i] = v;
        }
    }
}

// ---------------------------------------------------------------- launchers

cudaError_t launch_psym_packed(const ptsne_ctx* c, cudaStream_t s) {
    if (c->ntiles2 <= 0) return cudaSuccess;
    int k = 0;
    for (int64_t b = 0; b < c->ntiles2; b += 2147483647LL, ++k) {
        const int64_t cnt = (c->ntiles2 - b) < 2147483647LL ? (c->ntiles2 - b) : 2147483647LL;
        psym_packed_kernel<<<(unsigned)cnt, kPsymThreads, 0, s>>>(c->D, c->P2, make_layout(c), c->d_ptile_off, c->d_tiles2, b,
                                                         c->beta, c->mrow, c->Srow, c->ptile_nz);
    }
    return launched(c, k);
}

cudaError_t launch_export_packed(const ptsne_ctx* c, float* P_out, cudaStream_t s) {
    export_packed_kernel<<<(unsigned)c->ntiles2, 256, 0, s>>>(c->P2, make_layout(c), c->d_ptile_off, c->d_tiles2,
                                                              c->d_dense_off, c->loc_active ? c->src_row : nullptr,
                                                              P_out);
    return launched(c, 1);
}

// Number of stored tiles flagged nonzero by the last joint-P assembly.
__global__ void __launch_bounds__(256) count_nonzero_kernel(const uint8_t* __restrict__ nz, int64_t n,
                                                            unsigned long long* __restrict__ out) {
    unsigned long long cnt = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        cnt += nz[i] != 0;
    cnt = warp_sum((double)cnt);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(out, cnt);
}

cudaError_t launch_count_nonzero(const ptsne_ctx* c, unsigned long long* out, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess || c->ntiles2 <= 0) return e;
    int64_t g = (c->ntiles2 + 255) / 256;
    if (g > 152 * 8) g = 152 * 8;
    count_nonzero_kernel<<<(unsigned)g, 256, 0, s>>>(c->ptile_nz, c->ntiles2, out);
    return cudaGetLastError();   // a query: not counted among the context's kernel launches
}

}  // namespace ptsne
