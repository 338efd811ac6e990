// Pairwise squared Euclidean distances ||x_i - x_j||^2 within each chunk
// (ptSNE section, "Similarities in the input space"), FP32, by direct
// differences sum_k (x_ik - x_jk)^2: no ||x||^2 + ||y||^2 - 2 x.y cancellation,
// and bitwise symmetric because (a - b)^2 == (b - a)^2 with the same k order.
//
// Work unit: one 64 x 64 upper-triangular tile (I <= J) of one chunk; the
// block writes the tile and, off the diagonal, its transpose, so D is
// symmetric by construction and each pair is computed once.  Blocks are
// persistent (a grid-stride loop over the tile list) and skip the tiles that
// a TileSel leaves out: in the mixed-precision form the same kernel computes
// the chunks run in FP32 whole and, in the others, the tiles that hold window
// pairs of the dense window rows.
//
// Thread (ty, tx) of 16 x 16 owns rows 4ty..4ty+3 and columns 4tx..4tx+3.
// Each step of k stages 32 dimensions of both row blocks k-major in shared
// memory (8 lanes per row: coalesced 128-byte loads; the 4-row groups of
// dimension k sit at group g ^ ((k / 4) mod 8), so that the eight lanes of a
// row, which store dimensions 4m .. 4m + 3 for m = 0..7, and the warp's four
// rows hit 32 different banks, while the reads of four consecutive rows stay
// one aligned 16-byte load); the products run two
// rows per packed f32x2 instruction against a column value duplicated into
// both halves (IEEE round-to-nearest per lane, so every distance is the same
// sequence of roundings as the scalar sum over k in order).  The next step's
// rows are loaded into registers while the current one computes.
#include "ptsne_internal.cuh"

namespace ptsne {

namespace {
constexpr int KC = 32;            // dims staged per step
constexpr int SROW = kTile + 4;   // shared-memory row stride (floats) of the k-major blocks
// column of row `row` in the k-major block's line for dimension k (4-row groups swizzled)
__device__ __forceinline__ int swz(int k, int row) { return row ^ (((k >> 2) & 7) << 2); }

typedef unsigned long long f2;
__device__ __forceinline__ f2 pk(float a, float b) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk(f2 v, float& a, float& b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v)); }
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
}  // namespace

__device__ __forceinline__ bool tile_selected(const TileSel& sel, const TileDesc& td, int z) {
    if (!sel.chunk_fp32 || sel.chunk_fp32[td.chunk]) return true;
    if (!sel.tflag) return false;
    const int T = (z + kTile - 1) / kTile;
    const uint8_t* f = sel.tflag + sel.tflag_off[td.chunk];
    return (f[td.I * T + td.J] | f[td.J * T + td.I]) != 0;
}

__global__ void __launch_bounds__(256, 4)
dist_fp32_kernel(const float* __restrict__ Xg, float* __restrict__ D, Layout L, const TileDesc* __restrict__ tiles,
                 int64_t t0, int64_t nt, TileSel sel, unsigned long long* __restrict__ sel_pairs) {
    __shared__ __align__(16) float sI[KC][SROW];
    __shared__ __align__(16) float sJ[KC][SROW];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int dp = L.dp;
    unsigned long long npairs = 0;
    for (int64_t t = blockIdx.x; t < nt; t += gridDim.x) {
        const TileDesc td = tiles[t0 + t];
        const int c = td.chunk;
        const int64_t off = L.off[c];
        const int z = (int)(L.off[c + 1] - off);
        if (!tile_selected(sel, td, z)) continue;   // uniform over the block
        const int ld = L.ld[c];
        const int i0 = td.I * kTile, j0 = td.J * kTile;
        // staging: slot e = tid + 256 h holds row e >> 3, quad e & 7 of a step
        float4 ra[2], rb[2];
        auto load = [&](int k0) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int e = tid + 256 * h, row = e >> 3, k = k0 + 4 * (e & 7);
                float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
                if (k < dp) {   // dp is a multiple of 4
                    if (i0 + row < z) a = *reinterpret_cast<const float4*>(Xg + (off + i0 + row) * dp + k);
                    if (j0 + row < z) b = *reinterpret_cast<const float4*>(Xg + (off + j0 + row) * dp + k);
                }
                ra[h] = a;
                rb[h] = b;
            }
        };
        f2 acc[2][4];   // acc[rp][q]: rows 4ty + 2rp, 4ty + 2rp + 1 against column 4tx + q
#pragma unroll
        for (int rp = 0; rp < 2; ++rp)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[rp][q] = 0ull;
        load(0);
        for (int k0 = 0; k0 < dp; k0 += KC) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int e = tid + 256 * h, kk = 4 * (e & 7), col = swz(kk, e >> 3);
                sI[kk + 0][col] = ra[h].x; sI[kk + 1][col] = ra[h].y;
                sI[kk + 2][col] = ra[h].z; sI[kk + 3][col] = ra[h].w;
                sJ[kk + 0][col] = rb[h].x; sJ[kk + 1][col] = rb[h].y;
                sJ[kk + 2][col] = rb[h].z; sJ[kk + 3][col] = rb[h].w;
            }
            __syncthreads();
            if (k0 + KC < dp) load(k0 + KC);
            // (dimensions beyond dp are staged as zeros: fma(0, 0, acc) == acc exactly)
#pragma unroll 8
            for (int k = 0; k < KC; ++k) {
                const ulonglong2 a = *reinterpret_cast<const ulonglong2*>(&sI[k][swz(k, 4 * ty)]);   // rows in pairs
                const float4 b = *reinterpret_cast<const float4*>(&sJ[k][swz(k, 4 * tx)]);
                const f2 bq[4] = {pk(b.x, b.x), pk(b.y, b.y), pk(b.z, b.z), pk(b.w, b.w)};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    f2 d = sub2(a.x, bq[q]);
                    acc[0][q] = fma2(d, d, acc[0][q]);
                    d = sub2(a.y, bq[q]);
                    acc[1][q] = fma2(d, d, acc[1][q]);
                }
            }
            __syncthreads();
        }
        float v[4][4];   // v[r][q]: row 4ty + r, column 4tx + q
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            upk(acc[0][q], v[0][q], v[1][q]);
            upk(acc[1][q], v[2][q], v[3][q]);
        }
        float* base = D + L.moff[c];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int i = i0 + ty * 4 + r;
            if (i < z)
                *reinterpret_cast<float4*>(base + (int64_t)i * ld + j0 + tx * 4) =
                    make_float4(v[r][0], v[r][1], v[r][2], v[r][3]);
        }
        if (td.I != td.J) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int j = j0 + tx * 4 + q;
                if (j < z)
                    *reinterpret_cast<float4*>(base + (int64_t)j * ld + i0 + ty * 4) =
                        make_float4(v[0][q], v[1][q], v[2][q], v[3][q]);
            }
        }
        if (sel.chunk_fp32 && !sel.chunk_fp32[c] && tid == 0) {   // window tile of a mixed chunk
            const int hi = min(kTile, z - i0), hj = min(kTile, z - j0);
            npairs += (unsigned long long)hi * hj * (td.I != td.J ? 2 : 1);
        }
    }
    if (tid == 0 && npairs && sel_pairs) atomicAdd(sel_pairs, npairs);
}

cudaError_t launch_dist_fp32_sel(const ptsne_ctx* c, int64_t tile_begin, int64_t tile_end, const TileSel& sel,
                                 cudaStream_t s) {
    const int64_t nt = tile_end - tile_begin;
    if (nt <= 0) return cudaSuccess;
    int64_t g = (int64_t)c->num_sms * 4;
    if (g > nt) g = nt;
    dist_fp32_kernel<<<(unsigned)g, 256, 0, s>>>(c->Xg, c->D, make_layout(c), c->d_tiles, tile_begin, nt, sel,
                                                  &c->dstats->window_pairs);
    return launched(c, 1);
}

cudaError_t launch_dist_fp32(const ptsne_ctx* c, int64_t tile_begin, int64_t tile_end, cudaStream_t s) {
    return launch_dist_fp32_sel(c, tile_begin, tile_end, TileSel{}, s);
}

// Form of each chunk's distances in the mixed-precision mode.  A chunk whose
// window (the pairs that the FP32 recompute must cover) is most of the chunk
// costs less computed in FP32 whole than as a BF16 Gram matrix, a coarse
// search and the recompute; the window fraction of the chunk's size bin
// (measured by the last affinities' searches) against the threshold decides.
// One block; bins without rows in the last affinities keep their fraction.
__global__ void __launch_bounds__(256)
form_select_kernel(const int64_t* __restrict__ off, int nc, int zmin, int zmax, unsigned long long* __restrict__ acc,
                   float* __restrict__ frac, const float* __restrict__ fstar, uint8_t* __restrict__ chunk_fp32,
                   unsigned int* __restrict__ fp32_count) {
    __shared__ float sf[kFormBins];
    __shared__ unsigned int scount;
    const int tid = threadIdx.x;
    if (tid < kFormBins) {
        const unsigned long long w = acc[2 * tid], n = acc[2 * tid + 1];
        if (n > 0) frac[tid] = (float)((double)w / (double)n);
        acc[2 * tid] = 0ull;
        acc[2 * tid + 1] = 0ull;
        sf[tid] = frac[tid];
    }
    if (tid == 0) scount = 0u;
    __syncthreads();
    const float fs = *fstar;
    unsigned int cnt = 0;
    for (int k = tid; k < nc; k += blockDim.x) {
        const int z = (int)(off[k + 1] - off[k]);
        const int b = min(kFormBins - 1, (int)((int64_t)(z - zmin) * kFormBins / (zmax - zmin + 1)));
        const bool fp = sf[b] >= fs;
        chunk_fp32[k] = fp ? 1 : 0;
        cnt += fp ? 1u : 0u;
    }
    if (cnt) atomicAdd(&scount, cnt);
    __syncthreads();
    if (tid == 0 && scount) atomicAdd(fp32_count, scount);
}

cudaError_t launch_form_select(const ptsne_ctx* c, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(c->tflag, 0, (size_t)c->tflag_total, s);
    if (e != cudaSuccess) return e;
    form_select_kernel<<<1, 256, 0, s>>>(c->d_off, c->p.n_chunks, (int)c->zmin, (int)c->zmax, c->form_acc,
                                         c->form_frac, c->form_fstar, c->chunk_fp32, &c->dstats->fp32_chunks);
    return launched(c, 1);
}

}  // namespace ptsne
