// Pairwise squared Euclidean distances ||x_i - x_j||^2 within each chunk
// (ptSNE section, "Similarities in the input space"), FP32, by direct
// differences sum_k (x_ik - x_jk)^2: no ||x||^2 + ||y||^2 - 2 x.y cancellation,
// and bitwise symmetric because (a - b)^2 == (b - a)^2 with the same k order.
//
// Work unit: one 64 x 64 upper-triangular tile (I <= J) of one chunk; the
// block writes the tile and, off the diagonal, its transpose, so D is
// symmetric by construction and each pair is computed once.
#include "ptsne_internal.cuh"

namespace ptsne {

namespace {
constexpr int KC = 32;        // dims staged per pass
constexpr int SROW = kTile + 4;  // smem row stride (floats) of the k-major tiles
}

__global__ void __launch_bounds__(256)
dist_fp32_kernel(const float* __restrict__ Xg, float* __restrict__ D, Layout L,
                 const TileDesc* __restrict__ tiles, int64_t t0) {
    __shared__ __align__(16) float sI[KC][SROW];
    __shared__ __align__(16) float sJ[KC][SROW];
    const TileDesc td = tiles[t0 + blockIdx.x];
    const int c = td.chunk;
    const int64_t off = L.off[c];
    const int z = (int)(L.off[c + 1] - off);
    const int ld = L.ld[c];
    const int i0 = td.I * kTile, j0 = td.J * kTile;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int dp = L.dp;

    float acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[r][q] = 0.0f;

    for (int k0 = 0; k0 < dp; k0 += KC) {
        // stage 64 rows x KC dims of both row blocks, transposed to k-major
#pragma unroll
        for (int rep = 0; rep < 2; ++rep) {
            const int e = tid + rep * 256;      // 512 float4 slots: 64 rows x 8 quads
            const int row = e >> 3, quad = e & 7;
            const int k = k0 + quad * 4;
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
            if (k < dp) {
                if (i0 + row < z) a = *reinterpret_cast<const float4*>(Xg + (off + i0 + row) * dp + k);
                if (j0 + row < z) b = *reinterpret_cast<const float4*>(Xg + (off + j0 + row) * dp + k);
            }
            sI[quad * 4 + 0][row] = a.x; sI[quad * 4 + 1][row] = a.y;
            sI[quad * 4 + 2][row] = a.z; sI[quad * 4 + 3][row] = a.w;
            sJ[quad * 4 + 0][row] = b.x; sJ[quad * 4 + 1][row] = b.y;
            sJ[quad * 4 + 2][row] = b.z; sJ[quad * 4 + 3][row] = b.w;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < KC; ++k) {
            const float4 a = *reinterpret_cast<const float4*>(&sI[k][ty * 4]);
            const float4 b = *reinterpret_cast<const float4*>(&sJ[k][tx * 4]);
            const float av[4] = {a.x, a.y, a.z, a.w};
            const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float t = av[r] - bv[q];
                    acc[r][q] = fmaf(t, t, acc[r][q]);
                }
        }
        __syncthreads();
    }

    float* base = D + L.moff[c];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int i = i0 + ty * 4 + r;
        if (i < z)
            *reinterpret_cast<float4*>(base + (int64_t)i * ld + j0 + tx * 4) =
                make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
    }
    if (td.I != td.J) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = j0 + tx * 4 + q;
            if (j < z)
                *reinterpret_cast<float4*>(base + (int64_t)j * ld + i0 + ty * 4) =
                    make_float4(acc[0][q], acc[1][q], acc[2][q], acc[3][q]);
        }
    }
}

cudaError_t launch_dist_fp32(const ptsne_ctx* c, int64_t tile_begin, int64_t tile_end, cudaStream_t s) {
    const int64_t nt = tile_end - tile_begin;
    if (nt <= 0) return cudaSuccess;
    const Layout L = make_layout(c);
    int k = 0;
    for (int64_t b = 0; b < nt; b += 2147483647LL, ++k) {
        const int64_t cnt = (nt - b) < 2147483647LL ? (nt - b) : 2147483647LL;
        dist_fp32_kernel<<<(unsigned)cnt, 256, 0, s>>>(c->Xg, c->D, L, c->d_tiles, tile_begin + b);
    }
    return launched(c, k);
}

}  // namespace ptsne
