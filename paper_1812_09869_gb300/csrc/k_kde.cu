// Perplexity-adaptive kernel density estimate of a 2-D map (paKDE, the
// paper's Clustering section): the sample smoothing estimator with Gaussian
// kernels K_j(c) = exp(-beta_j |c - y_j|^2) / pi, h_j^2 = 1 / beta_j,
//     f(c) = (S / n) sum_j (beta_j / pi) exp(-beta_j |c - y_j|^2),
// evaluated at the centres of a regular grid of cells of area S.  The
// precisions beta_j come from the perplexity search on the map's own
// distances (ptsne_affinities on a 2-D context).
//
// One warp per point splats its kernel onto the cells within exp(-30) of
// its peak (FP32 atomic adds; the remaining tail is below FP32 resolution
// relative to the peak).  A point whose kernel would cover more than
// PTSNE_KDE_MAX_CELLS cells (a precision far too small for the grid, e.g. an
// isolated point of a widely spread map) is dropped and counted, so that the
// work per point stays bounded.
#include <float.h>
#include <stdio.h>

#include "ptsne_internal.cuh"

namespace {

constexpr float kKdeCut = 30.0f;   // beta r^2 beyond which a kernel is dropped

__global__ void __launch_bounds__(256)
kde_splat_kernel(const float* __restrict__ Y, const float* __restrict__ beta, int64_t n, int gx, int gy, float x0,
                 float y0, float dx, float dy, float scale, float* __restrict__ f,
                 unsigned long long* __restrict__ dropped) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < n; j += warps) {
        const float b = beta[j], yx = Y[2 * j], yy = Y[2 * j + 1];
        if (!(b > 0.f) || !isfinite(b) || !isfinite(yx) || !isfinite(yy)) continue;   // unusable point: dropped
        const float r = sqrtf(kKdeCut / b);
        // covered cells, clamped in floating point before the integer conversion
        const float fx0 = fminf(fmaxf(floorf((yx - r - x0) / dx), -1.f), (float)gx);
        const float fx1 = fminf(fmaxf(ceilf((yx + r - x0) / dx), -1.f), (float)gx);
        const float fy0 = fminf(fmaxf(floorf((yy - r - y0) / dy), -1.f), (float)gy);
        const float fy1 = fminf(fmaxf(ceilf((yy + r - y0) / dy), -1.f), (float)gy);
        const int ix0 = max(0, (int)fx0), ix1 = min(gx - 1, (int)fx1);
        const int iy0 = max(0, (int)fy0), iy1 = min(gy - 1, (int)fy1);
        if (ix1 < ix0 || iy1 < iy0) continue;
        const int w = ix1 - ix0 + 1;
        const int64_t cells = (int64_t)w * (iy1 - iy0 + 1);
        if (cells > PTSNE_KDE_MAX_CELLS) {
            if (lane == 0 && dropped) atomicAdd(dropped, 1ull);
            continue;
        }
        const float amp = scale * b;
        for (int64_t t = lane; t < cells; t += 32) {
            const int ix = ix0 + (int)(t % w), iy = iy0 + (int)(t / w);
            const float ex = x0 + ((float)ix + 0.5f) * dx - yx;
            const float ey = y0 + ((float)iy + 0.5f) * dy - yy;
            const float q = b * fmaf(ex, ex, ey * ey);
            if (q <= kKdeCut) atomicAdd(&f[(int64_t)iy * gx + ix], amp * __expf(-q));
        }
    }
}

}  // namespace

extern "C" int ptsne_kde_grid(const float* Y_dev, const float* beta_dev, int64_t n, int32_t gx, int32_t gy,
                              const float* box_host, float* density_dev, int64_t* dropped_dev, void* stream) {
    char msg[256];
    if (!Y_dev || !beta_dev || !density_dev || !box_host) {
        ptsne::set_last_error("ptsne_kde_grid: Y, beta, box and density must be non-NULL");
        return PTSNE_EINVAL;
    }
    if (n < 1 || gx < 1 || gy < 1 || gx > 16384 || gy > 16384) {
        snprintf(msg, sizeof msg, "ptsne_kde_grid: need n >= 1 and a grid of 1..16384 cells per axis (%lld, %d x %d)",
                 (long long)n, (int)gx, (int)gy);
        ptsne::set_last_error(msg);
        return PTSNE_EINVAL;
    }
    const float x0 = box_host[0], x1 = box_host[1], y0 = box_host[2], y1 = box_host[3];
    if (!(x1 > x0) || !(y1 > y0) || !isfinite(x0) || !isfinite(x1) || !isfinite(y0) || !isfinite(y1)) {
        ptsne::set_last_error("ptsne_kde_grid: box must be finite with xmax > xmin and ymax > ymin");
        return PTSNE_EINVAL;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const float dx = (x1 - x0) / (float)gx, dy = (y1 - y0) / (float)gy;
    const float scale = (float)((double)dx * (double)dy / ((double)n * 3.14159265358979323846));
    cudaError_t e = cudaMemsetAsync(density_dev, 0, sizeof(float) * (size_t)gx * (size_t)gy, s);
    if (e == cudaSuccess && dropped_dev) e = cudaMemsetAsync(dropped_dev, 0, sizeof(int64_t), s);
    if (e == cudaSuccess) {
        int64_t blocks = (n + 7) / 8;
        if (blocks > 152 * 16) blocks = 152 * 16;
        kde_splat_kernel<<<(unsigned)blocks, 256, 0, s>>>(Y_dev, beta_dev, n, gx, gy, x0, y0, dx, dy, scale,
                                                          density_dev,
                                                          reinterpret_cast<unsigned long long*>(dropped_dev));
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        ptsne::set_last_error(cudaGetErrorString(e));
        return PTSNE_ECUDA;
    }
    return PTSNE_OK;
}
