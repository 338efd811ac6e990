// Partition gather / pooling scatter (ptSNE section, "epochs": the master
// defines the chunks and pools the partial solutions back).  The partition is
// a permutation; chunk c is the contiguous run perm[off[c] .. off[c+1]) of it,
// so gathering rows by perm lays every chunk out contiguously.
#include "ptsne_internal.cuh"

namespace ptsne {

// X (n x d, original order) -> Xg (n x dp, permuted order, zero padded), one
// warp per row; counts non-finite inputs.
// Rows of X in partition order (with layers, entry v of the permutation is
// layer * npts + point, and the row is point = v mod npts).
__global__ void gather_x_kernel(const float* __restrict__ X, const int32_t* __restrict__ perm,
                                int64_t n, int64_t npts, int d, int dp, float* __restrict__ Xg,
                                unsigned long long* nonfinite, unsigned int* bad_index) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    unsigned int bad = 0;
    for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < n; r += warps) {
        const int64_t pr = perm[r];
        const bool ok = pr >= 0 && pr < n;
        if (!ok && lane == 0) atomicAdd(bad_index, 1u);
        const float* src = X + (ok ? pr % npts : 0) * d;
        float* dst = Xg + r * dp;
        for (int k = lane; k < dp; k += 32) {
            float v = (k < d && ok) ? __ldg(src + k) : 0.0f;
            if (!isfinite(v)) { bad++; v = 0.0f; }
            dst[k] = v;
        }
    }
    bad = __reduce_add_sync(0xffffffffu, bad);
    if (lane == 0 && bad) atomicAdd(nonfinite, (unsigned long long)bad);
}

// Copy `width` floats per row: dst[r] = src[perm[r]] (gather).
__global__ void gather_rows_kernel(const float* __restrict__ src, const int32_t* __restrict__ perm,
                                   int64_t n, int width, float* __restrict__ dst, unsigned int* bad_index) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * width;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = t / width;
        int k = (int)(t - r * width);
        const int64_t pr = perm[r];
        if (pr < 0 || pr >= n) {
            if (k == 0 && bad_index) atomicAdd(bad_index, 1u);
            dst[t] = 0.0f;
            continue;
        }
        dst[t] = src[pr * width + k];
    }
}

// dst[perm[r]] = src[r] (pool the chunk results back into original order).
__global__ void scatter_rows_kernel(const float* __restrict__ src, const int32_t* __restrict__ perm,
                                    int64_t n, int width, float* __restrict__ dst, unsigned int* bad_index) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * width;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = t / width;
        int k = (int)(t - r * width);
        const int64_t pr = perm[r];
        if (pr < 0 || pr >= n) {
            if (k == 0 && bad_index) atomicAdd(bad_index, 1u);
            continue;
        }
        dst[pr * width + k] = src[t];
    }
}

__global__ void reset_optim_kernel(float* vel, float* gains, int64_t m) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m;
         t += (int64_t)gridDim.x * blockDim.x) {
        vel[t] = 0.0f;
        gains[t] = 1.0f;
    }
}

// Internal z x ld chunk matrices -> dense z x z, chunks concatenated.
__global__ void export_P_kernel(const float* __restrict__ P, Layout L, const int64_t* __restrict__ dense_off,
                                float* __restrict__ out) {
    const int c = blockIdx.y;
    const int64_t z = L.off[c + 1] - L.off[c];
    const int ld = L.ld[c];
    const float* src = P + L.moff[c];
    float* dst = out + dense_off[c];
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < z * z;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = t / z, j = t - i * z;
        dst[t] = src[i * ld + j];
    }
}

static int grid_for(int64_t work, int block) {
    int64_t g = (work + block - 1) / block;
    if (g < 1) g = 1;
    if (g > 152 * 32) g = 152 * 32;
    return (int)g;
}

cudaError_t launch_gather(const ptsne_ctx* c, const float* X, const int32_t* perm, cudaStream_t s) {
    const int64_t n = c->p.n;
    gather_x_kernel<<<grid_for(n * 32, 256), 256, 0, s>>>(X, perm, n, c->npts, c->p.d, c->dp, c->Xg,
                                                          &c->dstats->nonfinite, &c->dstats->bad_index);
    return launched(c, 1);
}

cudaError_t launch_gather_y(const ptsne_ctx* c, const float* Y, const int32_t* perm, float* Yc,
                            cudaStream_t s) {
    const int64_t n = c->p.n;
    gather_rows_kernel<<<grid_for(n * c->p.out_dim, 256), 256, 0, s>>>(Y, perm, n, c->p.out_dim, Yc,
                                                                       &c->dstats->bad_index);
    return launched(c, 1);
}

cudaError_t launch_scatter_rows(const ptsne_ctx* c, const float* src, const int32_t* perm, int width,
                                float* dst, cudaStream_t s) {
    const int64_t n = c->p.n;
    scatter_rows_kernel<<<grid_for(n * width, 256), 256, 0, s>>>(src, perm, n, width, dst, &c->dstats->bad_index);
    return launched(c, 1);
}

// Precomputed dissimilarities: chunk blocks of the caller's n x n matrix
// (original point order, leading dimension ldd) gathered through the
// partition into the z x ld chunk layout of D.  One warp per chunk row;
// non-finite entries are counted; permutation entries were checked by the
// caller's gather of the same partition.
__global__ void gather_dist_kernel(const float* __restrict__ Dfull, int64_t ldd, const int32_t* __restrict__ perm,
                                   int64_t npts, Layout L, float* __restrict__ D, unsigned long long* nonfinite,
                                   unsigned int* bad_index) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < L.n; r += warps) {
        const int c = L.chunk_of_row[r];
        const int64_t off = L.off[c];
        const int z = (int)(L.off[c + 1] - off);
        const int i = (int)(r - off);
        float* drow = D + L.moff[c] + (int64_t)i * L.ld[c];
        const int64_t pv = perm[r];
        const bool pi_ok = pv >= 0 && pv < L.n;
        const int64_t pi = pi_ok ? pv % npts : 0;
        if (!pi_ok && lane == 0) atomicAdd(bad_index, 1u);
        unsigned long long bad = 0;
        for (int j = lane; j < z; j += 32) {
            const int64_t pw = perm[off + j];
            float v = 0.f;
            if (pi_ok && pw >= 0 && pw < L.n) v = Dfull[pi * ldd + pw % npts];
            if (!isfinite(v)) { ++bad; v = 0.f; }
            drow[j] = v;
        }
        if (bad) atomicAdd(nonfinite, bad);
    }
}

cudaError_t launch_gather_dist(const ptsne_ctx* c, const float* Dfull, int64_t ldd, const int32_t* perm,
                               cudaStream_t s) {
    gather_dist_kernel<<<grid_for(c->p.n * 32, 256), 256, 0, s>>>(Dfull, ldd, perm, c->npts, make_layout(c), c->D,
                                                                  &c->dstats->nonfinite, &c->dstats->bad_index);
    return launched(c, 1);
}

// Layers: thread row r takes point perm[vsrc[r]] of layer vbase[r] / npts.
// Entries of perm outside [0, npts) give -1 (counted by the gathers).
__global__ void virtual_perm_kernel(const int32_t* __restrict__ perm, const int32_t* __restrict__ vsrc,
                                    const int32_t* __restrict__ vbase, int64_t rows, int64_t npts,
                                    int32_t* __restrict__ vperm) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p = perm[vsrc[r]];
        vperm[r] = (p >= 0 && p < npts) ? vbase[r] + p : -1;
    }
}

const int32_t* virtual_perm(ptsne_ctx* c, const int32_t* perm, cudaStream_t s, cudaError_t* err) {
    *err = cudaSuccess;
    if (c->layers == 1) return perm;
    virtual_perm_kernel<<<grid_for(c->p.n, 256), 256, 0, s>>>(perm, c->d_vsrc, c->d_vbase, c->p.n, c->npts,
                                                              c->vperm);
    *err = launched(c, 1);
    return c->vperm;
}

// Per-point precisions of the previous epoch (original order) -> warm starts
// of this epoch's search (partition order), and back.  Bad permutation entries
// are counted by the X gather already.
cudaError_t launch_beta_warm(const ptsne_ctx* c, const int32_t* perm, cudaStream_t s) {
    const int64_t n = c->p.n;
    gather_rows_kernel<<<grid_for(n, 256), 256, 0, s>>>(c->beta_pt, perm, n, 1, c->beta, nullptr);
    return launched(c, 1);
}
cudaError_t launch_beta_keep(const ptsne_ctx* c, const int32_t* perm, cudaStream_t s) {
    const int64_t n = c->p.n;
    scatter_rows_kernel<<<grid_for(n, 256), 256, 0, s>>>(c->beta, perm, n, 1, c->beta_pt, nullptr);
    return launched(c, 1);
}

cudaError_t launch_reset_optim(const ptsne_ctx* c, cudaStream_t s) {
    const int64_t m = c->p.n * c->p.out_dim;
    reset_optim_kernel<<<grid_for(m, 256), 256, 0, s>>>(c->vel, c->gains, m);
    return launched(c, 1);
}

cudaError_t launch_export_dense(const ptsne_ctx* c, const float* src, float* out, cudaStream_t s) {
    dim3 grid(64, c->p.n_chunks);
    export_P_kernel<<<grid, 256, 0, s>>>(src, make_layout(c), c->d_dense_off, out);
    return launched(c, 1);
}

cudaError_t launch_export_P(const ptsne_ctx* c, float* P_out, cudaStream_t s) {
    return launch_export_dense(c, c->P, P_out, s);
}

}  // namespace ptsne
