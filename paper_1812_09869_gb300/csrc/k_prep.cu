// Partition gather / pooling scatter (ptSNE section, "epochs": the master
// defines the chunks and pools the partial solutions back).  The partition is
// a permutation; chunk c is the contiguous run perm[off[c] .. off[c+1]) of it,
// so gathering rows by perm lays every chunk out contiguously.
#include <float.h>

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

// ---- locality order within chunks -------------------------------------------
// The order of a chunk's rows changes none of the method's results (P, the
// gradient and the cost are equivariant under it; only FP32 summation order
// moves).  Rows of nearby points placed next to each other concentrate the
// joint P on few 32 x 32 tiles (leaving the others exactly zero: the FP32
// exponentials of far pairs underflow) and the window pairs of the
// mixed-precision distances on few 64 x 64 tiles, which are then the only
// ones recomputed in FP32.  The chunk's first kLandmarks rows (a random sample, the
// partition being random) serve as landmarks: each row's key is its nearest
// landmark (squared distance, ties to the smaller index); landmarks closer
// to each other than twice the median nearest-landmark distance are joined
// into groups (single linkage), so that the rows of one cluster, spread over
// several landmarks, stay together; the rows are then stably sorted by
// (group, landmark).
constexpr int kLandmarks = 64;
constexpr int kLandK = 32;          // dimensions staged per pass

// Block (row tile of 128, chunk): the chunk's landmarks are staged kLandK
// dimensions at a time in shared memory; the two threads of a row (adjacent
// lanes) keep its distances to landmarks 0..31 and 32..63 in registers and
// combine their nearest at the end (ties to the smaller index).
__global__ void __launch_bounds__(256)
landmark_key_kernel(const float* __restrict__ Xg, Layout L, uint8_t* __restrict__ key) {
    constexpr int kHalf = kLandmarks / 2;
    constexpr int kStride = kLandK + 4;   // 16-byte rows; the two halves' rows start 4 banks apart
    __shared__ __align__(16) float sl[kLandmarks][kStride];
    const int c = blockIdx.y;
    const int64_t off = L.off[c];
    const int z = (int)(L.off[c + 1] - off);
    const int half = threadIdx.x & 1;
    const int i = blockIdx.x * 128 + (threadIdx.x >> 1);
    if (blockIdx.x * 128 >= z) return;   // block-uniform
    const int nl = z < kLandmarks ? z : kLandmarks;
    const bool valid = i < z;
    const float* xr = Xg + (off + (valid ? i : 0)) * L.dp;
    float acc[kHalf];
#pragma unroll
    for (int l = 0; l < kHalf; ++l) acc[l] = 0.f;
    for (int k0 = 0; k0 < L.dp; k0 += kLandK) {
        const int kc = min(kLandK, L.dp - k0);
        __syncthreads();
        // landmark h * 32 + l at row 2 l + h: the two halves read different banks
        for (int e = threadIdx.x; e < kLandmarks * kLandK; e += 256) {
            const int l = e / kLandK, k = e % kLandK;
            sl[2 * (l % kHalf) + l / kHalf][k] = (l < nl && k < kc) ? Xg[(off + l) * L.dp + k0 + k] : 0.f;
        }
        float xv[kLandK];
#pragma unroll
        for (int k = 0; k < kLandK; ++k) xv[k] = k < kc ? xr[k0 + k] : 0.f;
        __syncthreads();
#pragma unroll
        for (int l = 0; l < kHalf; ++l) {
            const float4* lm = reinterpret_cast<const float4*>(sl[2 * l + half]);
            float d = 0.f;
#pragma unroll
            for (int k4 = 0; k4 < kLandK / 4; ++k4) {
                const float4 v = lm[k4];
                float t = xv[4 * k4] - v.x;
                d = fmaf(t, t, d);
                t = xv[4 * k4 + 1] - v.y;
                d = fmaf(t, t, d);
                t = xv[4 * k4 + 2] - v.z;
                d = fmaf(t, t, d);
                t = xv[4 * k4 + 3] - v.w;
                d = fmaf(t, t, d);
            }
            acc[l] += d;
        }
    }
    float bd = FLT_MAX;
    int bl = 0;
#pragma unroll
    for (int l = 0; l < kHalf; ++l)
        if (half * kHalf + l < nl && acc[l] < bd) { bd = acc[l]; bl = half * kHalf + l; }
    const float od = __shfl_xor_sync(0xffffffffu, bd, 1);
    const int ol = __shfl_xor_sync(0xffffffffu, bl, 1);
    if (half == 0 && valid) key[off + i] = (uint8_t)(od < bd ? ol : bl);
}

// One block of kLandmarks threads per chunk.  Thread l holds landmark l's
// squared distances to the others (staged like the rows above), links it to
// the landmarks within four times the median nearest-landmark distance
// (squared), and the groups are the connected components; landmarks are
// ranked by (smallest landmark of their group, index).  Then a stable
// counting sort of the rows by the rank of their key: thread k writes the
// rows of rank k in their original order.  perm_out[off + p] is the entry of
// perm_in that lands at position p; src_row[off + p] = off + (its position
// in perm_in), for mapping exported matrices back to the caller's order.
__global__ void __launch_bounds__(kLandmarks)
chunk_order_kernel(const float* __restrict__ Xg, const uint8_t* __restrict__ key, const int32_t* __restrict__ perm_in,
                   Layout L, int32_t* __restrict__ perm_out, int32_t* __restrict__ src_row) {
    __shared__ uint8_t sk[kMaxChunk];
    __shared__ float sl[kLandmarks][kLandK + 1];
    __shared__ float snn[kLandmarks];
    __shared__ unsigned long long sadj[kLandmarks];
    __shared__ int sgroup[kLandmarks], srank[kLandmarks];
    __shared__ int start[kLandmarks + 1];
    const int c = blockIdx.x, t = threadIdx.x;
    const int64_t off = L.off[c];
    const int z = (int)(L.off[c + 1] - off);
    const int nl = z < kLandmarks ? z : kLandmarks;
    // landmark distances
    float dl[kLandmarks];
#pragma unroll
    for (int m = 0; m < kLandmarks; ++m) dl[m] = 0.f;
    for (int k0 = 0; k0 < L.dp; k0 += kLandK) {
        const int kc = min(kLandK, L.dp - k0);
        __syncthreads();
        for (int e = t; e < kLandmarks * kLandK; e += kLandmarks) {
            const int l = e / kLandK, k = e % kLandK;
            sl[l][k] = (l < nl && k < kc) ? Xg[(off + l) * L.dp + k0 + k] : 0.f;
        }
        __syncthreads();
#pragma unroll 4
        for (int m = 0; m < kLandmarks; ++m) {
            float d = 0.f;
            for (int k = 0; k < kLandK; ++k) {
                const float v = sl[t][k] - sl[m][k];
                d = fmaf(v, v, d);
            }
            dl[m] += d;
        }
    }
    float nn = FLT_MAX;
#pragma unroll
    for (int m = 0; m < kLandmarks; ++m)
        if (m != t && m < nl && dl[m] < nn) nn = dl[m];
    snn[t] = t < nl ? nn : FLT_MAX;
    __syncthreads();
    // median of the nearest-landmark distances (rank counting; ties by index)
    int below = 0;
    for (int m = 0; m < nl; ++m) below += (snn[m] < snn[t] || (snn[m] == snn[t] && m < t)) ? 1 : 0;
    __shared__ float smed;
    if (t < nl && below == (nl - 1) / 2) smed = snn[t];
    __syncthreads();
    const float thr = 4.0f * smed;
    unsigned long long adj = 0ull;
#pragma unroll
    for (int m = 0; m < kLandmarks; ++m)
        if (t < nl && m < nl && dl[m] <= thr) adj |= 1ull << m;
    sadj[t] = adj;
    __syncthreads();
    if (t == 0) {   // connected components of the linkage graph, labelled by their smallest landmark
        unsigned long long left = nl == 64 ? ~0ull : ((1ull << nl) - 1ull);
        while (left) {
            const int root = __ffsll((long long)left) - 1;
            unsigned long long comp = 1ull << root, frontier = comp;
            while (frontier) {
                unsigned long long next = 0ull;
                unsigned long long f = frontier;
                while (f) {
                    const int v = __ffsll((long long)f) - 1;
                    f &= f - 1;
                    next |= sadj[v];
                }
                next &= ~comp;
                comp |= next;
                frontier = next;
            }
            unsigned long long cm = comp;
            while (cm) {
                const int v = __ffsll((long long)cm) - 1;
                cm &= cm - 1;
                sgroup[v] = root;
            }
            left &= ~comp;
        }
    }
    __syncthreads();
    if (t < nl) {
        int r = 0;
        for (int m = 0; m < nl; ++m) r += (sgroup[m] < sgroup[t] || (sgroup[m] == sgroup[t] && m < t)) ? 1 : 0;
        srank[t] = r;
    }
    for (int i = t; i < z; i += kLandmarks) sk[i] = key[off + i];
    __syncthreads();
    for (int i = t; i < z; i += kLandmarks) sk[i] = (uint8_t)srank[sk[i]];
    __syncthreads();
    int cnt = 0;
    for (int i = 0; i < z; ++i) cnt += sk[i] == t;
    start[t + 1] = cnt;
    __syncthreads();
    if (t == 0) {
        start[0] = 0;
        for (int j = 1; j <= kLandmarks; ++j) start[j] += start[j - 1];
    }
    __syncthreads();
    int p = start[t];
    for (int i = 0; i < z; ++i) {
        if (sk[i] == t) {
            perm_out[off + p] = perm_in[off + i];
            src_row[off + p] = (int32_t)(off + i);
            ++p;
        }
    }
}

// The rows of every chunk of the partition perm in locality order: keys from
// the X rows gathered in perm's order, then the sorted partition in
// c->perm_loc (and c->src_row); X is gathered again in that order.
cudaError_t launch_locality_order(ptsne_ctx* c, const float* X, const int32_t* perm, cudaStream_t s) {
    cudaError_t e = launch_gather(c, X, perm, s);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)((c->zmax + 127) / 128), (unsigned)c->p.n_chunks);
    landmark_key_kernel<<<grid, 256, 0, s>>>(c->Xg, make_layout(c), c->lkey);
    chunk_order_kernel<<<(unsigned)c->p.n_chunks, kLandmarks, 0, s>>>(c->Xg, c->lkey, perm, make_layout(c),
                                                                        c->perm_loc, c->src_row);
    c->launches += 2;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_gather(c, X, c->perm_loc, s);
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
