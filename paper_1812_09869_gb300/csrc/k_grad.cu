// Gradient iterations on the dense z x ld P of the plain per-chunk schedule
// (Eq. 4, Eq. 6, Eq. 12/13) and its cost evaluation (Eq. 5, Eq. 9).  The
// batched schedule uses the packed symmetric P of k_iter.cu instead.
//
// One pass per iteration: for each row i the warp accumulates
//   A_i = sum_j p_ij w_ij (y_i - y_j),  R_i = sum_j w_ij^2 (y_i - y_j),
//   Z_i = sum_{j != i} w_ij,            w_ij = (1 + ||y_i - y_j||^2)^-1,
// so that, once Z = sum_i Z_i is known, Eq. 6 is
//   dC/dy_i = 4 sum_j (p_ij - w_ij / Z) w_ij (y_i - y_j) = 4 (A_i - R_i / Z).
// Z is reduced in FP64 (per-row FP32 partials combined in double).
#include <float.h>

#include "ptsne_internal.cuh"

namespace ptsne {

namespace {
constexpr int kRowWarps = 8;
}

template <int OD>
struct PairAcc {
    float a[OD], r[OD], z;
    __device__ __forceinline__ void clear() {
#pragma unroll
        for (int k = 0; k < OD; ++k) { a[k] = 0.f; r[k] = 0.f; }
        z = 0.f;
    }
    // one ordered pair (i, j) with P_ij = p and y_i - y_j = yi - yj
    __device__ __forceinline__ void add(const float (&yi)[OD], const float* yj, float p) {
        float dx[OD];
        float q = 1.0f;
#pragma unroll
        for (int k = 0; k < OD; ++k) {
            dx[k] = yi[k] - yj[k];
            q = fmaf(dx[k], dx[k], q);
        }
        const float w = hw_rcp(q);
        z += w;
        const float pw = p * w, w2 = w * w;
#pragma unroll
        for (int k = 0; k < OD; ++k) {
            a[k] = fmaf(pw, dx[k], a[k]);
            r[k] = fmaf(w2, dx[k], r[k]);
        }
    }
};

// ---------------------------------------------------------------- per-row form

template <int OD>
__global__ void __launch_bounds__(kRowWarps * 32)
grad_rows_kernel(const float* __restrict__ P, const float* __restrict__ Yc, Layout L, int64_t r0,
                 int64_t r1, float* __restrict__ acc, double* __restrict__ rowz) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t r = r0 + (int64_t)blockIdx.x * kRowWarps + warp; r < r1;
         r += (int64_t)gridDim.x * kRowWarps) {
        const int c = L.chunk_of_row[r];
        const int64_t off = L.off[c];
        const int z = (int)(L.off[c + 1] - off);
        const int i = (int)(r - off);
        const float* prow = P + L.moff[c] + (int64_t)i * L.ld[c];
        const float* Ych = Yc + off * OD;
        float yi[OD];
#pragma unroll
        for (int k = 0; k < OD; ++k) yi[k] = Ych[i * OD + k];
        PairAcc<OD> s;
        s.clear();
        for (int j0 = lane * 4; j0 < z; j0 += 128) {
            const float4 p4 = __ldg(reinterpret_cast<const float4*>(prow + j0));
            const float pv[4] = {p4.x, p4.y, p4.z, p4.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int j = j0 + e;
                if (j < z) {
                    float yj[OD];
#pragma unroll
                    for (int k = 0; k < OD; ++k) yj[k] = Ych[j * OD + k];
                    s.add(yi, yj, pv[e]);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < OD; ++k) {
            s.a[k] = warp_sum(s.a[k]);
            s.r[k] = warp_sum(s.r[k]);
        }
        const double zr = warp_sum((double)s.z) - 1.0;  // drop w_ii = 1
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < OD; ++k) {
                acc[r * 2 * OD + k] = s.a[k];
                acc[r * 2 * OD + OD + k] = s.r[k];
            }
            rowz[r] = zr;
        }
    }
}

// Z of each chunk (FP64, fixed reduction order) and the extent of its map.
__global__ void __launch_bounds__(256)
zreduce_kernel(const double* __restrict__ rowz, const float* __restrict__ Yc, Layout L, int c0,
               double* __restrict__ Zc, float* __restrict__ ystat) {
    __shared__ double sd[8];
    __shared__ float smin[8], smax[8];
    const int c = c0 + blockIdx.x;
    const int64_t off = L.off[c], z = L.off[c + 1] - off;
    double zsum = 0.0;
    float mn = FLT_MAX, mx = -FLT_MAX;
    for (int64_t t = threadIdx.x; t < z; t += blockDim.x) zsum += rowz[off + t];
    for (int64_t t = threadIdx.x; t < z * L.od; t += blockDim.x) {
        const float v = Yc[off * L.od + t];
        mn = fminf(mn, v);
        mx = fmaxf(mx, v);
    }
    zsum = warp_sum(zsum);
    mn = warp_min(mn);
    mx = warp_max(mx);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { sd[warp] = zsum; smin[warp] = mn; smax[warp] = mx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double Z = 0.0;
        float a = FLT_MAX, b = -FLT_MAX;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            Z += sd[w];
            a = fminf(a, smin[w]);
            b = fmaxf(b, smax[w]);
        }
        Zc[c] = Z;
        ystat[2 * c] = a;
        ystat[2 * c + 1] = b;
    }
}

template <int OD>
__global__ void __launch_bounds__(256)
update_kernel(float* __restrict__ Yc, float* __restrict__ vel, float* __restrict__ gains,
              const float* __restrict__ acc, const double* __restrict__ Zc, const float* __restrict__ ystat,
              Layout L, int64_t r0, int64_t r1, Optim opt, float* __restrict__ grad_perm) {
    for (int64_t r = r0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < r1;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int c = L.chunk_of_row[r];
        const int z = (int)(L.off[c + 1] - L.off[c]);
        const float invZ = (float)(1.0 / Zc[c]);
        const float eta = step_eta(opt, z, ystat[2 * c], ystat[2 * c + 1]);
        update_point<OD>(Yc + r * OD, vel + r * OD, gains + r * OD, acc + r * 2 * OD, acc + r * 2 * OD + OD,
                         invZ, eta, opt, grad_perm ? grad_perm + r * OD : nullptr);
    }
}

// ---------------------------------------------------------------- cost (Eq. 5, Eq. 9)
// Per row: sum p ln p, sum p ln w, sum p, sum_{j != i} w.  Then per chunk
//   KL = sum p ln p - sum p ln w + (sum p) ln Z,
//   normalised cost = (-sum p ln w + (sum p) ln Z) / (ln z + ln(z - 1)),
// and the average over chunks.

template <int OD>
__global__ void __launch_bounds__(kRowWarps * 32)
cost_rows_kernel(const float* __restrict__ P, const float* __restrict__ Yc, Layout L,
                 double* __restrict__ out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float kLn2 = 0.69314718055994531f;
    for (int64_t r = (int64_t)blockIdx.x * kRowWarps + warp; r < L.n; r += (int64_t)gridDim.x * kRowWarps) {
        const int c = L.chunk_of_row[r];
        const int64_t off = L.off[c];
        const int z = (int)(L.off[c + 1] - off);
        const int i = (int)(r - off);
        const float* prow = P + L.moff[c] + (int64_t)i * L.ld[c];
        const float* Ych = Yc + off * OD;
        float yi[OD];
#pragma unroll
        for (int k = 0; k < OD; ++k) yi[k] = Ych[i * OD + k];
        float plp = 0.f, plw = 0.f, ps = 0.f, zs = 0.f;
        for (int j = lane; j < z; j += 32) {
            if (j == i) continue;
            float q = 1.0f;
#pragma unroll
            for (int k = 0; k < OD; ++k) {
                const float d = yi[k] - Ych[j * OD + k];
                q = fmaf(d, d, q);
            }
            const float w = 1.0f / q;
            zs += w;
            const float p = prow[j];
            if (p >= FLT_MIN) {
                plp += p * (hw_lg2(p) * kLn2);
                plw += p * (-hw_lg2(q) * kLn2);
                ps += p;
            }
        }
        const double a = warp_sum((double)plp), b = warp_sum((double)plw), s = warp_sum((double)ps),
                     zz = warp_sum((double)zs);
        if (lane == 0) {
            out[r * 4 + 0] = a;
            out[r * 4 + 1] = b;
            out[r * 4 + 2] = s;
            out[r * 4 + 3] = zz;
        }
    }
}

__global__ void __launch_bounds__(256)
cost_chunk_kernel(const double* __restrict__ rows, Layout L, double* __restrict__ chunk_out) {
    __shared__ double sd[8][4];
    const int c = blockIdx.x;
    const int64_t off = L.off[c], z = L.off[c + 1] - off;
    double v[4] = {0, 0, 0, 0};
    for (int64_t t = threadIdx.x; t < z; t += blockDim.x)
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] += rows[(off + t) * 4 + k];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[k] = warp_sum(v[k]);
        if (lane == 0) sd[warp][k] = v[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0, s = 0, Z = 0;
        for (int w = 0; w < 8; ++w) { a += sd[w][0]; b += sd[w][1]; s += sd[w][2]; Z += sd[w][3]; }
        const double lnZ = log(Z);
        chunk_out[2 * c] = a - b + s * lnZ;
        chunk_out[2 * c + 1] = (-b + s * lnZ) / (log((double)z) + log((double)(z - 1)));
    }
}

__global__ void cost_final_kernel(const double* __restrict__ chunk, int n_chunks, double* __restrict__ out2) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double a = 0, b = 0;
        for (int c = 0; c < n_chunks; ++c) { a += chunk[2 * c]; b += chunk[2 * c + 1]; }
        out2[0] = a / n_chunks;
        out2[1] = b / n_chunks;
    }
}

// ---------------------------------------------------------------- embedding size
// The paper monitors, next to the cost, the size of the embedding: the length
// of the diagonal of the map's bounding box, sqrt(sum_k (max_i y_ik - min_i
// y_ik)^2), taken over every row of the pooled map.  Each block reduces a
// grid-stride share of the rows to per-coordinate extremes; the last block to
// finish (counted in `done`) combines the blocks' extremes and writes the
// size in FP64, then re-arms the counter for the next launch.  Minimum and
// maximum are exact in any order, so the result does not depend on the
// schedule.  NaN coordinates are ignored (fminf / fmaxf).
constexpr int kSizeThreads = 256;

template <int OD>
__global__ void __launch_bounds__(kSizeThreads)
embedding_size_kernel(const float* __restrict__ Y, int64_t rows, float* __restrict__ part, unsigned int* done,
                      double* __restrict__ out) {
    __shared__ float s_ext[kSizeThreads / 32][2 * OD];
    __shared__ bool s_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float lo[OD], hi[OD];
#pragma unroll
    for (int k = 0; k < OD; ++k) { lo[k] = FLT_MAX; hi[k] = -FLT_MAX; }
    for (int64_t i = (int64_t)blockIdx.x * kSizeThreads + threadIdx.x; i < rows;
         i += (int64_t)gridDim.x * kSizeThreads) {
        float v[OD];
        if constexpr (OD == 2) {
            const float2 t = reinterpret_cast<const float2*>(Y)[i];
            v[0] = t.x;
            v[1] = t.y;
        } else {
#pragma unroll
            for (int k = 0; k < OD; ++k) v[k] = Y[i * OD + k];
        }
#pragma unroll
        for (int k = 0; k < OD; ++k) { lo[k] = fminf(lo[k], v[k]); hi[k] = fmaxf(hi[k], v[k]); }
    }
#pragma unroll
    for (int k = 0; k < OD; ++k) {
        lo[k] = warp_min(lo[k]);
        hi[k] = warp_max(hi[k]);
        if (lane == 0) { s_ext[warp][k] = lo[k]; s_ext[warp][OD + k] = hi[k]; }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < OD; ++k) {
            float a = FLT_MAX, b = -FLT_MAX;
            for (int w = 0; w < kSizeThreads / 32; ++w) { a = fminf(a, s_ext[w][k]); b = fmaxf(b, s_ext[w][OD + k]); }
            part[blockIdx.x * 2 * OD + k] = a;
            part[blockIdx.x * 2 * OD + OD + k] = b;
        }
        __threadfence();
        s_last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
#pragma unroll
    for (int k = 0; k < OD; ++k) { lo[k] = FLT_MAX; hi[k] = -FLT_MAX; }
    for (int b = threadIdx.x; b < (int)gridDim.x; b += kSizeThreads) {
#pragma unroll
        for (int k = 0; k < OD; ++k) {
            lo[k] = fminf(lo[k], __ldcg(part + b * 2 * OD + k));
            hi[k] = fmaxf(hi[k], __ldcg(part + b * 2 * OD + OD + k));
        }
    }
#pragma unroll
    for (int k = 0; k < OD; ++k) {
        lo[k] = warp_min(lo[k]);
        hi[k] = warp_max(hi[k]);
    }
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < OD; ++k) { s_ext[warp][k] = lo[k]; s_ext[warp][OD + k] = hi[k]; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < OD; ++k) {
            float a = FLT_MAX, b = -FLT_MAX;
            for (int w = 0; w < kSizeThreads / 32; ++w) { a = fminf(a, s_ext[w][k]); b = fmaxf(b, s_ext[w][OD + k]); }
            const double e = (double)b - (double)a;
            s += e * e;
        }
        *out = sqrt(s);
        *done = 0u;
    }
}

// ---------------------------------------------------------------- launchers

static Optim optim_of(const ptsne_ctx* c) {
    Optim o;
    o.lr = c->p.lr;
    o.momentum = c->p.momentum;
    o.lr_mode = c->p.lr_mode;
    o.use_gains = c->p.use_gains;
    return o;
}

static unsigned row_blocks(int64_t rows, int per_block) {
    int64_t b = (rows + per_block - 1) / per_block;
    if (b > 152 * 64) b = 152 * 64;
    return (unsigned)(b < 1 ? 1 : b);
}

cudaError_t launch_grad_rows(const ptsne_ctx* c, int64_t row_begin, int64_t row_end, cudaStream_t s) {
    const int64_t rows = row_end - row_begin;
    if (rows <= 0) return cudaSuccess;
    const Layout L = make_layout(c);
    if (c->p.out_dim == 2)
        grad_rows_kernel<2><<<row_blocks(rows, kRowWarps), kRowWarps * 32, 0, s>>>(c->P, c->Yc, L, row_begin,
                                                                                   row_end, c->acc, c->rowz);
    else
        grad_rows_kernel<3><<<row_blocks(rows, kRowWarps), kRowWarps * 32, 0, s>>>(c->P, c->Yc, L, row_begin,
                                                                                   row_end, c->acc, c->rowz);
    return launched(c, 1);
}

cudaError_t launch_zreduce(const ptsne_ctx* c, int chunk_begin, int chunk_end, cudaStream_t s) {
    if (chunk_end <= chunk_begin) return cudaSuccess;
    zreduce_kernel<<<chunk_end - chunk_begin, 256, 0, s>>>(c->rowz, c->Yc, make_layout(c), chunk_begin, c->Zc,
                                                           c->ystat);
    return launched(c, 1);
}

cudaError_t launch_update(const ptsne_ctx* c, int64_t row_begin, int64_t row_end, float* grad_perm,
                          cudaStream_t s) {
    const int64_t rows = row_end - row_begin;
    if (rows <= 0) return cudaSuccess;
    const Layout L = make_layout(c);
    const unsigned g = row_blocks(rows, 256);
    if (c->p.out_dim == 2)
        update_kernel<2><<<g, 256, 0, s>>>(c->Yc, c->vel, c->gains, c->acc, c->Zc, c->ystat, L, row_begin, row_end,
                                          optim_of(c), grad_perm);
    else
        update_kernel<3><<<g, 256, 0, s>>>(c->Yc, c->vel, c->gains, c->acc, c->Zc, c->ystat, L, row_begin, row_end,
                                          optim_of(c), grad_perm);
    return launched(c, 1);
}

cudaError_t launch_cost(const ptsne_ctx* c, double* out2, cudaStream_t s) {
    const Layout L = make_layout(c);
    const unsigned g = row_blocks(c->p.n, kRowWarps);
    if (c->p.out_dim == 2)
        cost_rows_kernel<2><<<g, kRowWarps * 32, 0, s>>>(c->P, c->Yc, L, c->cost_rows);
    else
        cost_rows_kernel<3><<<g, kRowWarps * 32, 0, s>>>(c->P, c->Yc, L, c->cost_rows);
    cost_chunk_kernel<<<c->p.n_chunks, 256, 0, s>>>(c->cost_rows, L, c->cost_chunk);
    cost_final_kernel<<<1, 32, 0, s>>>(c->cost_chunk, c->p.n_chunks, out2);
    return launched(c, 3);
}

cudaError_t launch_cost_final(const ptsne_ctx* c, double* out2, cudaStream_t s) {
    cost_final_kernel<<<1, 32, 0, s>>>(c->cost_chunk, c->p.n_chunks, out2);
    return launched(c, 1);
}

cudaError_t launch_embedding_size(const ptsne_ctx* c, const float* Y, double* out, cudaStream_t s) {
    const int64_t rows = c->p.n;
    int64_t b = (rows + kSizeThreads - 1) / kSizeThreads;
    if (b > kSizeBlocks) b = kSizeBlocks;
    if (b < 1) b = 1;
    if (c->p.out_dim == 2)
        embedding_size_kernel<2><<<(unsigned)b, kSizeThreads, 0, s>>>(Y, rows, c->size_part, c->size_done, out);
    else
        embedding_size_kernel<3><<<(unsigned)b, kSizeThreads, 0, s>>>(Y, rows, c->size_part, c->size_done, out);
    return launched(c, 1);
}

}  // namespace ptsne
