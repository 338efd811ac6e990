// Mixed-precision distances (PTSNE_PREC_BF16_WINDOW): a BF16 Gram matrix on
// the tensor cores with FP32 accumulation, then FP32 recomputation of every
// distance that can matter to a row's conditional distribution (Eq. 1).
//
//   d~_ij = |x~_i|^2 + |x~_j|^2 - 2 x~_i . x~_j     (x~ = x rounded to BF16)
//
// One thread block per 128 x 128 upper tile (I <= J) of one chunk: TMA loads
// the two BF16 row blocks (128-byte swizzle), one thread issues tcgen05.mma
// (M = N = 128, K = 16 per instruction) into a 128-column FP32 accumulator in
// tensor memory, and four warps read it back (tcgen05.ld) to write d~ to the
// tile and its transpose.
//
// Window: with u = 2^-8 the BF16 unit roundoff and e = u max_i |x_i| (x~ =
// x + delta, |delta_i| <= u |x_i|), every true distance satisfies
//   |d_ij - d~_ij| <= E(d~_ij),  E(d) = 4 e sqrt(d) + 4 e^2 + (accumulation slack),
// so j can carry weight exp(-beta (d_ij - m_i)) >= exp(-T) only if
//   d~_ij - E(d~_ij) <= m~_i + E(m~_i) + T / beta~_i.
// Those distances are recomputed in FP32 by direct differences and written to
// row i only (each row owns its entries; the joint-P assembly reads d_ij for
// p_{j|i} and d_ji for p_{i|j}); the perplexity search then runs again from
// beta~.
#include <float.h>

#include "ptsne_internal.cuh"
#include "tc_common.cuh"

namespace ptsne {

namespace tc {
bool make_bf16_tmap(CUtensorMap* out, const void* base, uint64_t rows, uint64_t cols) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return false;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {cols * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kTileK, (cuuint32_t)kTileRows};
    const cuuint32_t estr[2] = {1, 1};
    return encode(out, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
}  // namespace tc


// Xg (FP32, permuted) -> Xb (BF16, K padded to kp with zeros) and |x~|^2;
// also the largest |x~| (as float bits) for the window bound.
__global__ void gather_bf16_kernel(const float* __restrict__ Xg, int64_t n, int dp, int kp,
                                   __nv_bfloat16* __restrict__ Xb, float* __restrict__ xnorm, unsigned int* maxnorm) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    float mx = 0.f;
    for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < n; r += warps) {
        float s = 0.f;
        for (int k = lane; k < kp; k += 32) {
            const float v = k < dp ? Xg[r * dp + k] : 0.f;
            const __nv_bfloat16 b = __float2bfloat16_rn(v);
            const float f = __bfloat162float(b);
            Xb[r * kp + k] = b;
            s = fmaf(f, f, s);
        }
        s = warp_sum(s);
        if (lane == 0) xnorm[r] = s;
        mx = fmaxf(mx, s);
    }
    if (lane == 0) atomicMax(maxnorm, __float_as_uint(sqrtf(mx)));
}

__global__ void __launch_bounds__(128)
dist_bf16_kernel(const __grid_constant__ CUtensorMap tmX, float* __restrict__ D, Layout L,
                 const TileDesc* __restrict__ tiles, int64_t t0, const float* __restrict__ xnorm, int kblocks,
                 unsigned int* timeouts, const uint8_t* __restrict__ skip) {
    extern __shared__ unsigned char dsmem[];
    __shared__ uint64_t full_bar[2], done_bar[2], drain_bar;
    __shared__ uint32_t tmem_base;
    __shared__ float nj[tc::kTileRows];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // operand stages: 2 x (A 16 KB + B 16 KB), 1024-byte aligned for the 128-byte swizzle
    const uint32_t sbase = (tc::smem_addr(dsmem) + 1023u) & ~1023u;
    const TileDesc td = tiles[t0 + blockIdx.x];
    const int c = td.chunk;
    if (skip && skip[c]) return;   // a chunk computed in FP32 whole (before any barrier or TMEM use)
    const int64_t off = L.off[c];
    const int z = (int)(L.off[c + 1] - off);
    const int ld = L.ld[c];
    const int i0 = td.I * tc::kTileRows, j0 = td.J * tc::kTileRows;

    if (warp == 0) tc::tmem_alloc(tc::smem_addr(&tmem_base), tc::kTileRows);
    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            tc::mbar_init(tc::smem_addr(&full_bar[s]), 1);
            tc::mbar_init(tc::smem_addr(&done_bar[s]), 1);
        }
        tc::mbar_init(tc::smem_addr(&drain_bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    nj[tid] = (j0 + tid < z) ? xnorm[off + j0 + tid] : 0.f;
    // this thread's accumulator row: its norm is loaded before the main loop
    const int row = warp * 32 + lane, i = i0 + row;
    const float ni = i < z ? xnorm[off + i] : 0.f;
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (tid == 0) {
        const uint32_t idesc = tc::idesc_bf16_f32(tc::kTileRows, tc::kTileRows);
        bool ok = true;
        int issued = 0;   // K blocks whose loads were issued
        for (int kb = 0; kb < kblocks; ++kb) {
            const int s = kb & 1;
            const uint32_t fb = tc::smem_addr(&full_bar[s]), db = tc::smem_addr(&done_bar[s]);
            if (kb >= 2 && !(ok = tc::mbar_wait(db, (uint32_t)((kb - 2) >> 1) & 1u))) break;   // stage free again
            const uint32_t sa = sbase + (uint32_t)s * 2u * tc::kTileBytes, sb = sa + tc::kTileBytes;
            tc::mbar_expect_tx(fb, 2u * tc::kTileBytes);
            tc::tma_load_2d(sa, &tmX, kb * tc::kTileK, (int)(off + i0), fb);
            tc::tma_load_2d(sb, &tmX, kb * tc::kTileK, (int)(off + j0), fb);
            issued = kb + 1;
            if (!(ok = tc::mbar_wait(fb, (uint32_t)(kb >> 1) & 1u))) break;
            tc::tc_fence_after();
            const uint64_t da = tc::sw128_desc(sa), dbd = tc::sw128_desc(sb);
#pragma unroll
            for (int k16 = 0; k16 < tc::kTileK / 16; ++k16)   // advance 32 bytes (16 BF16) along K
                tc::mma_bf16(tmem, da + 2 * k16, dbd + 2 * k16, idesc, (kb > 0 || k16 > 0) ? 1u : 0u);
            tc::mma_commit(db);
        }
        const int last = kblocks - 1;
        if (ok) ok = tc::mbar_wait(tc::smem_addr(&done_bar[last & 1]), (uint32_t)(last >> 1) & 1u);
        if (!ok) {   // the host reports the count; nothing issued stays in flight
            atomicAdd(timeouts, 1u);
            tc::drain_issued(tc::smem_addr(&full_bar[0]), 2, issued, tc::smem_addr(&drain_bar));
        }
    }
    __syncthreads();
    tc::tc_fence_after();

    // epilogue: warp w owns accumulator lanes (tile rows) 32w .. 32w + 31
    float* base = D + L.moff[c];
    for (int cc = 0; cc < tc::kTileRows / 32; ++cc) {
        float v[32];
        tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cc * 32), v);
        const int jb = j0 + cc * 32;
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = ni + nj[cc * 32 + k] - 2.0f * v[k];
        if (i < z) {
            if (jb + 31 < z) {
#pragma unroll
                for (int k = 0; k < 32; k += 4)
                    *reinterpret_cast<float4*>(base + (int64_t)i * ld + jb + k) =
                        make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
            } else {
#pragma unroll
                for (int k = 0; k < 32; ++k)
                    if (jb + k < z) base[(int64_t)i * ld + jb + k] = v[k];
            }
        }
        if (td.I != td.J && i < z) {
#pragma unroll
            for (int k = 0; k < 32; ++k)
                if (jb + k < z) base[(int64_t)(jb + k) * ld + i] = v[k];   // lanes: consecutive i
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, tc::kTileRows);
}

// Exact FP32 squared distance by direct differences (row xi staged in shared
// memory), dimensions in order k = 0, 1, ...: KR > 0 is the padded dimension
// count known at compile time (every load of xj issued at once), KR = 0 a
// runtime dp.
template <int KR>
__device__ __forceinline__ float exact_d2(const float* __restrict__ xi, const float* __restrict__ xj, int dp) {
    float s = 0.f;
    if constexpr (KR > 0) {
        float4 q[KR / 4];
#pragma unroll
        for (int k = 0; k < KR / 4; ++k) q[k] = k * 4 < dp ? *reinterpret_cast<const float4*>(xj + 4 * k) : float4{};
#pragma unroll
        for (int k = 0; k < KR / 4; ++k) {
            if (k * 4 >= dp) break;
            const float4 a = *reinterpret_cast<const float4*>(xi + 4 * k);
            float t = a.x - q[k].x; s = fmaf(t, t, s);
            t = a.y - q[k].y; s = fmaf(t, t, s);
            t = a.z - q[k].z; s = fmaf(t, t, s);
            t = a.w - q[k].w; s = fmaf(t, t, s);
        }
    } else {
        for (int k = 0; k < dp; k += 4) {
            const float4 a = *reinterpret_cast<const float4*>(xi + k);
            const float4 q = *reinterpret_cast<const float4*>(xj + k);
            float t = a.x - q.x; s = fmaf(t, t, s);
            t = a.y - q.y; s = fmaf(t, t, s);
            t = a.z - q.z; s = fmaf(t, t, s);
            t = a.w - q.w; s = fmaf(t, t, s);
        }
    }
    return s;
}

// Window recompute of the sparse rows (the coarse search has flagged the
// 64 x 64 tiles holding the window pairs of the rows whose window covers
// >= 1/16 of the chunk; those tiles are recomputed whole by the FP32 distance
// kernel, which also computes the chunks run in FP32 whole): one warp per row.  The row of D is scanned 256 entries per step (two float4 per
// lane, the next step's loads issued before this step's are used);
// candidates d~_ij <= window_dmax(...) are compacted with ballots into a
// per-warp list and recomputed 32 at a time, one per lane, by direct
// differences.  Only the row's own entries (i, j) are rewritten; the order in
// which candidates are recomputed does not matter.
constexpr int kWinStep = 256;                 // D entries scanned per step
constexpr int kWinSlots = 32 + kWinStep;      // candidate list: < 32 left over + one step
template <int KR>
__global__ void __launch_bounds__(256)
window_kernel(float* __restrict__ D, const float* __restrict__ Xg, Layout L, int64_t r0, int64_t r1,
              const float* __restrict__ beta, const float* __restrict__ mrow, const unsigned int* maxnorm,
              unsigned long long* pairs, const uint8_t* __restrict__ row_dense,
              const uint8_t* __restrict__ chunk_fp32) {
    extern __shared__ float wsm[];   // per warp: one staged row of Xg (dp floats) + kWinSlots candidate slots
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int dp = L.dp;
    float* xi = wsm + (size_t)warp * (dp + kWinSlots);
    int* cand = reinterpret_cast<int*>(xi + dp);
    const float xmax = __uint_as_float(*maxnorm);
    const unsigned lt = (1u << lane) - 1u;
    unsigned long long count = 0;
    for (int64_t r = r0 + (int64_t)blockIdx.x * nw + warp; r < r1; r += (int64_t)gridDim.x * nw) {
        const int c = L.chunk_of_row[r];
        const int64_t off = L.off[c];
        const int z = (int)(L.off[c + 1] - off);
        if (chunk_fp32[c]) {   // computed in FP32 whole: on to this warp's first row past the chunk
            const int64_t G = (int64_t)gridDim.x * nw;
            r += (L.off[c + 1] - r - 1) / G * G;
            continue;
        }
        if (row_dense[r]) continue;   // a dense row: its window tiles are recomputed whole
        const int i = (int)(r - off);
        const int ld = L.ld[c];
        float* Drow = D + L.moff[c] + (int64_t)i * ld;
        for (int k = lane; k < dp; k += 32) xi[k] = Xg[r * dp + k];
        __syncwarp();
        const float dmax = window_dmax(beta[r], mrow[r], xmax, dp);
        // a float4 at entry j (a multiple of 4 below z) ends within the row: ld is a multiple of 64 >= z
        auto load = [&](int j) {
            return j < z ? *reinterpret_cast<const float4*>(Drow + j) : make_float4(FLT_MAX, FLT_MAX, FLT_MAX, FLT_MAX);
        };
        float4 v0 = load(4 * lane), v1 = load(128 + 4 * lane);
        int nbuf = 0;
        for (int j0 = 0; j0 < z; j0 += kWinStep) {
            const float4 c0 = v0, c1 = v1;
            v0 = load(j0 + kWinStep + 4 * lane);
            v1 = load(j0 + kWinStep + 128 + 4 * lane);
            const float vals[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int j = j0 + (e >> 2) * 128 + 4 * lane + (e & 3);
                const bool is_c = j < z && j != i && vals[e] <= dmax;
                const unsigned mask = __ballot_sync(0xffffffffu, is_c);
                if (is_c) cand[nbuf + __popc(mask & lt)] = j;
                nbuf += __popc(mask);
            }
            __syncwarp();
            // recompute full batches of 32, and the remainder after the last step
            while (nbuf >= 32 || (j0 + kWinStep >= z && nbuf > 0)) {
                const int take = nbuf < 32 ? nbuf : 32;
                const int rest = nbuf - take;
                int jj = 0;
                if (lane < take) jj = cand[rest + lane];   // take from the top of the list
                __syncwarp();
                if (lane < take) Drow[jj] = exact_d2<KR>(xi, Xg + (off + jj) * dp, dp);
                count += (lane < take) ? 1 : 0;
                nbuf = rest;
            }
            __syncwarp();
        }
        __syncwarp();
    }
    count = __reduce_add_sync(0xffffffffu, (unsigned)count);
    if (lane == 0 && count) atomicAdd(pairs, count);
}

cudaError_t launch_gather_bf16(const ptsne_ctx* c, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(c->maxnorm, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    int64_t g = (c->p.n * 32 + 255) / 256;
    if (g > 152 * 32) g = 152 * 32;
    gather_bf16_kernel<<<(unsigned)g, 256, 0, s>>>(c->Xg, c->p.n, c->dp, c->kp, c->Xb, c->xnorm, c->maxnorm);
    return launched(c, 1);
}

cudaError_t launch_dist_bf16(const ptsne_ctx* c, int64_t tile_begin, int64_t tile_end, cudaStream_t s,
                             const uint8_t* skip) {
    const int64_t nt = tile_end - tile_begin;
    if (nt <= 0) return cudaSuccess;
    CUtensorMap tm;
    if (!tc::make_bf16_tmap(&tm, c->Xb, (uint64_t)c->p.n, (uint64_t)c->kp)) return cudaErrorInvalidValue;
    // two operand stages; with a single K block (D <= 64) only stage 0 is used,
    // and 48 KB per block lets 4 blocks share an SM — as many as the TMEM holds
    // (4 x 128 accumulator columns) — where two stages allow 3
    const int kblocks = (int)(c->kp / tc::kTileK);
    const size_t smem = kblocks == 1 ? (size_t)48 * 1024 : 2 * 2 * tc::kTileBytes + 1024;
    cudaError_t e = cudaFuncSetAttribute(dist_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dist_bf16_kernel<<<(unsigned)nt, 128, smem, s>>>(tm, c->D, make_layout(c), c->d_tiles128, tile_begin, c->xnorm,
                                                     kblocks, &c->dstats->timeouts, skip);
    return launched(c, 1);
}

cudaError_t launch_window_recompute(const ptsne_ctx* c, int64_t row_begin, int64_t row_end, cudaStream_t s) {
    const int64_t rows = row_end - row_begin;
    if (rows <= 0) return cudaSuccess;
    // sparse rows: their candidates one by one
    const size_t smem = (size_t)8 * (c->dp + kWinSlots) * sizeof(float);
    void (*wk)(float*, const float*, Layout, int64_t, int64_t, const float*, const float*, const unsigned int*,
               unsigned long long*, const uint8_t*, const uint8_t*) = c->dp <= 16   ? window_kernel<16>
                                                                      : c->dp <= 32 ? window_kernel<32>
                                                                      : c->dp <= 64 ? window_kernel<64>
                                                                                    : window_kernel<0>;
    cudaError_t e = cudaFuncSetAttribute(wk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int64_t blocks = (rows + 7) / 8;
    if (blocks > 152 * 16) blocks = 152 * 16;
    wk<<<(unsigned)blocks, 256, smem, s>>>(c->D, c->Xg, make_layout(c), row_begin, row_end, c->beta, c->mrow,
                                           c->maxnorm, &c->dstats->window_pairs, c->row_dense, c->chunk_fp32);
    e = launched(c, 1);
    if (e != cudaSuccess) return e;
    // dense rows' window tiles, and the chunks computed in FP32 whole
    const int c0 = c->chunk_of(row_begin), c1 = c->chunk_of(row_end - 1);
    TileSel sel;
    sel.chunk_fp32 = c->chunk_fp32;
    sel.tflag = c->tflag;
    sel.tflag_off = c->d_tflag_off;
    return launch_dist_fp32_sel(c, c->tile_start[c0], c->tile_start[c1 + 1], sel, s);
}

}  // namespace ptsne
