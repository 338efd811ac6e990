// Internal declarations of libptsne: context, device layout and launchers.
// Every kernel lives in one .cu file together with its host launcher; the
// entry points in ptsne_api.cu only validate, allocate and enqueue.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "ptsne.h"   // include/ptsne.h (the build passes -I include)

namespace ptsne {

// Square tile edge used by the pair kernels (distances, P assembly).  Chunk
// matrices are stored z rows x ld columns with ld = z rounded up to kTile, so
// every row starts 256-byte aligned and float4 loads never straddle rows.
constexpr int kTile = 64;
constexpr int kMaxChunk = 8192;
// Blocks of the embedding-size reduction (4 per SM of a GB300); the context
// keeps one set of per-coordinate extremes per block.
constexpr int kSizeBlocks = 608;

// One upper-triangular tile (I <= J) of one chunk's z x z pair matrix.
struct TileDesc {
    int32_t chunk;
    int16_t I, J;
};

// Which 64 x 64 distance tiles an FP32 pass computes.  chunk_fp32 NULL: every
// tile.  Otherwise every tile of a chunk with chunk_fp32[c] != 0, and of the
// other chunks the tiles (I, J) whose flag (I, J) or (J, I) is set in that
// chunk's T x T flags (T = ceil(z / 64)) at tflag + tflag_off[c].
struct TileSel {
    const uint8_t* chunk_fp32 = nullptr;
    const uint8_t* tflag = nullptr;
    const int64_t* tflag_off = nullptr;
};

// Mixed-precision form choice: chunk sizes are split into kFormBins equal
// bins over [zmin, zmax]; each bin keeps the window fraction of the last
// affinities (window pairs / (z - 1) per row, summed over its rows).
constexpr int kFormBins = 8;

// ---- packed symmetric P for the batched iteration kernel ---------------------
// Each chunk's joint P is stored once per unordered pair of 32-row blocks as
// 32 x 32 FP32 tiles (row block a <= column block b), row block by row block
// (a = 0: b = 0, 1, ..., then a = 1: b = 1, 2, ...), so that the tiles a warp
// takes from the stream often share their row block.  Inside a tile the 1024
// values are ordered for the warp that evaluates it (see packed_index, which
// depends on the map's dimension): lane L owns 32 floats, read as 8 float4.
constexpr int kPT = 32;                      // packed tile edge
constexpr int kPTileFloats = kPT * kPT;      // 1024 floats = 4 KB of P
// Stored tile: the 4 KB of P followed by a 16-byte trailer {a, b, 0, 0} (int
// bits) naming its row and column blocks, so a consumer learns the pair from
// the tile itself.
constexpr int kPTileStride = kPTileFloats + 4;

struct TileDesc2 {
    int32_t chunk;
    int16_t a, b;      // row block a <= column block b
    int32_t pos;       // tile index inside the chunk's packed block
};

// Position of element (r, c) of a stored tile, in the order of the warp that
// evaluates it: lane L owns 32 values, read as 8 float4; float4 f of lane L
// sits at float4 index 32 f + L, so that a warp-wide read of float4 f is 512
// contiguous bytes (no bank conflict, compile-time offsets).  Two lane
// layouts:
//
// 3-D maps (packed_index_ring16): lane L = 16 h + g owns rows 2g and 2g + 1
// and the ring h of columns 16h..16h+15, which it meets in the order
// (g + t) & 15, t = 0..15; float4 f = t / 2 holds {(2g, 2f), (2g, 2f+1),
// (2g+1, 2f), (2g+1, 2f+1)} in (row, step) terms.
//
// 2-D maps (packed_index_ring8): lane L = 8 q + g owns rows 4g .. 4g+3 and
// the ring q of columns 8q..8q+7, which it meets as natural column pairs:
// pair (g / 2 + s) & 3 at step s = 0..3; float4 2s + h holds rows 4g + 2h,
// 4g + 2h + 1 against the two columns of that step's pair.
__host__ __device__ inline int packed_index_ring16(int r, int c) {
    const int g = r >> 1, L = (c & 16) | g;
    const int t = ((c & 15) - g) & 15;
    return (((t >> 1) * kPT + L) << 2) | ((r & 1) << 1) | (t & 1);
}
__host__ __device__ inline int packed_index_ring8(int r, int c) {
    const int g = r >> 2, q = c >> 3, L = 8 * q + g;
    const int s = (((c & 7) >> 1) - (g >> 1)) & 3;
    const int f = 2 * s + ((r >> 1) & 1);
    return ((f * kPT + L) << 2) | ((r & 1) << 1) | (c & 1);
}
__host__ __device__ inline int packed_index(int r, int c, int od) {
    return od == 2 ? packed_index_ring8(r, c) : packed_index_ring16(r, c);
}

// Device view of the chunk layout, passed by value to kernels.
struct Layout {
    int64_t n;                     // points
    int32_t n_chunks;
    int32_t d, dp;                 // input dims and row stride of the gathered X (multiple of 4)
    int32_t od;                    // embedding dims
    const int64_t* off;            // n_chunks+1 row offsets (permuted order)
    const int64_t* moff;           // n_chunks offsets (floats) of each chunk's z x ld matrix
    const int32_t* ld;             // n_chunks leading dimensions
    const int32_t* chunk_of_row;   // n: chunk of each permuted row
    const int32_t* order;          // n_chunks: chunks by decreasing size (work-queue order)
};

// Records the message that ptsne_last_error(NULL) returns on the calling thread.
void set_last_error(const char* msg);

struct DeviceStats {               // device-side counters, reset per affinities call
    unsigned long long fp64_rows;
    unsigned long long failed_rows;
    unsigned long long window_pairs;
    unsigned long long nonfinite;
    unsigned long long bisect_evals;  // entropy evaluations, all rows
    unsigned int max_herr_bits;    // float bits of max |H - ln perp| (non-negative floats order as ints)
    unsigned int bad_index;        // permutation entries outside [0, n) (skipped)
    unsigned int timeouts;         // bounded device waits that ran out
    unsigned int fp32_chunks;      // mixed precision: chunks whose distances were computed in FP32 whole
    unsigned long long ptiles_nonzero;  // stored P tiles with a nonzero entry (batched schedule)
};

struct Optim {                     // optimiser settings
    float lr, momentum;
    int lr_mode, use_gains;
};

// Launch shape of the batched iteration kernel (chosen by the autotuner).
struct IterTune {
    int cluster = 2;               // blocks sharing one chunk (1, 2 or 4)
    int group = 1;                 // warps per tile (1: each warp evaluates whole tiles)
    int consumer_warps = 20;       // warps per block (1 .. 21)
};

}  // namespace ptsne

struct ptsne_ctx {
    ptsne_params p{};                  // p.n is the number of ROWS: layers x points
    int64_t npts = 0;                  // points (the caller's n)
    int layers = 1;
    int n_elem = 0;                    // elementary chunks of the caller's offsets
    // layers > 1: thread row r holds point perm[vsrc[r]] of layer vlayer[r]
    int32_t* d_vsrc = nullptr;         // rows
    int32_t* d_vbase = nullptr;        // rows: layer * npts
    int32_t* vperm = nullptr;          // rows: the virtual permutation of the current call
    std::vector<int64_t> off, moff;
    std::vector<int32_t> ld, order;
    int64_t zmin = 0, zmax = 0, mtotal = 0, ntiles = 0;
    std::vector<int64_t> tile_start;   // per chunk, first entry in the tile table (n_chunks+1)
    int dp = 0, kp = 0;                // padded X row (fp32) and bf16 K (multiple of 64)

    // device layout tables
    int64_t* d_off = nullptr;
    int64_t* d_moff = nullptr;
    int32_t* d_ld = nullptr;
    int32_t* d_chunk_of_row = nullptr;
    int32_t* d_order = nullptr;
    int64_t* d_dense_off = nullptr;    // n_chunks: sum of z^2 of the preceding chunks (P export)
    ptsne::TileDesc* d_tiles = nullptr;
    // packed symmetric P (batched schedule)
    int64_t ntiles2 = 0;               // stored 32 x 32 tiles over all chunks
    int64_t* d_ptile_off = nullptr;    // n_chunks: first packed tile of each chunk
    ptsne::TileDesc2* d_tiles2 = nullptr;
    float* P2 = nullptr;               // ntiles2 x kPTileStride floats
    uint8_t* ptile_nz = nullptr;       // ntiles2: 1 if the stored tile has a nonzero entry
    ptsne::IterTune tune;
    // BF16 Gram matrix (PTSNE_PREC_BF16_WINDOW): 128 x 128 upper tiles per chunk
    int64_t ntiles128 = 0;
    std::vector<int64_t> tile_start128;
    ptsne::TileDesc* d_tiles128 = nullptr;
    unsigned int* maxnorm = nullptr;   // largest |x~| (float bits), for the window bound
    // window rows recomputed whole: per chunk, a list of rows and its length,
    // and the chunks' 128-column blocks (TileDesc{chunk, 0, block})
    uint8_t* row_dense = nullptr;      // n: 1 = the row's window pairs are recomputed by whole tiles
    // the form of each chunk's distances and the window tiles of the dense rows
    int num_sms = 0;
    uint8_t* chunk_fp32 = nullptr;     // n_chunks: 1 = this affinities computes the chunk in FP32 whole
    uint8_t* tflag = nullptr;          // sum of T^2 over chunks: 64-tiles holding a dense row's window pairs
    int64_t* d_tflag_off = nullptr;    // n_chunks
    int64_t tflag_total = 0;
    unsigned long long* form_acc = nullptr;  // kFormBins x 2: window pairs and (z - 1), summed over rows
    float* form_frac = nullptr;        // kFormBins: window fraction of each size bin (last measured)
    float* form_fstar = nullptr;       // 1: chunks whose bin fraction is >= this run in FP32 whole
    float form_fstar_host = 2.0f;      // host copy (> 1: never)
    double form_ms[3] = {0, 0, 0};     // autotuner: affinities ms all mixed, all FP32, and the window recompute
    int chunk_of(int64_t r) const {     // chunk holding row r (off is sorted)
        return (int)(std::upper_bound(off.begin(), off.end(), r) - off.begin()) - 1;
    }

    // workspace
    float* Xg = nullptr;               // n x dp gathered X (permuted order)
    __nv_bfloat16* Xb = nullptr;       // n x kp gathered X in bf16 (BF16_WINDOW)
    float* xnorm = nullptr;            // n squared norms of the bf16 rows (BF16_WINDOW)
    float* D = nullptr;                // mtotal pair distances
    float* P = nullptr;                // mtotal joint probabilities
    float* beta = nullptr;             // n (permuted)
    float* beta_pt = nullptr;          // n, original order: last search's beta of each point (ptsne_run warm starts)
    float* mrow = nullptr;             // n row minima of the distances
    float* Srow = nullptr;             // n row normalisers at beta
    float* Yc = nullptr;               // n x od (permuted)
    float* vel = nullptr;              // n x od
    float* gains = nullptr;            // n x od
    float* acc = nullptr;              // n x 2od: attractive and repulsive sums
    float* gradp = nullptr;            // n x od gradient in permuted order (ptsne_step output)
    double* rowz = nullptr;            // n: per-row sum of w
    double* Zc = nullptr;              // n_chunks
    float* ystat = nullptr;            // n_chunks x 2 (min, max coordinate)
    double* cost_rows = nullptr;       // n x 3 per-row cost partials
    double* cost_chunk = nullptr;      // n_chunks x 2
    double* cost_hist = nullptr;       // 3 x kCostHist per-epoch {KL, cost, size} of ptsne_run
    float* size_part = nullptr;        // kSizeBlocks x 2 od: per-block extremes of the map
    unsigned int* size_done = nullptr; // blocks of the embedding-size reduction done (0 between launches)
    int* queue = nullptr;              // work-queue counters
    ptsne::DeviceStats* dstats = nullptr;

    // ptsne_run_host staging (lazily allocated)
    float* hX = nullptr;
    int32_t* hperms = nullptr;
    int64_t hperms_cap = 0;
    float* hY = nullptr;
    float* ycold = nullptr;            // ptsne_mlp_warm_start: the cold start's map (lazily allocated)
    // locality order of the rows within each chunk (batched schedule)
    bool locality = false;             // on: each affinities call orders the chunks' rows (ptsne_set_locality_order)
    bool deterministic = false;        // on: fixed-point accumulators in the batched kernel (ptsne_set_deterministic)
    bool loc_active = false;           // the kept affinities were computed in locality order
    int32_t* perm_loc = nullptr;       // n: the partition in locality order
    int32_t* src_row = nullptr;        // n: position in the caller's partition of each row of perm_loc
    uint8_t* lkey = nullptr;           // n: landmark key of each row

    bool have_P = false;
    size_t ws_bytes = 0;
    std::string err;

    // graph-captured epoch of ptsne_run: it reads the partition from perm_cur
    // and leaves the epoch's cost in cost_cur, so one graph serves every epoch
    int32_t* perm_cur = nullptr;       // n
    double* cost_cur = nullptr;        // 3: {avg KL, avg normalised cost, embedding size}
    cudaStream_t cap_stream = nullptr; // private stream the epoch is captured on
    cudaGraphExec_t graph = nullptr;
    const float* graph_X = nullptr;
    const float* graph_Y = nullptr;
    int graph_cost = -1;
    int graph_prof = -1;               // profiling marks captured as event nodes
    bool capturing = false;
    int graph_loc = -1;                // locality order captured in the graph
    ptsne::IterTune graph_tune{};
    long long graph_launches = 0;      // kernels per replay

    // tracing: kernels enqueued, and per-stage event timing of ptsne_run
    mutable long long launches = 0;
    bool profiling = false;
    cudaEvent_t ev[PTSNE_N_STAGES + 1] = {};
    double stage_ms[PTSNE_N_STAGES] = {};
    long long stage_calls[PTSNE_N_STAGES] = {};
};

namespace ptsne {

// --- launchers (host side, defined next to their kernels) -------------------
cudaError_t launch_gather(const ptsne_ctx* c, const float* X, const int32_t* perm, cudaStream_t s);
// rows of each chunk in locality order: partition -> c->perm_loc / c->src_row, X gathered in that order
cudaError_t launch_locality_order(ptsne_ctx* c, const float* X, const int32_t* perm, cudaStream_t s);
cudaError_t launch_gather_y(const ptsne_ctx* c, const float* Y, const int32_t* perm, float* Yc, cudaStream_t s);
// all gathers and scatters skip (and count in DeviceStats::bad_index) perm entries outside [0, n)
cudaError_t launch_scatter_rows(const ptsne_ctx* c, const float* src, const int32_t* perm, int width,
                                float* dst, cudaStream_t s);
cudaError_t launch_reset_optim(const ptsne_ctx* c, cudaStream_t s);
cudaError_t launch_export_P(const ptsne_ctx* c, float* P_out, cudaStream_t s);
// z x ld chunk matrices (src) -> dense z x z per chunk, chunks concatenated
cudaError_t launch_export_dense(const ptsne_ctx* c, const float* src, float* out, cudaStream_t s);

cudaError_t launch_dist_fp32(const ptsne_ctx* c, int64_t tile_begin, int64_t tile_end, cudaStream_t s);
cudaError_t launch_dist_fp32_sel(const ptsne_ctx* c, int64_t tile_begin, int64_t tile_end, const TileSel& sel,
                                 cudaStream_t s);
// mixed precision: each chunk's form for this affinities (c->chunk_fp32) from
// its size bin's last window fraction; clears the tile flags
cudaError_t launch_form_select(const ptsne_ctx* c, cudaStream_t s);
// skip (optional, n_chunks): tiles of chunks with skip[c] != 0 are left alone
cudaError_t launch_dist_bf16(const ptsne_ctx* c, int64_t tile_begin, int64_t tile_end, cudaStream_t s,
                             const uint8_t* skip = nullptr);
cudaError_t launch_window_recompute(const ptsne_ctx* c, int64_t row_begin, int64_t row_end, cudaStream_t s);
// beta_init (optional): start each row's search from this beta instead of 1 / mean(d - m)
// layers > 1: the caller's permutation (npts entries) -> the virtual one of
// the thread rows (layer * npts + point); returns the pointer to use.
const int32_t* virtual_perm(ptsne_ctx* c, const int32_t* perm, cudaStream_t s, cudaError_t* err);
cudaError_t launch_gather_dist(const ptsne_ctx* c, const float* Dfull, int64_t ldd, const int32_t* perm,
                               cudaStream_t s);
cudaError_t launch_beta_warm(const ptsne_ctx* c, const int32_t* perm, cudaStream_t s);
cudaError_t launch_beta_keep(const ptsne_ctx* c, const int32_t* perm, cudaStream_t s);
cudaError_t launch_bisect(const ptsne_ctx* c, int64_t row_begin, int64_t row_end, cudaStream_t s,
                          const float* beta_init = nullptr, int coarse = 0, int form = 0);
// (form 1: mixed precision bookkeeping — the coarse search skips the chunks
// run in FP32 whole and flags its dense rows' window tiles; both searches add
// their rows' window sizes to the size-bin fractions.  form 2: the same, and
// the fine search's beta_init holds a warm start for the FP32 chunks' rows)
cudaError_t launch_gather_bf16(const ptsne_ctx* c, cudaStream_t s);
cudaError_t launch_psym(const ptsne_ctx* c, int64_t tile_begin, int64_t tile_end, cudaStream_t s);

cudaError_t launch_grad_rows(const ptsne_ctx* c, int64_t row_begin, int64_t row_end, cudaStream_t s);
cudaError_t launch_zreduce(const ptsne_ctx* c, int chunk_begin, int chunk_end, cudaStream_t s);
cudaError_t launch_update(const ptsne_ctx* c, int64_t row_begin, int64_t row_end, float* grad_perm,
                          cudaStream_t s);
cudaError_t launch_cost(const ptsne_ctx* c, double* out2, cudaStream_t s);
cudaError_t launch_cost_final(const ptsne_ctx* c, double* out2, cudaStream_t s);
// embedding size of the map Y (all c->p.n rows, original order) into *out
cudaError_t launch_embedding_size(const ptsne_ctx* c, const float* Y, double* out, cudaStream_t s);

// batched schedule (packed symmetric P)
cudaError_t launch_psym_packed(const ptsne_ctx* c, cudaStream_t s);
// (with the locality order active, rows and columns go back to the caller's order)
cudaError_t launch_export_packed(const ptsne_ctx* c, float* P_out, cudaStream_t s);
// stored tiles flagged nonzero by the last joint P (into *out, device)
cudaError_t launch_count_nonzero(const ptsne_ctx* c, unsigned long long* out, cudaStream_t s);
cudaError_t launch_iterate(const ptsne_ctx* c, int iters, int cost_pass, float* gradp, double* Zc,
                           double* cost_chunk, cudaStream_t s);
// Warps of the batched iteration kernel that fit its shared memory for the
// largest chunk zmax (0: not even one), deterministic or not, on clusters of
// K blocks (the deterministic build splits its accumulators over the cluster).
int iterate_warps(int od, int64_t zmax, int want, bool det, int K);
int iterate_smem_bytes(int od, int64_t zmax, int warps, bool det, int K);

Layout make_layout(const ptsne_ctx* c);

// Count k kernels enqueued by a launcher and return the launch status.
inline cudaError_t launched(const ptsne_ctx* c, int k) {
    c->launches += k;
    return cudaGetLastError();
}

// --- device helpers ----------------------------------------------------------
#ifdef __CUDACC__
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
// Hardware approximations (PTX ex2.approx / rcp.approx / lg2.approx).
__device__ __forceinline__ float hw_ex2(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float hw_rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float hw_lg2(float x) {
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Position update, Eq. 12 in the descent direction, with gains or Eq. 13:
//   g = 4 (A - R / Z);  gains (+0.2 if sign(g) != sign(vel), else x0.8, >= 0.01)
//   vel = momentum * vel - eta * gains * g;  y += vel.
template <int OD>
__device__ __forceinline__ void update_point(float* y, float* vel, float* gains, const float* A, const float* R,
                                             float invZ, float eta, const Optim& opt, float* gout) {
#pragma unroll
    for (int k = 0; k < OD; ++k) {
        const float g = 4.0f * (A[k] - R[k] * invZ);
        if (gout) gout[k] = g;
        float v = vel[k];
        float gm = 1.0f;
        if (opt.use_gains) {
            float gn = ((g > 0.f) != (v > 0.f)) ? gains[k] + 0.2f : gains[k] * 0.8f;
            gn = fmaxf(gn, 0.01f);
            gains[k] = gn;
            gm = gn;
        }
        v = opt.momentum * v - eta * gm * g;
        vel[k] = v;
        y[k] += v;
    }
}

// Window of the mixed-precision distances: the largest d~ whose true distance
// can still carry weight exp(-beta (d - m)) >= exp(-T) of the row's largest.
// With u = 2^-8 (BF16 unit roundoff), e = u max|x| (1.01 margin) and the FP32
// accumulation slack s, |d - d~| <= E(d~) = 4 e sqrt(d~) + 4 e^2 + s; entry j
// is a candidate when d~ - E(d~) <= lim = T / (0.8 beta~) + m~ + E(m~), i.e.
// (solving in sqrt d~) d~ <= (2e + sqrt(8 e^2 + s + lim))^2, widened by 1e-6
// relative.  beta~ comes from a coarse search (|H - ln perp| <= 1e-3 nats);
// the 1/0.8 widening covers its error.  FLT_MAX (everything) when beta~ <= 0.
constexpr float kWindowT = 25.0f;      // e^-25 ~ 1.4e-11 of the row's largest weight
constexpr float kBf16U = 0.00390625f;  // 2^-8
__device__ __forceinline__ float window_dmax(float beta, float m, float xmax, int dp) {
    if (!(beta > 0.f)) return 3.0e38f;
    const float e = kBf16U * xmax * 1.01f;
    const float slack = 4.0f * (float)dp * 6.0e-8f * xmax * xmax;
    const float Em = 4.0f * e * sqrtf(fmaxf(m, 0.f)) + 4.0f * e * e + slack;
    const float lim = kWindowT / (0.8f * beta) + m + Em;
    const float u = 2.0f * e + sqrtf(8.0f * e * e + slack + lim);
    return u * u * (1.0f + 1e-6f);
}

// Learning rate: fixed, or Eq. 13 from the extent [ymin, ymax] of the chunk's map.
__device__ __forceinline__ float step_eta(const Optim& opt, int z, float ymin, float ymax) {
    return opt.lr_mode == PTSNE_LR_PAPER ? logf((float)(z - 1)) * (ymax - ymin) * 0.5f : opt.lr;
}
#endif

}  // namespace ptsne
