// C-ABI entry points of libptsne (declared and documented in include/ptsne.h).
// They validate arguments on the host, own the device workspace, and enqueue
// the kernels of k_*.cu on the caller's stream.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <numeric>

#include "ptsne_internal.cuh"

using namespace ptsne;

namespace ptsne {

Layout make_layout(const ptsne_ctx* c) {
    Layout L;
    L.n = c->p.n;
    L.n_chunks = c->p.n_chunks;
    L.d = c->p.d;
    L.dp = c->dp;
    L.od = c->p.out_dim;
    L.off = c->d_off;
    L.moff = c->d_moff;
    L.ld = c->d_ld;
    L.chunk_of_row = c->d_chunk_of_row;
    L.order = c->d_order;
    return L;
}
}  // namespace ptsne

namespace {

constexpr int kCostHist = 4096;
thread_local std::string g_create_err;  // message of the last failed ptsne_create on this thread

int fail(ptsne_ctx* c, int code, const char* fmt, const char* a = "", long long b = 0) {
    if (c) {
        char buf[512];
        snprintf(buf, sizeof buf, fmt, a, b);
        c->err = buf;
    }
    return code;
}

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) return fail(c, PTSNE_ECUDA, "%s: %lld", cudaGetErrorString(e_), \
                                           (long long)__LINE__);                          \
    } while (0)

// The permutation the kernels use: the caller's, or with layers the virtual
// one of the thread rows (enqueued on s).
#define VPERM(var, perm, s)                                                              \
    const int32_t* var;                                                                  \
    do {                                                                                 \
        cudaError_t ve_;                                                                 \
        var = virtual_perm(c, (perm), (s), &ve_);                                        \
        if (ve_ != cudaSuccess) return fail(c, PTSNE_ECUDA, "%s: %lld", cudaGetErrorString(ve_), \
                                            (long long)__LINE__);                        \
    } while (0)

template <class T>
int dalloc(ptsne_ctx* c, T** p, size_t count) {
    const size_t bytes = sizeof(T) * (count ? count : 1);
    cudaError_t e = cudaMalloc((void**)p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(c, PTSNE_ENOMEM, "device allocation of %s bytes failed (%lld)", "", (long long)bytes);
    }
    c->ws_bytes += bytes;
    return PTSNE_OK;
}

void free_all(ptsne_ctx* c) {
    void* ptrs[] = {c->d_off,  c->d_moff,  c->d_ld,   c->d_chunk_of_row, c->d_order, c->d_dense_off,
                    c->d_tiles, c->Xg,     c->Xb,     c->xnorm,          c->D,       c->P,
                    c->beta,   c->mrow,    c->Srow,   c->Yc,             c->vel,     c->gains,
                    c->acc,    c->gradp,   c->rowz,   c->Zc,             c->ystat,   c->cost_rows,
                    c->cost_chunk, c->cost_hist, c->queue, c->dstats, c->hX,   c->hperms,
                    c->hY,     c->P2,      c->d_ptile_off, c->d_tiles2, c->d_tiles128, c->maxnorm,
                    c->perm_cur, c->cost_cur, c->chunk_fp32, c->tflag, c->d_tflag_off, c->row_dense,
                    c->beta_pt, c->d_vsrc, c->d_vbase, c->vperm, c->size_part, c->size_done, c->ycold,
                    c->perm_loc, c->src_row, c->lkey, c->ptile_nz, c->form_acc, c->form_frac, c->form_fstar};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    c->graph = nullptr;
    c->cap_stream = nullptr;
    for (auto& e : c->ev)
        if (e) {
            cudaEventDestroy(e);
            e = nullptr;
        }
}

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

}  // namespace

void ptsne::set_last_error(const char* msg) { g_create_err = msg; }

extern "C" {

const char* ptsne_last_error(const ptsne_ctx* ctx) {
    if (!ctx) return g_create_err.c_str();
    return ctx->err.c_str();
}

size_t ptsne_workspace_bytes(const ptsne_ctx* ctx) { return ctx ? ctx->ws_bytes : 0; }

int ptsne_create(ptsne_ctx** out, const ptsne_params* prm) {
    if (!out || !prm) return PTSNE_EINVAL;
    *out = nullptr;
    ptsne_ctx* c = new (std::nothrow) ptsne_ctx();
    if (!c) return PTSNE_ENOMEM;
    g_create_err.clear();
    auto bad = [&](const char* msg, long long v) {
        fail(c, PTSNE_EINVAL, "invalid parameter: %s (%lld)", msg, v);
        g_create_err = c->err;
        delete c;
        return PTSNE_EINVAL;
    };
    const ptsne_params& p = *prm;
    if (p.n < 2) return bad("n must be >= 2", p.n);
    if (p.d < 1 || p.d > 4096) return bad("d must be in [1, 4096]", p.d);
    if (p.out_dim != 2 && p.out_dim != 3) return bad("out_dim must be 2 or 3", p.out_dim);
    if (p.n_chunks < 1) return bad("n_chunks must be >= 1", p.n_chunks);
    if (!p.chunk_offsets) return bad("chunk_offsets is NULL", 0);
    if (p.chunk_offsets[0] != 0 || p.chunk_offsets[p.n_chunks] != p.n)
        return bad("chunk offsets must start at 0 and end at n", p.chunk_offsets[p.n_chunks]);
    if (p.layers < 1 || p.layers > p.n_chunks) return bad("layers must be in [1, n_chunks]", p.layers);
    if ((double)p.layers * (double)p.n >= 2147483647.0) return bad("layers x n must be < 2^31", p.layers);
    for (int k = 0; k < p.n_chunks; ++k)
        if (p.chunk_offsets[k + 1] < p.chunk_offsets[k]) return bad("chunk offsets must not decrease", k);
    // threads: chunk t chained with the next layers - 1 chunks
    std::vector<int64_t> toff(p.n_chunks + 1, 0);
    int64_t zmin = INT64_MAX, zmax = 0;
    for (int t = 0; t < p.n_chunks; ++t) {
        int64_t z = 0;
        for (int k = 0; k < p.layers; ++k) {
            const int e = (t + k) % p.n_chunks;
            z += p.chunk_offsets[e + 1] - p.chunk_offsets[e];
        }
        if (z < 2 || z > kMaxChunk) return bad("every chunk (thread) size must be in [2, 8192]", z);
        toff[t + 1] = toff[t] + z;
        zmin = std::min(zmin, z);
        zmax = std::max(zmax, z);
    }
    if (!(p.perplexity > 1.0) || !(p.perplexity < (double)(zmin - 1)) || !isfinite(p.perplexity))
        return bad("perplexity must satisfy 1 < perplexity < min chunk size - 1", zmin);
    if (p.iters < 0) return bad("iters must be >= 0", p.iters);
    if (!(p.lr > 0.f) || !isfinite(p.lr)) return bad("lr must be > 0", 0);
    if (!(p.momentum >= 0.f && p.momentum < 1.f)) return bad("momentum must be in [0, 1)", 0);
    if (p.lr_mode != PTSNE_LR_FIXED && p.lr_mode != PTSNE_LR_PAPER) return bad("lr_mode", p.lr_mode);
    if (p.use_gains != 0 && p.use_gains != 1) return bad("use_gains must be 0 or 1", p.use_gains);
    if (p.precision != PTSNE_PREC_FP32 && p.precision != PTSNE_PREC_BF16_WINDOW)
        return bad("precision", p.precision);
    if (p.schedule != PTSNE_SCHED_BATCHED && p.schedule != PTSNE_SCHED_PER_CHUNK) return bad("schedule", p.schedule);
    if (p.use_graph != 0 && p.use_graph != 1) return bad("use_graph must be 0 or 1", p.use_graph);
    if (p.schedule == PTSNE_SCHED_BATCHED && iterate_warps(p.out_dim, zmax, 1, false, 1) < 1)
        return bad("largest chunk too large for the batched schedule at this out_dim", zmax);

    c->p = p;
    c->p.chunk_offsets = nullptr;
    c->npts = p.n;
    {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
        c->num_sms = sms;
    }
    c->layers = p.layers;
    c->n_elem = p.n_chunks;
    c->p.n = toff[p.n_chunks];   // rows: layers x points
    c->zmin = zmin;
    c->zmax = zmax;
    const int nc = p.n_chunks;
    c->off = toff;
    // layers: thread row -> (layer, position in the caller's permutation)
    std::vector<int32_t> vsrc, vbase;
    if (p.layers > 1) {
        vsrc.reserve((size_t)c->p.n);
        vbase.reserve((size_t)c->p.n);
        for (int t = 0; t < nc; ++t)
            for (int k = 0; k < p.layers; ++k) {
                const int e = (t + k) % nc;
                for (int64_t i = p.chunk_offsets[e]; i < p.chunk_offsets[e + 1]; ++i) {
                    vsrc.push_back((int32_t)i);
                    vbase.push_back((int32_t)(k * p.n));
                }
            }
    }
    c->ld.resize(nc);
    c->moff.resize(nc);
    c->tile_start.resize(nc + 1);
    std::vector<int64_t> dense(nc);
    int64_t m = 0, t = 0, dz = 0;
    std::vector<TileDesc> tiles;
    for (int k = 0; k < nc; ++k) {
        const int64_t z = c->off[k + 1] - c->off[k];
        const int64_t ld = (z + kTile - 1) / kTile * kTile;
        c->ld[k] = (int32_t)ld;
        c->moff[k] = m;
        m += z * ld;
        dense[k] = dz;
        dz += z * z;
        c->tile_start[k] = t;
        const int nb = (int)(ld / kTile);
        for (int I = 0; I < nb; ++I)
            for (int J = I; J < nb; ++J) tiles.push_back(TileDesc{k, (int16_t)I, (int16_t)J});
        t = (int64_t)tiles.size();
    }
    c->tile_start[nc] = t;
    c->mtotal = m;
    c->ntiles = t;
    // BF16 Gram matrix: 128 x 128 upper tiles of each chunk
    std::vector<TileDesc> tiles128;
    if (p.precision == PTSNE_PREC_BF16_WINDOW) {
        c->tile_start128.resize(nc + 1);
        for (int k = 0; k < nc; ++k) {
            c->tile_start128[k] = (int64_t)tiles128.size();
            const int nb = (int)((c->off[k + 1] - c->off[k] + 127) / 128);
            for (int I = 0; I < nb; ++I)
                for (int J = I; J < nb; ++J) tiles128.push_back(TileDesc{k, (int16_t)I, (int16_t)J});
        }
        c->tile_start128[nc] = (int64_t)tiles128.size();
        c->ntiles128 = (int64_t)tiles128.size();
    }
    // 64-tile flags of each chunk (window tiles of the dense window rows)
    std::vector<int64_t> tfoff(nc);
    if (p.precision == PTSNE_PREC_BF16_WINDOW) {
        int64_t acc = 0;
        for (int k = 0; k < nc; ++k) {
            const int64_t T = (c->off[k + 1] - c->off[k] + kTile - 1) / kTile;
            tfoff[k] = acc;
            acc += T * T;
        }
        c->tflag_total = acc;
    }
    // packed symmetric P: the 32 x 32 tiles (a <= b) of each chunk, row block
    // by row block
    std::vector<TileDesc2> tiles2;
    std::vector<int64_t> ptoff(nc);
    if (p.schedule == PTSNE_SCHED_BATCHED) {
        int64_t acc2 = 0;
        for (int k = 0; k < nc; ++k) {
            const int nb = (int)((c->off[k + 1] - c->off[k] + kPT - 1) / kPT);
            ptoff[k] = acc2;
            int32_t pos = 0;
            for (int a = 0; a < nb; ++a)
                for (int b = a; b < nb; ++b) tiles2.push_back(TileDesc2{k, (int16_t)a, (int16_t)b, pos++});
            acc2 += (int64_t)nb * (nb + 1) / 2;
        }
        c->ntiles2 = acc2;
    }
    c->order.resize(nc);
    std::iota(c->order.begin(), c->order.end(), 0);
    std::stable_sort(c->order.begin(), c->order.end(), [&](int a, int b) {
        return (c->off[a + 1] - c->off[a]) > (c->off[b + 1] - c->off[b]);
    });
    std::vector<int32_t> cor(c->p.n);
    for (int k = 0; k < nc; ++k)
        for (int64_t r = c->off[k]; r < c->off[k + 1]; ++r) cor[r] = k;
    c->dp = (p.d + 3) & ~3;
    c->kp = (p.d + 63) & ~63;

    const int64_t n = c->p.n, od = p.out_dim;
    int st = PTSNE_OK;
#define AL(ptr, count)                                               \
    do {                                                             \
        if ((st = dalloc(c, &(ptr), (size_t)(count))) != PTSNE_OK) { \
            g_create_err = c->err;                                   \
            free_all(c);                                             \
            delete c;                                                \
            return st;                                               \
        }                                                            \
    } while (0)
    AL(c->d_off, nc + 1);
    AL(c->d_moff, nc);
    AL(c->d_ld, nc);
    AL(c->d_chunk_of_row, n);
    AL(c->d_order, nc);
    AL(c->d_dense_off, nc);
    AL(c->d_tiles, t);
    AL(c->Xg, n * c->dp);
    if (p.precision == PTSNE_PREC_BF16_WINDOW) {
        AL(c->Xb, n * c->kp);
        AL(c->xnorm, n);
        AL(c->d_tiles128, c->ntiles128);
        AL(c->maxnorm, 1);
        AL(c->row_dense, n);
        AL(c->chunk_fp32, nc);
        AL(c->tflag, c->tflag_total);
        AL(c->d_tflag_off, nc);
        AL(c->form_acc, 2 * kFormBins);
        AL(c->form_frac, kFormBins);
        AL(c->form_fstar, 1);
    }
    AL(c->D, m);
    if (p.schedule == PTSNE_SCHED_BATCHED) {
        AL(c->perm_loc, n);
        AL(c->src_row, n);
        AL(c->lkey, n);
        AL(c->P2, c->ntiles2 * kPTileStride);
        AL(c->ptile_nz, c->ntiles2);
        AL(c->d_ptile_off, nc);
        AL(c->d_tiles2, c->ntiles2);
    } else {
        AL(c->P, m);
    }
    AL(c->beta, n);
    AL(c->beta_pt, n);
    AL(c->mrow, n);
    AL(c->Srow, n);
    AL(c->Yc, n * od);
    AL(c->vel, n * od);
    AL(c->gains, n * od);
    AL(c->acc, n * 2 * od);
    AL(c->gradp, n * od);
    AL(c->rowz, n);
    AL(c->Zc, nc);
    AL(c->ystat, 2 * nc);
    AL(c->cost_rows, 4 * n);
    AL(c->cost_chunk, 2 * nc);
    AL(c->cost_hist, 3 * kCostHist);
    AL(c->size_part, (int64_t)kSizeBlocks * 2 * od);
    AL(c->size_done, 1);
    AL(c->queue, 4);
    AL(c->dstats, 1);
    AL(c->perm_cur, c->npts);
    if (p.layers > 1) {
        AL(c->d_vsrc, n);
        AL(c->d_vbase, n);
        AL(c->vperm, n);
    }
    AL(c->cost_cur, 3);
#undef AL
    auto up = [&](void* dst, const void* src, size_t bytes) {
        return cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
    };
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = up(c->d_off, c->off.data(), sizeof(int64_t) * (nc + 1));
    if (e == cudaSuccess) e = up(c->d_moff, c->moff.data(), sizeof(int64_t) * nc);
    if (e == cudaSuccess) e = up(c->d_ld, c->ld.data(), sizeof(int32_t) * nc);
    if (e == cudaSuccess) e = up(c->d_chunk_of_row, cor.data(), sizeof(int32_t) * n);
    if (e == cudaSuccess) e = up(c->d_order, c->order.data(), sizeof(int32_t) * nc);
    if (e == cudaSuccess) e = up(c->d_dense_off, dense.data(), sizeof(int64_t) * nc);
    if (e == cudaSuccess) e = up(c->d_tiles, tiles.data(), sizeof(TileDesc) * tiles.size());
    if (e == cudaSuccess && c->ntiles128)
        e = up(c->d_tiles128, tiles128.data(), sizeof(TileDesc) * tiles128.size());
    if (e == cudaSuccess && c->tflag) {
        e = up(c->d_tflag_off, tfoff.data(), sizeof(int64_t) * nc);
        if (e == cudaSuccess) e = cudaMemset(c->form_acc, 0, sizeof(unsigned long long) * 2 * kFormBins);
        if (e == cudaSuccess) e = cudaMemset(c->form_frac, 0, sizeof(float) * kFormBins);
        if (e == cudaSuccess) e = up(c->form_fstar, &c->form_fstar_host, sizeof(float));
        if (e == cudaSuccess) e = cudaMemset(c->chunk_fp32, 0, (size_t)nc);
    }
    if (e == cudaSuccess && p.layers > 1) {
        e = up(c->d_vsrc, vsrc.data(), sizeof(int32_t) * vsrc.size());
        if (e == cudaSuccess) e = up(c->d_vbase, vbase.data(), sizeof(int32_t) * vbase.size());
    }
    if (e == cudaSuccess && c->ntiles2) {
        e = up(c->d_ptile_off, ptoff.data(), sizeof(int64_t) * nc);
        if (e == cudaSuccess) e = up(c->d_tiles2, tiles2.data(), sizeof(TileDesc2) * tiles2.size());
    }
    if (e == cudaSuccess) e = cudaMemset(c->dstats, 0, sizeof(DeviceStats));
    if (e == cudaSuccess) e = cudaMemset(c->size_done, 0, sizeof(unsigned int));
    // zero P once so that padded columns read as exact zeros before the first assembly
    if (e == cudaSuccess && c->P) e = cudaMemset(c->P, 0, sizeof(float) * (size_t)m);
    if (e != cudaSuccess) {
        g_create_err = cudaGetErrorString(e);
        free_all(c);
        delete c;
        return PTSNE_ECUDA;
    }
    *out = c;
    return PTSNE_OK;
}

void ptsne_destroy(ptsne_ctx* c) {
    if (!c) return;
    cudaDeviceSynchronize();
    free_all(c);
    delete c;
}

// Record the event that opens stage k (profiling only).
static void mark(ptsne_ctx* c, int k, cudaStream_t s) {
    if (!c->profiling) return;
    // inside an epoch capture the record becomes an event node of the graph
    if (c->capturing) cudaEventRecordWithFlags(c->ev[k], s, cudaEventRecordExternal);
    else cudaEventRecord(c->ev[k], s);
}

// Gather (and, for ptsne_run, the chunk maps), then the affinities of every
// chunk of the partition *perm_io.  With the locality order on, the rows of
// each chunk are first put in locality order and *perm_io becomes that
// partition (c->perm_loc), which the caller then uses for everything of this
// partition.  Opens stages GATHER..JOINT_P; the caller opens ITERATE.
static int affinities_impl(ptsne_ctx* c, const float* X, const int32_t** perm_io, cudaStream_t s, bool reset_stats,
                           const float* Y_run) {
    if (reset_stats) CK(cudaMemsetAsync(c->dstats, 0, sizeof(DeviceStats), s));
    // BF16_WINDOW with a threshold <= 0 puts every chunk in FP32 whole: the
    // plain FP32 path (the form choice still records its chunks)
    const bool all_fp32 = c->p.precision == PTSNE_PREC_BF16_WINDOW && c->form_fstar_host <= 0.f;
    const bool mixed = c->p.precision == PTSNE_PREC_BF16_WINDOW && !all_fp32;
    mark(c, PTSNE_STAGE_GATHER, s);
    c->loc_active = c->locality && c->p.schedule == PTSNE_SCHED_BATCHED;
    if (c->loc_active) {
        CK(launch_locality_order(c, X, *perm_io, s));
        *perm_io = c->perm_loc;
    } else {
        CK(launch_gather(c, X, *perm_io, s));
    }
    const int32_t* perm = *perm_io;
    if (mixed) CK(launch_gather_bf16(c, s));
    if (Y_run) CK(launch_gather_y(c, Y_run, perm, c->Yc, s));
    CK(launch_reset_optim(c, s));
    // ptsne_run: each row's search starts from its point's beta of the last
    // epoch (the root is unique; only the number of evaluations changes)
    const float* warm = nullptr;
    if (Y_run) {
        CK(launch_beta_warm(c, perm, s));
        warm = c->beta;
    }
    mark(c, PTSNE_STAGE_DISTANCES, s);
    // mixed precision: each chunk's form (BF16 Gram + window, or FP32 whole)
    if (mixed || all_fp32) CK(launch_form_select(c, s));
    if (c->p.schedule == PTSNE_SCHED_BATCHED) {
        if (mixed) CK(launch_dist_bf16(c, 0, c->ntiles128, s, c->chunk_fp32));
        else CK(launch_dist_fp32(c, 0, c->ntiles, s));
        mark(c, PTSNE_STAGE_PERPLEXITY, s);
        // mixed precision: a coarse search on d~ only places the windows
        CK(launch_bisect(c, 0, c->p.n, s, warm, mixed ? 1 : 0, mixed ? 1 : 0));
        if (mixed) {
            // FP32 distances inside each row's window (and of the FP32 chunks),
            // then the search again from beta~
            CK(launch_window_recompute(c, 0, c->p.n, s));
            CK(launch_bisect(c, 0, c->p.n, s, c->beta, 0, warm ? 2 : 1));
        }
        mark(c, PTSNE_STAGE_JOINT_P, s);
        CK(launch_psym_packed(c, s));
    } else {
        for (int k = 0; k < c->p.n_chunks; ++k) {
            if (mixed) CK(launch_dist_bf16(c, c->tile_start128[k], c->tile_start128[k + 1], s, c->chunk_fp32));
            else CK(launch_dist_fp32(c, c->tile_start[k], c->tile_start[k + 1], s));
            CK(launch_bisect(c, c->off[k], c->off[k + 1], s, warm, mixed ? 1 : 0, mixed ? 1 : 0));
            if (mixed) {
                CK(launch_window_recompute(c, c->off[k], c->off[k + 1], s));
                CK(launch_bisect(c, c->off[k], c->off[k + 1], s, c->beta, 0, warm ? 2 : 1));
            }
            CK(launch_psym(c, c->tile_start[k], c->tile_start[k + 1], s));
        }
        mark(c, PTSNE_STAGE_PERPLEXITY, s);
        mark(c, PTSNE_STAGE_JOINT_P, s);
    }
    if (Y_run) CK(launch_beta_keep(c, perm, s));
    c->have_P = true;
    return PTSNE_OK;
}

static int iterate_rows(ptsne_ctx* c, float* grad_perm, cudaStream_t s);

// One epoch of ptsne_run on the partition perm: affinities, every gradient
// iteration of every chunk, the pool back into Y and, if want_cost, the
// epoch's average costs and the pooled map's embedding size into cost_dst
// (3 doubles).
static int run_epoch(ptsne_ctx* c, const float* X, const int32_t* perm_in, float* Y, bool want_cost, double* cost_dst,
                     cudaStream_t s) {
    VPERM(perm0, perm_in, s);
    const int32_t* perm = perm0;
    int st = affinities_impl(c, X, &perm, s, false, Y);
    if (st != PTSNE_OK) return st;
    mark(c, PTSNE_STAGE_ITERATE, s);
    if (c->p.schedule == PTSNE_SCHED_BATCHED) {
        // every iteration of every chunk, then (if requested) one cost pass, in one launch
        CK(launch_iterate(c, c->p.iters, want_cost ? 1 : 0, nullptr, nullptr, c->cost_chunk, s));
    } else {
        for (int it = 0; it < c->p.iters; ++it) {
            st = iterate_rows(c, nullptr, s);
            if (st != PTSNE_OK) return st;
        }
    }
    mark(c, PTSNE_STAGE_POOL, s);
    CK(launch_scatter_rows(c, c->Yc, perm, c->p.out_dim, Y, s));
    mark(c, PTSNE_STAGE_COST, s);
    if (want_cost) {
        if (c->p.schedule == PTSNE_SCHED_BATCHED) CK(launch_cost_final(c, cost_dst, s));
        else CK(launch_cost(c, cost_dst, s));
        CK(launch_embedding_size(c, Y, cost_dst + 2, s));
    }
    return PTSNE_OK;
}

static bool same_tune(const IterTune& a, const IterTune& b) {
    return a.cluster == b.cluster && a.group == b.group && a.consumer_warps == b.consumer_warps;
}

// Capture one epoch (partition read from perm_cur, cost left in cost_cur) on
// the context's private stream and instantiate it; replays then run on the
// caller's stream, which may be the legacy default stream.
static int capture_epoch(ptsne_ctx* c, const float* X, float* Y, bool want_cost) {
    if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    const long long l0 = c->launches;
    CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeRelaxed));
    c->capturing = true;
    const int st = run_epoch(c, X, c->perm_cur, Y, want_cost, c->cost_cur, c->cap_stream);
    c->capturing = false;
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
    c->graph_launches = c->launches - l0;
    c->launches = l0;
    if (st != PTSNE_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return st != PTSNE_OK ? st : fail(c, PTSNE_ECUDA, "epoch capture failed (%s, line %lld)", cudaGetErrorString(e), __LINE__);
    }
    const cudaError_t ei = cudaGraphInstantiate(&c->graph, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
        c->graph = nullptr;
        return fail(c, PTSNE_ECUDA, "epoch graph instantiation failed (%s, line %lld)", cudaGetErrorString(ei), __LINE__);
    }
    c->graph_X = X;
    c->graph_Y = Y;
    c->graph_cost = want_cost ? 1 : 0;
    c->graph_tune = c->tune;
    c->graph_prof = c->profiling ? 1 : 0;
    c->graph_loc = c->locality ? 1 : 0;
    return PTSNE_OK;
}

int ptsne_affinities(ptsne_ctx* c, const float* X, const int32_t* perm_in, float* P_out, float* beta_out,
                     void* stream) {
    if (!c) return PTSNE_EINVAL;
    if (!X || !perm_in) return fail(c, PTSNE_EINVAL, "X and perm must be device pointers%s%lld");
    cudaStream_t s = as_stream(stream);
    CK(cudaMemsetAsync(c->dstats, 0, sizeof(DeviceStats), s));
    VPERM(perm0, perm_in, s);
    const int32_t* perm = perm0;
    int st = affinities_impl(c, X, &perm, s, false, nullptr);
    if (st != PTSNE_OK) return st;
    if (P_out) CK(c->P2 ? launch_export_packed(c, P_out, s) : launch_export_P(c, P_out, s));
    if (beta_out) CK(launch_scatter_rows(c, c->beta, perm, 1, beta_out, s));
    return PTSNE_OK;
}

int ptsne_affinities_from_distances(ptsne_ctx* c, const float* D_dev, int64_t ldd, const int32_t* perm_in,
                                    float* P_out, float* beta_out, void* stream) {
    if (!c) return PTSNE_EINVAL;
    if (!D_dev || !perm_in) return fail(c, PTSNE_EINVAL, "D and perm must be device pointers%s%lld");
    if (ldd < c->npts) return fail(c, PTSNE_EINVAL, "ldd must be >= n%s (%lld)", "", ldd);
    cudaStream_t s = as_stream(stream);
    CK(cudaMemsetAsync(c->dstats, 0, sizeof(DeviceStats), s));
    VPERM(perm, perm_in, s);
    c->loc_active = false;   // the dissimilarities are used in the caller's order
    CK(launch_gather_dist(c, D_dev, ldd, perm, s));
    CK(launch_reset_optim(c, s));
    // the given dissimilarities are final: one fine search, then the joint P
    if (c->p.schedule == PTSNE_SCHED_BATCHED) {
        CK(launch_bisect(c, 0, c->p.n, s));
        CK(launch_psym_packed(c, s));
    } else {
        for (int k = 0; k < c->p.n_chunks; ++k) {
            CK(launch_bisect(c, c->off[k], c->off[k + 1], s));
            CK(launch_psym(c, c->tile_start[k], c->tile_start[k + 1], s));
        }
    }
    c->have_P = true;
    if (P_out) CK(c->P2 ? launch_export_packed(c, P_out, s) : launch_export_P(c, P_out, s));
    if (beta_out) CK(launch_scatter_rows(c, c->beta, perm, 1, beta_out, s));
    return PTSNE_OK;
}

int ptsne_distances(ptsne_ctx* c, const float* X, const int32_t* perm_in, float* D_out, void* stream) {
    if (!c) return PTSNE_EINVAL;
    if (!X || !perm_in || !D_out) return fail(c, PTSNE_EINVAL, "X, perm and D_out must be device pointers%s%lld");
    cudaStream_t s = as_stream(stream);
    VPERM(perm, perm_in, s);
    CK(launch_gather(c, X, perm, s));
    if (c->p.precision == PTSNE_PREC_BF16_WINDOW) {
        CK(launch_gather_bf16(c, s));
        CK(launch_dist_bf16(c, 0, c->ntiles128, s));
    } else {
        CK(launch_dist_fp32(c, 0, c->ntiles, s));
    }
    CK(launch_export_dense(c, c->D, D_out, s));
    return PTSNE_OK;
}

static int iterate_rows(ptsne_ctx* c, float* grad_perm, cudaStream_t s) {
    if (c->p.schedule == PTSNE_SCHED_BATCHED) {
        CK(launch_grad_rows(c, 0, c->p.n, s));
        CK(launch_zreduce(c, 0, c->p.n_chunks, s));
        CK(launch_update(c, 0, c->p.n, grad_perm, s));
    } else {
        for (int k = 0; k < c->p.n_chunks; ++k) {
            CK(launch_grad_rows(c, c->off[k], c->off[k + 1], s));
            CK(launch_zreduce(c, k, k + 1, s));
            CK(launch_update(c, c->off[k], c->off[k + 1], grad_perm, s));
        }
    }
    return PTSNE_OK;
}

int ptsne_step(ptsne_ctx* c, const int32_t* perm_in, float* Y, float* grad_out, double* Z_out, void* stream) {
    if (!c) return PTSNE_EINVAL;
    if (!perm_in || !Y) return fail(c, PTSNE_EINVAL, "perm and Y must be device pointers%s%lld");
    if (!c->have_P) return fail(c, PTSNE_ESTATE, "ptsne_step before ptsne_affinities%s%lld");
    cudaStream_t s = as_stream(stream);
    VPERM(perm0, perm_in, s);
    // the partition of the kept affinities, in the row order they were computed in
    const int32_t* perm = c->loc_active ? c->perm_loc : perm0;
    CK(launch_gather_y(c, Y, perm, c->Yc, s));
    if (c->p.schedule == PTSNE_SCHED_BATCHED) {
        CK(launch_iterate(c, 1, 0, grad_out ? c->gradp : nullptr, c->Zc, nullptr, s));
    } else {
        int st = iterate_rows(c, grad_out ? c->gradp : nullptr, s);
        if (st != PTSNE_OK) return st;
    }
    CK(launch_scatter_rows(c, c->Yc, perm, c->p.out_dim, Y, s));
    if (grad_out) CK(launch_scatter_rows(c, c->gradp, perm, c->p.out_dim, grad_out, s));
    if (Z_out)
        CK(cudaMemcpyAsync(Z_out, c->Zc, sizeof(double) * c->p.n_chunks, cudaMemcpyDeviceToDevice, s));
    return PTSNE_OK;
}

int ptsne_cost(ptsne_ctx* c, const int32_t* perm_in, const float* Y, double* out_dev, void* stream) {
    if (!c) return PTSNE_EINVAL;
    if (!perm_in || !Y || !out_dev) return fail(c, PTSNE_EINVAL, "perm, Y and out must be device pointers%s%lld");
    if (!c->have_P) return fail(c, PTSNE_ESTATE, "ptsne_cost before ptsne_affinities%s%lld");
    cudaStream_t s = as_stream(stream);
    VPERM(perm0, perm_in, s);
    const int32_t* perm = c->loc_active ? c->perm_loc : perm0;
    CK(launch_gather_y(c, Y, perm, c->Yc, s));
    if (c->p.schedule == PTSNE_SCHED_BATCHED) {
        CK(launch_iterate(c, 0, 1, nullptr, nullptr, c->cost_chunk, s));
        CK(launch_cost_final(c, out_dev, s));
    } else {
        CK(launch_cost(c, out_dev, s));
    }
    return PTSNE_OK;
}

int ptsne_embedding_size(ptsne_ctx* c, const float* Y, double* out_dev, void* stream) {
    if (!c) return PTSNE_EINVAL;
    if (!Y || !out_dev) return fail(c, PTSNE_EINVAL, "Y and out must be device pointers%s%lld");
    CK(launch_embedding_size(c, Y, out_dev, as_stream(stream)));
    return PTSNE_OK;
}

int ptsne_run(ptsne_ctx* c, const float* X, const int32_t* perms, int32_t epochs, float* Y, double* cost_out,
              void* stream) {
    if (!c) return PTSNE_EINVAL;
    if (!X || !perms || !Y) return fail(c, PTSNE_EINVAL, "X, perms and Y must be device pointers%s%lld");
    if (epochs < 0) return fail(c, PTSNE_EINVAL, "epochs must be >= 0%s (%lld)", "", epochs);
    cudaStream_t s = as_stream(stream);
    const int64_t n = c->p.n, npts = c->npts;   // rows, points
    const bool want_cost = cost_out != nullptr;
    const bool use_graph = c->p.use_graph != 0;
    if (use_graph && (!c->graph || c->graph_X != X || c->graph_Y != Y || c->graph_cost != (int)want_cost ||
                      c->graph_prof != (c->profiling ? 1 : 0) || c->graph_loc != (c->locality ? 1 : 0) ||
                      !same_tune(c->graph_tune, c->tune))) {
        const int st = capture_epoch(c, X, Y, want_cost);
        if (st != PTSNE_OK) return st;
    }
    // counters accumulate over the whole run; the first epoch's search starts cold
    CK(cudaMemsetAsync(c->dstats, 0, sizeof(DeviceStats), s));
    CK(cudaMemsetAsync(c->beta_pt, 0, sizeof(float) * n, s));
    for (int e = 0; e < epochs; ++e) {
        const int32_t* perm = perms + (int64_t)e * npts;
        const int slot = e % kCostHist;
        if (use_graph) {
            CK(cudaMemcpyAsync(c->perm_cur, perm, sizeof(int32_t) * npts, cudaMemcpyDeviceToDevice, s));
            CK(cudaGraphLaunch(c->graph, s));
            c->launches += c->graph_launches;
            if (want_cost)
                CK(cudaMemcpyAsync(c->cost_hist + 3 * slot, c->cost_cur, 3 * sizeof(double), cudaMemcpyDeviceToDevice,
                                   s));
        } else {
            const int st = run_epoch(c, X, perm, Y, want_cost, c->cost_hist + 3 * slot, s);
            if (st != PTSNE_OK) return st;
        }
        if (want_cost && (slot == kCostHist - 1 || e == epochs - 1))
            CK(cudaMemcpyAsync(cost_out + 3 * (int64_t)(e - slot), c->cost_hist, sizeof(double) * 3 * (slot + 1),
                               cudaMemcpyDeviceToHost, s));
        if (c->profiling) {
            CK(cudaEventRecord(c->ev[PTSNE_N_STAGES], s));
            CK(cudaEventSynchronize(c->ev[PTSNE_N_STAGES]));
            for (int k = 0; k < PTSNE_N_STAGES; ++k) {
                if (k == PTSNE_STAGE_COST && !want_cost) continue;
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, c->ev[k], c->ev[k + 1]));
                c->stage_ms[k] += ms;
                c->stage_calls[k] += 1;
            }
        }
    }
    DeviceStats h;
    CK(cudaMemcpyAsync(&h, c->dstats, sizeof h, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (h.timeouts) return fail(c, PTSNE_ETIMEOUT, "%s%lld bounded device waits ran out", "", (long long)h.timeouts);
    if (h.bad_index) return fail(c, PTSNE_EINVAL, "%s%lld permutation entries outside [0, n)", "", (long long)h.bad_index);
    if (h.nonfinite) return fail(c, PTSNE_ENONFINITE, "%s%lld non-finite values in X", "", (long long)h.nonfinite);
    if (h.failed_rows) {
        fail(c, PTSNE_WBISECT, "%s%lld rows missed the perplexity tolerance", "", (long long)h.failed_rows);
        return PTSNE_WBISECT;
    }
    return PTSNE_OK;
}

int ptsne_run_host(ptsne_ctx* c, const float* X_host, const int32_t* perms_host, int32_t epochs, float* Y_host,
                   double* cost_out, void* stream) {
    if (!c) return PTSNE_EINVAL;
    if (!X_host || !perms_host || !Y_host) return fail(c, PTSNE_EINVAL, "host buffers must be non-NULL%s%lld");
    if (epochs < 0) return fail(c, PTSNE_EINVAL, "epochs must be >= 0%s (%lld)", "", epochs);
    cudaStream_t s = as_stream(stream);
    const int64_t n = c->p.n, npts = c->npts, d = c->p.d, od = c->p.out_dim;   // n: map rows
    int st;
    if (!c->hX && (st = dalloc(c, &c->hX, (size_t)(npts * d))) != PTSNE_OK) return st;
    if (!c->hY && (st = dalloc(c, &c->hY, (size_t)(n * od))) != PTSNE_OK) return st;
    if (c->hperms_cap < (int64_t)epochs * npts) {
        if (c->hperms) { cudaFree(c->hperms); c->ws_bytes -= sizeof(int32_t) * c->hperms_cap; c->hperms = nullptr; }
        if ((st = dalloc(c, &c->hperms, (size_t)epochs * npts)) != PTSNE_OK) return st;
        c->hperms_cap = (int64_t)epochs * npts;
    }
    CK(cudaMemcpyAsync(c->hX, X_host, sizeof(float) * npts * d, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->hperms, perms_host, sizeof(int32_t) * epochs * npts, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->hY, Y_host, sizeof(float) * n * od, cudaMemcpyHostToDevice, s));
    st = ptsne_run(c, c->hX, c->hperms, epochs, c->hY, cost_out, stream);
    if (st < 0) return st;
    CK(cudaMemcpyAsync(Y_host, c->hY, sizeof(float) * n * od, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return st;
}

int ptsne_get_stats(ptsne_ctx* c, ptsne_stats* out, void* stream) {
    if (!c || !out) return PTSNE_EINVAL;
    cudaStream_t s = as_stream(stream);
    if (c->ptile_nz && c->have_P) CK(launch_count_nonzero(c, &c->dstats->ptiles_nonzero, s));
    DeviceStats h;
    CK(cudaMemcpyAsync(&h, c->dstats, sizeof h, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    out->bisect_rows = c->p.n;
    out->bisect_fp64_rows = (int64_t)h.fp64_rows;
    out->bisect_failed_rows = (int64_t)h.failed_rows;
    out->window_pairs = (int64_t)h.window_pairs;
    out->nonfinite_inputs = (int64_t)h.nonfinite;
    out->bad_perm_entries = (int64_t)h.bad_index;
    out->wait_timeouts = (int64_t)h.timeouts;
    out->bisect_evals = (int64_t)h.bisect_evals;
    out->ptiles_total = c->ntiles2;
    out->ptiles_nonzero = (int64_t)h.ptiles_nonzero;
    out->fp32_chunks = (int64_t)h.fp32_chunks;
    out->form_threshold = c->form_fstar ? (double)c->form_fstar_host : 0.0;
    for (int k = 0; k < 8; ++k) out->window_fraction[k] = 0.0;
    if (c->form_frac) {   // the last measurement: sums not yet taken by a form choice, else the kept fraction
        static_assert(kFormBins == 8, "ptsne_stats.window_fraction has 8 bins");
        float fr[kFormBins];
        unsigned long long acc[2 * kFormBins];
        CK(cudaMemcpy(fr, c->form_frac, sizeof fr, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(acc, c->form_acc, sizeof acc, cudaMemcpyDeviceToHost));
        for (int k = 0; k < kFormBins; ++k)
            out->window_fraction[k] = acc[2 * k + 1] ? (double)acc[2 * k] / (double)acc[2 * k + 1] : (double)fr[k];
    }
    out->form_ms_mixed = c->form_ms[0];
    out->form_ms_fp32 = c->form_ms[1];
    out->form_ms_window = c->form_ms[2];
    out->locality_order = c->locality ? 1 : 0;
    float herr;
    memcpy(&herr, &h.max_herr_bits, sizeof herr);
    out->max_abs_entropy_err = herr;
    out->kernel_launches = c->launches;
    for (int k = 0; k < PTSNE_N_STAGES; ++k) {
        out->stage_ms[k] = c->stage_ms[k];
        out->stage_calls[k] = c->stage_calls[k];
    }
    return PTSNE_OK;
}

int ptsne_set_form_threshold(ptsne_ctx* c, double threshold) {
    if (!c) return PTSNE_EINVAL;
    if (!c->form_fstar) return fail(c, PTSNE_EINVAL, "the form threshold needs PTSNE_PREC_BF16_WINDOW%s%lld");
    if (!(threshold == threshold)) return fail(c, PTSNE_EINVAL, "threshold must not be NaN%s%lld");
    c->form_fstar_host = (float)threshold;
    CK(cudaMemcpy(c->form_fstar, &c->form_fstar_host, sizeof(float), cudaMemcpyHostToDevice));
    return PTSNE_OK;
}

int ptsne_set_profiling(ptsne_ctx* c, int on) {
    if (!c) return PTSNE_EINVAL;
    if (on && !c->ev[0]) {
        for (int k = 0; k <= PTSNE_N_STAGES; ++k) CK(cudaEventCreate(&c->ev[k]));
    }
    c->profiling = on != 0;
    return PTSNE_OK;
}

int ptsne_set_tuning(ptsne_ctx* c, const ptsne_tuning* t) {
    if (!c || !t) return PTSNE_EINVAL;
    const bool ok_k = t->cluster == 1 || t->cluster == 2 || t->cluster == 4;
    if (!ok_k || t->group != 1 || t->consumer_warps < 1 || t->consumer_warps > 21)
        return fail(c, PTSNE_EINVAL, "invalid tuning%s (cluster %lld)", "", t->cluster);
    if (c->deterministic && c->p.schedule == PTSNE_SCHED_BATCHED &&
        iterate_warps(c->p.out_dim, c->zmax, 1, true, t->cluster) < 1)
        return fail(c, PTSNE_EINVAL, "largest chunk too large for the deterministic kernel on clusters of%s %lld",
                    "", t->cluster);
    c->tune.cluster = t->cluster;
    c->tune.group = t->group;
    c->tune.consumer_warps = t->consumer_warps;
    return PTSNE_OK;
}

int ptsne_set_locality_order(ptsne_ctx* c, int on) {
    if (!c) return PTSNE_EINVAL;
    if (c->p.schedule != PTSNE_SCHED_BATCHED)
        return fail(c, PTSNE_EINVAL, "the locality order needs the batched schedule%s%lld");
    c->locality = on != 0;
    return PTSNE_OK;
}

int ptsne_set_deterministic(ptsne_ctx* c, int on) {
    if (!c) return PTSNE_EINVAL;
    if (on && c->p.schedule == PTSNE_SCHED_BATCHED && iterate_warps(c->p.out_dim, c->zmax, 1, true, c->tune.cluster) < 1)
        return fail(c, PTSNE_EINVAL, "largest chunk too large for the deterministic batched kernel%s (%lld)", "",
                    (long long)c->zmax);
    c->deterministic = on != 0;
    return PTSNE_OK;
}

int ptsne_get_tuning(const ptsne_ctx* c, ptsne_tuning* t) {
    if (!c || !t) return PTSNE_EINVAL;
    t->cluster = c->tune.cluster;
    t->group = c->tune.group;
    t->consumer_warps = c->tune.consumer_warps;
    return PTSNE_OK;
}

int ptsne_reset_counters(ptsne_ctx* c) {
    if (!c) return PTSNE_EINVAL;
    c->launches = 0;
    for (int k = 0; k < PTSNE_N_STAGES; ++k) {
        c->stage_ms[k] = 0.0;
        c->stage_calls[k] = 0;
    }
    return PTSNE_OK;
}

}  // extern "C"
