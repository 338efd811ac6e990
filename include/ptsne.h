/*
 * ptsne.h — C ABI of libptsne.so, the GB300 (sm_103a) implementation of the
 * hot path of parallelized t-SNE (ptSNE; Garriga & Bartumeus, "bigMap: Big
 * Data Mapping with parallelized t-SNE", arXiv 1812.09869).
 *
 * A ptSNE epoch cuts a random permutation of the n points into chunks (the
 * paper's "threads"; one layer), runs one partial t-SNE per chunk and pools
 * the partial maps back (ptSNE section, subsections "threads" and "epochs").
 * For each chunk of z points:
 *   affinities  — squared Euclidean distances, per-row precision beta_i such
 *                 that the perplexity 2^H of p_{.|i} (Eq. 1, Eq. 2) equals the
 *                 target, joint P_ij = (p_{j|i} + p_{i|j}) / (2z) (Eq. 3);
 *   iterations  — Cauchy kernel w_ij and normaliser Z (Eq. 4), exact gradient
 *                 4 sum_j (p_ij - w_ij/Z) w_ij (y_i - y_j) (Eq. 6), momentum
 *                 update in the descent direction (Eq. 12) with optional gains
 *                 or the auto-adaptive learning rate (Eq. 13);
 *   evaluation  — KL (Eq. 5) and pseudo-normalised cost (Eq. 9) averaged over
 *                 chunks, and the embedding size (the diagonal of the map's
 *                 bounding box) that the paper monitors beside the cost.
 *
 * Conventions for every entry point:
 *   - Pointers named *_dev are device pointers on the current CUDA device;
 *     *_host are host pointers.  Arrays are dense and row-major.
 *   - Points are addressed in their ORIGINAL order (0..n-1) in X, Y, beta and
 *     grad.  A partition is a device int32 permutation perm of [0, n); chunk c
 *     holds the points perm[off[c] .. off[c+1]) with off the chunk offsets
 *     given at creation.  Permutations are inputs (drawn by the caller).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  All work is enqueued on it; entry points marked "async"
 *     return before the GPU work completes.
 *   - The caller owns every array it passes.  The context owns its device
 *     workspace (allocated once by ptsne_create) and frees it in
 *     ptsne_destroy.
 *   - Return codes: PTSNE_OK (0), a negative error, or a positive warning.
 *     Argument errors are detected on the host before any work is enqueued;
 *     ptsne_last_error() then describes the first failure.  Permutation
 *     entries outside [0, n) are detected on the device, skipped, and counted
 *     (ptsne_get_stats); ptsne_run then fails with PTSNE_EINVAL.
 */
#ifndef PTSNE_H
#define PTSNE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PTSNE_OK 0
#define PTSNE_EINVAL (-1)     /* bad argument (null pointer, size, layout, perplexity) */
#define PTSNE_ENONFINITE (-2) /* NaN or Inf found in X */
#define PTSNE_ENOMEM (-3)     /* device allocation failed */
#define PTSNE_ECUDA (-4)      /* a CUDA call failed */
#define PTSNE_ESTATE (-5)     /* call order violated (e.g. step before affinities) */
#define PTSNE_ETIMEOUT (-6)   /* a bounded wait inside a kernel ran out (results invalid) */
#define PTSNE_WBISECT 1       /* some rows' perplexity search missed its tolerance */

#define PTSNE_LR_FIXED 0      /* eta = lr (with gains if use_gains) */
#define PTSNE_LR_PAPER 1      /* eta = ln(z-1) (Ymax - Ymin) / 2 per chunk (Eq. 13) */

#define PTSNE_PREC_FP32 0        /* distances in FP32 by direct differences */
#define PTSNE_PREC_BF16_WINDOW 1 /* BF16 tensor-core Gram matrix, FP32 recompute in the
                                    perplexity window of each row */

#define PTSNE_SCHED_BATCHED 0    /* all chunks per launch; one persistent launch per epoch
                                    runs every gradient iteration of every chunk */
#define PTSNE_SCHED_PER_CHUNK 1  /* plain form: each chunk and iteration launched separately */

/* Stages of a ptsne_run epoch, for per-stage timing (ptsne_set_profiling). */
#define PTSNE_STAGE_GATHER 0     /* gather X and Y rows by the partition, reset the optimiser */
#define PTSNE_STAGE_DISTANCES 1  /* pairwise distances (all chunks; the per-chunk schedule
                                    counts its whole affinity phase here) */
#define PTSNE_STAGE_PERPLEXITY 2 /* per-row beta search (and window recompute) */
#define PTSNE_STAGE_JOINT_P 3    /* symmetric joint P */
#define PTSNE_STAGE_ITERATE 4    /* all gradient iterations of the epoch */
#define PTSNE_STAGE_POOL 5       /* scatter the partial maps back */
#define PTSNE_STAGE_COST 6       /* per-epoch cost evaluation (if requested) */
#define PTSNE_N_STAGES 7

typedef struct ptsne_ctx ptsne_ctx;

typedef struct {
    int64_t n;                    /* points, >= 2 */
    int32_t d;                    /* input dimensions, 1..4096 */
    int32_t out_dim;              /* embedding dimensions: 2 or 3 (Eq. 4 text: d in {2,3}) */
    double perplexity;            /* target perplexity; 1 < perplexity < z_min - 1 (Eq. 2:
                                     the maximum perplexity of a chunk of z points is z-1) */
    int32_t n_chunks;             /* >= 1 */
    const int64_t* chunk_offsets; /* host, n_chunks+1 entries, off[0]=0, off[n_chunks]=n,
                                     every chunk size in [2, 8192]; copied by ptsne_create */
    int32_t iters;                /* gradient iterations per epoch (ptsne_run), >= 0 */
    float lr;                     /* learning rate eta for PTSNE_LR_FIXED, > 0 */
    float momentum;               /* alpha of Eq. 12, in [0, 1) */
    int32_t lr_mode;              /* PTSNE_LR_FIXED or PTSNE_LR_PAPER */
    int32_t use_gains;            /* 1: per-coordinate gains (+0.2 on sign change of grad
                                     versus velocity, x0.8 otherwise, floor 0.01) */
    int32_t precision;            /* PTSNE_PREC_* */
    int32_t schedule;             /* PTSNE_SCHED_* */
    int32_t use_graph;            /* 1: ptsne_run replays each epoch from one captured CUDA
                                     graph (captured on the first call, and again whenever
                                     X, Y, the tuning, profiling or the cost request
                                     change); 0: plain launches.  Profiling marks are
                                     captured as event nodes of the graph. */
    int32_t layers;               /* L >= 1 (at most n_chunks): the chunks of chunk_offsets are
                                     the elementary chunks of a partition; thread t runs
                                     elementary chunks t, t+1, ..., t+L-1 (mod n_chunks)
                                     together (ptSNE section, "layers"), so each point runs
                                     in L threads and keeps L maps.  With L > 1 every Y,
                                     grad and beta array holds L layers of n rows,
                                     layer-major (row k n + i = point i in layer k; the
                                     point in slot k of a thread reads and writes layer k);
                                     P_out holds one z x z block per thread and Z_out one
                                     value per thread; permutations stay n entries.
                                     Thread sizes z_t = sum of its L chunk sizes must be
                                     in [2, 8192].  1: the plain scheme. */
} ptsne_params;

typedef struct {
    int64_t bisect_rows;          /* rows searched by the last ptsne_affinities */
    int64_t bisect_fp64_rows;     /* rows whose FP32 search stalled and were redone in FP64 */
    int64_t bisect_failed_rows;   /* rows that missed the tolerance even in FP64 */
    int64_t window_pairs;         /* BF16_WINDOW: distances recomputed in FP32 (the window
                                     candidates of sparse rows, and every pair of the 64 x 64
                                     tiles recomputed whole for dense rows; chunks computed in
                                     FP32 whole are not counted) */
    int64_t nonfinite_inputs;     /* NaN/Inf entries seen in X by the last gather */
    int64_t bad_perm_entries;     /* permutation entries outside [0, n): skipped, never dereferenced */
    int64_t wait_timeouts;        /* bounded in-kernel waits that ran out (PTSNE_ETIMEOUT) */
    double max_abs_entropy_err;   /* max |H(beta_i) - ln perplexity| (nats) of the last search */
    int64_t kernel_launches;      /* kernels this context enqueued since creation / last reset */
    double stage_ms[PTSNE_N_STAGES];     /* profiling on: device time per stage of ptsne_run */
    int64_t stage_calls[PTSNE_N_STAGES]; /* profiling on: epochs accumulated into stage_ms */
    int64_t bisect_evals;         /* entropy evaluations (FP32 and FP64) of the last search, all rows */
    int64_t ptiles_total;         /* batched schedule: stored 32 x 32 tiles of the joint P */
    int64_t ptiles_nonzero;       /* of those, tiles with a nonzero entry in the last affinities
                                     (FP32 exponentials of far pairs underflow to exactly 0);
                                     counted on the stats call's stream, not among kernel_launches */
    int64_t fp32_chunks;          /* BF16_WINDOW: chunks computed in FP32 whole (see
                                     ptsne_set_form_threshold), summed like window_pairs */
    double form_threshold;        /* BF16_WINDOW: the window fraction at or above which a chunk
                                     runs in FP32 whole (> 1: never) */
    double window_fraction[8];    /* BF16_WINDOW: window fraction (window pairs / (z - 1) per
                                     row) last measured in each of 8 equal chunk-size bins
                                     over [zmin, zmax] */
    double form_ms_mixed;         /* ptsne_autotune on BF16_WINDOW: affinities time with every
                                     chunk in the mixed form, */
    double form_ms_fp32;          /* ... with every chunk in FP32 whole, */
    double form_ms_window;        /* ... and of the window recompute alone (0: not tuned) */
    int64_t locality_order;       /* 1: the locality order is on (ptsne_set_locality_order, or
                                     ptsne_autotune_form's choice) */
} ptsne_stats;

/* Turn on (1) or off (0) per-stage timing of ptsne_run: CUDA events are
 * recorded between its stages on the caller's stream and, after each epoch,
 * the elapsed times are added to stage_ms (the host waits for each epoch to
 * finish while profiling).  Off by default. */
int ptsne_set_profiling(ptsne_ctx* ctx, int on);

/* Zero kernel_launches, stage_ms and stage_calls. */
int ptsne_reset_counters(ptsne_ctx* ctx);

/* Launch shape of the batched iteration kernel (no effect on results beyond
 * FP32 summation order).  cluster: thread blocks sharing one chunk through
 * distributed shared memory (1, 2 or 4); group: warps per P tile, 1 (each
 * warp evaluates whole tiles; other values are rejected); consumer_warps:
 * warps per block, each evaluating tiles and copying its own, 1 .. 21 (2-D
 * maps use at most 16, the four rows per lane of their evaluation need 128
 * registers; 3-D maps at most 21; the largest chunks leave shared memory for
 * fewer warps' tile buffers).  Defaults {2, 1, 20}; ptsne_autotune picks by
 * timing. */
typedef struct {
    int32_t cluster;
    int32_t group;
    int32_t consumer_warps;
} ptsne_tuning;

int ptsne_set_tuning(ptsne_ctx* ctx, const ptsne_tuning* tuning);

/* Locality order of the rows within each chunk (batched schedule; off by
 * default).  The order of a chunk's rows changes none of the method's
 * results (Eq. 1-6 are equivariant under it; only the FP32 summation order
 * moves).  With it on, every affinities computation first places each row
 * of a chunk next to the rows nearest it (the rows are sorted by their
 * nearest of the chunk's first 64 rows, a random sample), so that the joint
 * P concentrates on few 32 x 32 tiles and many tiles are exactly zero (the
 * FP32 exponentials of far pairs underflow; ptsne_get_stats counts the
 * nonzero ones).  Exported P and every per-point output stay in the caller's
 * order; ptsne_step and ptsne_cost use the order of the kept affinities.
 * ptsne_affinities_from_distances never reorders.  PTSNE_EINVAL on the
 * per-chunk schedule. */
int ptsne_set_locality_order(ptsne_ctx* ctx, int on);

/* Summation order of the batched iteration kernel (Eq. 6 sums A_i and R_i).
 * 0 (default): FP32 atomic adds in shared memory, whose order varies from
 * run to run, so that two identical runs agree to about 1e-7 relative per
 * iteration, not bit for bit.  1: the sums are kept in 64-bit fixed point
 * (A at 2^-61, R at 2^-48; integer adds do not depend on their order), so
 * that identical runs on one GPU give bitwise identical maps and costs.  The
 * 8-byte sums need twice the shared memory; where that would leave a block
 * fewer warps than the tuning asks for, on clusters of 2 or 4 blocks
 * (ptsne_set_tuning) each block holds only the sums of the rows it updates
 * and adds to the other rows' sums in their block's shared memory, so the
 * footprint is that of the FP32 sums on 2 blocks and less on 4.  The
 * per-chunk schedule sums in a fixed order in either mode.  PTSNE_EINVAL if
 * the largest chunk does not fit the deterministic kernel for the current
 * cluster size (on 1 block per chunk: 2-D maps up to z of about 5600, 3-D
 * about 3700; on 2 or 4 blocks every chunk the batched schedule takes; all
 * 16 warps of a 2-D block up to about 4100, 6800 and 10200 on 1, 2 and 4
 * blocks), and ptsne_set_tuning refuses a cluster size that would not fit
 * while the mode is on. */
int ptsne_set_deterministic(ptsne_ctx* ctx, int on);

/* Form of each chunk's distances under PTSNE_PREC_BF16_WINDOW.  A row's
 * window (the pairs whose weight exp(-beta (d - m)) can reach e^-25 of the
 * row's largest, the BF16 error bound included) is what the FP32 recompute
 * must cover; when windows are most of a chunk, computing the chunk's
 * distances in FP32 whole (direct differences, as PTSNE_PREC_FP32) costs less
 * than the BF16 Gram matrix, the coarse search and the recompute.  Each
 * affinities computation gives every chunk whose size bin's last measured
 * window fraction (ptsne_stats.window_fraction) is >= threshold the FP32 form
 * (no Gram tiles, no coarse search; the fine search and everything after it
 * are the same).  Either form yields the same distances wherever they matter:
 * results differ only by FP32 rounding.  Default 2 (never); ptsne_autotune
 * measures both forms and sets it; a negative value puts every chunk in FP32.
 * PTSNE_EINVAL unless the context is BF16_WINDOW, or for NaN.  Synchronous;
 * a captured ptsne_run graph reads the threshold from device memory. */
int ptsne_set_form_threshold(ptsne_ctx* ctx, double threshold);
int ptsne_get_tuning(const ptsne_ctx* ctx, ptsne_tuning* tuning);

typedef struct {
    ptsne_tuning tuning;
    double ms_per_iter;           /* device time per gradient iteration (all chunks) */
} ptsne_tune_trial;

/* Form of the distances under BF16_WINDOW (A1 of the autotuner; no
 * counterpart in the paper, which computes distances in double precision):
 * the affinities of perm_dev are timed with every chunk in the mixed form and
 * with every chunk in FP32 whole (each the faster of two runs after an
 * untimed one), and the window recompute alone; the break-even window
 * fraction goes to ptsne_set_form_threshold (times in ptsne_stats.form_ms_*).
 * On the batched schedule the mixed form is timed with the locality order off
 * and on (it gathers a dense window row's pairs on few tiles) and the faster
 * setting is applied, unless every chunk goes to FP32 whole (then the
 * caller's setting stays).  Leaves the affinities of perm_dev in ctx.
 * Synchronous.  PTSNE_EINVAL unless the context is BF16_WINDOW. */
int ptsne_autotune_form(ptsne_ctx* ctx, const float* X_dev, const int32_t* perm_dev, void* stream);

/* Autotuner of the batched iteration kernel's launch shape (no counterpart in
 * the paper, whose kernels are CPU threads).  Under BF16_WINDOW it first runs
 * ptsne_autotune_form (timed on every call, cache or not).  Then it computes
 * the affinities of the partition perm_dev and times `iters` gradient iterations from the map
 * Y_dev (n x out_dim, not modified) for every candidate shape with CUDA
 * events (best of two), restoring the optimiser state between trials, and
 * applies the fastest to ctx.  cache_path (optional): a text file of one
 * record per line, keyed by device name, SM count, out_dim and the chunk-size
 * layout; a matching record is applied without timing, a new result is
 * appended.  trials_out (optional, host, capacity max_trials) receives every
 * timed trial; *n_trials_out their count (0 on a cache hit).  Leaves the
 * affinities of perm_dev in ctx with a reset optimiser state.  Synchronous.
 * Per-chunk schedule: PTSNE_EINVAL (nothing to tune). */
int ptsne_autotune(ptsne_ctx* ctx, const float* X_dev, const int32_t* perm_dev, const float* Y_dev, int32_t iters,
                   const char* cache_path, ptsne_tune_trial* trials_out, int32_t max_trials,
                   int32_t* n_trials_out, void* stream);

/* Create a context for one problem shape and allocate its device workspace
 * on the current device.  Validates every field (PTSNE_EINVAL), then
 * allocates (PTSNE_ENOMEM).  On success *out owns the workspace. */
int ptsne_create(ptsne_ctx** out, const ptsne_params* params);

/* Release the context and its workspace (NULL is a no-op).  Synchronises the
 * device first so that no enqueued work still uses the workspace. */
void ptsne_destroy(ptsne_ctx* ctx);

/* Text of the last error recorded on ctx (never NULL).  With ctx == NULL:
 * the reason of the last failed ptsne_create, ptsne_gradient_static or
 * ptsne_kde_grid on the calling thread. */
const char* ptsne_last_error(const ptsne_ctx* ctx);

/* Input affinities for the partition perm_dev (Eq. 1-3 per chunk, n := z).
 * X_dev: n x d float32.  perm_dev: n int32.  P_out_dev (optional, NULL to
 * skip): receives every chunk's z x z joint P, row-major, chunks concatenated
 * in chunk order (sum_c z_c^2 floats; rows and columns in chunk order, i.e.
 * P_out[c][r][s] couples points perm[off[c]+r] and perm[off[c]+s]).
 * beta_out_dev (optional): n floats, beta of each point in original order.
 * Keeps P for later ptsne_step / ptsne_cost calls and resets the optimiser
 * state (velocity 0, gains 1): each partition starts fresh partial t-SNEs.
 * Async. */
int ptsne_affinities(ptsne_ctx* ctx, const float* X_dev, const int32_t* perm_dev,
                     float* P_out_dev, float* beta_out_dev, void* stream);

/* ptsne_affinities from precomputed dissimilarities instead of points (for
 * instance shortest-path lengths of a graph, the paper's non-vector input):
 * D_dev is n x n float32, row-major with leading dimension ldd >= n, D[i][j]
 * the dissimilarity of points i and j in ORIGINAL order (need not be
 * symmetric; the diagonal is ignored).  Each chunk's block is gathered through
 * perm_dev; the search and joint P follow as in ptsne_affinities, at FP32
 * whatever the context's precision (there is nothing to recompute).
 * Non-finite entries are counted in nonfinite_inputs and read as 0.  P_out,
 * beta_out, the kept P and the optimiser reset as ptsne_affinities; follow
 * with ptsne_step / ptsne_cost.  Async. */
int ptsne_affinities_from_distances(ptsne_ctx* ctx, const float* D_dev, int64_t ldd, const int32_t* perm_dev,
                                    float* P_out_dev, float* beta_out_dev, void* stream);

/* Pairwise squared distances of every chunk of the partition perm_dev, at
 * the context's precision and before any window recompute: FP32 direct
 * differences (PTSNE_PREC_FP32), or |x~_i|^2 + |x~_j|^2 - 2 x~_i . x~_j from
 * the BF16-rounded rows on the tensor cores (PTSNE_PREC_BF16_WINDOW).
 * D_out_dev: sum_c z_c^2 floats, dense z x z per chunk in chunk order (as
 * P_out of ptsne_affinities; diagonal entries unspecified).  Does not change
 * the affinities kept by the context.  Async. */
int ptsne_distances(ptsne_ctx* ctx, const float* X_dev, const int32_t* perm_dev, float* D_out_dev,
                    void* stream);

/* One gradient iteration on every chunk of the partition of the last
 * ptsne_affinities call (Eq. 4, 6, 12/13).  Y_dev: n x out_dim float32 in
 * original order, updated in place.  grad_out_dev (optional): n x out_dim,
 * the gradient of Eq. 6 at the input Y.  Z_out_dev (optional): n_chunks
 * doubles, each chunk's Z of Eq. 4 at the input Y.  perm_dev must be the same
 * permutation.  Async. */
int ptsne_step(ptsne_ctx* ctx, const int32_t* perm_dev, float* Y_dev,
               float* grad_out_dev, double* Z_out_dev, void* stream);

/* Average over chunks of KL (Eq. 5) and pseudo-normalised cost (Eq. 9) for
 * the P of the last ptsne_affinities and the map Y_dev (original order).
 * out_dev: 2 doubles {avg KL, avg normalised cost} on the device.  Async. */
int ptsne_cost(ptsne_ctx* ctx, const int32_t* perm_dev, const float* Y_dev,
               double* out_dev, void* stream);

/* Embedding size of a map (ptSNE section, the monitoring of cost and size at
 * the end of each epoch): the length of the diagonal of the map's bounding
 * box, sqrt(sum_k (max_i Y[i][k] - min_i Y[i][k])^2), over every row of Y_dev
 * (the context's rows x out_dim floats: n rows, or layers x n with layers > 1).
 * The extremes are exact; the sum and square root run in FP64.  NaN
 * coordinates are ignored.  out_dev: 1 double on the device.  Uses the
 * context's workspace, so calls on one context must be ordered (one stream).
 * Async. */
int ptsne_embedding_size(ptsne_ctx* ctx, const float* Y_dev, double* out_dev, void* stream);

/* The ptSNE cycle: for e in [0, epochs): affinities for perms_dev[e] (n int32
 * each, epochs x n), `iters` gradient iterations of every chunk from the
 * current map, pooling into Y_dev (n x out_dim, in: start map, out: result).
 * cost_out_host (optional): epochs x 3 doubles, {avg KL, avg normalised cost,
 * embedding size of the pooled map} at the end of each epoch.  From the second epoch on, each row's perplexity
 * search starts from the precision its point had in the previous epoch (the
 * root is unique, so only the number of evaluations changes); the first
 * epoch of every call starts cold, so identical calls give identical results.
 * Synchronous: returns after the work completes, with PTSNE_WBISECT if some
 * row missed the perplexity tolerance. */
int ptsne_run(ptsne_ctx* ctx, const float* X_dev, const int32_t* perms_dev,
              int32_t epochs, float* Y_dev, double* cost_out_host, void* stream);

/* ptsne_run on HOST buffers: copies X_host (n x d), perms_host (epochs x n)
 * and Y_host (n x out_dim) to context-owned device buffers, runs, and copies
 * the map back into Y_host.  Page-locked host memory makes the copies
 * asynchronous.  Synchronous. */
int ptsne_run_host(ptsne_ctx* ctx, const float* X_host, const int32_t* perms_host,
                   int32_t epochs, float* Y_host, double* cost_out_host, void* stream);

/* Counters of the last ptsne_affinities / ptsne_run.  Synchronises stream. */
int ptsne_get_stats(ptsne_ctx* ctx, ptsne_stats* out, void* stream);

/* Bytes of device workspace held by ctx. */
size_t ptsne_workspace_bytes(const ptsne_ctx* ctx);

/* Perplexity-adaptive kernel density estimate of a 2-D map (paKDE, the
 * paper's Clustering section): the sample smoothing estimator with Gaussian
 * kernels, f(c) = (S / n) sum_j (beta_j / pi) exp(-beta_j |c - y_j|^2), at the
 * centres of a gx x gy grid of cells of area S over box_host = {xmin, xmax,
 * ymin, ymax} (host, 4 floats).  Y_dev: n x 2 float32 map; beta_dev: n
 * precisions, obtained with the same perplexity search as the input
 * affinities applied to the map (ptsne_affinities on a context with d = 2,
 * X := Y).  density_dev: gy x gx float32 (row = y cell), overwritten; its sum
 * is the kernel mass inside the box (1 when the box covers the map).  Kernels
 * are dropped beyond beta r^2 = 30, and points with a non-positive or
 * non-finite beta or position are ignored.  A point whose kernel would cover
 * more than PTSNE_KDE_MAX_CELLS cells of the grid is left out (its precision is
 * far too small for the grid; this bounds the work per point) and counted in
 * *dropped_dev (optional, 1 int64 on the device, overwritten).  n >= 1,
 * 1 <= gx, gy <= 16384; else PTSNE_EINVAL with the reason in
 * ptsne_last_error(NULL).  Async. */
#define PTSNE_KDE_MAX_CELLS (1 << 20)
int ptsne_kde_grid(const float* Y_dev, const float* beta_dev, int64_t n, int32_t gx, int32_t gy,
                   const float* box_host, float* density_dev, int64_t* dropped_dev, void* stream);

/* k-nearest-neighbour preservation of a map (the measure of a map's local
 * structure, used on the learned mapper's placements): for each query q (an
 * index into the n points), the k nearest neighbours of q among the rows of
 * X_dev (n x d) and among the rows of Y_dev (n x od), by squared Euclidean
 * distance in FP32 (direct differences), q itself excluded and ties broken by
 * the smaller index.  overlap_out_dev (nq int32): the size of the overlap of
 * the two sets (the preservation of q is overlap / k; -1 for a query outside
 * [0, n)).  nbr_x_out_dev, nbr_y_out_dev (optional, nq x k int32): the two
 * sets, nearest first.  1 <= k <= 32, k < n < 2^31, 1 <= d, od <= 4096,
 * nq >= 0; else PTSNE_EINVAL with the reason in ptsne_last_error(NULL).
 * Async. */
int ptsne_knn_preservation(const float* X_dev, const float* Y_dev, int64_t n, int32_t d, int32_t od,
                           const int32_t* queries_dev, int32_t nq, int32_t k, int32_t* overlap_out_dev,
                           int32_t* nbr_x_out_dev, int32_t* nbr_y_out_dev, void* stream);

/* Largest chunk ptsne_gradient_static accepts. */
#define PTSNE_STATIC_MAX_ROWS 32768

/* The exact gradient of one chunk WITHOUT any device allocation and without a
 * context.  The paper has no counterpart: it exists for callers that cannot
 * call cudaMalloc (a host framework that owns the whole device memory pool
 * and forbids allocations outside its own accounting, callers that must not
 * block on an allocation, which may synchronise the device).
 *   P_dev:    z rows of ld floats (ld >= z), the symmetric joint P of the
 *             chunk (e.g. one block of ptsne_affinities' P_out, ld = z);
 *             the diagonal is ignored.
 *   Y_dev:    z x out_dim floats, the chunk's map in the same row order.
 *   grad_out_dev: z x out_dim floats, dC/dy_i = 4 (A_i - R_i / Z) as ptsne_step
 *             computes it.
 *   Z_out_dev (optional): 1 double, Z of the chunk.
 * z in [2, PTSNE_STATIC_MAX_ROWS], out_dim 2 or 3; anything else returns
 * PTSNE_EINVAL before any work, with the reason in ptsne_last_error(NULL).
 * Scratch (1 MiB of per-row sums) is a fixed array in the library's device
 * memory, shared by every call on a device: calls that can overlap on the GPU
 * race on it; calls ordered on one stream are safe, and nothing needs
 * clearing between them.  The first call on each device looks up the array's
 * address (and the SM count) and may load the module.  The address is kept
 * per device together with the CUDA
 * context it was taken in, and looked up again after that context has been
 * destroyed and re-created (cudaDeviceReset).  Async. */
int ptsne_gradient_static(const float* P_dev, int64_t ld, const float* Y_dev, int32_t z, int32_t out_dim,
                          float* grad_out_dev, double* Z_out_dev, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PTSNE_H */
