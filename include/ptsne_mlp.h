/*
 * ptsne_mlp.h — the learned out-of-sample mapper of libptsne.so.
 *
 * The paper maps new points only by re-running ptSNE.  This library adds a
 * small network trained on the maps that ptSNE itself produces: it places
 * held-out points directly, and its output warm-starts ptsne_run (pass it as
 * the start map Y).  Plain ptSNE stays the fallback and the measure of the
 * mapper's quality (KL of Eq. 5 and k-nearest-neighbour preservation).
 *
 * Network: y = W3 g(W2 g(W1 x + b1) + b2) + b3 with g the exact GELU
 * g(u) = u (1 + erf(u / sqrt 2)) / 2 (the normal CDF evaluated with the
 * approximations of Abramowitz & Stegun, formulas 7.1.26 and 7.1.28, absolute
 * error <= 3e-7, far below the BF16 rounding of the hidden activations),
 * x in R^d_in (d_in <= 64), hidden width
 * 256, y in R^out_dim.  Weights are kept in FP32 (master copy, AdamW state)
 * and used in BF16; the products accumulate in FP32 on the tensor cores
 * (tcgen05, 128-row tiles).  Training minimises
 *     L = sum_b sum_k (y_bk - t_bk)^2 / (2 B)
 * over batches of B rows, t the target map standardised per coordinate
 * (t = (Y - mean) / std, mean and std from ptsne_mlp_fit_scaler), with AdamW
 * (decoupled weight decay on W1, W2, W3 only).  Inference returns
 * y * std + mean.
 *
 * Packed parameter layout (float32, host or device as stated), in order:
 *   W1 [256][d_in], b1 [256], W2 [256][256], b2 [256], W3 [out_dim][256],
 *   b3 [out_dim]                     (PTSNE_MLP_NPARAMS(d_in, out_dim) floats)
 *
 * Conventions as in ptsne.h: *_dev device pointers, row-major arrays, the
 * caller owns every array it passes, the handle owns its workspace, work is
 * enqueued on `stream` (cudaStream_t as void*).  Random numbers (initial
 * weights, sample orders) are inputs.
 */
#ifndef PTSNE_MLP_H
#define PTSNE_MLP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PTSNE_MLP_HIDDEN 256
#define PTSNE_MLP_NPARAMS(d_in, out_dim) \
    (256 * (d_in) + 256 + 256 * 256 + 256 + (out_dim) * 256 + (out_dim))

typedef struct ptsne_mlp ptsne_mlp;

typedef struct {
    int32_t d_in;            /* input features, 1 .. 64 */
    int32_t out_dim;         /* 2 or 3 */
    int32_t batch;           /* training rows per step, a multiple of 128, <= 65536 */
    int64_t infer_rows;      /* rows per inference launch, multiple of 128, <= 2^24 */
    float lr;                /* AdamW step size (e.g. 1e-3) */
    float beta1, beta2, eps; /* AdamW moments (0.9, 0.999, 1e-8) */
    float weight_decay;      /* decoupled decay on W1, W2, W3 (e.g. 1e-4) */
} ptsne_mlp_params;

/* Create a mapper with the initial parameters init_host (packed layout,
 * FP32, host).  The scaler starts as the identity (mean 0, std 1). */
int ptsne_mlp_create(ptsne_mlp** out, const ptsne_mlp_params* prm, const float* init_host);

/* Release the handle (NULL is a no-op).  Synchronises the device first. */
void ptsne_mlp_destroy(ptsne_mlp* m);

/* Text of the last error on m, or of the last failed create on this thread
 * when m is NULL (never NULL). */
const char* ptsne_mlp_last_error(const ptsne_mlp* m);

/* Copy the FP32 master parameters (packed layout) to out_host.  Synchronous. */
int ptsne_mlp_get_params(ptsne_mlp* m, float* out_host, void* stream);

/* Per-coordinate mean and standard deviation (population, FP64 sums) of the
 * n x out_dim target map T_dev, kept for training and inference.  Async. */
int ptsne_mlp_fit_scaler(ptsne_mlp* m, const float* T_dev, int64_t n, void* stream);

/* Loss and gradient of one batch without updating the parameters.  X_dev
 * (n x d_in) and T_dev (n x out_dim) are the data; rows_dev holds the batch's
 * `batch` row indices into them (int32, each in [0, n)).  grad_out_dev
 * (optional): packed gradient of L with respect to the FP32 parameters as
 * used (BF16-rounded weights).  loss_out_dev (optional): 1 double.  Async. */
int ptsne_mlp_grad(ptsne_mlp* m, const float* X_dev, const float* T_dev, int64_t n, const int32_t* rows_dev,
                   float* grad_out_dev, double* loss_out_dev, void* stream);

/* ptsne_mlp_grad followed by one AdamW step.  Async. */
int ptsne_mlp_train_step(ptsne_mlp* m, const float* X_dev, const float* T_dev, int64_t n,
                         const int32_t* rows_dev, double* loss_out_dev, void* stream);

/* `epochs` passes over the data: epoch e visits the rows in the order
 * orders_dev[e * n .. e * n + n) (a permutation of [0, n)), floor(n / batch)
 * steps of `batch` rows (the remainder is skipped).  loss_out_host
 * (optional): epochs doubles, each epoch's mean batch loss.  Synchronous. */
int ptsne_mlp_train(ptsne_mlp* m, const float* X_dev, const float* T_dev, int64_t n, const int32_t* orders_dev,
                    int32_t epochs, double* loss_out_host, void* stream);

/* Autotuner of the weight-gradient GEMMs (K = batch): times the forward and
 * backward pass of the batch rows_dev (parameters untouched) for 1, 2, 4, ...
 * CTAs along K (at most batch / 64 and 64) and keeps the fastest for this
 * handle.  cache_path (optional): text file of earlier choices keyed by
 * device, d_in, out_dim and batch; a hit skips the timing and a new choice is
 * appended.  split_out (optional): the choice.  Synchronous. */
int ptsne_mlp_autotune(ptsne_mlp* m, const float* X_dev, const float* T_dev, int64_t n, const int32_t* rows_dev,
                       const char* cache_path, int32_t* split_out, void* stream);

/* Map n points: X_dev (n x d_in) -> Y_out_dev (n x out_dim), de-standardised
 * by the scaler.  One fused kernel launch per infer_rows rows (X is read
 * in place, FP32, rounded to BF16 on chip).  Async. */
int ptsne_mlp_infer(ptsne_mlp* m, const float* X_dev, int64_t n, float* Y_out_dev, void* stream);

struct ptsne_ctx;

/* Warm start with plain ptSNE as the fallback and the arbiter.  The mapper
 * places the n points of X_dev (n x d_in, d_in = the context's d) into Y_dev
 * (n x out_dim); then one ptSNE epoch on the partition perm_dev runs from
 * that placement and one from the cold start Y_random_dev (n x out_dim, not
 * modified; e.g. the N(0, 1e-4) or unit-disk start), both with the context's
 * settings, so at equal iterations.  If the warm epoch ends at a larger
 * average KL (Eq. 5) than the cold one, the mapper did worse than no mapper
 * and Y_dev receives the cold epoch's map; else it keeps the warm epoch's.
 * Either way Y_dev then holds a map one epoch into the run: continue with
 * ptsne_run.  kl_out_host (optional, 2 doubles): {warm KL, cold KL};
 * used_mapper_out (optional): 1 if the warm map was kept, 0 on fallback.
 * Needs a context with layers = 1, n points, d = d_in and the mapper's
 * out_dim; else PTSNE_EINVAL.  The context keeps a second n x out_dim map
 * (allocated on the first call).  Synchronous. */
int ptsne_mlp_warm_start(ptsne_mlp* m, struct ptsne_ctx* ctx, const float* X_dev, const int32_t* perm_dev,
                         const float* Y_random_dev, float* Y_dev, double* kl_out_host, int32_t* used_mapper_out,
                         void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PTSNE_MLP_H */
