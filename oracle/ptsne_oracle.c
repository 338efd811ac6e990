/*
 * ptSNE oracle: a plain, slow, FP64 CPU implementation of what the GPU path
 * computes, used ONLY as test infrastructure (tests, the smoke check and the
 * CPU-baseline leg of the benchmark).  The product path never calls it.
 *
 * It follows the paper (Garriga & Bartumeus, "bigMap: Big Data Mapping with
 * parallelized t-SNE", arXiv 1812.09869) step by step:
 *   - input similarities: squared Euclidean distances, Gaussian conditional
 *     probabilities with per-row precision beta_i (Eq. 1), perplexity 2^H
 *     (Eq. 2), symmetric joint P (Eq. 3);
 *   - output similarities: Cauchy kernel q_ij (Eq. 4);
 *   - cost: KL(P||Q) (Eq. 5) and its exact gradient (Eq. 6);
 *   - pseudo-normalised cost (Eq. 9), averaged over partial t-SNEs;
 *   - position update with momentum (Eq. 12, descent direction) and the
 *     auto-adaptive learning rate (Eq. 13);
 *   - the ptSNE epoch cycle: partition, partial t-SNEs, pooling (ptSNE
 *     section, "threads", "epochs").
 * Readings where the paper is silent (the beta search of its missing
 * Supplement S1, gains, velocity reset per epoch) are stated at each function.
 *
 * Parity status: every function here is pinned by a CPU test against closed
 * forms, brute force or finite differences, except the multi-epoch trajectory
 * of orc_ptsne_run beyond the first step (chaotic; pinned only through the
 * monotone decrease of the cost).
 *
 * Plain C11, doubles throughout, no fast-math.  OpenMP only spreads
 * independent rows over cores; every sum runs in a fixed sequential order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOMEM -3

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Squared Euclidean distances ||x_i - x_j||^2 by direct differences (ptSNE
 * section, "Similarities in the input space").  D is z x z, row-major. */
int orc_sqdist(const double* X, int64_t z, int32_t d, double* D) {
    if (!X || !D || z < 1 || d < 1) return ORC_EINVAL;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < z; ++i) {
        for (int64_t j = 0; j < z; ++j) {
            double s = 0.0;
            for (int32_t k = 0; k < d; ++k) {
                double t = X[i * d + k] - X[j * d + k];
                s += t * t;
            }
            D[i * z + j] = s;
        }
    }
    return ORC_OK;
}

/* Entropy H (nats) of the conditional distribution of row i at precision beta
 * (Eq. 1), and the row's normaliser.  t_j = d_ij - m with m = min_{j!=i} d_ij;
 * the shift cancels in Eq. 1 and only keeps exp() in range.
 *   p_{j|i} = exp(-beta t_j) / S,  S = sum_{j!=i} exp(-beta t_j)
 *   H = -sum_j p_{j|i} ln p_{j|i} = ln S + beta * sum_j t_j exp(-beta t_j) / S */
static double row_entropy(const double* drow, int64_t z, int64_t i, double m,
                          double beta, double* S_out) {
    double S = 0.0, T = 0.0;
    for (int64_t j = 0; j < z; ++j) {
        if (j == i) continue;
        double t = drow[j] - m;
        double e = exp(-beta * t);
        S += e;
        T += t * e;
    }
    if (S_out) *S_out = S;
    return log(S) + beta * T / S;
}

/* Per-row search for beta_i such that the perplexity 2^H of p_{.|i} (Eq. 2)
 * equals `perp`.  The paper defers the procedure to its Supplement S1, which is
 * not available; this is plain bisection on beta (H is non-increasing in beta):
 * start at beta = 1/mean_j(t_j), double beta until the target is bracketed from
 * above, then halve the bracket, stopping when |H - ln(perp)| <= tol (nats) or
 * after maxit evaluations.  Returns 0 when converged, 1 when not (the row's
 * best beta is still written).
 * Degenerate rows: when every t_j is 0 (all neighbours equidistant) the
 * distribution is uniform for every beta; beta = 0 is returned with H =
 * ln(z-1), converged only if that equals the target.  */
int orc_row_beta(const double* drow, int64_t z, int64_t i, double perp,
                 double tol, int32_t maxit, double* beta_out, double* H_out,
                 int32_t* iters_out) {
    if (!drow || z < 2 || i < 0 || i >= z || !(perp > 0.0)) return ORC_EINVAL;
    double m = INFINITY, tsum = 0.0;
    for (int64_t j = 0; j < z; ++j)
        if (j != i && drow[j] < m) m = drow[j];
    for (int64_t j = 0; j < z; ++j)
        if (j != i) tsum += drow[j] - m;
    const double target = log(perp);
    double beta, H;
    int32_t it = 0;
    int conv = 0;
    if (tsum == 0.0) {
        beta = 0.0;
        H = log((double)(z - 1));
        conv = fabs(H - target) <= tol;
    } else {
        double lo = 0.0, hi = INFINITY;
        beta = (double)(z - 1) / tsum;
        H = row_entropy(drow, z, i, m, beta, NULL);
        for (it = 1; it < maxit; ++it) {
            double f = H - target;
            if (fabs(f) <= tol) { conv = 1; break; }
            double next;
            if (f > 0.0) {            /* too flat: sharpen the kernel */
                lo = beta;
                next = isinf(hi) ? 2.0 * beta : 0.5 * (lo + hi);
            } else {                  /* too peaked: widen the kernel */
                hi = beta;
                next = 0.5 * (lo + hi);
            }
            /* unreachable target (several nearest neighbours tied and a
             * perplexity below their count): stop before beta overflows */
            if (!(next < 1e300) || next == beta) break;
            beta = next;
            H = row_entropy(drow, z, i, m, beta, NULL);
        }
        if (!conv && fabs(H - target) <= tol) conv = 1;
    }
    if (beta_out) *beta_out = beta;
    if (H_out) *H_out = H;
    if (iters_out) *iters_out = it;
    return conv ? 0 : 1;
}

/* Conditional probabilities p_{j|i} of Eq. 1 for row i at precision beta. */
static void row_conditional(const double* drow, int64_t z, int64_t i,
                            double beta, double* out) {
    double m = INFINITY, S = 0.0;
    for (int64_t j = 0; j < z; ++j)
        if (j != i && drow[j] < m) m = drow[j];
    for (int64_t j = 0; j < z; ++j) {
        if (j == i) { out[j] = 0.0; continue; }
        out[j] = exp(-beta * (drow[j] - m));
        S += out[j];
    }
    for (int64_t j = 0; j < z; ++j) out[j] /= S;
}

/* Joint P (Eq. 3, n := z) of one chunk from its z x z matrix of dissimilarities
 * D (squared Euclidean distances, or any precomputed ones such as graph path
 * lengths): beta_i by the search of orc_row_beta on row i of D (Eq. 1, Eq. 2),
 * conditionals p_{j|i}, then P_ij = (p_{j|i} + p_{i|j}) / (2z).  P is z x z
 * row-major with zero diagonal; beta (optional) has z entries; Pcond (z x z,
 * optional) receives p_{j|i} at [i*z + j].  Returns the number of rows whose
 * search missed the tolerance (>= 0) or a negative error. */
int orc_affinities_from_distances(const double* D, int64_t z, double perp, double tol, int32_t maxit,
                                  double* P, double* beta, double* Pcond) {
    if (!D || !P || z < 2) return ORC_EINVAL;
    double* C = Pcond ? Pcond : (double*)malloc(sizeof(double) * (size_t)(z * z));
    if (!C) return ORC_ENOMEM;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+:bad)
    for (int64_t i = 0; i < z; ++i) {
        double b;
        int r = orc_row_beta(D + i * z, z, i, perp, tol, maxit, &b, NULL, NULL);
        if (r != 0) bad += 1;
        if (beta) beta[i] = b;
        row_conditional(D + i * z, z, i, b, C + i * z);
    }
    const double inv2n = 1.0 / (2.0 * (double)z);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < z; ++i)
        for (int64_t j = 0; j < z; ++j)
            P[i * z + j] = (i == j) ? 0.0 : (C[i * z + j] + C[j * z + i]) * inv2n;
    if (!Pcond) free(C);
    return bad;
}

/* Input affinities of one chunk of z points Xc (z x d; a partial t-SNE:
 * ptSNE section, "threads"), with n := z in Eq. 3: D_ij = ||x_i - x_j||^2 (the
 * input-space similarities of the ptSNE section), then
 * orc_affinities_from_distances on D.  Same outputs and return value. */
int orc_affinities(const double* Xc, int64_t z, int32_t d, double perp,
                   double tol, int32_t maxit, double* P, double* beta,
                   double* Pcond) {
    if (!Xc || !P || z < 2 || d < 1) return ORC_EINVAL;
    double* D = (double*)malloc(sizeof(double) * (size_t)(z * z));
    if (!D) return ORC_ENOMEM;
    orc_sqdist(Xc, z, d, D);
    const int bad = orc_affinities_from_distances(D, z, perp, tol, maxit, P, beta, Pcond);
    free(D);
    return bad;
}

/* Cauchy kernel w_ij = (1 + ||y_i - y_j||^2)^-1 (Eq. 4 numerator). */
static double cauchy(const double* Y, int32_t od, int64_t i, int64_t j) {
    double s = 0.0;
    for (int32_t k = 0; k < od; ++k) {
        double t = Y[i * od + k] - Y[j * od + k];
        s += t * t;
    }
    return 1.0 / (1.0 + s);
}

/* Normaliser of Eq. 4: Z = sum_{k != l} w_kl over ordered pairs. */
double orc_cauchy_Z(const double* Y, int64_t z, int32_t od) {
    double* rows = (double*)malloc(sizeof(double) * (size_t)z);
    if (!rows) return NAN;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < z; ++k) {
        double s = 0.0;
        for (int64_t l = 0; l < z; ++l)
            if (l != k) s += cauchy(Y, od, k, l);
        rows[k] = s;
    }
    double Z = 0.0;
    for (int64_t k = 0; k < z; ++k) Z += rows[k];
    free(rows);
    return Z;
}

/* Exact KL gradient, Eq. 6, as printed:
 *   dC/dy_i = 4 sum_j (p_ij - q_ij) (y_i - y_j) (1 + ||y_i - y_j||^2)^-1
 * with q_ij from Eq. 4.  grad is z x od; Z_out (optional) receives Z. */
int orc_gradient(const double* P, const double* Y, int64_t z, int32_t od,
                 double* grad, double* Z_out) {
    if (!P || !Y || !grad || z < 2 || od < 1) return ORC_EINVAL;
    const double Z = orc_cauchy_Z(Y, z, od);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < z; ++i) {
        for (int32_t k = 0; k < od; ++k) grad[i * od + k] = 0.0;
        for (int64_t j = 0; j < z; ++j) {
            if (j == i) continue;
            double w = cauchy(Y, od, i, j);
            double q = w / Z;
            double c = 4.0 * (P[i * z + j] - q) * w;
            for (int32_t k = 0; k < od; ++k)
                grad[i * od + k] += c * (Y[i * od + k] - Y[j * od + k]);
        }
    }
    if (Z_out) *Z_out = Z;
    return ORC_OK;
}

/* Eq. 6 for selected rows only, for chunks whose z x z P is too large to
 * hold in FP64: grad_r = 4 sum_{j != i} (p_ij - w_ij / Z) w_ij (y_i - y_j)
 * for i = rows[r], with Prows[r * z + j] = p_ij (the rows' P entries) and Z
 * the chunk's normaliser of Eq. 4 (orc_cauchy_Z).  grad is nr x od. */
int orc_gradient_rows(const double* Prows, const int64_t* rows, int64_t nr, const double* Y, int64_t z,
                      int32_t od, double Z, double* grad) {
    if (!Prows || !rows || !Y || !grad || z < 2 || od < 1 || nr < 0 || !(Z > 0.0)) return ORC_EINVAL;
    for (int64_t r = 0; r < nr; ++r)
        if (rows[r] < 0 || rows[r] >= z) return ORC_EINVAL;
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < nr; ++r) {
        const int64_t i = rows[r];
        for (int32_t k = 0; k < od; ++k) grad[r * od + k] = 0.0;
        for (int64_t j = 0; j < z; ++j) {
            if (j == i) continue;
            double w = cauchy(Y, od, i, j);
            double c = 4.0 * (Prows[r * z + j] - w / Z) * w;
            for (int32_t k = 0; k < od; ++k)
                grad[r * od + k] += c * (Y[i * od + k] - Y[j * od + k]);
        }
    }
    return ORC_OK;
}

/* KL(P||Q), Eq. 5, natural log, with 0 log 0 = 0. */
double orc_kl(const double* P, const double* Y, int64_t z, int32_t od) {
    const double Z = orc_cauchy_Z(Y, z, od);
    double* rows = (double*)malloc(sizeof(double) * (size_t)z);
    if (!rows) return NAN;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < z; ++i) {
        double s = 0.0;
        for (int64_t j = 0; j < z; ++j) {
            if (j == i || P[i * z + j] <= 0.0) continue;
            double q = cauchy(Y, od, i, j) / Z;
            s += P[i * z + j] * log(P[i * z + j] / q);
        }
        rows[i] = s;
    }
    double C = 0.0;
    for (int64_t i = 0; i < z; ++i) C += rows[i];
    free(rows);
    return C;
}

/* Pseudo-normalised cost, Eq. 9: -sum p_ij ln q_ij / (ln z + ln(z - 1)). */
double orc_normalized_cost(const double* P, const double* Y, int64_t z, int32_t od) {
    const double Z = orc_cauchy_Z(Y, z, od);
    double* rows = (double*)malloc(sizeof(double) * (size_t)z);
    if (!rows) return NAN;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < z; ++i) {
        double s = 0.0;
        for (int64_t j = 0; j < z; ++j) {
            if (j == i || P[i * z + j] == 0.0) continue;
            s += P[i * z + j] * log(cauchy(Y, od, i, j) / Z);
        }
        rows[i] = s;
    }
    double H = 0.0;
    for (int64_t i = 0; i < z; ++i) H += rows[i];
    free(rows);
    return -H / (log((double)z) + log((double)(z - 1)));
}

/* Embedding size: length of the diagonal of the bounding box of Y (ptSNE
 * section, cost and size monitoring). */
double orc_embedding_size(const double* Y, int64_t n, int32_t od) {
    double s = 0.0;
    for (int32_t k = 0; k < od; ++k) {
        double lo = INFINITY, hi = -INFINITY;
        for (int64_t i = 0; i < n; ++i) {
            double v = Y[i * od + k];
            if (v < lo) lo = v;
            if (v > hi) hi = v;
        }
        s += (hi - lo) * (hi - lo);
    }
    return sqrt(s);
}

#define ORC_LR_FIXED 0
#define ORC_LR_PAPER 1

/* Auto-adaptive learning rate, Eq. 13: eta = ln(z - 1) (Ymax - Ymin) / 2,
 * where Ymax / Ymin are the largest / smallest coordinate of the chunk's map. */
double orc_paper_lr(const double* Y, int64_t z, int32_t od) {
    double lo = INFINITY, hi = -INFINITY;
    for (int64_t i = 0; i < z * od; ++i) {
        if (Y[i] < lo) lo = Y[i];
        if (Y[i] > hi) hi = Y[i];
    }
    return log((double)(z - 1)) * (hi - lo) * 0.5;
}

/* One position update, Eq. 12 read as gradient DESCENT (the paper prints
 * "+eta dC/dY"; the minimisation of Eq. 5 needs the minus sign):
 *   vel <- momentum * vel - eta * gains * grad;  y <- y + vel
 * so that y(t) = y(t-1) - eta g + momentum (y(t-1) - y(t-2)).
 * Gains (not in the paper; the delta-bar-delta rule of the standard t-SNE
 * optimiser): per coordinate, gains += 0.2 when grad and vel have different
 * signs (grad > 0 versus vel > 0), else gains *= 0.8; floor 0.01.
 * eta is `lr` (lr_mode 0) or Eq. 13 evaluated on the current Y (lr_mode 1). */
void orc_update(double* Y, double* vel, double* gains, const double* grad,
                int64_t z, int32_t od, double lr, double momentum,
                int32_t lr_mode, int32_t use_gains) {
    const double eta = (lr_mode == ORC_LR_PAPER) ? orc_paper_lr(Y, z, od) : lr;
    for (int64_t i = 0; i < z * od; ++i) {
        double g = grad[i];
        if (use_gains) {
            int differ = (g > 0.0) != (vel[i] > 0.0);
            gains[i] = differ ? gains[i] + 0.2 : gains[i] * 0.8;
            if (gains[i] < 0.01) gains[i] = 0.01;
        }
        double gm = use_gains ? gains[i] : 1.0;
        vel[i] = momentum * vel[i] - eta * gm * g;
        Y[i] += vel[i];
    }
}

typedef struct {
    double perplexity;
    double lr;
    double momentum;
    int32_t lr_mode;
    int32_t use_gains;
    int32_t iters;
    int32_t epochs;
    double bisect_tol;
    int32_t bisect_maxit;
} orc_params;

/* One partial t-SNE (one chunk, one epoch): affinities of the chunk, then
 * `iters` gradient steps from Yc with velocity 0 and gains 1 (a fresh partial
 * t-SNE per epoch).  Writes P (z x z) if given; kl / ncost (optional) get
 * Eq. 5 and Eq. 9 at the final Yc.  Returns the affinity status. */
int orc_partial_tsne(const double* Xc, int64_t z, int32_t d, int32_t od,
                     const orc_params* prm, double* Yc, double* P_out,
                     double* kl, double* ncost) {
    double* P = P_out ? P_out : (double*)malloc(sizeof(double) * (size_t)(z * z));
    double* g = (double*)malloc(sizeof(double) * (size_t)(z * od));
    double* vel = (double*)calloc((size_t)(z * od), sizeof(double));
    double* gains = (double*)malloc(sizeof(double) * (size_t)(z * od));
    if (!P || !g || !vel || !gains) {
        if (!P_out) free(P);
        free(g); free(vel); free(gains);
        return ORC_ENOMEM;
    }
    for (int64_t i = 0; i < z * od; ++i) gains[i] = 1.0;
    int st = orc_affinities(Xc, z, d, prm->perplexity, prm->bisect_tol,
                            prm->bisect_maxit, P, NULL, NULL);
    if (st >= 0) {
        for (int32_t t = 0; t < prm->iters; ++t) {
            orc_gradient(P, Yc, z, od, g, NULL);
            orc_update(Yc, vel, gains, g, z, od, prm->lr, prm->momentum,
                       prm->lr_mode, prm->use_gains);
        }
        if (kl) *kl = orc_kl(P, Yc, z, od);
        if (ncost) *ncost = orc_normalized_cost(P, Yc, z, od);
    }
    if (!P_out) free(P);
    free(g); free(vel); free(gains);
    return st;
}

/* The ptSNE cycle with layers (ptSNE section, subsections "layers" and
 * "thread-size"): each epoch's permutation and the offsets define T
 * elementary chunks; thread t runs the L chunks t, t+1, ..., t+L-1 (mod T)
 * together, so consecutive threads share L-1 chunks, and every point takes
 * part in L threads.  The point of elementary chunk (t + k) mod T sits in slot
 * k of thread t and reads and writes layer k of the map: Y holds L maps of n
 * points, layer-major (row k n + p).  The threads of an epoch all start from
 * the epoch's maps and never write the same row.  cost: per epoch, the
 * averages over threads.  With layers = 1 this is orc_ptsne_run. */
int orc_ptsne_run_layers(const double* X, int64_t n, int32_t d, int32_t od,
                         const int32_t* perms, const int64_t* offsets, int32_t n_chunks, int32_t layers,
                         const orc_params* prm, double* Y, double* cost) {
    if (!X || !Y || !perms || !offsets || n_chunks < 1 || !prm) return ORC_EINVAL;
    if (layers < 1 || layers > n_chunks) return ORC_EINVAL;
    if (offsets[0] != 0 || offsets[n_chunks] != n) return ORC_EINVAL;
    int bad = 0;
    for (int32_t e = 0; e < prm->epochs; ++e) {
        const int32_t* perm = perms + (int64_t)e * n;
        double kl_sum = 0.0, nc_sum = 0.0;
        for (int32_t t = 0; t < n_chunks; ++t) {
            int64_t z = 0;
            for (int32_t k = 0; k < layers; ++k) {
                const int32_t c = (t + k) % n_chunks;
                z += offsets[c + 1] - offsets[c];
            }
            double* Xc = (double*)malloc(sizeof(double) * (size_t)(z * d));
            double* Yc = (double*)malloc(sizeof(double) * (size_t)(z * od));
            int64_t* row = (int64_t*)malloc(sizeof(int64_t) * (size_t)z);   // row of Y of each thread row
            if (!Xc || !Yc || !row) { free(Xc); free(Yc); free(row); return ORC_ENOMEM; }
            int64_t r = 0;
            for (int32_t k = 0; k < layers; ++k) {
                const int32_t c = (t + k) % n_chunks;
                for (int64_t i = offsets[c]; i < offsets[c + 1]; ++i, ++r) {
                    const int64_t p = perm[i];
                    row[r] = (int64_t)k * n + p;
                    memcpy(Xc + r * d, X + p * d, sizeof(double) * (size_t)d);
                    memcpy(Yc + r * od, Y + row[r] * od, sizeof(double) * (size_t)od);
                }
            }
            double kl = 0.0, nc = 0.0;
            int st = orc_partial_tsne(Xc, z, d, od, prm, Yc, NULL, &kl, &nc);
            if (st < 0) { free(Xc); free(Yc); free(row); return st; }
            bad += st;
            /* the rows this thread writes are read by no other thread */
            for (int64_t q = 0; q < z; ++q)
                memcpy(Y + row[q] * od, Yc + q * od, sizeof(double) * (size_t)od);
            free(Xc); free(Yc); free(row);
            kl_sum += kl;
            nc_sum += nc;
        }
        if (cost) {
            cost[2 * e] = kl_sum / n_chunks;
            cost[2 * e + 1] = nc_sum / n_chunks;
        }
    }
    return bad;
}

/* The ptSNE epoch cycle (ptSNE section, "epochs"): for every epoch e the
 * partition perms[e] (n entries) is cut at `offsets` into n_chunks chunks;
 * each chunk runs a partial t-SNE from its current positions and the results
 * are pooled back into Y (n x od, in/out).  cost (optional, epochs x 2)
 * receives the average over chunks of KL (Eq. 5) and of the pseudo-normalised
 * cost (Eq. 9) at the end of each epoch.  One layer (each point in exactly one
 * chunk per epoch). */
int orc_ptsne_run(const double* X, int64_t n, int32_t d, int32_t od,
                  const int32_t* perms, const int64_t* offsets, int32_t n_chunks,
                  const orc_params* prm, double* Y, double* cost) {
    if (!X || !Y || !perms || !offsets || n_chunks < 1 || !prm) return ORC_EINVAL;
    if (offsets[0] != 0 || offsets[n_chunks] != n) return ORC_EINVAL;
    int bad = 0;
    for (int32_t e = 0; e < prm->epochs; ++e) {
        const int32_t* perm = perms + (int64_t)e * n;
        double kl_sum = 0.0, nc_sum = 0.0;
        for (int32_t c = 0; c < n_chunks; ++c) {
            int64_t o = offsets[c], z = offsets[c + 1] - offsets[c];
            double* Xc = (double*)malloc(sizeof(double) * (size_t)(z * d));
            double* Yc = (double*)malloc(sizeof(double) * (size_t)(z * od));
            if (!Xc || !Yc) { free(Xc); free(Yc); return ORC_ENOMEM; }
            for (int64_t r = 0; r < z; ++r) {
                int64_t src = perm[o + r];
                memcpy(Xc + r * d, X + src * d, sizeof(double) * (size_t)d);
                memcpy(Yc + r * od, Y + src * od, sizeof(double) * (size_t)od);
            }
            double kl = 0.0, nc = 0.0;
            int st = orc_partial_tsne(Xc, z, d, od, prm, Yc, NULL, &kl, &nc);
            if (st < 0) { free(Xc); free(Yc); return st; }
            bad += st;
            for (int64_t r = 0; r < z; ++r)
                memcpy(Y + (int64_t)perm[o + r] * od, Yc + r * od, sizeof(double) * (size_t)od);
            kl_sum += kl;
            nc_sum += nc;
            free(Xc); free(Yc);
        }
        if (cost) {
            cost[2 * e] = kl_sum / n_chunks;
            cost[2 * e + 1] = nc_sum / n_chunks;
        }
    }
    return bad;
}
