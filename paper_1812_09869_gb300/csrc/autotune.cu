// Autotuner of the batched iteration kernel's launch shape: times every
// candidate (blocks per chunk x warps per block; one warp per tile) on the
// caller's chunk layout and keeps the fastest; results persist in a small text
// cache keyed by device and layout.  Under BF16_WINDOW it first chooses the
// form of the distances (ptsne_set_form_threshold) by timing the affinities
// with every chunk in each form on the caller's data.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "ptsne_internal.cuh"

using namespace ptsne;

namespace ptsne {
cudaError_t launch_gather_y(const ptsne_ctx* c, const float* Y, const int32_t* perm, float* Yc, cudaStream_t s);
}

namespace {

// Key of a tuning record: the device and everything of the layout that the
// kernel's speed depends on.
std::string tune_key(const ptsne_ctx* c) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) prop.name[0] = 0;
    long double z2 = 0;
    for (int k = 0; k < c->p.n_chunks; ++k) {
        const long double z = (long double)(c->off[k + 1] - c->off[k]);
        z2 += z * z;
    }
    char buf[512];
    std::string name(prop.name);
    for (char& ch : name)
        if (ch == ' ' || ch == '|') ch = '_';
    snprintf(buf, sizeof buf, "%s|sm%d|od%d|chunks%d|zmin%lld|zmax%lld|z2_%.4Le", name.c_str(), sms, c->p.out_dim,
             c->p.n_chunks, (long long)c->zmin, (long long)c->zmax, z2);
    return buf;
}

bool cache_lookup(const char* path, const std::string& key, IterTune* out) {
    FILE* f = fopen(path, "r");
    if (!f) return false;
    char line[1024];
    bool found = false;
    while (fgets(line, sizeof line, f)) {
        char k[600];
        int cl = 0, g = 0, w = 0;
        // records of launch shapes the kernel no longer has are skipped
        if (sscanf(line, "%599s %d %d %d", k, &cl, &g, &w) == 4 && key == k && (cl == 1 || cl == 2 || cl == 4) &&
            g == 1 && w >= 1 && w <= 20) {
            out->cluster = cl;
            out->group = g;
            out->consumer_warps = w;
            found = true;  // the last matching record wins
        }
    }
    fclose(f);
    return found;
}

void cache_append(const char* path, const std::string& key, const IterTune& t, double ms) {
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d %d %d %.6f\n", key.c_str(), t.cluster, t.group, t.consumer_warps, ms);
    fclose(f);
}

}  // namespace

extern "C" int ptsne_affinities(ptsne_ctx* c, const float* X, const int32_t* perm, float* P_out, float* beta_out,
                                void* stream);
extern "C" int ptsne_set_form_threshold(ptsne_ctx* c, double threshold);

namespace {

// Mixed-precision form choice.  With every chunk in the mixed form the
// affinities take Tm, of which Tw is the window recompute of a measured
// window fraction f; with every chunk in FP32 whole they take Tf.  Taking the
// recompute as proportional to the window fraction, a chunk of fraction f
// costs (Tm - Tw) + Tw f / f_meas mixed and Tf in FP32 (per unit of z^2), so
// the mixed form pays below f* = f_meas (Tf - Tm + Tw) / Tw.  Each time is
// the faster of two runs after one untimed run.  On the batched schedule the
// mixed form is timed with the locality order off and on (it gathers a dense
// row's window pairs on few tiles), and the faster setting is kept.
int tune_form(ptsne_ctx* c, const float* X, const int32_t* perm, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
    auto timed = [&](double fstar, double* ms) {
        int st = ptsne_set_form_threshold(c, fstar);
        if (st == PTSNE_OK) st = ptsne_affinities(c, X, perm, nullptr, nullptr, s);   // untimed: fills the bins
        float best = 1e30f;
        for (int rep = 0; rep < 2 && st == PTSNE_OK; ++rep) {
            cudaEventRecord(e0, s);
            st = ptsne_affinities(c, X, perm, nullptr, nullptr, s);
            cudaEventRecord(e1, s);
            if (st == PTSNE_OK && cudaEventSynchronize(e1) != cudaSuccess) st = PTSNE_ECUDA;
            float t = 0.f;
            if (st == PTSNE_OK) cudaEventElapsedTime(&t, e0, e1);
            best = t < best ? t : best;
        }
        *ms = best;
        return st;
    };
    double tm = 0, tf = 0;
    const bool user_loc = c->locality;
    int st = PTSNE_OK;
    if (c->p.schedule == PTSNE_SCHED_BATCHED) {
        double tl[2] = {0, 0};
        for (int loc = 0; loc < 2 && st == PTSNE_OK; ++loc) {
            c->locality = loc != 0;
            st = timed(2.0, &tl[loc]);
        }
        c->locality = tl[1] < tl[0];
        tm = tl[1];
        // the window recompute is timed below on the state of the last run: the kept setting's
        if (st == PTSNE_OK && !c->locality) st = timed(2.0, &tm);
    } else {
        st = timed(2.0, &tm);
    }
    if (st != PTSNE_OK) {
        c->locality = user_loc;
        return st;
    }
    // the window fraction of the last (mixed) run, before the next one consumes it
    unsigned long long acc[2 * kFormBins];
    if (cudaMemcpy(acc, c->form_acc, sizeof acc, cudaMemcpyDeviceToHost) != cudaSuccess) return PTSNE_ECUDA;
    double w = 0, nrow = 0, fmin = 2.0;
    for (int b = 0; b < kFormBins; ++b) {
        w += (double)acc[2 * b];
        nrow += (double)acc[2 * b + 1];
        if (acc[2 * b + 1]) fmin = std::min(fmin, (double)acc[2 * b] / (double)acc[2 * b + 1]);
    }
    const double fmeas = nrow > 0 ? w / nrow : 0.0;
    // the window recompute alone, on the state the last run left
    float tw = 1e30f;
    for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(e0, s);
        const cudaError_t e = launch_window_recompute(c, 0, c->p.n, s);
        cudaEventRecord(e1, s);
        if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return PTSNE_ECUDA;
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        tw = t < tw ? t : tw;
    }
    const bool loc_mixed = c->locality;
    c->locality = user_loc;   // FP32 whole gains nothing from the order
    st = timed(-1.0, &tf);
    if (st != PTSNE_OK) return st;
    double fstar;
    if (tf <= tm - tw) fstar = -1.0;                  // FP32 whole is faster even with no window at all
    else if (tw <= 0.0 || fmeas <= 0.0) fstar = tf < tm ? -1.0 : 2.0;
    else fstar = fmeas * (tf - tm + tw) / tw;
    if (fstar > 1.0) fstar = 2.0;
    // every measured size bin on the FP32 side: the plain FP32 path (no Gram
    // matrix, coarse search or window launches at all)
    if (fstar <= fmin) fstar = -1.0;
    if (fstar > 0.0) c->locality = loc_mixed;   // some chunks may run mixed
    c->form_ms[0] = tm;
    c->form_ms[1] = tf;
    c->form_ms[2] = tw;
    return ptsne_set_form_threshold(c, fstar);
}

}  // namespace

extern "C" int ptsne_autotune_form(ptsne_ctx* c, const float* X, const int32_t* perm, void* stream) {
    if (!c) return PTSNE_EINVAL;
    if (!X || !perm) {
        c->err = "autotune_form: X and perm must be device pointers";
        return PTSNE_EINVAL;
    }
    if (!c->form_fstar) {
        c->err = "autotune_form: the distances' form needs PTSNE_PREC_BF16_WINDOW";
        return PTSNE_EINVAL;
    }
    cudaEvent_t f0 = nullptr, f1 = nullptr;
    int st = cudaEventCreate(&f0) == cudaSuccess && cudaEventCreate(&f1) == cudaSuccess ? PTSNE_OK : PTSNE_ECUDA;
    if (st == PTSNE_OK) st = tune_form(c, X, perm, reinterpret_cast<cudaStream_t>(stream), f0, f1);
    if (f0) cudaEventDestroy(f0);
    if (f1) cudaEventDestroy(f1);
    return st;
}

extern "C" int ptsne_autotune(ptsne_ctx* c, const float* X, const int32_t* perm, const float* Y, int32_t iters,
                              const char* cache_path, ptsne_tune_trial* trials, int32_t max_trials, int32_t* n_trials,
                              void* stream) {
    if (!c) return PTSNE_EINVAL;
    if (n_trials) *n_trials = 0;
    if (!X || !perm || !Y || iters < 1) {
        c->err = "autotune: X, perm, Y must be device pointers and iters >= 1";
        return PTSNE_EINVAL;
    }
    if (c->p.schedule != PTSNE_SCHED_BATCHED) {
        c->err = "autotune: only the batched schedule has launch shapes to tune";
        return PTSNE_EINVAL;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (c->form_fstar) {   // BF16_WINDOW: the distances' form first
        const int st = ptsne_autotune_form(c, X, perm, stream);
        if (st != PTSNE_OK) return st;
    }
    const std::string key = tune_key(c);
    IterTune cached;
    if (cache_path && cache_lookup(cache_path, key, &cached)) {
        c->tune = cached;
        return ptsne_affinities(c, X, perm, nullptr, nullptr, stream);
    }
    int st = ptsne_affinities(c, X, perm, nullptr, nullptr, stream);
    if (st != PTSNE_OK) return st;
    const size_t m = (size_t)c->p.n * c->p.out_dim;
    float *y0 = nullptr, *v0 = nullptr, *g0 = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&]() {
        if (y0) cudaFree(y0);
        if (v0) cudaFree(v0);
        if (g0) cudaFree(g0);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    auto cuda_fail = [&](cudaError_t e) {
        c->err = std::string("autotune: ") + cudaGetErrorString(e);
        cleanup();
        return PTSNE_ECUDA;
    };
    cudaError_t e;
    if ((e = cudaMalloc(&y0, m * sizeof(float))) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaMalloc(&v0, m * sizeof(float))) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaMalloc(&g0, m * sizeof(float))) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) return cuda_fail(e);
    const int32_t* vperm = virtual_perm(c, perm, s, &e);   // the thread rows' permutation (layers)
    if (e != cudaSuccess) return cuda_fail(e);
    if ((e = launch_gather_y(c, Y, vperm, c->Yc, s)) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaMemcpyAsync(y0, c->Yc, m * sizeof(float), cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return cuda_fail(e);
    if ((e = cudaMemcpyAsync(v0, c->vel, m * sizeof(float), cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return cuda_fail(e);
    if ((e = cudaMemcpyAsync(g0, c->gains, m * sizeof(float), cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return cuda_fail(e);
    auto restore = [&]() {
        cudaMemcpyAsync(c->Yc, y0, m * sizeof(float), cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(c->vel, v0, m * sizeof(float), cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(c->gains, g0, m * sizeof(float), cudaMemcpyDeviceToDevice, s);
    };

    const IterTune keep = c->tune;
    IterTune best = keep;
    double best_ms = 1e300;
    int nt = 0;
    // warps per block: the 2-D evaluation runs with at most 16
    const int clusters[] = {1, 2, 4}, groups[] = {1};
    const int warps2[] = {8, 12, 16}, warps3[] = {12, 17, 20, 21};
    const bool two_d = c->p.out_dim == 2;
    const int nwarps = two_d ? 3 : 4;
    for (int cl : clusters)
        for (int g : groups)
            for (int wi = 0; wi < nwarps; ++wi) {
                const int w = two_d ? warps2[wi] : warps3[wi];
                c->tune = IterTune{cl, g, w};
                double ms = 1e300;
                for (int rep = 0; rep < 2; ++rep) {
                    restore();
                    cudaEventRecord(e0, s);
                    e = launch_iterate(c, iters, 0, nullptr, nullptr, nullptr, s);
                    cudaEventRecord(e1, s);
                    if (e != cudaSuccess) break;
                    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
                    float t = 0.f;
                    cudaEventElapsedTime(&t, e0, e1);
                    ms = t / iters < ms ? t / iters : ms;
                }
                if (e != cudaSuccess) {
                    // a shape that cannot launch here (e.g. cluster occupancy) is skipped
                    cudaGetLastError();
                    continue;
                }
                if (trials && nt < max_trials) {
                    trials[nt].tuning.cluster = cl;
                    trials[nt].tuning.group = g;
                    trials[nt].tuning.consumer_warps = w;
                    trials[nt].ms_per_iter = ms;
                }
                ++nt;
                if (ms < best_ms) {
                    best_ms = ms;
                    best = c->tune;
                }
            }
    restore();
    cudaStreamSynchronize(s);
    DeviceStats h;
    cudaMemcpy(&h, c->dstats, sizeof h, cudaMemcpyDeviceToHost);
    cleanup();
    if (h.timeouts) {
        c->tune = keep;
        c->err = "autotune: a bounded device wait ran out";
        return PTSNE_ETIMEOUT;
    }
    if (nt == 0) {
        c->tune = keep;
        c->err = "autotune: no launch shape could run";
        return PTSNE_ECUDA;
    }
    c->tune = best;
    if (n_trials) *n_trials = nt;
    if (cache_path) cache_append(cache_path, key, best, best_ms);
    // leave a fresh optimiser state for the caller's next step / run
    cudaError_t er = launch_reset_optim(c, s);
    return er == cudaSuccess ? PTSNE_OK : PTSNE_ECUDA;
}
