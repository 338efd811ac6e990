#!/usr/bin/env python3
"""ptSNE benchmark: point-iterations/s on the uneven-chunk workload
(N = 1,000,000 points, D = 64, chunk sizes drawn U[1000, 5000], perplexity 30,
100 gradient iterations per epoch, 2-D map), one step = one ptSNE epoch
(partition gather, distances, perplexity search, joint P, all gradient
iterations of every chunk, pooling, cost evaluation).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With --gpus N > 1 (launched by
torch.distributed.run) every rank runs its own replica of the workload (weak
scaling, no collective on the data path); the timed region is bracketed by a
barrier and the slowest rank's time is reported.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ptSNE point-iterations/s at N=1M, D=64 vs plain FP32 GPU; % of roofline"
UNIT = "point-iter/s"
WORKLOAD = "uneven-1m-d64"
PERM_POOL = 4          # distinct epoch partitions cycled through the steps
DOMINANT = "iterate_kernel"


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--precision", choices=["fp32", "bf16_window"], default=None,
                    help="distance precision (default: the workload's own)")
    ap.add_argument("--no-plain", action="store_true",
                    help="skip the comparison of forms (plain FP32, batched, mixed precision, learned)")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned (mapper) form")
    ap.add_argument("--no-eq13", action="store_true", help="skip the Eq. 13 study (adaptive vs fixed learning rate)")
    ap.add_argument("--mapper-kernels", type=int, default=0, metavar="ROWS",
                    help="only time the mapper's kernels: inference of ROWS points (one launch) and training "
                         "epochs over them (batch 4096); prints one JSON line")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the oracle CPU sample")
    ap.add_argument("--tuning", default=None,
                    help="fixed launch shape 'cluster,group,warps' of the iteration kernel, group 1 (skips the autotuner)")
    ap.add_argument("--form", default=None, metavar="THRESHOLD[,LOCALITY]",
                    help="BF16_WINDOW: fixed distance-form threshold (a chunk whose window fraction is >= it runs in "
                         "FP32 whole; 2 = every chunk mixed) and locality order 0/1, instead of ptsne_autotune_form "
                         "(for profiling runs, whose timings the profiler distorts)")
    return ap.parse_args(argv)


# ----------------------------------------------------------------- distributed helpers

def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def dist_init(world: int, backend: str):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(x: float, world: int) -> float:
    """Max of a per-rank scalar over all ranks (identity for one rank)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(units_per_rank: float, seconds_per_rank: float, world: int) -> tuple[float, float]:
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    t = reduce_max(seconds_per_rank, world)
    return units_per_rank * world / t, t


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(s):
            try:
                return float(s)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((num(r[3]) or 0.0) for r in rows)}


# ----------------------------------------------------------------- roofline bookkeeping

def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": d["hbm_gbs"], "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


def algorithmic_iterate_bytes(sizes: np.ndarray, iters: int) -> float:
    """Minimum DRAM bytes of one launch of the iteration kernel: the symmetric
    FP32 joint P read once per iteration (z (z - 1) / 2 stored pairs x 4 B per
    chunk); map, velocity and gains are O(z) per chunk and are neglected."""
    z = sizes.astype(np.float64)
    return float(iters * np.sum(z * (z - 1) / 2 * 4.0))


def recorded_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from a committed ncu summary, if the kernel source
    it was taken on is unchanged (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    rec = json.load(open(p)).get(f"{kernel}@{workload}")
    if not rec:
        return None
    src = os.path.join(ROOT, "paper_1812_09869_gb300", "csrc", rec["source"])
    if not os.path.exists(src) or hashlib.sha1(open(src, "rb").read()).hexdigest() != rec["source_sha1"]:
        return None
    return float(rec["bytes_per_launch"])


# ----------------------------------------------------------------- CPU baseline (the oracle)

def oracle_sample(w, seconds: float, max_chunks: int = 64):
    """Time the FP64 oracle on whole chunks of epoch 0 (affinities, all
    iterations, cost) until `seconds` of CPU time have been spent."""
    from oracle import oracle as O
    prm = O.params(perplexity=w.perplexity, lr=w.lr, momentum=w.momentum, iters=w.iters, epochs=1)
    perm = w.perms[0]
    units, spent, chunks = 0, 0.0, 0
    for c in range(min(max_chunks, len(w.offsets) - 1)):
        idx = perm[w.offsets[c]:w.offsets[c + 1]]
        t0 = time.perf_counter()
        O.partial_tsne(w.X[idx], w.Y0[idx], prm)
        spent += time.perf_counter() - t0
        units += len(idx) * w.iters
        chunks += 1
        if spent >= seconds:
            break
    return {"value": units / spent, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
            "sample": f"{chunks} chunk(s) of epoch 0 ({units // w.iters} points), affinities + {w.iters} "
                      f"iterations + cost each, FP64 C with OpenMP over rows; {spent:.1f} s"}


# ----------------------------------------------------------------- forms of the method

def _timed_epochs(ctx, Xd, perm_rows, Y, stream, record=None):
    """Run one epoch per partition row, timing all of them with CUDA events;
    returns (seconds, avg KL after each epoch).  record (optional list)
    receives per epoch {ms, kl, size} and the search counters."""
    import torch
    kls = []
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    secs = 0.0
    for pr in perm_rows:
        cost = np.zeros((1, 3))
        a.record(stream)
        ctx.run(Xd, pr, 1, Y, cost_out=cost)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        secs += ms / 1000.0
        kls.append(float(cost[0, 0]))
        if record is not None:
            st = ctx.stats()
            record.append({"ms": ms, "kl": float(cost[0, 0]), "size": float(cost[0, 2]),
                           "window_pairs": int(st.window_pairs), "fp64_rows": int(st.bisect_fp64_rows),
                           "max_abs_entropy_err": float(st.max_abs_entropy_err)})
    return secs, kls


def compare_forms(w, Xd, perms, dev, stream, tuning):
    """Plain FP32 (per-chunk launches, FP32 SIMT distances, dense P), batched
    FP32, batched mixed precision, and batched mixed precision with the
    paper's Eq. 13 learning rate, each running the same two epochs
    (partitions 0 and 1) from the same start map; the second epoch is timed
    and the final KL compared."""
    import torch
    from paper_1812_09869_gb300 import ptsne
    # "form": how the mixed-precision contexts pick each chunk's distance form
    # ("auto": ptsne_autotune_form; "all_mixed": BF16 Gram + window for every chunk)
    kinds = {"plain_fp32": dict(precision="fp32", schedule="per_chunk", use_graph=0),
             "batched_fp32": dict(precision="fp32", schedule="batched", use_graph=1),
             # fixed-point accumulators: bitwise repeatable (fewer warps on the largest chunks)
             "batched_fp32_deterministic": dict(precision="fp32", schedule="batched", use_graph=1, det=True),
             "batched_bf16_window": dict(precision="bf16_window", schedule="batched", use_graph=1, form="auto"),
             "batched_bf16_window_all_mixed": dict(precision="bf16_window", schedule="batched", use_graph=1,
                                                   form="all_mixed"),
             # the paper's own update: adaptive learning rate of Eq. 13, no gains
             "batched_bf16_window_lr_eq13": dict(precision="bf16_window", schedule="batched", use_graph=1,
                                                 lr_mode=ptsne.LR_PAPER, use_gains=0, form="auto")}
    out = {}
    for name, kw in kinds.items():
        kw = dict(kw)
        form = kw.pop("form", None)
        det = kw.pop("det", False)
        cfg = ptsne.Config(n=w.n, d=w.d, offsets=w.offsets, perplexity=w.perplexity, iters=w.iters, lr=w.lr,
                           momentum=w.momentum, **kw)
        with ptsne.Context(cfg) as c:
            if kw["schedule"] == "batched":
                c.set_tuning(*tuning)
            if det:
                c.set_deterministic(True)
            if form == "auto":
                c.autotune_form(Xd, perms[0])
            frec = c.form_record() if form else None
            Y = torch.from_numpy(w.Y0.copy()).to(dev)
            _timed_epochs(c, Xd, [perms[0]], Y, stream)
            rec = []
            secs, kls = _timed_epochs(c, Xd, [perms[1]], Y, stream, record=rec)
            if frec is not None:
                frec["fp32_chunks_per_epoch"] = int(c.stats().fp32_chunks)
        out[name] = {"value": w.n * w.iters / secs, "unit": UNIT, "ms_per_epoch": secs * 1e3,
                     "final_kl_after_2_epochs": kls[-1], "window_pairs_per_epoch": rec[-1]["window_pairs"],
                     "fp64_rows_per_epoch": rec[-1]["fp64_rows"],
                     "max_abs_entropy_err": rec[-1]["max_abs_entropy_err"], **kw}
        if form:
            out[name]["form"] = form
            out[name]["distance_form"] = frec
        if det:
            out[name]["deterministic"] = True
    base = out["plain_fp32"]
    for name, r in out.items():
        r["speedup_vs_plain"] = r["value"] / base["value"]
        r["kl_rel_diff_vs_plain"] = abs(r["final_kl_after_2_epochs"] - base["final_kl_after_2_epochs"]) / \
            base["final_kl_after_2_epochs"]
    return out


def knn_block(X, maps: dict, k: int = 10, nq: int = 1000, seed: int = 705) -> dict:
    """k-NN preservation (ptsne_knn_preservation on the GPU) of each map on
    one seeded sample of nq query points."""
    import torch
    from paper_1812_09869_gb300 import ptsne
    n = int(X.shape[0])
    q = torch.from_numpy(np.random.default_rng(seed).choice(n, nq, replace=False).astype(np.int32)).to(X.device)
    out = {"k": k, "queries": nq}
    for name, Y in maps.items():
        ov = torch.zeros(nq, dtype=torch.int32, device=X.device)
        ptsne.knn_preservation(X, Y, q, k, ov)
        torch.cuda.synchronize()
        out[name] = float(ov.double().mean().item() / k)
    return out


def learned_form(dev, stream, train_epochs=10, mapper_epochs=20, warm_iters=25, max_warm_epochs=16):
    """The learned form on the 1M + 1M, D = 50 mixture: ptSNE maps the training
    half, the mapper is trained on that map and places the held-out half, and
    the library's warm start (one epoch from the placement against one from
    the random start, plain ptSNE keeping the better) is continued until it
    reaches the KL that the full schedule (train_epochs x 100 iterations) from
    the random start reaches.  10-NN preservation of the mapper's placement,
    the warm map and the cold map on 1000 sampled held-out points."""
    import torch
    from paper_1812_09869_gb300 import mapper as M
    from paper_1812_09869_gb300 import ptsne, synth
    w = synth.workload("mapper-1m+1m-d50", epochs=train_epochs)
    half = w.n // 2
    Xtr = torch.from_numpy(np.ascontiguousarray(w.X[:half])).to(dev)
    Xte = torch.from_numpy(np.ascontiguousarray(w.X[half:])).to(dev)
    perms_tr = torch.from_numpy(w.perms).to(dev)
    perms_te = torch.from_numpy(synth.permutations(half, max(max_warm_epochs, train_epochs), seed=405)).to(dev)

    def ctx(iters):
        return ptsne.Context(ptsne.Config(n=half, d=w.d, offsets=w.offsets, perplexity=w.perplexity, iters=iters,
                                          lr=w.lr, momentum=w.momentum))

    with ctx(w.iters) as c:
        Ytr = torch.from_numpy(w.Y0.copy()).to(dev)
        t_ptsne_tr, kl_tr = _timed_epochs(c, Xtr, [perms_tr[e] for e in range(train_epochs)], Ytr, stream)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    Yrand = torch.from_numpy(synth.init_gaussian(half, 2, 1e-4, seed=705)).to(dev)
    m = M.Mapper(w.d, synth.mlp_init(w.d, 2, seed=505), batch=4096)
    orders = torch.from_numpy(synth.permutations(half, mapper_epochs, seed=605)).to(dev)
    split = m.autotune(Xtr, Ytr, orders[0][:4096].contiguous())   # split-K of the weight gradients
    t0 = time.perf_counter()
    m.fit_scaler(Ytr)
    loss = m.train(Xtr, Ytr, orders, mapper_epochs)
    t_train = time.perf_counter() - t0
    Ymap = torch.zeros((half, 2), dtype=torch.float32, device=dev)
    m.infer(Xte, Ymap)   # warm-up
    a.record(stream)
    m.infer(Xte, Ymap)
    b.record(stream)
    torch.cuda.synchronize()
    t_infer = a.elapsed_time(b) / 1000.0
    with ctx(w.iters) as c:
        Yc = Yrand.clone()
        t_cold, kl_cold = _timed_epochs(c, Xte, [perms_te[e] for e in range(train_epochs)], Yc, stream)
    target = kl_cold[-1]
    with ctx(warm_iters) as c:
        Yw = torch.zeros((half, 2), dtype=torch.float32, device=dev)
        t0 = time.perf_counter()
        used, kl_w0, kl_c0 = m.warm_start(c, Xte, perms_te[0], Yrand, Yw)   # includes the inference
        t_ws = time.perf_counter() - t0
        t_warm, kls = 0.0, [min(kl_w0, kl_c0)]
        for e in range(1, max_warm_epochs):
            if kls[-1] <= target:
                break
            t, k = _timed_epochs(c, Xte, [perms_te[e]], Yw, stream)
            t_warm += t
            kls += k
    m.close()
    reached = kls[-1] <= target
    knn = knn_block(Xte, {"mapper": Ymap, "warm": Yw, "cold": Yc})
    return {"workload": "mapper-1m+1m-d50", "mlp": "50-256-256-2 GELU, BF16 tcgen05, AdamW",
            "train_ptsne": {"epochs": train_epochs, "iters": train_epochs * w.iters, "seconds": t_ptsne_tr,
                            "final_kl": kl_tr[-1]},
            "mapper_train": {"epochs": mapper_epochs, "batch": 4096, "seconds": t_train, "split_k": split,
                             "loss_first_last": [float(loss[0]), float(loss[-1])]},
            "mapper_infer": {"points": half, "seconds": t_infer, "points_per_s": half / t_infer},
            "cold": {"iters": train_epochs * w.iters, "seconds": t_cold, "final_kl": target},
            "warm": {"iters": warm_iters * len(kls), "seconds_incl_infer": t_ws + t_warm,
                     "warm_start": {"mapper_placement_kl_after_1_epoch": kl_w0, "random_start_kl_after_1_epoch": kl_c0,
                                    "seconds": t_ws},
                     "kl_per_epoch": kls, "reached_cold_kl": reached},
            "fallback_used": not used, "knn": knn,
            "speedup_at_equal_kl": (t_cold / (t_ws + t_warm)) if reached else None}


def eq13_study(w, Xd, dev, stream, tuning, ref_epochs=10, epochs=24):
    """The paper's auto-adaptive learning rate (Eq. 13, no gains) against the
    fixed rate with gains, both from the paper's start in the disk of radius
    1, each for `epochs` epochs.  Each form's target is the other's KL after
    ref_epochs; a form reaches it at the first epoch from which its KL stays
    at or below the target for the rest of the run (a run's first epoch can
    sit deceptively low: every chunk relaxes on its own from the disk, and the
    pooled map only becomes consistent over later epochs)."""
    import torch
    from paper_1812_09869_gb300 import ptsne, synth
    perms = torch.from_numpy(synth.permutations(w.n, epochs, seed=903)).to(dev)
    Y0 = synth.init_disk(w.n, seed=904)
    forms = {"fixed_lr_gains": dict(lr_mode=ptsne.LR_FIXED, use_gains=1),
             "eq13_lr": dict(lr_mode=ptsne.LR_PAPER, use_gains=0)}
    recs = {}
    for name, kw in forms.items():
        cfg = ptsne.Config(n=w.n, d=w.d, offsets=w.offsets, perplexity=w.perplexity, iters=w.iters, lr=w.lr,
                           momentum=w.momentum, precision=w.precision, schedule="batched", **kw)
        with ptsne.Context(cfg) as c:
            c.set_tuning(*tuning)
            if w.precision == "bf16_window":
                c.autotune_form(Xd, perms[0])
            Y = torch.from_numpy(Y0.copy()).to(dev)
            rec = []
            _timed_epochs(c, Xd, [perms[e] for e in range(epochs)], Y, stream, record=rec)
            recs[name] = rec
    out = {"init": "disk of radius 1", "epochs": epochs, "ref_epochs": ref_epochs, "iters_per_epoch": w.iters}
    names = list(forms)
    for me, other in ((names[0], names[1]), (names[1], names[0])):
        target = recs[other][ref_epochs - 1]["kl"]
        kl = [r["kl"] for r in recs[me]]
        hit = None
        for e in range(len(kl) - 1, -1, -1):
            if kl[e] > target:
                break
            hit = e
        out[me] = {"kl_per_epoch": kl, "size_per_epoch": [r["size"] for r in recs[me]],
                   "ms_per_epoch": float(np.mean([r["ms"] for r in recs[me]])),
                   "target_kl": target, "target_from": f"{other} after {ref_epochs} epochs",
                   "epochs_to_target": (hit + 1) if hit is not None else None,
                   "seconds_to_target": (sum(r["ms"] for r in recs[me][:hit + 1]) / 1e3) if hit is not None else None}
    return out


def mapper_kernels(rows: int, dev, stream, reps: int = 5, train_epochs: int = 2) -> dict:
    """The learned mapper's kernels alone (MLP 50-256-256-2): inference of
    `rows` points of the D = 50 mixture in one launch, timed over `reps` calls
    after one warm-up call, and `train_epochs` training epochs over them."""
    import torch
    from paper_1812_09869_gb300 import mapper as M
    from paper_1812_09869_gb300 import synth
    X, _ = synth.gaussian_mixture(rows, 50, 20, seed=5, anisotropic=True)
    Xd = torch.from_numpy(X).to(dev)
    T = torch.from_numpy(synth.init_gaussian(rows, 2, 5.0, seed=6)).to(dev)
    Y = torch.zeros((rows, 2), dtype=torch.float32, device=dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with M.Mapper(50, synth.mlp_init(50, 2, seed=7), batch=4096, infer_rows=rows) as m:
        m.fit_scaler(T)
        m.infer(Xd, Y)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(reps):
            m.infer(Xd, Y)
        b.record(stream)
        torch.cuda.synchronize()
        t_inf = a.elapsed_time(b) / reps / 1e3
        orders = torch.from_numpy(synth.permutations(rows, train_epochs, seed=10)).to(dev)
        a.record(stream)
        m.train(Xd, T, orders, train_epochs)
        b.record(stream)
        torch.cuda.synchronize()
        t_tr = a.elapsed_time(b) / 1e3
    flop = 2.0 * rows * (64 * 256 + 256 * 256 + 256 * 2)   # K padded to 64 in layer 1
    steps = train_epochs * (rows // 4096)
    return {"metric": "mapper inference points/s", "value": rows / t_inf, "unit": "points/s",
            "infer_ms": t_inf * 1e3, "infer_tflops": flop / t_inf / 1e12,
            "train_us_per_step": t_tr / steps * 1e6, "train_steps": steps, "batch": 4096,
            "config": {"mlp": "50-256-256-2 GELU, BF16 tcgen05", "rows": rows}}


# ----------------------------------------------------------------- our arm

def bench_ours(args, rank, world, local_rank):
    import torch
    from paper_1812_09869_gb300 import build as pbuild
    from paper_1812_09869_gb300 import ptsne, synth

    if rank == 0:
        pbuild.build()
    barrier(world)
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = synth.workload(args.workload, epochs=PERM_POOL)
    sizes = np.diff(w.offsets)
    precision = args.precision or w.precision
    cfg = ptsne.Config(n=w.n, d=w.d, offsets=w.offsets, perplexity=w.perplexity, iters=w.iters, lr=w.lr,
                       momentum=w.momentum, precision=precision, schedule="batched")
    ctx = ptsne.Context(cfg)
    Xd = torch.from_numpy(w.X).to(dev)
    perms = torch.from_numpy(w.perms).to(dev)
    Y = torch.from_numpy(w.Y0.copy()).to(dev)
    cost = np.zeros((1, 3))
    stream = torch.cuda.current_stream()

    def epochs_from(k0, count):
        """Partitions of steps k0 .. k0 + count - 1 (cycling through the pool), contiguous."""
        return torch.stack([perms[(k0 + k) % PERM_POOL] for k in range(count)]).contiguous()

    # launch shape of the iteration kernel (and, under BF16_WINDOW, the form of
    # the distances), chosen by the library's autotuner
    if args.tuning:
        if precision == "bf16_window":
            if args.form:
                f = args.form.split(",")
                ctx.set_form_threshold(float(f[0]))
                ctx.set_locality_order(len(f) > 1 and f[1] == "1")
            else:
                ctx.autotune_form(Xd, perms[0])
        ctx.set_tuning(*[int(v) for v in args.tuning.split(",")])
        trials = []
    else:
        trials = ctx.autotune(Xd, perms[0], Y, iters=3)
    tuning = ctx.tuning()
    form = ctx.form_record() if precision == "bf16_window" else None
    # profiling marks are part of the captured epoch graph: turn them on before
    # the warm-up steps so that the timed steps replay the same graph
    ctx.set_profiling(True)
    warm_perms, timed_perms = epochs_from(0, args.warmup), epochs_from(args.warmup, args.steps)
    ctx.run(Xd, warm_perms, args.warmup, Y, cost_out=np.zeros((args.warmup, 3)))
    cost = np.zeros((args.steps, 3))
    ctx.reset_counters()
    sampler = ClockSampler(local_rank)
    torch.cuda.synchronize()
    barrier(world)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    # the K timed steps are K epochs of one ptsne_run call (each epoch's
    # perplexity search starts from the previous epoch's precisions)
    ctx.run(Xd, timed_perms, args.steps, Y, cost_out=cost)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop()
    ctx.set_profiling(False)
    secs = e0.elapsed_time(e1) / 1000.0
    st = ctx.stats()
    launches = int(st.kernel_launches)
    stages = {name: (st.stage_ms[k] / st.stage_calls[k] if st.stage_calls[k] else None)
              for k, name in enumerate(ptsne.STAGES)}
    # search counters of the timed call, per epoch
    if form is not None:
        form["fp32_chunks_per_epoch"] = st.fp32_chunks / args.steps
    search = {"evals_per_row": st.bisect_evals / w.n / args.steps,
              "fp64_rows_per_epoch": st.bisect_fp64_rows / args.steps,
              "failed_rows": int(st.bisect_failed_rows), "window_pairs_per_epoch": st.window_pairs / args.steps,
              "max_abs_entropy_err": st.max_abs_entropy_err}
    units = float(w.n * w.iters * args.steps)
    value, tmax = aggregate(units, secs, world)
    final_cost = cost[-1].tolist()

    # dominant kernel: one persistent launch per epoch runs every iteration
    it_ms = stages["iterate"]
    peaks = measured_peaks()
    # the launch also runs the per-epoch cost pass over P: iters + 1 passes
    alg = algorithmic_iterate_bytes(sizes, w.iters + 1)
    achieved = alg / (it_ms / 1000.0) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": recorded_traffic(DOMINANT, args.workload),
                "kernel": DOMINANT, "kernel_ms": it_ms, "algorithmic_bytes": alg,
                "peak_source": peaks["source"]}

    # end to end through the public API on host buffers (copies inside the timed region)
    Xh = torch.from_numpy(w.X).pin_memory()
    Ph = torch.from_numpy(w.perms).pin_memory()
    Yh = torch.from_numpy(w.Y0.copy()).pin_memory()
    cost = np.zeros((1, 3))
    ctx.run_host(Xh, Ph[0], 1, Yh)   # first call allocates the staging buffers
    e2e_steps = max(1, min(args.steps, 3))
    barrier(world)
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        ctx.run_host(Xh, Ph[k % PERM_POOL], 1, Yh, cost_out=cost)
    t_e2e = time.perf_counter() - t0
    e2e_value, _ = aggregate(float(w.n * w.iters * e2e_steps), t_e2e, world)
    e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(w.X.nbytes + w.n * 4 + w.Y0.nbytes),
           "d2h_bytes_per_step": int(w.Y0.nbytes + 16)}
    ctx.close()
    del Xh, Ph, Yh

    # the forms of the method at equal work: same partitions, same start map
    forms = learned = None
    if not args.no_plain and world == 1:
        forms = compare_forms(w, Xd, perms, dev, stream, tuning)
        if not args.no_eq13:
            forms["lr_eq13_study"] = eq13_study(w, Xd, dev, stream, tuning)
        if not args.no_learned:
            learned = learned_form(dev, stream)
    plain = forms["plain_fp32"] if forms else None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(w, args.cpu_seconds)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tmax / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "n": w.n, "d": w.d, "chunks": int(len(sizes)),
                   "chunk_size_range": [int(sizes.min()), int(sizes.max())], "perplexity": w.perplexity,
                   "iters_per_epoch": w.iters, "out_dim": 2, "schedule": "batched persistent, graph-captured epoch",
                   "distances": {"fp32": "fp32 direct differences",
                                 "bf16_window": "bf16 tcgen05 Gram + fp32 window recompute, per-chunk form "
                                                "autotuned (chunks whose window covers most of the chunk "
                                                "computed in fp32 whole)"}[precision],
                   "distance_form": form,
                   "step": "one epoch (the K timed epochs run as one ptsne_run call)", "parallelism": f"replicas{world}",
                   "tuning": {"cluster": tuning[0], "group": tuning[1], "consumer_warps": tuning[2]},
                   "autotune_ms_per_iter": {f"{t[0]}x{t[1]}x{t[2]}": round(ms, 4) for t, ms in trials},
                   "l2": "inputs larger than L2 (joint P %.1f GB per epoch)" % (4 * float((sizes ** 2).sum()) / 1e9)},
        "e2e": e2e, "gpu_launches": launches, "roofline": roofline, "cpu_baseline": cpu, "clocks": clocks,
        "plain_fp32": plain, "forms": forms, "learned": learned, "stages_ms": stages, "perplexity_search": search, "final_cost": {"avg_kl": final_cost[0], "avg_norm_cost": final_cost[1]},
        "impl": "ours",
    }
    return out


# ----------------------------------------------------------------- reference arm (the oracle)

def bench_reference(args, rank, world):
    if rank != 0:
        return None
    from oracle import build as obuild
    from oracle import oracle as O
    from paper_1812_09869_gb300 import synth
    obuild.build()
    w = synth.workload(args.workload, epochs=1)
    prm = O.params(perplexity=w.perplexity, lr=w.lr, momentum=w.momentum, iters=w.iters, epochs=1)
    perm, off = w.perms[0], w.offsets

    def one(c):
        idx = perm[off[c]:off[c + 1]]
        t0 = time.perf_counter()
        O.partial_tsne(w.X[idx], w.Y0[idx], prm)
        return len(idx) * w.iters, time.perf_counter() - t0

    nck = len(off) - 1
    for k in range(args.warmup):
        one(k % nck)
    units, secs = 0, 0.0
    for k in range(args.steps):
        u, s = one((args.warmup + k) % nck)
        units += u
        secs += s
    value = units / secs
    sample = (f"{args.steps} timed chunk(s) of epoch 0 (one per step: affinities + {w.iters} iterations + cost), "
              f"FP64 C oracle with OpenMP")
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "n": w.n, "d": w.d, "perplexity": w.perplexity,
                       "iters_per_epoch": w.iters, "step": "one chunk's partial t-SNE"},
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main(argv=None):
    args = parse_args(argv)
    rank, world, local_rank = dist_env()
    if args.impl == "reference":
        out = bench_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out), flush=True)
        return 0
    import torch
    if args.mapper_kernels:
        from paper_1812_09869_gb300 import build as pbuild
        pbuild.build()
        dev = torch.device("cuda", local_rank)
        torch.cuda.set_device(dev)
        if rank == 0:
            print(json.dumps(mapper_kernels(args.mapper_kernels, dev, torch.cuda.current_stream())), flush=True)
        return 0
    dist_init(world, "nccl" if torch.cuda.is_available() else "gloo")
    out = bench_ours(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
