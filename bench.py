#!/usr/bin/env python
"""Benchmark of batched Seismic search on GB300: QPS at recall@10 >= 0.9.

A step is one pass of the whole query path (list selection, summary scoring,
block ordering, skipping, forward-index scoring, top-k; kappa-NN expansion
where the workload has a graph) over the batch of synthetic queries, with the
index and the queries resident in HBM.  The operating point is the fastest
(cut, heap_factor) of the workload's grid whose mean recall@10 against the
exact top-10 (computed on the device by brute force) is >= 0.9.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c2] [--impl reference]

Prints one JSON line.  Under torchrun each rank holds a full replica and
searches the full batch (the path does not shard); `value` is all ranks'
queries over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # the tiny configuration: fp32 summaries, fixed (cut, heap_factor)
    "c1": dict(desc="Seismic 100k docs, vocab 30522, lambda=2000, beta=100, alpha=0.4, fp32 summaries, "
                    "1k queries (lognormal nnz), k=10", n_docs=100_000, n_q=1000, uneven=False, lam=2000,
               beta=100, alpha=0.4, quant=False, cuts=(10,), hfs=(0.8,), kappa=0, cpu_sample=1000),
    # the batched configuration the metric is quoted on
    "c2": dict(desc="Seismic 1M docs, vocab 30522, lambda=6000, beta=400, alpha=0.4, u8 summaries, "
                    "10k queries (uniform nnz 10-150), k=10, grid cut {5,10,20} x hf {0.6..0.9}",
               n_docs=1_000_000, n_q=10_000, uneven=True, lam=6000, beta=400, alpha=0.4, quant=True,
               cuts=(5, 10, 20), hfs=(0.6, 0.7, 0.8, 0.9), kappa=0, cpu_sample=200, n_train=20_000,
               serve_rates=(5_000, 50_000, 100_000, 200_000)),
    # the c2 shape at 300k documents and 2k queries: small enough for multi-pass ncu captures
    "c2s": dict(desc="Seismic 300k docs, vocab 30522, lambda=6000, beta=400, alpha=0.4, u8 summaries, "
                     "2k queries (uniform nnz 10-150), k=10, cut=5, heap_factor=0.9", n_docs=300_000, n_q=2000,
                uneven=True, lam=6000, beta=400, alpha=0.4, quant=True, cuts=(5,), hfs=(0.9,), kappa=0,
                cpu_sample=100, n_train=4000, serve_rates=(20_000, 200_000)),
    "c3": dict(desc="Seismic 8.8M docs, vocab 30522, lambda=6000, beta=400, alpha=0.4, u8 summaries, kappa=10, "
                    "10k queries (uniform nnz 10-150), k=10", n_docs=8_800_000, n_q=10_000, uneven=True, lam=6000,
               beta=400, alpha=0.4, quant=True, cuts=(5, 10, 20), hfs=(0.6, 0.7, 0.8, 0.9), kappa=10,
               cpu_sample=100, n_train=20_000, serve_rates=(5_000, 50_000, 100_000, 200_000),
               fine_cuts=(5, 8, 10, 12, 16, 20, 25, 30)),
}
RECALL_TARGET = 0.9
K = 10
METRIC = "QPS at recall@10>=0.9 (batched Seismic search, fixed parameters)"
# DRAM bytes (read + write) of one search launch, from one ncu capture of this kernel version on the
# named workload and launch configuration; any other case: null
MEASURED_TRAFFIC = {}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev, self.proc, self.lines = dev, None, []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self, t0=None, t1=None):
        """Summary of the samples taken in [t0, t1] (all samples if none fall there)."""
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        inside = [ln for ts, ln in self.lines if t0 is not None and t0 <= ts <= t1]
        for ln in (inside or [ln for _, ln in self.lines]):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x: float, dist, device) -> float:
    """The largest value over all ranks (the slowest rank's time); x itself
    when there is one process."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_qps(world: int, queries_per_rank: int, ms_slowest: float) -> float:
    """Whole-job throughput: every rank searches its own full batch (replicas),
    so the job answers world x queries_per_rank queries in the slowest rank's time."""
    return world * queries_per_rank / ms_slowest * 1e3


def make_data(w, seed=0):
    import synth
    t = time.time()
    docs = synth.docs(w["n_docs"], seed=seed)
    queries = synth.queries(w["n_q"], seed=seed, uneven=w["uneven"])
    log(f"data: {docs.n_rows} docs / {docs.nnz} nnz, {queries.n_rows} queries in {time.time() - t:.1f}s")
    return docs, queries


def cpu_baseline(w, docs, queries, cut, hf, steps=1):
    """The oracle, as it stands, on the host cores: sequential Seismic search
    (one query per thread) over a bounded sample of the same workload; the
    index lists those queries traverse are built first (untimed)."""
    import oracle
    n = min(w["cpu_sample"], queries.n_rows)
    sample = queries.slice(0, n)
    threads = os.cpu_count() or 1
    t = time.time()
    terms = oracle.query_list_terms(sample, cut)
    ox = oracle.Index(docs, w["lam"], w["beta"], w["alpha"], w["quant"], seed=0, threads=threads,
                      terms=terms)
    log(f"cpu baseline: oracle lists for {len(terms)} terms built in {time.time() - t:.1f}s")
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        ox.search(sample, K, cut=cut, heap_factor=float(np.float32(hf)), threads=threads)
        times.append(time.perf_counter() - t0)
    qps = n / float(np.median(times))
    # the paper's protocol: one thread, mean time per query (a smaller sample)
    n1 = max(1, min(n, 20))
    t0 = time.perf_counter()
    ox.search(sample.slice(0, n1), K, cut=cut, heap_factor=float(np.float32(hf)), threads=1)
    us1 = (time.perf_counter() - t0) / n1 * 1e6
    return {"value": qps, "unit": "queries/s", "cores": threads, "kind": "oracle",
            "sample": f"first {n} of the {queries.n_rows} queries, cut={cut}, heap_factor={hf}, one query per "
                      f"thread; lists built untimed", "times_s": times,
            "single_thread_us_per_query": us1, "single_thread_sample": n1}


def sample_parity(w, ix, docs, queries, gt_ids, gt_sc, ids, sc, sz, n_q=200, n_nodes=1000):
    """Full-size parity on sampled outputs, against the oracle: the device's
    exact top-10 (the recall judge) and the timed configuration's returned
    scores on a sample of queries, and the kappa-NN graph on a sample of nodes."""
    import oracle
    t = time.time()
    rng = np.random.default_rng(7)
    qs = np.sort(rng.choice(queries.n_rows, min(n_q, queries.n_rows), replace=False))
    sub = queries.take(qs)
    ei, es = oracle.exact_topk(docs, sub, K)
    gi = gt_ids[qs].view(np.uint32)
    gs = gt_sc[qs].astype(np.float64)
    # exact top-10: ids equal up to near-ties, scores within 1e-5 of fp64
    qi = np.repeat(np.arange(len(qs), dtype=np.uint64), K)
    ex = oracle.pair_dots(docs, sub, qi, gi.reshape(-1)).reshape(gi.shape)
    rel_exact = float(np.max(np.abs(gs - ex) / np.maximum(np.abs(ex), 1e-30)))
    same = gi == ei
    tie_ok = bool(np.all(same | (np.abs(ex - es) <= 2e-5 * np.abs(es))))
    # the timed configuration: each returned score is the exact inner product of its id
    ri = ids[qs].view(np.uint32)
    valid = ri != oracle.NONE_ID
    rs = oracle.pair_dots(docs, sub, np.repeat(np.arange(len(qs), dtype=np.uint64), K)[valid.reshape(-1)],
                          ri[valid])
    rel_search = float(np.max(np.abs(sc[qs][valid] - rs) / np.maximum(np.abs(rs), 1e-30), initial=0.0))
    out = {"queries": int(len(qs)), "exact_ids_equal": float(same.mean()), "exact_ties_only": tie_ok,
           "exact_max_rel_err": rel_exact, "search_scores_max_rel_err": rel_search}
    if w["kappa"]:
        nodes = np.sort(rng.choice(docs.n_rows, min(n_nodes, docs.n_rows), replace=False))
        ni, _ = oracle.exact_topk(docs, docs.take(nodes), w["kappa"] + 1)
        g = sz.seismic_get_knn(ix)[nodes]
        rec = []
        for r, row in enumerate(ni):
            truth = [x for x in row if x != nodes[r]][: w["kappa"]]
            rec.append(len(set(truth) & set(g[r].tolist())) / w["kappa"])
        out["knn_nodes"] = int(len(nodes))
        out["knn_graph_recall"] = float(np.mean(rec))
        out["knn_self_loops"] = int(np.sum(g == nodes[:, None]))
    out["seconds"] = time.time() - t
    log(f"sample parity: {out}")
    return out


def learned_eval(args, w, sz, ix, dq, gt_sc, stream, time_runs, launch):
    """Trains the per-query parameter MLP on separate synthetic training
    queries (labels from the method's own runs), then measures the learned form
    on the benchmark's queries against the fixed form at equal recall."""
    import torch
    import synth
    from paper_2509_24815_gb300 import learn, metrics
    t = time.time()
    tq = synth.queries(w["n_train"], seed=0, uneven=w["uneven"], stream=synth.TRAIN_STREAM)
    dtq = sz.DeviceCSR.from_host(tq)
    base = dict(launch)
    res = learn.fit(ix, dtq, tq, k=K, target=args.learn_target, quantized=w["quant"], steps=3000, base_params=base)
    t_fit = time.time() - t
    log(f"learned: labels + training on {tq.n_rows} queries in {t_fit:.1f}s, final loss {res['trace'][-1][1]:.4f}")

    def measure(**kw):
        p = sz.search_params(k=K, max_query_nnz=dq.max_row_nnz, **base, **kw)
        ids, sc = sz.seismic_search(ix, dq, p)
        torch.cuda.synchronize()
        rec = float(metrics.recall_at_k(ids.cpu().numpy().view(np.uint32), sc.cpu().numpy(), gt_sc, K).mean())
        for _ in range(2):
            sz.seismic_search(ix, dq, p, stream=stream)
        ms = float(np.median(time_runs(p, max(3, args.steps))))
        return dict(recall=rec, ms=ms, qps=dq.n_rows / ms * 1e3)

    lr = measure(cut=10, heap_factor=0.8, learned=True)
    fine = []
    for cut in w.get("fine_cuts", (3, 4, 5, 6, 8, 10)):
        for hf in (0.6, 0.7, 0.8, 0.9, 1.0):
            fine.append(dict(cut=cut, heap_factor=hf, **measure(cut=cut, heap_factor=hf)))
    at = [f for f in fine if f["recall"] >= lr["recall"] - 1e-9]
    ref = max(at, key=lambda f: f["qps"]) if at else max(fine, key=lambda f: f["recall"])
    # the fixed form's recall/QPS frontier, interpolated linearly at the learned recall
    front = sorted(fine, key=lambda f: f["recall"])
    front = [f for i, f in enumerate(front) if all(g["qps"] < f["qps"] for g in front[i + 1:])]
    interp = None
    for f0, f1 in zip(front, front[1:]):
        if f0["recall"] <= lr["recall"] <= f1["recall"]:
            t = (lr["recall"] - f0["recall"]) / max(f1["recall"] - f0["recall"], 1e-12)
            interp = f0["qps"] + t * (f1["qps"] - f0["qps"])
    log(f"learned: recall {lr['recall']:.4f} at {lr['qps']:,.0f} q/s; best fixed at >= that recall: "
        f"cut={ref['cut']} hf={ref['heap_factor']} recall {ref['recall']:.4f} at {ref['qps']:,.0f} q/s; "
        f"fixed frontier at that recall: {interp if interp is None else round(interp)} q/s")
    return {"value": lr["qps"], "unit": "queries/s", "recall@10": lr["recall"], "ms_per_step": lr["ms"],
            "fixed_at_equal_recall": ref, "qps_gain_vs_fixed": lr["qps"] / ref["qps"],
            "fixed_frontier_qps_at_learned_recall": interp,
            "qps_gain_vs_fixed_frontier": (lr["qps"] / interp) if interp else None,
            "train_queries": tq.n_rows, "label_target_recall": args.learn_target, "fit_seconds": t_fit,
            "final_loss": res["trace"][-1][1], "label_mean_recall": res["label_recall"],
            "calibration_shift": res["calib_shift"], "validation_recall": res["val_recall"],
            "fixed_fine_grid": fine}


def serving_eval(args, w, sz, ix, best, learned, launch):
    """Poisson arrivals replayed through the continuous-batching server:
    p50/p99 latency (arrival to results on the host) and achieved QPS per
    offered rate, with recall@10 of the served k=10 requests."""
    import synth
    from paper_2509_24815_gb300 import metrics, serve
    sp = sz.search_params(cut=best["cut"], heap_factor=best["heap_factor"], learned=learned,
                          use_knn=bool(w["kappa"]), **launch)
    srv = sz.Server(ix, sp, max_batch=1024, streams=16, max_query_nnz=160)
    out = []
    for rate in w["serve_rates"]:
        n = int(min(20_000, max(2_000, rate * 2.0)))
        q = synth.queries(n, seed=0, uneven=True, stream=synth.SERVE_STREAM)
        ids, sc, kq, summ = serve.run_trace(ix, q, rate, search=sp, server=srv)
        gi, gs = sz.seismic_search_exact(ix, q, K)
        m10 = kq == 10
        rec = metrics.recall_at_k(ids[m10][:, :K], sc[m10][:, :K], gs[m10], K).mean() if m10.any() else None
        summ["recall@10_k10_requests"] = float(rec) if rec is not None else None
        out.append(summ)
        log(f"serving {rate:>9,.0f} q/s offered: achieved {summ['achieved_qps']:,.0f} q/s, "
            f"p50 {summ['p50_ms']:.3f} ms, p99 {summ['p99_ms']:.3f} ms, recall@10 {summ['recall@10_k10_requests']:.4f}")
    srv.close()
    return {"params": "learned (fixed fallback)" if learned else "fixed", "rates": out}


def run_reference(args, w):
    """The reference arm: the oracle timed on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    docs, queries = make_data(w)
    cut, hf = (5, 0.9) if len(w["cuts"]) > 1 else (w["cuts"][0], w["hfs"][0])
    cb = cpu_baseline(w, docs, queries, cut, hf, steps=max(1, args.steps))
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"],
            "unit": "queries/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.median(cb["times_s"])), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w["desc"], "cut": cut, "heap_factor": hf, "k": K, "queries_per_step": queries.n_rows,
                       "sample_per_step": min(w["cpu_sample"], queries.n_rows)},
            "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": cb["value"], "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="c2", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--group", type=int, default=1, help="1: chunk-flattened scoring, 8/16/32: lane groups")
    ap.add_argument("--cta-warps", type=int, default=0)
    ap.add_argument("--wave", type=int, default=16)
    ap.add_argument("--persistent", type=int, default=1)
    ap.add_argument("--shape", type=int, default=1, help="1 (or 0): CTA per query, 2: warp per query")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--learn-target", type=float, default=0.9)
    ap.add_argument("--prefetch", type=int, default=0, help="TMA L2 prefetch of the wave's rows (when not autotuned)")
    ap.add_argument("--autotune", type=int, default=1, help="tune the launch configuration at the operating point")
    ap.add_argument("--graph", type=int, default=1, help="time the step as a CUDA graph replay")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, w)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    import paper_2509_24815_gb300 as sz
    from paper_2509_24815_gb300 import autotune, metrics

    docs, queries = make_data(w)
    t = time.time()
    ix = sz.seismic_build(docs, lambda_=w["lam"], beta=w["beta"], alpha=w["alpha"], quantize_u8=w["quant"], seed=0,
                          keep_full_lists=True)
    torch.cuda.synchronize()
    info = sz.seismic_info(ix)
    log(f"build {time.time() - t:.1f}s; index {info['device_bytes'] / 2**30:.2f} GiB on device, "
        f"{info['n_blocks']} blocks, {info['n_summary_entries']} summary entries")
    dq = sz.DeviceCSR.from_host(queries)
    t = time.time()
    gt_ids, gt_sc = sz.seismic_search_exact(ix, dq, K)
    torch.cuda.synchronize()
    gt_sc = gt_sc.cpu().numpy()
    log(f"exact top-{K} (device brute force) in {time.time() - t:.1f}s")
    if w["kappa"]:
        t = time.time()
        sz.seismic_build_knn(ix, w["kappa"], sz.search_params(k=w["kappa"] + 1, cut=10, heap_factor=0.9, shape=1,
                                                              group=1, wave=16, persistent=True))
        log(f"kappa-NN graph built in {time.time() - t:.1f}s")

    stream = torch.cuda.Stream()
    ids = torch.empty((dq.n_rows, K), dtype=torch.int32, device="cuda")
    sc = torch.empty((dq.n_rows, K), dtype=torch.float32, device="cuda")

    def params(cut, hf):
        return sz.search_params(k=K, cut=cut, heap_factor=hf, use_knn=bool(w["kappa"]), wave=args.wave,
                                group=args.group, cta_warps=args.cta_warps, persistent=bool(args.persistent),
                                max_query_nnz=dq.max_row_nnz, shape=args.shape, no_prefetch=not args.prefetch)

    def run(p):
        sz.seismic_search(ix, dq, p, ids_out=ids, scores_out=sc, stream=stream)

    def time_runs(p, n, fn=None):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * n)]
        with torch.cuda.stream(stream):
            for i in range(n):
                ev[2 * i].record(stream)
                if fn is None:
                    run(p)
                else:
                    fn()
                ev[2 * i + 1].record(stream)
        stream.synchronize()
        return [ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(n)]

    # operating point: fastest grid point reaching the recall target
    grid = []
    for cut in w["cuts"]:
        for hf in w["hfs"]:
            p = params(cut, hf)
            run(p)
            stream.synchronize()
            rec = float(metrics.recall_at_k(ids.cpu().numpy().view(np.uint32), sc.cpu().numpy(), gt_sc, K).mean())
            ms = float(np.median(time_runs(p, 2)))
            grid.append(dict(cut=cut, heap_factor=hf, recall=rec, ms=ms, qps=dq.n_rows / ms * 1e3))
            log(f"  cut={cut:2d} hf={hf:.1f}: recall@10 {rec:.4f}  {ms:7.2f} ms  {grid[-1]['qps']:,.0f} q/s")
    ok = [g for g in grid if g["recall"] >= RECALL_TARGET]
    best = max(ok, key=lambda g: g["qps"]) if ok else max(grid, key=lambda g: g["recall"])
    p = params(best["cut"], best["heap_factor"])
    launch = dict(shape=args.shape, group=args.group, cta_warps=args.cta_warps, wave=args.wave,
                  persistent=bool(args.persistent), no_prefetch=not args.prefetch)
    tuned = None
    if args.autotune:
        # launch configuration (kernel shape, lane group, warps, wave) at the chosen operating point
        base = dict(k=K, cut=best["cut"], heap_factor=best["heap_factor"], use_knn=bool(w["kappa"]))
        floor = min(RECALL_TARGET, best["recall"])

        def rec_fn(i, s):
            return metrics.recall_at_k(i.cpu().numpy().view(np.uint32), s.cpu().numpy(), gt_sc, K).mean()
        kw, table = autotune.autotune(ix, dq, base, recall_fn=rec_fn, min_recall=floor, stream=stream, log=log)
        launch = {x: kw[x] for x in launch}
        p = sz.search_params(max_query_nnz=dq.max_row_nnz, **dict(base, **launch))
        run(p)
        stream.synchronize()
        best["recall"] = float(rec_fn(ids, sc))
        tuned = {"chosen": launch, "candidates": len(table),
                 "table": [{x: t.get(x) for x in ("shape", "group", "cta_warps", "wave", "no_prefetch", "ms", "recall")}
                           for t in table]}
        log(f"autotune: {launch}, recall@10 {best['recall']:.4f}")

    # work counters for the algorithmic byte count (deterministic at wave = 1)
    _, _, st = sz.seismic_search(ix, dq, p, stats=True)
    alg_bytes = float(metrics.algorithmic_bytes(st, K, w["quant"], w["kappa"]).sum())

    for _ in range(args.warmup):
        run(p)
    stream.synchronize()
    step, graph_note = (lambda: run(p)), "direct launches"
    if args.graph:
        # the whole step (queue reset, work-queue order, search) as one CUDA graph
        g = torch.cuda.CUDAGraph()
        try:
            with torch.cuda.graph(g, stream=stream, capture_error_mode="thread_local"):
                run(p)
            stream.synchronize()
            step, graph_note = g.replay, "CUDA graph replay"
            for _ in range(args.warmup):
                with torch.cuda.stream(stream):
                    step()
            stream.synchronize()
        except Exception as e:  # capture unsupported here: direct launches of the same kernels
            graph_note = f"direct launches (graph capture failed: {e})"
            log(graph_note)
    # the clock sampler starts (and finishes initialising) before the warm-up
    # steps, so it never competes with the timed launches
    clocks = Clocks(local)
    clocks.start()
    time.sleep(1.0)
    for _ in range(args.warmup):
        with torch.cuda.stream(stream):
            step()
    stream.synchronize()
    barrier()
    torch.cuda.synchronize()
    t_timed = time.time()
    per = time_runs(p, args.steps, step)  # events bracket each step on its stream
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop(t_timed, time.time())
    ms_step = max_over_ranks(float(np.mean(per)), dist, "cuda")
    qps = job_qps(world, dq.n_rows, ms_step)

    # end to end through the public call with host buffers (pinned), copies inside the timed region
    pin = {f: torch.from_numpy(np.ascontiguousarray(getattr(queries, f))).pin_memory()
           for f in ("indptr", "terms", "vals")}
    hq = type(queries)(pin["indptr"].numpy(), pin["terms"].numpy(), pin["vals"].numpy(), queries.dim)
    hid = torch.empty((queries.n_rows, K), dtype=torch.int32).pin_memory()
    hsc = torch.empty((queries.n_rows, K), dtype=torch.float32).pin_memory()
    pe = sz.search_params(k=K, cut=best["cut"], heap_factor=best["heap_factor"], use_knn=bool(w["kappa"]),
                          **launch)
    for _ in range(2):
        sz.seismic_search(ix, hq, pe, ids_out=hid, scores_out=hsc, stream=stream)
    e2e_t = []
    for _ in range(max(3, args.steps)):
        t0 = time.perf_counter()
        sz.seismic_search(ix, hq, pe, ids_out=hid, scores_out=hsc, stream=stream)
        e2e_t.append(time.perf_counter() - t0)
    e2e_qps = job_qps(world, queries.n_rows, 1e3 * max_over_ranks(float(np.median(e2e_t)), dist, "cuda"))
    h2d = queries.indptr.nbytes + queries.terms.nbytes + queries.vals.nbytes
    d2h = hid.numel() * 4 + hsc.numel() * 4

    # kernels per step: the search, plus the work-queue order (keys, sort) ahead of a persistent launch
    launches_per_step = 1 + (2 if (launch["persistent"] or launch["shape"] == 2) and dq.n_rows > 1 else 0)
    peak, peak_kind = peaks()
    achieved = alg_bytes / (float(np.mean(per)) * 1e-3) / 1e9  # this rank's kernel, per launch
    line = {
        "metric": METRIC,
        "value": qps, "unit": "queries/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": w["desc"], "cut": best["cut"], "heap_factor": best["heap_factor"],
                   "recall@10": best["recall"], "queries_per_step": dq.n_rows, "k": K,
                   "l2": "index resident in HBM, larger than L2 (no flush)", **launch,
                   "launch": graph_note, "parallelism": f"replicas x{world}"},
        "grid": grid,
        "autotune": tuned,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": MEASURED_TRAFFIC.get((args.workload, launch["group"], launch["cta_warps"] or 8,
                                                      launch["wave"], launch["no_prefetch"])),
                     "peak_source": peak_kind,
                     "alg_bytes_per_launch": alg_bytes, "kernel": "k_search"},
        "e2e": {"value": e2e_qps, "unit": "queries/s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": args.steps * launches_per_step,
        "clocks": clk,
        "index": {k: info[k] for k in ("n_docs", "nnz", "n_postings", "n_blocks", "n_summary_entries",
                                       "device_bytes")},
    }
    run(p)
    stream.synchronize()
    line["parity_sample"] = sample_parity(w, ix, docs, queries, gt_ids.cpu().numpy(), gt_sc, ids.cpu().numpy(),
                                          sc.cpu().numpy(), sz)
    if not args.no_learned and w.get("n_train"):
        line["learned"] = learned_eval(args, w, sz, ix, dq, gt_sc, stream, time_runs, launch)
    if not args.no_serve and w.get("serve_rates"):
        line["serving"] = serving_eval(args, w, sz, ix, best, bool(line.get("learned")), launch)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(w, docs, queries, best["cut"], best["heap_factor"])
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample",
                                                   "single_thread_us_per_query", "single_thread_sample")}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
