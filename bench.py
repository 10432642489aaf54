"""Benchmark of the streaming IVF-Flat hot path on GB300.

One step = one pass of the whole hot path over one batch of the SIFT-shaped
sliding window (1,000,000 live vectors, d=128, nlist=1024, slab 64):
insert 10,000 new vectors (coarse assignment + slot claim + append), delete
the 10,000 oldest (address-table lookup, bit clear, slab reclaim), and search
10,000 fresh queries (coarse probe selection, list scan, top-10) at the
smallest nprobe of {1, 2, 3, 4, 6, 8, 16, 32, 64, 128} whose recall@10,
against the FP64 oracle's exact k nearest neighbours of 1,000 sampled
queries, reaches 0.95.
Each scan form is measured (FP32 direct form; BF16 and FP8 scans on the
tensor cores with an FP32 re-rank of the best 4k); the headline is the
fastest form that reaches recall 0.95, and every form is reported.

Prints one JSON line.  `value` is queries per second of whole steps (each
step also absorbs its insert and delete batch), timed with no
instrumentation: each step's add, remove and search run as one recorded
CUDA graph through the library's executor (sivf_exec_*), the step's fresh
inputs copied into the executor's buffers inside the timed region, and the
graph's results checked against an eager search.  The components (search
QPS alone, insert and delete vectors/s, the p99 update latency, per-kernel
times) and the scan roofline come from an instrumented eager pass of other
steps (CUDA events around every phase and kernel group).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl sivf|reference]

Under torchrun (N > 1) every rank runs its own replica of the index on its
own GPU (the path has no cross-GPU exchange); rank 0 reports the sum of
queries over the max time.  `--impl reference` times the FP64 CPU oracle on
the host cores on a bounded sample of the same steps.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2601_11808_gb300 import workloads as W  # noqa: E402

METRIC = "QPS@recall@10=0.95; insert/delete vec/s; p99 update ms (1×GB300)"
NPROBES = (1, 2, 3, 4, 6, 8, 16, 32, 64, 128)
N_TRUTH = 1000          # sampled queries with FP64 exact ground truth
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP32 ALU peak: 152 SMs x 128 FP32 lanes x 2 flops (FMA) x 2070 MHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# ncu capture of the reduced-precision list scan on this workload (nprobe
# 1, FP8): the hash of the scan kernel's source (scan_tc.cu up to the
# per-query merge: the kernel and every device helper it calls) it was
# taken of, and the mean dram__bytes_read.sum + dram__bytes_write.sum per
# launch
E2E_PASSES = 3
TC_KERNEL_END = "// ------------------------------------------------------- per-query merge"
TC_PROFILED = {"fp8": ("b33352ac939cf1f0", 149_527_808)}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="sivf", choices=["sivf", "reference"])
    p.add_argument("--workload", default="sift_window")
    p.add_argument("--nprobe", type=int, default=0, help="0 = calibrate for recall 0.95")
    p.add_argument("--gpu-truth", action="store_true",
                   help="recall against the GPU's FP32 search over every list instead of "
                        "the FP64 oracle (quick runs only)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-mixed", action="store_true",
                   help="skip the mixed-batch executor workload")
    p.add_argument("--mixed-replays", type=int, default=5)
    p.add_argument("--mixed-form", default="bf16")
    p.add_argument("--no-serving", action="store_true",
                   help="skip the serving-loop workload")
    p.add_argument("--serving-window", type=int, default=0,
                   help="live vectors of the serving window (0 = 100,000,000)")
    p.add_argument("--serving-seconds", type=float, default=2.0)
    p.add_argument("--deep-vectors", type=int, default=None,
                   help="precision component on a reduced copy of this many vectors (profiling)")
    p.add_argument("--deep-queries", type=int, default=None,
                   help="precision component with this many queries (profiling)")
    p.add_argument("--no-deep", action="store_true",
                   help="skip the deep-precision (k=100) workload")
    p.add_argument("--no-train", action="store_true",
                   help="skip the quantizer-training measurement")
    p.add_argument("--no-compact", action="store_true",
                   help="skip the compaction measurement")
    p.add_argument("--no-delete-window", action="store_true",
                   help="skip the delete-latency-vs-window-size component")
    p.add_argument("--no-zipf", action="store_true",
                   help="skip the Zipf-skewed ingestion workload")
    p.add_argument("--forms", default="fp32,bf16,fp8",
                   help="scan forms to measure; the fastest that reaches recall 0.95 "
                        "is the headline")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi clock / throttle samples taken during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu, self.proc, self.path = gpu, None, None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [t.strip() for t in line.split(",")]
            if len(f) >= 9 and f[1].replace(".", "").isdigit():
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9])
                          if v.lower() == "active"})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(rows[0][2]),
                "samples": len(rows), "reasons": reasons}


def peaks():
    try:
        return json.load(open(PEAKS_PATH))
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}


# ------------------------------------------------------------- data
def make_data(w: W.Workload, n_steps: int, n_calib: int, rank: int):
    ctr = W.centers(w)
    cent = W.index_centroids(w, ctr)
    # each replica draws its own stream and queries (weak scaling)
    wr = W.small(w.name, seed=w.seed + rank) if rank else w
    ctr_r = ctr
    total = w.window + n_steps * w.step
    X = W.vectors(wr, 0, total, ctr_r)
    Q = W.queries(wr, 0, n_steps * w.n_queries + n_calib, ctr_r)
    return cent, X, Q


def oracle_window(w, cent, X, n_max):
    """The FP64 oracle holding the initial window (positions 0 .. window),
    built with every host core; returns (oracle, cores, seconds)."""
    import oracle
    cores = oracle.num_threads(os.cpu_count() or 1)
    S = int(1.25 * (w.window // w.slab_size + 2 * w.nlist))
    o = oracle.OracleIVF(w.d, w.nlist, w.slab_size, n_max, S)
    o.set_centroids(cent)
    t0 = time.time()
    for b in range(0, w.window, 100_000):
        n = min(100_000, w.window - b)
        o.add(W.stream_ids(b, n, n_max), X[b:b + n])
    return o, cores, time.time() - t0


def oracle_sample(w, cent, X, Q, n_max, nprobe, n_ins, n_del, n_q, steps, o=None,
                  threads=0, at=(0, 0, 0)):
    """FP64 oracle on the host cores: full window built with all cores
    (untimed, or the given oracle holding it), then `steps` bounded samples
    of a step (n_ins inserts, n_del deletes of the oldest, n_q queries) with
    `threads` OpenMP threads (0 = every core), each scaled to the full
    step.  `at` = (inserted, deleted, queried) by earlier samples on the
    same oracle: the stream continues from there."""
    import oracle
    build_s = 0.0
    if o is None:
        o, _, build_s = oracle_window(w, cent, X, n_max)
    cores = oracle.num_threads(threads or (os.cpu_count() or 1))
    per_step = []
    for s in range(steps):
        new = w.window + at[0] + s * n_ins
        t0 = time.time()
        o.add(W.stream_ids(new, n_ins, n_max), X[new:new + n_ins])
        t_ins = time.time() - t0
        t0 = time.time()
        o.remove(W.stream_ids(at[1] + s * n_del, n_del, n_max))
        t_del = time.time() - t0
        t0 = time.time()
        q0 = at[2] + s * n_q
        o.search(Q[q0:q0 + n_q], w.k, nprobe)
        t_q = time.time() - t0
        per_step.append((t_ins * w.step / n_ins, t_del * w.step / n_del,
                         t_q * w.n_queries / n_q))
    a = np.array(per_step)
    step_s = a.sum(axis=1)
    oracle.num_threads(os.cpu_count() or 1)
    return {
        "qps": float(w.n_queries / np.mean(step_s)),
        "search_qps": float(w.n_queries / np.mean(a[:, 2])),
        "insert_vec_s": float(w.step / np.mean(a[:, 0])),
        "delete_vec_s": float(w.step / np.mean(a[:, 1])),
        "p99_update_ms": float(np.percentile((a[:, 0] + a[:, 1]) * 1e3, 99)),
        "cores": cores, "build_s": build_s, "step_s": step_s.tolist(),
    }


# ------------------------------------------------------- reference arm
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w = W.CONFIGS[args.workload]
    n_ins, n_del, n_q, n_cal = 1000, 1000, 200, 200
    steps = args.steps + args.warmup
    cent, X, Q = make_data(w, (steps * n_ins) // w.step + 1, n_cal, 0)
    n_max = w.window + (steps * n_ins // w.step + 3) * w.step
    t0 = time.time()
    orc, _, _ = oracle_window(w, cent, X, n_max)
    # nprobe by the sivf arm's rule: the smallest of the sweep whose
    # recall@10 reaches 0.95 against the exact k nearest neighbours of
    # sampled queries over the initial window (here the oracle's own IVF
    # search against its brute force, on n_cal queries)
    rec = {}
    if args.nprobe:
        nprobe = args.nprobe
    else:
        Qc = Q[-n_cal:]
        _, gt = orc.exact_knn(Qc, w.k)
        nprobe = NPROBES[-1]
        for P in NPROBES:
            _, got = orc.search(Qc, w.k, P)
            rec[P] = float(np.mean([len(set(a) & set(b)) / w.k
                                    for a, b in zip(got.tolist(), gt.tolist())]))
            if rec[P] >= 0.95:
                nprobe = P
                break
    r = oracle_sample(w, cent, X, Q, n_max, nprobe, n_ins, n_del, n_q, steps, o=orc)
    wall = time.time() - t0
    sample = (f"oracle index holding the full {w.window:,}-vector window (built with "
              f"{r['cores']} threads, untimed); per step {n_ins} inserts, {n_del} deletes "
              f"of the oldest and {n_q} queries (k={w.k}, nprobe={nprobe}), each scaled to "
              f"the full step ({w.step} / {w.step} / {w.n_queries})")
    st = r["step_s"][args.warmup:]
    val = float(w.n_queries / np.mean(st))
    line = {
        "impl": "reference", "metric": METRIC, "value": round(val, 3), "unit": "queries/s",
        "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(float(np.mean(st)) * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(w, nprobe),
        "recall_at_10": rec.get(nprobe), "recall_by_nprobe": rec,
        "recall_truth": (f"the oracle's exact k nearest neighbours of {n_cal} sampled queries "
                         "over the initial window" if rec else None),
        "components": {k: r[k] for k in ("search_qps", "insert_vec_s", "delete_vec_s",
                                           "p99_update_ms")},
        "cpu_baseline": {"value": round(val, 3), "unit": "queries/s", "cores": r["cores"],
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(val, 3), "unit": "queries/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "wall_s": round(wall, 1),
    }
    print(json.dumps(line), flush=True)


def config_of(w, nprobe, form="fp32"):
    return {"workload": w.name, "window": w.window, "d": w.d, "nlist": w.nlist,
            "slab": w.slab_size, "insert_per_step": w.step, "delete_per_step": w.step,
            "queries_per_step": w.n_queries, "k": w.k, "nprobe": nprobe,
            "scan_dtype": form if form == "fp32" else f"{form} scan + fp32 re-rank of 4k",
            "l2": "inputs larger than L2: 512 MB index, fresh insert/query batches "
                  "every step",
            "parallelism": "replicas"}


# ---------------------------------------------------- mixed-batch queue
def run_mixed(torch, sivf, dev, stream, replays, warmup, form="bf16"):
    """The mixed-batch workload: a 5,000,000-vector index (d=128, nlist=2048,
    slab 64) and a queue of 64 insert, 64 delete and 64 query batches of
    log-uniform sizes (inserts 1..50,000, deletes 1..100,000 random live ids,
    queries 1..4,096 with nprobe drawn from {8,...,128}, k=10), interleaved
    1:1:1.  The queue is recorded once into a CUDA graph (scan tiles tuned per
    batch bucket first) and replayed with fresh data written in place; one
    replay of the same queue as single calls is timed beside it."""
    from paper_2601_11808_gb300 import autotune
    w = W.CONFIGS["mixed_batches"]
    sched = W.mixed_schedule(64, 4096, 100_000, 50_000, w.nprobes, seed=w.seed)
    n_ins = sum(n for k, n, _ in sched if k == "add")
    n_rep = warmup + replays + 3
    n_max = w.window + n_ins * (n_rep + 1) + 1
    S = w.window // w.slab_size + 2 * w.nlist + n_rep * (n_ins // w.slab_size + w.nlist)
    ctr = W.centers(w)
    g = sivf.Index(w.d, w.nlist, w.slab_size, n_max, S,
                   scan_dtypes=(form,) if form != "fp32" else ())
    g.set_centroids(torch.from_numpy(W.index_centroids(w, ctr)).to(dev))
    alive = np.zeros(n_max, bool)
    t_fill = time.time()
    for b in range(0, w.window, 250_000):
        n = min(250_000, w.window - b)
        g.add(torch.from_numpy(W.stream_ids(b, n, n_max)).to(dev),
              torch.from_numpy(W.vectors(w, b, n, ctr)).to(dev))
    alive[:w.window] = True
    g.sync()
    t_fill = time.time() - t_fill
    state = {"pos": w.window, "qpos": 0, "rnd": 0}

    def fresh(kind, n):
        if kind == "add":
            ids = W.stream_ids(state["pos"], n, n_max)
            x = W.vectors(w, state["pos"], n, ctr)
            state["pos"] += n
            alive[ids] = True
            return ids, x
        if kind == "remove":
            state["rnd"] += 1
            ids = W.sample_ids(w.seed, 8, state["rnd"], np.flatnonzero(alive), n)
            alive[ids] = False
            return (ids,)
        q = W.queries(w, state["qpos"] % 1_000_000, n, ctr)
        state["qpos"] += n
        return (q,)

    ops = []
    for kind, n, P in sched:
        if kind == "add":
            ops.append({"kind": "add", "ids": torch.empty(n, dtype=torch.int64, device=dev),
                        "x": torch.empty((n, w.d), dtype=torch.float32, device=dev)})
        elif kind == "remove":
            ops.append({"kind": "remove", "ids": torch.empty(n, dtype=torch.int64, device=dev)})
        else:
            ops.append({"kind": "search", "q": torch.empty((n, w.d), dtype=torch.float32,
                                                           device=dev),
                        "k": w.k, "nprobe": P, "dtype": form,
                        "dist": torch.empty((n, w.k), dtype=torch.float32, device=dev),
                        "labels": torch.empty((n, w.k), dtype=torch.int64, device=dev)})

    def refill():
        for op, (kind, n, _) in zip(ops, sched):
            data = fresh(kind, n)
            if kind == "add":
                op["ids"].copy_(torch.from_numpy(data[0]))
                op["x"].copy_(torch.from_numpy(data[1]))
            elif kind == "remove":
                op["ids"].copy_(torch.from_numpy(data[0]))
            else:
                op["q"].copy_(torch.from_numpy(data[0]))
        torch.cuda.synchronize()

    # tiles: one autotune per bucket the queue's query batches fall in
    t_tune = time.time()
    qs = torch.from_numpy(W.queries(w, 2_000_000, 4096, ctr)).to(dev)
    tuned = autotune.tune(g, qs, [(n, w.k, P, form) for k, n, P in sched if k == "search"],
                          reps=3)
    t_tune = time.time() - t_tune
    refill()
    t_rec = time.time()
    ex = g.executor(ops)
    t_rec = time.time() - t_rec

    def check(res):
        for (kind, n, _), r in zip(sched, res):
            want = n
            if r[0] != 0 or r[1] != want:
                raise RuntimeError(f"mixed batch {kind} n={n}: status/count {r}")

    for _ in range(warmup):
        ex.launch(stream)
        torch.cuda.synchronize()
        check(ex.results(stream))
        refill()
    graph_ms, per = [], {"add": [], "remove": [], "search": []}
    for _ in range(replays):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ex.launch(stream)
        e1.record(stream)
        torch.cuda.synchronize()
        graph_ms.append(e0.elapsed_time(e1))
        res = ex.results(stream)
        check(res)
        for (kind, n, _), r in zip(sched, res):
            per[kind].append(r[2])
        refill()
    # the same queue as single calls (scratch reserved, one untimed pass first)
    g.reserve(max(n for k, n, _ in sched if k == "add"),
              max(n for k, n, _ in sched if k == "remove"),
              max(n for k, n, _ in sched if k == "search"), w.k, max(w.nprobes), stream)

    def eager():
        for op in ops:
            if op["kind"] == "add":
                g.add(op["ids"], op["x"])
            elif op["kind"] == "remove":
                g.remove(op["ids"])
            else:
                g.search(op["q"], op["k"], op["nprobe"], op["dtype"], dist=op["dist"],
                         labels=op["labels"])

    eager()
    refill()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    eager()
    e1.record(stream)
    torch.cuda.synchronize()
    eager_ms = e0.elapsed_time(e1)
    g.sync()
    # the scans of the queue's small query batches (under 256 queries, the
    # memory-bound regime) against the HBM roof: each batch searched once
    # more on its own with the library's CUDA events; unique bytes of the
    # lists its scan probed over the scan launches' device time
    small = [op for op in ops if op["kind"] == "search" and op["q"].shape[0] < 256]
    sb, sms, sn = 0, 0.0, 0
    for op in small:
        st0 = g.stats()
        g.profile(True)
        g.search(op["q"], op["k"], op["nprobe"], op["dtype"], dist=op["dist"],
                 labels=op["labels"])
        n1, ms1 = g.profile_read("scan")
        g.profile(False)
        sb += g.stats()["list_bytes_scanned"] - st0["list_bytes_scanned"]
        sms += ms1
        sn += n1
    small_gbs = sb / (sms / 1e3) / 1e9 if sms > 0 else 0.0
    kernels = ex.kernels
    ex.close()
    live = g.stats()["ntotal"]
    g.close()
    nq = sum(n for k, n, _ in sched if k == "search")
    nd = sum(n for k, n, _ in sched if k == "remove")
    gm = float(np.mean(graph_ms))
    pct = {k: {"p50_ms": round(float(np.percentile(v, 50)), 4),
               "p99_ms": round(float(np.percentile(v, 99)), 4)} for k, v in per.items()}
    return {
        "workload": "mixed_batches: 5,000,000 vectors d=128 (64-component mixture, "
                    "centers U[-1,1], sigma 0.1), nlist=2048, slab 64; 64 insert + 64 delete "
                    "+ 64 query batches, log-uniform sizes, nprobe per query batch from "
                    "{8,16,32,64,128}, k=10, " + form + " scan + fp32 re-rank",
        "batches": len(sched), "queries": nq, "inserted": n_ins, "deleted": nd,
        "graph_launches_per_queue": 1, "kernels_per_queue": int(kernels),
        "graph_ms_per_queue": round(gm, 3), "eager_ms_per_queue": round(eager_ms, 3),
        "graph_speedup": round(eager_ms / gm, 3),
        "queries_per_s": round(nq / (gm / 1e3), 1),
        "ops_per_s": round((nq + n_ins + nd) / (gm / 1e3), 1),
        "per_batch_device_ms": pct, "replays": replays,
        "small_query_scans": {"batches": len(small), "launches": int(sn), "ms": round(sms, 3),
                              "unique_list_bytes": int(sb), "achieved_gbs": round(small_gbs, 1),
                              "frac_of_hbm": round(small_gbs / peaks().get("hbm_gbs", 6695.5),
                                                   4)},
        "tuned_buckets": len(tuned), "tune_s": round(t_tune, 2), "record_s": round(t_rec, 3),
        "prefill_s": round(t_fill, 1), "live_after": int(live),
    }


# ------------------------------------------------- delete vs window size
def run_delete_window(torch, sivf, dev, windows=(1_000_000, 10_000_000, 100_000_000),
                      batches=(1000, 10_000), steps=200):
    """Delete latency as the window grows (the paper's O(1) delete, Sec.
    3.5.2, and its tail-latency table for batches of 1,000, Sec. 5.5): the
    serving workload's vectors (d=128, 16,384-component mixture, nlist
    16384, slab 128) in one index grown from 1 M to 10 M to 100 M live
    vectors; at each size and batch B, `steps` sliding-window steps insert
    B new vectors and delete the B oldest; the delete alone is timed with
    CUDA events on its stream (device time, p50 / p99 / max)."""
    w = W.CONFIGS["serving"]
    top = max(windows)
    n_max = top + (1 << 22)
    S = int(1.02 * top / w.slab_size) + 3 * w.nlist + (1 << 14)
    ctr = W.centers(w)
    pool = W.noise_pool(w, 1 << 20)
    g = sivf.Index(w.d, w.nlist, w.slab_size, n_max, S)
    g.set_centroids(torch.from_numpy(W.index_centroids(w, ctr)).to(dev))
    ctr_d, pool_d = torch.from_numpy(ctr).to(dev), torch.from_numpy(pool).to(dev)
    sig = float(np.float32(w.sigma))
    stream = torch.cuda.current_stream()

    def add_range(b, n):
        for c0 in range(b, b + n, 2_000_000):
            m = min(2_000_000, b + n - c0)
            c, r = W.pooled_parts(w, c0, m, len(pool))
            x = ctr_d[torch.from_numpy(c).to(dev)] + pool_d[torch.from_numpy(r).to(dev)] * sig
            g.add(torch.from_numpy(W.stream_ids(c0, m, n_max)).to(dev), x)

    lo, hi, out = 0, 0, {}
    t_fill = time.time()
    for Wn in sorted(windows):
        add_range(hi, Wn - (hi - lo))
        hi = lo + Wn
        g.sync()
        res = {}
        for B in batches:
            ms = []
            for st in range(steps + 3):
                add_range(hi, B)
                hi += B
                ids = torch.from_numpy(W.stream_ids(lo, B, n_max)).to(dev)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                g.remove(ids)
                e1.record(stream)
                lo += B
                e1.synchronize()
                if st >= 3:
                    ms.append(e0.elapsed_time(e1))
            a = np.array(ms)
            res[f"B{B}"] = {"p50_ms": round(float(np.percentile(a, 50)), 4),
                            "p99_ms": round(float(np.percentile(a, 99)), 4),
                            "max_ms": round(float(a.max()), 4),
                            "delete_vec_s": round(B / (a.mean() / 1e3), 1)}
        assert g.sync() >= 0
        res["live"] = int(g.stats()["ntotal"])
        out[f"W{Wn}"] = res
    t_fill = time.time() - t_fill
    g.close()
    del ctr_d, pool_d
    torch.cuda.empty_cache()
    lo_w, hi_w = f"W{min(windows)}", f"W{max(windows)}"
    out["p99_ratio_largest_vs_smallest"] = {
        f"B{B}": round(out[hi_w][f"B{B}"]["p99_ms"] / out[lo_w][f"B{B}"]["p99_ms"], 3)
        for B in batches}
    out["workload"] = ("serving mixture (d=128, 16,384 components, nlist=16384, slab 128), one "
                       "index grown 1M -> 10M -> 100M live vectors; per size and batch B, "
                       f"{steps} steps of insert B new + delete the B oldest, the delete timed "
                       "with CUDA events (device time)")
    out["seconds"] = round(t_fill, 1)
    return out


# ----------------------------------------------------------- serving loop
def run_serving(torch, sivf, dev, window=0, seconds=2.0, loads=(0.5, 0.8, 0.95)):
    """The serving workload: a sliding window of 100,000,000 vectors (d=128,
    16,384-component mixture, nlist=16384, slab 128, FP32 payload + BF16
    copy) served by the library's serving loop.  Requests arrive as a Poisson
    stream: 70% inserts of 1..10,000 fresh vectors (each evicting the oldest
    ids beyond the window), 10% deletes of the 1..10,000 oldest ids, 20%
    queries of 1..256 vectors (k=10, nprobe=32, BF16 scan + FP32 re-rank),
    sizes log-uniform.  The saturation rate is measured first (a burst served
    as fast as possible), then each offered load runs for `seconds`;
    latency is measured from each request's scheduled arrival."""
    w = W.CONFIGS["serving"]
    Wn = window or w.window
    n_max = Wn + (1 << 22)
    S = int(1.02 * Wn / w.slab_size) + 3 * w.nlist + (1 << 14)
    ctr = W.centers(w)
    pool = W.noise_pool(w, 1 << 20)
    g = sivf.Index(w.d, w.nlist, w.slab_size, n_max, S, scan_dtypes=("bf16",))
    g.set_centroids(torch.from_numpy(W.index_centroids(w, ctr)).to(dev))
    ctr_d, pool_d = torch.from_numpy(ctr).to(dev), torch.from_numpy(pool).to(dev)
    sig = float(np.float32(w.sigma))
    t_fill = time.time()
    ch = 2_000_000
    for b in range(0, Wn, ch):
        n = min(ch, Wn - b)
        c, r = W.pooled_parts(w, b, n, len(pool))
        x = ctr_d[torch.from_numpy(c).to(dev)] + pool_d[torch.from_numpy(r).to(dev)] * sig
        g.add(torch.from_numpy(W.stream_ids(b, n, n_max)).to(dev), x)
        del x
    g.sync()
    t_fill = time.time() - t_fill
    del ctr_d, pool_d
    torch.cuda.empty_cache()
    # page-locked payload pools: inserts reuse pool vectors under fresh ids
    xpool = torch.from_numpy(W.pooled_vectors(w, 0, 1 << 20, ctr, pool)).pin_memory().numpy()
    qpool = torch.from_numpy(W.queries(w, 0, 1 << 16, ctr)).pin_memory().numpy()
    k, P = w.k, w.nprobes[0]
    sv = sivf.Server(g, k=k, nprobe=P, dtype="bf16", depth=4, max_query_batch=2048,
                     max_insert_batch=40_000, max_delete_batch=40_000)
    win = {"lo": 0, "hi": Wn, "xo": 0, "qo": 0}

    def submit(kind, n, t_arr):
        if kind == 0:
            ids = np.arange(win["hi"], win["hi"] + n, dtype=np.int64) % n_max
            win["hi"] += n
            over = max(0, win["hi"] - win["lo"] - Wn)
            ev = np.arange(win["lo"], win["lo"] + over, dtype=np.int64) % n_max
            win["lo"] += over
            if win["xo"] + n > len(xpool):
                win["xo"] = 0
            x = xpool[win["xo"]:win["xo"] + n]
            win["xo"] += n
            return sv.add(ids, x, evict=ev, arrival_ns=t_arr)
        if kind == 1:
            n = min(n, win["hi"] - win["lo"])
            ids = np.arange(win["lo"], win["lo"] + n, dtype=np.int64) % n_max
            win["lo"] += n
            return sv.remove(ids, arrival_ns=t_arr)
        if win["qo"] + n > len(qpool):
            win["qo"] = 0
        q = qpool[win["qo"]:win["qo"] + n]
        win["qo"] += n
        return sv.search(q, arrival_ns=t_arr)

    def run(n_req, rate, stream):
        t_off, kinds, sizes = W.request_stream(n_req, rate, seed=w.seed, stream=stream)
        g.profile(True)          # CUDA events around the library's kernel groups
        gs0 = g.stats()
        st0 = sv.stats()
        t0 = sivf.Server.now_ns() + 2_000_000
        reqs = []
        for off, kd, sz in zip(t_off.tolist(), kinds.tolist(), sizes.tolist()):
            t_arr = t0 + off
            while True:
                now = sivf.Server.now_ns()
                if now >= t_arr:
                    break
                if t_arr - now > 300_000:
                    time.sleep((t_arr - now - 200_000) / 1e9)
            reqs.append((kd, submit(kd, sz, t_arr)))
        sv.drain()
        infos = [(kd, sv.wait(r)) for kd, r in reqs]
        st1 = sv.stats()
        done = [t0 + off + 1e6 * i["latency_ms"] for off, (_, i) in zip(t_off.tolist(), infos)]
        span = (max(done) - t0) / 1e9
        out = {"offered_req_s": round(rate, 1), "requests": n_req,
               "achieved_req_s": round(n_req / span, 1)}
        for kd, name in enumerate(("insert", "delete", "query")):
            lat = np.asarray([i["latency_ms"] for k2, i in infos if k2 == kd])
            if len(lat):
                out[name] = {"n": int(len(lat)), "p50_ms": round(float(np.percentile(lat, 50)), 3),
                             "p99_ms": round(float(np.percentile(lat, 99)), 3),
                             "items_per_s": round((st1["items"][kd] - st0["items"][kd]) / span, 1),
                             "batches": st1["batches"][kd] - st0["batches"][kd]}
        out["rejected"] = st1["rejected"] - st0["rejected"]
        out["deferred"] = st1["deferred"] - st0["deferred"]
        out["max_in_flight"] = st1["max_in_flight"]
        bad = [i for _, i in infos if i["status"] != 0]
        out["failed"] = len(bad)
        # the query scans against the HBM roof: unique bytes of the lists
        # the scans probed over the scan launches' summed device time
        gs1 = g.stats()
        n_scan, scan_ms = g.profile_read("scan")
        g.profile(False)
        ub = gs1["list_bytes_scanned"] - gs0["list_bytes_scanned"]
        gbs = ub / (scan_ms / 1e3) / 1e9 if scan_ms > 0 else 0.0
        out["scan"] = {"launches": int(n_scan), "ms": round(scan_ms, 3),
                       "unique_list_bytes": int(ub), "achieved_gbs": round(gbs, 1),
                       "frac_of_hbm": round(gbs / peaks().get("hbm_gbs", 6695.5), 4)}
        return out

    # saturation: a burst with every arrival at once
    burst = run(3000, 1e12, 30)
    sat = burst["achieved_req_s"]
    res = {"saturation": burst}
    for i, ld in enumerate(loads):
        n_req = max(200, int(sat * ld * seconds))
        res[f"load_{ld}"] = run(n_req, sat * ld, 31 + i)
    sv.close()
    live = g.stats()["ntotal"]
    g.close()
    torch.cuda.empty_cache()
    res.update({
        "workload": f"serving: {Wn:,}-vector window d=128 (16,384-component mixture, centers "
                    "U[-1,1], sigma 0.1, noise rows from a 2^20-vector pool), nlist=16384, slab "
                    "128, FP32 + BF16 copy; Poisson 70% insert (1..10k, evicting beyond the "
                    "window) / 10% delete-oldest (1..10k) / 20% query (1..256, k=10, nprobe=32, "
                    "bf16 scan + fp32 re-rank), sizes log-uniform",
        "prefill_s": round(t_fill, 1), "live_after": int(live), "seconds_per_load": seconds,
        "latency": "from each request's scheduled arrival to its completion on the host"})
    return res


# ------------------------------------------------------- deep precision
def run_train(torch, sivf, dev, n=200_000, iters=10, reps=3):
    """Lloyd's k-means of the coarse quantizer (sivf_train) on n rows of the
    SIFT-shaped stream, nlist 1024, `iters` iterations: device time per run
    (CUDA events on the stream; the call synchronises the stream at entry,
    so a run's time includes that host round trip)."""
    w = W.CONFIGS["sift_window"]
    ctr = W.centers(w)
    x = W.vectors(w, 0, n, ctr)
    xd = torch.from_numpy(x).to(dev)
    g = sivf.Index(w.d, w.nlist, w.slab_size, 1024, 4 * w.nlist)
    g.train(xd, 1, 1)
    torch.cuda.synchronize()
    times = []
    for r in range(reps):
        t0 = time.time()
        g.train(xd, iters, r)
        torch.cuda.synchronize()
        times.append(time.time() - t0)
    g.close()
    best = min(times)
    return {"rows": n, "d": w.d, "nlist": w.nlist, "iters": iters,
            "seconds": round(best, 4), "row_iters_per_s": round(n * iters / best, 1)}


def oracle_train_sample(n=10_000, iters=2):
    """The oracle's k-means on a bounded sample of the same rows (host cores)."""
    import oracle
    w = W.CONFIGS["sift_window"]
    x = W.vectors(w, 0, n, W.centers(w))
    t0 = time.time()
    oracle.kmeans(x, w.nlist, iters, 0)
    s = time.time() - t0
    return {"rows": n, "iters": iters, "seconds": round(s, 3),
            "row_iters_per_s": round(n * iters / s, 1)}


def run_deep(torch, sivf, dev, steps=3, n_truth=100, n_vec=None, n_q=None):
    """The precision workload: 10,000,000 unit-norm vectors d=96 from a
    4,096-component mixture, nlist=4096, slab 32, with FP32, BF16 and FP8
    E4M3 (per-list scale) payloads; 10,000 queries, k=100, nprobe=64; the
    reduced forms keep the best 400 candidates per query and re-rank them in
    FP32.  Per form: QPS, recall@100 against exact FP64 brute force on a
    sample of queries, and the largest relative error of the returned
    distances against their FP64 values."""
    w = W.CONFIGS["deep_precision"]
    n, k, P = n_vec or w.window, w.k, w.nprobes[0]
    nq = n_q or w.n_queries
    ctr = W.centers(w)
    cent = W.index_centroids(w, ctr)
    S = int(1.05 * (n // w.slab_size)) + 2 * w.nlist
    g = sivf.Index(w.d, w.nlist, w.slab_size, n, S, scan_dtypes=("bf16", "fp8"))
    g.set_centroids(torch.from_numpy(cent).to(dev))
    t_fill = time.time()
    X = np.empty((n, w.d), np.float32)
    ch = 1_000_000
    for b in range(0, n, ch):
        X[b:b + ch] = W.vectors_threaded(w, b, min(ch, n - b), ctr)
        g.add(torch.from_numpy(W.stream_ids(b, min(ch, n - b), n)).to(dev),
              torch.from_numpy(X[b:b + ch]).to(dev))
    g.sync()
    t_fill = time.time() - t_fill
    Q = W.vectors_threaded(w, 0, nq, ctr, stream=2)
    Qd = torch.from_numpy(Q).to(dev)
    # exact FP64 top-k of a query sample (brute force, ties to the lower id)
    t_gt = time.time()
    qs = Q[:n_truth].astype(np.float64)
    best_d = np.full((n_truth, k), np.inf)
    best_i = np.full((n_truth, k), -1, np.int64)
    qn = (qs ** 2).sum(1)
    for b in range(0, n, 500_000):
        xb = X[b:b + 500_000].astype(np.float64)
        dd = qn[:, None] + (xb ** 2).sum(1)[None, :] - 2.0 * (qs @ xb.T)
        rows = np.arange(n_truth)[:, None]
        part = np.argpartition(dd, k, axis=1)[:, :k]
        cd = np.concatenate([best_d, dd[rows, part]], axis=1)
        ci = np.concatenate([best_i, b + part], axis=1)
        order = np.lexsort((ci, cd), axis=1)[:, :k]
        best_d, best_i = cd[rows, order], ci[rows, order]
    t_gt = time.time() - t_gt
    out = {}
    stream = torch.cuda.current_stream()
    for form in ("fp32", "bf16", "fp8"):
        dist = torch.empty((nq, k), dtype=torch.float32, device=dev)
        lab = torch.empty((nq, k), dtype=torch.int64, device=dev)
        for _ in range(2):
            g.search(Qd, k, P, form, dist=dist, labels=lab)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            g.search(Qd, k, P, form, dist=dist, labels=lab)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        gi = lab[:n_truth].cpu().numpy()
        gd = dist[:n_truth].cpu().numpy().astype(np.float64)
        rec = float(np.mean([len(set(a) & set(b)) / k for a, b in zip(gi.tolist(),
                                                                     best_i.tolist())]))
        err = 0.0
        for r in range(n_truth):
            ok = gi[r] >= 0
            ex = ((X[gi[r][ok]].astype(np.float64) - Q[r].astype(np.float64)) ** 2).sum(1)
            err = max(err, float(np.max(np.abs(gd[r][ok] - ex) / np.maximum(ex, 1e-30))))
        out[form] = {"qps": round(nq / (ms / 1e3), 1), "ms_per_search": round(ms, 3),
                     "recall_at_100": round(rec, 4), "max_rel_dist_err": err}
    g.close()
    del X
    torch.cuda.empty_cache()
    out.update({
        "workload": f"deep_precision: {n:,} unit-norm vectors d=96 (4,096-component "
                    "mixture, sigma 0.02), nlist=4096, slab 32, FP32 + BF16 + FP8 E4M3 payloads; "
                    f"{nq:,} queries, k=100, nprobe=64, re-rank depth 400",
        "truth": f"exact FP64 brute force over all vectors for {n_truth} sampled queries",
        "prefill_s": round(t_fill, 1), "truth_s": round(t_gt, 1)})
    return out


def run_zipf(torch, sivf, dev, reps=3, n_truth=100, batch=10_000):
    """Skewed ingestion: 1,000,000 SIFT-shaped vectors whose 1,024 mixture
    components are drawn with P(rank r) ~ 1/r (the heaviest list takes 13 %
    of the rows, about 2,100 slabs of 64), nlist=1024.  Ingestion time of
    the whole set in one call and in batches of 10,000 (device-resident
    input, CUDA events; best of `reps` fresh indexes), beside the same
    ingestion with components drawn uniformly; then 10,000 queries from the
    same skewed law, k=10, nprobe=8, per scan form: QPS and recall@10
    against exact FP64 brute force on a sample of queries."""
    w = W.CONFIGS["zipf_ingest"]
    n, k, P = w.window, w.k, w.nprobes[0]
    ctr = W.centers(w)
    cent = W.index_centroids(w, ctr)
    S = int(1.25 * (n // w.slab_size + 2 * w.nlist))
    stream = torch.cuda.current_stream()
    ids = torch.from_numpy(W.stream_ids(0, n, n)).to(dev)
    cent_d = torch.from_numpy(cent).to(dev)

    def ingest(xd, step):
        best = None
        for _ in range(reps):
            g = sivf.Index(w.d, w.nlist, w.slab_size, n, S, scan_dtypes=("bf16", "fp8"))
            g.set_centroids(cent_d)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for b in range(0, n, step):
                g.add(ids[b:b + step], xd[b:b + step])
            e1.record(stream)
            torch.cuda.synchronize()
            g.sync()
            assert g.stats()["ntotal"] == n
            ms = e0.elapsed_time(e1)
            if best is None or ms < best[0]:
                if best is not None:
                    best[1].close()
                best = (ms, g)
            else:
                g.close()
        return best

    Xu = torch.from_numpy(W.vectors_threaded(W.small("zipf_ingest", zipf=0.0), 0, n, ctr)).to(dev)
    uni_ms, gu = ingest(Xu, n)
    gu.close()
    del Xu
    X = W.vectors_threaded(w, 0, n, ctr)
    Xd = torch.from_numpy(X).to(dev)
    bat_ms, gb = ingest(Xd, batch)
    gb.close()
    one_ms, g = ingest(Xd, n)
    sizes = np.asarray(g.list_sizes())
    Q = W.queries(w, 0, w.n_queries, ctr)
    Qd = torch.from_numpy(Q).to(dev)
    # exact FP64 top-k of a query sample
    qs = Q[:n_truth].astype(np.float64)
    x64 = X.astype(np.float64)
    dd = (qs ** 2).sum(1)[:, None] + (x64 ** 2).sum(1)[None, :] - 2.0 * (qs @ x64.T)
    truth = np.argsort(dd, axis=1, kind="stable")[:, :k]
    del dd, x64
    out = {}
    for form in ("fp32", "bf16", "fp8"):
        dist = torch.empty((w.n_queries, k), dtype=torch.float32, device=dev)
        lab = torch.empty((w.n_queries, k), dtype=torch.int64, device=dev)
        for _ in range(2):
            g.search(Qd, k, P, form, dist=dist, labels=lab)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            g.search(Qd, k, P, form, dist=dist, labels=lab)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 3
        gi = lab[:n_truth].cpu().numpy()
        rec = float(np.mean([len(set(a) & set(b)) / k for a, b in zip(gi.tolist(),
                                                                     truth.tolist())]))
        out[form] = {"qps": round(w.n_queries / (ms / 1e3), 1), "ms_per_search": round(ms, 3),
                     "recall_at_10": round(rec, 4)}
    g.close()
    del Xd, Qd
    torch.cuda.empty_cache()
    return {
        "workload": "zipf_ingest: 1,000,000 SIFT-shaped vectors d=128 from 1,024 components "
                    "with P(rank r) ~ 1/r, nlist=1024, slab 64; 10,000 queries of the same law, "
                    "k=10, nprobe=8",
        "ingest_one_call_s": round(one_ms / 1e3, 4),
        "ingest_one_call_vec_s": round(n / (one_ms / 1e3), 1),
        f"ingest_batches_{batch}_s": round(bat_ms / 1e3, 4),
        "uniform_ingest_one_call_s": round(uni_ms / 1e3, 4),
        "largest_list": int(sizes.max()), "mean_list": round(float(sizes.mean()), 1),
        "search": out,
        "truth": f"exact FP64 brute force over all vectors for {n_truth} sampled queries",
    }


def run_compact(torch, sivf, dev, frac=0.5, reps=3):
    """Compaction of partly-live slabs: the SIFT-shaped window (1,000,000
    vectors d=128, nlist=1024, slab 64, FP8 copy) with a uniformly random
    half of its ids deleted, then one full pass (min_free 1, no budget):
    kernel time of the pass (the library's CUDA-event profile), slabs freed,
    members moved, and the FP8 search (10,000 queries, k=10, nprobe=8)
    before and after it."""
    w = W.CONFIGS["sift_window"]
    n, P = w.window, 8
    ctr = W.centers(w)
    S = int(1.25 * (n // w.slab_size + 2 * w.nlist))
    g = sivf.Index(w.d, w.nlist, w.slab_size, n, S, scan_dtypes=("fp8",))
    g.set_centroids(torch.from_numpy(W.index_centroids(w, ctr)).to(dev))
    X = W.vectors_threaded(w, 0, n, ctr)
    g.add(torch.from_numpy(W.stream_ids(0, n, n)).to(dev), torch.from_numpy(X).to(dev))
    del X
    gone = W.sample_ids(w.seed, 14, 0, W.stream_ids(0, n, n), int(frac * n))
    g.remove(torch.from_numpy(gone).to(dev))
    g.sync()
    Qd = torch.from_numpy(W.queries(w, 0, w.n_queries, ctr)).to(dev)
    stream = torch.cuda.current_stream()

    def search_ms():
        for _ in range(2):
            g.search(Qd, w.k, P, "fp8")
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            g.search(Qd, w.k, P, "fp8")
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    used0 = g.stats()["used_slabs"]
    before = search_ms()
    g.profile(True)
    freed, moved = g.compact(1, 1 << 40, sync=True)
    pass_ms = g.profile_read("compact")[1]
    g.profile(False)
    used1 = g.stats()["used_slabs"]
    after = search_ms()
    g.close()
    del Qd
    torch.cuda.empty_cache()
    return {
        "workload": f"sift_window (1,000,000 vectors, nlist 1024, slab 64) with a random "
                    f"{frac:.0%} of ids deleted; one compaction pass (min_free 1, no budget); "
                    f"FP8 search of 10,000 queries, k=10, nprobe=8",
        "pass_ms": round(pass_ms, 3), "slabs_freed": int(freed), "members_moved": int(moved),
        "moved_per_s": round(moved / (pass_ms / 1e3), 1) if pass_ms > 0 else None,
        "slabs_used_before": int(used0), "slabs_used_after": int(used1),
        "search_ms_before": round(before, 3), "search_ms_after": round(after, 3),
    }


def oracle_zipf_sample(n=100_000):
    """The oracle's ingestion of the first n rows of the skewed stream."""
    import oracle
    w = W.CONFIGS["zipf_ingest"]
    ctr = W.centers(w)
    x = W.vectors(w, 0, n, ctr)
    o = oracle.OracleIVF(w.d, w.nlist, w.slab_size, n, 2 * (n // w.slab_size + w.nlist))
    o.set_centroids(W.index_centroids(w, ctr))
    t0 = time.time()
    o.add(W.stream_ids(0, n, n), x)
    s = time.time() - t0
    return {"rows": n, "seconds": round(s, 3), "vec_s": round(n / s, 1)}


# ------------------------------------------------------------ our arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    rank, world, local = dist_env()
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2601_11808_gb300 import build as B
    B.build()
    from paper_2601_11808_gb300 import sivf

    w = W.CONFIGS[args.workload]
    forms = [f for f in args.forms.split(",") if f]
    K, Wm = args.steps, args.warmup
    # warm-up, then per form an instrumented eager pass, two graph warm-up
    # steps and the graph pass, then the e2e pass
    n_steps = Wm + len(forms) * (2 * K + 2) + E2E_PASSES * K + 1
    n_calib = N_TRUTH
    cent, X, Q = make_data(w, n_steps, n_calib, rank)
    n_max = w.window + (n_steps + 2) * w.step
    S = int(1.25 * (w.window // w.slab_size + 2 * w.nlist))
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    g = sivf.Index(w.d, w.nlist, w.slab_size, n_max, S,
                   scan_dtypes=tuple(f for f in forms if f != "fp32"))
    g.set_centroids(torch.from_numpy(cent).to(dev))
    for b in range(0, w.window, 100_000):
        n = min(100_000, w.window - b)
        g.add(torch.from_numpy(W.stream_ids(b, n, n_max)).to(dev),
              torch.from_numpy(X[b:b + n]).to(dev))
    g.sync()

    # per form: the smallest nprobe of the sweep whose recall@10 reaches
    # 0.95 against the exact k nearest neighbours of N_TRUTH sampled queries
    # (the FP64 oracle's brute force over the same window, computed on the
    # host cores outside any timed region), and the nprobe interpolated
    # linearly between the last sweep point below the target and the first
    # at or above it
    Qc_h = Q[-n_calib:]
    Qc = torch.from_numpy(Qc_h).to(dev)
    orc = None
    t_truth = time.time()
    if args.gpu_truth or args.impl != "sivf" or world > 1:
        _, gt = g.search(Qc, w.k, w.nlist)
        gt = gt.cpu().numpy()
        truth = "the GPU's FP32 search over every list"
    else:
        orc, _, _ = oracle_window(w, cent, X, n_max)
        _, gt = orc.exact_knn(Qc_h, w.k)
        truth = (f"exact FP64 k nearest neighbours (the oracle's brute force) of {n_calib} "
                 "sampled queries over the initial window")
    t_truth = time.time() - t_truth
    calib = {}
    for f in forms:
        rec, chosen, interp, prev = {}, None, None, None
        for P in ([args.nprobe] if args.nprobe else NPROBES):
            _, got = g.search(Qc, w.k, P, f)
            got = got.cpu().numpy()
            rec[P] = float(np.mean([len(set(a) & set(b)) / w.k
                                    for a, b in zip(got.tolist(), gt.tolist())]))
            if chosen is None and rec[P] >= 0.95:
                chosen = P
                if prev is None:
                    interp = float(P)
                else:
                    p0, r0 = prev
                    interp = p0 + (0.95 - r0) / max(rec[P] - r0, 1e-12) * (P - p0)
            if chosen is None:
                prev = (P, rec[P])
        calib[f] = {"recall_by_nprobe": rec, "nprobe": chosen or NPROBES[-1],
                    "nprobe_interpolated": interp, "meets_target": chosen is not None,
                    "recall_at_10": rec[chosen or NPROBES[-1]]}

    def step_inputs(s):
        new = w.window + s * w.step
        return (torch.from_numpy(W.stream_ids(new, w.step, n_max)).to(dev),
                torch.from_numpy(X[new:new + w.step]).to(dev),
                torch.from_numpy(W.stream_ids(s * w.step, w.step, n_max)).to(dev),
                torch.from_numpy(Q[s * w.n_queries:(s + 1) * w.n_queries]).to(dev))

    dist_out = torch.empty((w.n_queries, w.k), dtype=torch.float32, device=dev)
    lab_out = torch.empty((w.n_queries, w.k), dtype=torch.int64, device=dev)
    g.reserve(w.step, w.step, w.n_queries, w.k, max(c["nprobe"] for c in calib.values()))

    def record_step(form, nprobe, dist=None, labels=None):
        """An executor holding one step (add, remove, search) on fixed
        device buffers."""
        ins_ids, ins_x, del_ids, q = step_inputs(0)
        bufs = [torch.empty_like(ins_ids), torch.empty_like(ins_x), torch.empty_like(del_ids),
                torch.empty_like(q)]
        ex = g.executor([{"kind": "add", "ids": bufs[0], "x": bufs[1]},
                         {"kind": "remove", "ids": bufs[2]},
                         {"kind": "search", "q": bufs[3], "k": w.k, "nprobe": nprobe,
                          "dtype": form, "dist": dist_out if dist is None else dist,
                          "labels": lab_out if labels is None else labels}])
        return ex, bufs

    def graph_step(ex, bufs, inp):
        for dst, src in zip(bufs, inp):
            dst.copy_(src, non_blocking=True)
        ex.launch(stream)

    def run_step(form, nprobe, ins_ids, ins_x, del_ids, q, ev=None):
        if ev:
            ev[0].record(stream)
        g.add(ins_ids, ins_x)
        if ev:
            ev[1].record(stream)
        g.remove(del_ids)
        if ev:
            ev[2].record(stream)
        g.search(q, w.k, nprobe, form, dist=dist_out, labels=lab_out)
        if ev:
            ev[3].record(stream)

    step_no = 0
    for s in range(Wm):
        for f in forms:
            run_step(f, calib[f]["nprobe"], *step_inputs(step_no))
        step_no += 1
    torch.cuda.synchronize()
    g.sync()

    results, execs = {}, {}
    for f in forms:
        P = calib[f]["nprobe"]
        inputs = [step_inputs(step_no + s) for s in range(K)]
        step_no += K
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
        st0 = g.stats()
        launches0 = g.profile_read("all")[0]
        g.profile(True)
        clocks = Clocks(local)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clocks.start()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for s in range(K):
            run_step(f, P, *inputs[s], ev=evs[s])
        t1.record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        if world > 1:
            torch.distributed.barrier()
        total_ms = t0.elapsed_time(t1)
        st1 = g.stats()
        launches = g.profile_read("all")[0] - launches0
        prof = {k: g.profile_read(k) for k in ("coarse", "insert", "remove", "group", "scan",
                                               "merge", "rerank")}
        g.profile(False)
        g.sync()
        if world > 1:
            t = torch.tensor([total_ms], device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            total_ms = float(t.item())
        ins_ms = np.array([a[0].elapsed_time(a[1]) for a in evs])
        del_ms = np.array([a[1].elapsed_time(a[2]) for a in evs])
        srch_ms = np.array([a[2].elapsed_time(a[3]) for a in evs])
        upd = ins_ms + del_ms
        results[f] = {
            "qps": world * K * w.n_queries / (total_ms / 1e3), "total_ms": total_ms,
            "search_qps": world * K * w.n_queries / (srch_ms.sum() / 1e3),
            "insert_vec_s": world * K * w.step / (ins_ms.sum() / 1e3),
            "delete_vec_s": world * K * w.step / (del_ms.sum() / 1e3),
            "p50_update_ms": float(np.percentile(upd, 50)),
            "p99_update_ms": float(np.percentile(upd, 99)),
            "insert_ms": float(ins_ms.mean()), "delete_ms": float(del_ms.mean()),
            "search_ms": float(srch_ms.mean()),
            "kernel_ms_per_step": {k: round(v[1] / K, 4) for k, v in prof.items()},
            "scan": prof["scan"], "launches": launches, "clocks": clk,
            "pairs": st1["pairs_scanned"] - st0["pairs_scanned"],
            "sbytes": st1["slab_bytes_scanned"] - st0["slab_bytes_scanned"],
            "ubytes": st1["list_bytes_scanned"] - st0["list_bytes_scanned"],
        }

        # the headline pass, with no instrumentation: the same steps (fresh
        # batches) through the library's executor, the step's add, remove
        # and search recorded once into one CUDA graph whose input buffers
        # are refilled by device copies inside the timed region
        ex, bufs = record_step(f, P)
        for s in range(2):
            graph_step(ex, bufs, step_inputs(step_no + s))
        step_no += 2
        inputs = [step_inputs(step_no + s) for s in range(K)]
        step_no += K
        launches0 = g.profile_read("all")[0]
        clocks = Clocks(local)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clocks.start()
        t0.record(stream)
        for s in range(K):
            graph_step(ex, bufs, inputs[s])
        t1.record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        if world > 1:
            torch.distributed.barrier()
        gms = t0.elapsed_time(t1)
        glaunch = g.profile_read("all")[0] - launches0
        if world > 1:
            t = torch.tensor([gms], device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            gms = float(t.item())
        st = ex.results(stream)
        # the graph's last search equals an eager search of the same queries
        # on the same state (nothing changes the index after it)
        gd, gl = dist_out.clone(), lab_out.clone()
        g.search(inputs[-1][3], w.k, P, f, dist=dist_out, labels=lab_out)
        same = bool(torch.equal(gd, dist_out) and torch.equal(gl, lab_out))
        results[f].update({
            "eager_instrumented_qps": results[f]["qps"],
            "eager_instrumented_ms": total_ms,
            "qps": world * K * w.n_queries / (gms / 1e3), "total_ms": gms,
            "launches": glaunch, "clocks": clk,
            "graph_kernels": int(ex.kernels), "graph_equals_eager": same,
            "graph_status_ok": all(x[0] == 0 for x in st)})
        execs[f] = (ex, bufs)

    ok = [f for f in forms if calib[f]["meets_target"]] or forms
    head = max(ok, key=lambda f: results[f]["qps"])
    r = results[head]
    nprobe = calib[head]["nprobe"]
    pk = peaks()
    scan_n, scan_ms = r["scan"]
    if head == "fp32":
        flops = 3.0 * w.d * r["pairs"]
        achieved = flops / (scan_ms / 1e3) / 1e12 if scan_ms > 0 else 0.0
        roofline = {"bound": "alu", "achieved": round(achieved, 3),
                    "peak": round(FP32_PEAK_TFLOPS, 1), "unit": "TFLOP/s",
                    "frac": round(achieved / FP32_PEAK_TFLOPS, 4),
                    "peak_note": "FP32 FMA peak 152 SMs x 128 lanes x 2 x 2070 MHz; the direct "
                                 "form issues 2 instructions per 3 flops, so its ceiling is 0.75",
                    "kernel": "k_scan (FP32 direct form)"}
    else:
        # algorithmic bytes: the unique bytes of the lists each launch probes
        # (payload copy, norms, bitmaps), the list-centric lower bound
        gbs = r["ubytes"] / (scan_ms / 1e3) / 1e9 if scan_ms > 0 else 0.0
        roofline = {"bound": "hbm", "achieved": round(gbs, 1), "peak": pk.get("hbm_gbs"),
                    "unit": "GB/s", "frac": round(gbs / pk.get("hbm_gbs", 6695.5), 4),
                    "peak_note": "measured HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs), "
                                 "of measured",
                    "kernel": f"k_scan_tc<{head}> (tcgen05 scan of the {head} copy)",
                    "tensor_view": {"tflops": round(2.0 * w.d * r["pairs"] / (scan_ms / 1e3) / 1e12, 2),
                                    "peak_bf16_tflops": pk.get("bf16_tflops")},
                    "tile_read_bytes_per_launch": r["sbytes"] / max(scan_n, 1)}
    traffic = None
    if head != "fp32":
        # DRAM bytes per launch of this kernel from one ncu capture on this
        # workload, valid while the kernel source is the one it was taken of
        import hashlib
        src = os.path.join(ROOT, "paper_2601_11808_gb300", "csrc", "scan_tc.cu")
        sha, nbytes = TC_PROFILED.get(head, (None, None))
        text = open(src).read()
        if sha and TC_KERNEL_END in text and \
                hashlib.sha256(text[:text.index(TC_KERNEL_END)].encode()).hexdigest()[:16] == sha:
            traffic = nbytes
    roofline.update({"traffic": traffic, "launches": scan_n,
                     "ms_per_launch": round(scan_ms / max(scan_n, 1), 4),
                     "algorithmic_bytes_per_launch": (r["ubytes"] if head != "fp32" else r["sbytes"])
                     / max(scan_n, 1),
                     "flops_per_launch": (3.0 if head == "fp32" else 2.0) * w.d * r["pairs"]
                     / max(scan_n, 1)})

    line = {
        "metric": METRIC, "value": round(r["qps"], 3), "unit": "queries/s", "n_gpus": world,
        "steps": K, "warmup": Wm, "ms_per_step": round(r["total_ms"] / K, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if head == "fp32" else f"{head}+f32",
        "data": "synthetic: seeded 1,024-component Gaussian mixture shaped like SIFT "
                "(d=128, integers 0..255); stands in for SIFT1M",
        "config": config_of(w, nprobe, head),
        "recall_at_10": calib[head]["recall_at_10"],
        "nprobe": nprobe,
        "recall_truth": truth,
        "components": {
            **{k: round(r[k], 4) for k in ("search_qps", "insert_vec_s", "delete_vec_s",
                                           "p50_update_ms", "p99_update_ms", "insert_ms",
                                           "delete_ms", "search_ms")},
            "truth_s": round(t_truth, 1),
            "kernel_ms_per_step": r["kernel_ms_per_step"],
            "forms": {f: {"qps": round(results[f]["qps"], 1),
                          "search_qps": round(results[f]["search_qps"], 1),
                          "nprobe": calib[f]["nprobe"],
                          "nprobe_interpolated": calib[f]["nprobe_interpolated"],
                          "recall_at_10": calib[f]["recall_at_10"],
                          "meets_recall_0.95": calib[f]["meets_target"],
                          "recall_by_nprobe": calib[f]["recall_by_nprobe"],
                          "scan_ms": round(results[f]["scan"][1] / K, 4),
                          "eager_instrumented_qps": round(results[f]["eager_instrumented_qps"], 1),
                          "graph_kernels_per_step": results[f]["graph_kernels"],
                          "graph_equals_eager": results[f]["graph_equals_eager"],
                          "graph_status_ok": results[f]["graph_status_ok"]} for f in forms},
            "timing": ("value and ms_per_step: the steps replayed as one recorded CUDA graph "
                       "per step through the library's executor (inputs copied into its "
                       "buffers inside the timed region), no instrumentation; the per-phase "
                       "times, kernel_ms_per_step and the roofline come from an instrumented "
                       "eager pass of K other steps (CUDA events around every phase and kernel "
                       "group)"),
        },
        "gpu_launches": int(r["launches"]),
        "roofline": roofline,
        "clocks": r["clocks"],
    }

    if not args.no_e2e:
        # a client that streams its batches from host memory: two executors
        # with their own input and result buffers, an upload stream and a
        # read-back stream; the inputs of step s + 1 are copied (pinned host
        # -> device) while step s runs, step s's results are read back while
        # step s + 1 runs; every step's copy in and read-back are inside the
        # timed region
        host = []
        for s in range(E2E_PASSES * K):
            host.append([x.cpu().pin_memory() for x in step_inputs(step_no + s)])
        step_no += E2E_PASSES * K
        sets = []
        for i in range(2):
            if i == 0:
                ex, bufs = execs[head]
                dd, ll = dist_out, lab_out
            else:
                dd, ll = torch.empty_like(dist_out), torch.empty_like(lab_out)
                ex, bufs = record_step(head, nprobe, dd, ll)
            hd = torch.empty((w.n_queries, w.k), dtype=torch.float32).pin_memory()
            hl = torch.empty((w.n_queries, w.k), dtype=torch.int64).pin_memory()
            sets.append((ex, bufs, dd, ll, hd, hl))
        h2d = sum(x.numel() * x.element_size() for x in host[0])
        d2h = sum(x.numel() * x.element_size() for x in sets[0][4:6])
        # one untimed copy of every pinned buffer first: the first DMA to or
        # from a freshly pinned buffer pays its one-time mapping
        for hs in host:
            for dst, src in zip(sets[0][1], hs):
                dst.copy_(src, non_blocking=True)
        for ex, bufs, dd, ll, hd, hl in sets:
            hd.copy_(dd, non_blocking=True)
            hl.copy_(ll, non_blocking=True)
        torch.cuda.synchronize()
        up, down = torch.cuda.Stream(), torch.cuda.Stream()
        passes = []
        for pss in range(E2E_PASSES):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            up.wait_stream(stream)
            down.wait_stream(stream)
            ran, read = [None, None], [None, None]  # per set: its last step, read-back

            def upload(s):
                # step s's inputs into its set, once the set's previous step ran
                with torch.cuda.stream(up):
                    if ran[s % 2] is not None:
                        up.wait_event(ran[s % 2])
                    for dst, src in zip(sets[s % 2][1], host[s]):
                        dst.copy_(src, non_blocking=True)
                    ev = torch.cuda.Event()
                    ev.record(up)
                return ev

            s0, s1 = pss * K, (pss + 1) * K
            copied = upload(s0)
            for s in range(s0, s1):
                ex, bufs, dd, ll, hd, hl = sets[s % 2]
                stream.wait_event(copied)
                if read[s % 2] is not None:
                    stream.wait_event(read[s % 2])  # the set's results were read back
                ex.launch(stream)
                ev = torch.cuda.Event()
                ev.record(stream)
                ran[s % 2] = ev
                if s + 1 < s1:
                    copied = upload(s + 1)
                with torch.cuda.stream(down):
                    down.wait_event(ev)
                    hd.copy_(dd, non_blocking=True)
                    hl.copy_(ll, non_blocking=True)
                    rb = torch.cuda.Event()
                    rb.record(down)
                    read[s % 2] = rb
            stream.wait_stream(up)
            stream.wait_stream(down)
            e1.record(stream)
            torch.cuda.synchronize()
            passes.append(e0.elapsed_time(e1))
        sets[1][0].close()
        e2e_ms = float(np.median(passes))
        if world > 1:
            t = torch.tensor([e2e_ms], device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            e2e_ms = float(t.item())
        line["e2e"] = {"value": round(world * K * w.n_queries / (e2e_ms / 1e3), 3),
                       "unit": "queries/s", "h2d_bytes_per_step": int(h2d),
                       "d2h_bytes_per_step": int(d2h),
                       "passes_ms": [round(x, 3) for x in passes],
                       "timing": (f"median of {E2E_PASSES} passes of {K} steps; the next "
                                  "step's inputs are uploaded and the last step's results "
                                  "read back while a step runs (two executors, an upload and "
                                  "a read-back stream)")}

    for ex, _ in execs.values():
        ex.close()
    g.close()
    torch.cuda.empty_cache()
    if not args.no_mixed:
        line["components"]["mixed_batches"] = run_mixed(
            torch, sivf, dev, stream, max(1, min(args.mixed_replays, K)), max(1, min(Wm, 2)),
            args.mixed_form)
        torch.cuda.empty_cache()
    if not args.no_deep:
        line["components"]["deep_precision"] = run_deep(torch, sivf, dev, n_vec=args.deep_vectors,
                                                        n_q=args.deep_queries)
    if not args.no_train:
        line["components"]["train"] = run_train(torch, sivf, dev)
    if not args.no_zipf:
        line["components"]["zipf_ingest"] = run_zipf(torch, sivf, dev)
    if not args.no_compact:
        line["components"]["compaction"] = run_compact(torch, sivf, dev)
    if not args.no_delete_window:
        line["components"]["delete_vs_window"] = run_delete_window(torch, sivf, dev)
        torch.cuda.empty_cache()
    if not args.no_serving:
        line["components"]["serving"] = run_serving(
            torch, sivf, dev, args.serving_window, args.serving_seconds)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n_ins, n_del, n_q = 1000, 1000, 200
        if orc is None:
            orc, _, _ = oracle_window(w, cent, X, n_max)
        rr = oracle_sample(w, cent, X, Q, n_max, nprobe, n_ins, n_del, n_q, 2, o=orc)
        r1 = oracle_sample(w, cent, X, Q, n_max, nprobe, n_ins // 2, n_del // 2, n_q // 2, 1,
                           o=orc, threads=1, at=(2 * n_ins, 2 * n_del, 2 * n_q))
        line["cpu_baseline"] = {
            "value": round(rr["qps"], 3), "unit": "queries/s", "cores": rr["cores"],
            "kind": "oracle",
            "sample": (f"FP64 oracle holding the full {w.window:,}-vector window (built with "
                       f"every core, untimed); 2 steps of {n_ins} inserts, {n_del} deletes of "
                       f"the oldest and {n_q} queries (k={w.k}, nprobe={nprobe}), each scaled "
                       f"to the full step"),
            "components": {k: round(rr[k], 3) for k in ("search_qps", "insert_vec_s",
                                                        "delete_vec_s", "p99_update_ms")},
            "single_thread": {
                "value": round(r1["qps"], 3), "unit": "queries/s", "cores": r1["cores"],
                "sample": (f"the same oracle on one thread: 1 step of {n_ins // 2} inserts, "
                           f"{n_del // 2} deletes and {n_q // 2} queries, scaled to the full "
                           f"step"),
                **{k: round(r1[k], 3) for k in ("search_qps", "insert_vec_s", "delete_vec_s")}},
        }
        if not args.no_train:
            line["cpu_baseline"]["components"]["train"] = oracle_train_sample()
        if not args.no_zipf:
            line["cpu_baseline"]["components"]["zipf_ingest"] = oracle_zipf_sample()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
