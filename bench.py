"""Throughput benchmark: Hugin propagation over the large-clique tree
(64 cliques x 10 variables of cardinality 4 = 2^20 entries each, separators
of 4-6 variables, depth <= 8, FP32, 5% of the variables observed).

One step = one jt_propagate over a batch of evidence cases (collect and
distribute, every message by Eq. 1-3), inputs resident in HBM.  The metric
is clique-entries per second: each case counts the numerator of Eq. 4 over
its 2(n-1) messages, sum of |phi_src| + |phi_dst|.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--batch B] [--impl cuda|reference]
                    [--no-serving] [--no-cpu-baseline] [--no-ablation]

Under torchrun every rank runs its own replica on its own evidence cases
(the path shards by case; there is no data-path collective), and rank 0
prints one JSON line with the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1202_3777_gb300 import synth  # noqa: E402

WORKLOAD = "large_clique"
METRIC = "propagation clique-entries/s (batched FP32 vs plain); p50/p99 query latency"
UNIT = "clique-entries/s"


def _json_default(o):
    """numpy scalars in the JSON line."""
    if hasattr(o, "item"):
        return o.item()
    raise TypeError(type(o))


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


class Clocks:
    """nvidia-smi sampling (every 200 ms) while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# DRAM traffic of the propagation kernel from an ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum, summarised in
# profiles/k_propagate_large_clique.md), valid only while the kernel and
# planner sources are the ones it was taken on.  One-case launch: bytes per
# launch.  Case-block launch: bytes per case block (16 cases = 2 case blocks
# captured; every case block streams the tables again, so traffic grows with
# their number).
TRAFFIC = {
    "sources_sha256": "2b7ffdc46295254912ef5a082dcc0cce3cfa097de2460c4308983a50f7b4168e",
    "plain": 470387584 + 1843136,       # mean of 4 launches
    "per_case_block": (965038208 + 15660672) / 2,   # mean of 2 launches
}
TRAFFIC_SOURCES = ["paper_1202_3777_gb300/csrc/jt_kernels.cu", "paper_1202_3777_gb300/csrc/jt_kernels.h",
                   "paper_1202_3777_gb300/csrc/jt_internal.h", "paper_1202_3777_gb300/csrc/jt_plan.cpp"]


def measured_traffic(cases):
    """ncu DRAM bytes per launch for `cases` cases, or None once the kernel
    or planner sources differ from the profiled ones."""
    import hashlib
    h = hashlib.sha256()
    try:
        for f in TRAFFIC_SOURCES:
            with open(os.path.join(ROOT, f), "rb") as fh:
                h.update(fh.read())
    except OSError:
        return None
    if h.hexdigest() != TRAFFIC["sources_sha256"]:
        return None
    if cases == 1:
        return int(TRAFFIC["plain"])
    return int(TRAFFIC["per_case_block"] * ((cases + 7) // 8))


def evidence_seed(rank: int) -> int:
    """Seed of a rank's evidence cases: every replica propagates its own."""
    return 7000 + 100000 * rank


def max_over_ranks(x: float, world: int, device: str = "cpu") -> float:
    """The largest of every rank's value (the job's time is its slowest
    rank's); `device` is where the collective's tensor lives (cuda for NCCL,
    cpu for gloo)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(work_per_case: int, cases_per_rank: int, world: int, ms_per_step: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (each rank propagates its own cases: weak scaling)."""
    return work_per_case * cases_per_rank * world / (ms_per_step * 1e-3)


def msg_total(tree):
    """Entries of all separator tables (the per-case message arrays)."""
    from math import prod
    n = 1
    for c in range(1, tree.n_cliques):
        sv = set(tree.cliques[c].tolist()) & set(tree.cliques[tree.parent[c]].tolist())
        n += prod(int(tree.card[v]) for v in sv)
    return n


def oracle_rate(tree, cases, budget_s=20.0, gpu=None):
    """The FP64 oracle, as it stands, on a bounded sample of the cases; with
    `gpu` = (log Z array, marginal rows) of the same cases from the GPU, also
    the GPU's error against the oracle on that sample (rel_errors)."""
    from oracle import hugin
    w = tree.work_per_case()
    t0 = time.perf_counter()
    done = 0
    refs = []
    for v, s in cases:
        refs.append(hugin.propagate_tree(tree, hugin.evidence_dict(v, s)))
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    err = None
    if gpu is not None:
        err = rel_errors(tree, refs, gpu[0], gpu[1])
    return w * done / dt, done, dt, err


def rel_errors(tree, refs, lz_gpu, marg_rows, floor=1e-30):
    """The parity metric on a sample: max relative error over normalised
    marginal entries the oracle puts at or above `floor` (an entry the oracle
    gives as exactly 0 must be 0; one below the floor counts its absolute
    error in units of the floor), and the relative log Z error
    |dlogZ| / max(1, |log Z|)."""
    card = np.asarray(tree.card, dtype=np.int64)
    off = np.concatenate([[0], np.cumsum(card)])
    worst, worst_lz = 0.0, 0.0
    for i, ref in enumerate(refs):
        row = np.asarray(marg_rows[i], dtype=np.float64)
        for v in range(len(card)):
            g = row[off[v]:off[v + 1]]
            o = np.asarray(ref.marginals[v], dtype=np.float64)
            big = o >= floor
            if np.any(big):
                worst = max(worst, float(np.max(np.abs(g[big] - o[big]) / o[big])))
            small = ~big
            if np.any(small):
                worst = max(worst, float(np.max(np.abs(g[small] - o[small]))) / floor)
        worst_lz = max(worst_lz, abs(float(lz_gpu[i]) - ref.log_z) / max(1.0, abs(ref.log_z)))
    return {"cases": len(refs), "max_rel_err": worst, "logz_rel_err": worst_lz,
            "tolerance": 1e-5, "oracle": "FP64 numpy oracle (oracle/hugin.py)"}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    tree = synth.WORKLOADS[WORKLOAD]["build"]().as_dtype(np.float32)
    ev = synth.evidence_matrix(tree, args.steps + args.warmup, 0.05, 9000)
    cases = [synth.case_from_row(r) for r in ev]
    from oracle import hugin
    w = tree.work_per_case()
    for i in range(args.warmup):
        hugin.propagate_tree(tree, hugin.evidence_dict(*cases[i]))
    t0 = time.perf_counter()
    for i in range(args.warmup, args.warmup + args.steps):
        hugin.propagate_tree(tree, hugin.evidence_dict(*cases[i]))
    dt = time.perf_counter() - t0
    val = w * args.steps / dt
    sample = f"one evidence case per step of the {tree.name} workload (FP64 oracle, numpy, single thread)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": tree.name, "cases_per_step": 1, "observed_frac": 0.05},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                         "host_cores": host_cores()},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)
    return 0


def measure_per_message(tree, ev_row):
    """The paper's own propagation (one kernel launch pair per message, index-
    mapping tables; Algorithm 1) for one case of the workload, in the naive
    and the interleaved mapping-table layout: device time of the whole
    propagation, best of three after a first run that also builds the
    tables."""
    from paper_1202_3777_gb300 import jt
    h = jt.jt_load_synth(tree, compute=jt.JT_F32, max_cases=1, flags=jt.JT_MATERIALIZE_CLIQUES)
    jt.jt_set_evidence_dense(h, 0, ev_row[None, :])
    out = {}
    for layout, name in ((0, "naive"), (1, "interleaved")):
        jt.jt_propagate_per_message(h, 0, layout)
        out[name + "_ms"] = min(jt.jt_propagate_per_message(h, 0, layout) for _ in range(3))
    assert jt.jt_get_status(h, 0, 1)[0] == jt.JT_OK
    h.free()
    return out


def measure_cpt_init(tree, hbm):
    """Algorithm 4's initialisation on the device: the workload's tree loaded
    without tables, then every clique table built from a Bayesian network's
    CPTs (one per variable, up to three parents).  Device time of the
    initialisation kernel, best of three after a first call; algorithmic
    bytes = every table entry written once plus every CPT entry read once."""
    from paper_1202_3777_gb300 import jt
    fams, vals = synth.bn_for_tree(tree, 7, max_parents=3)
    h = jt.jt_load_tree(tree.card, tree.cliques, tree.parent, None, compute=jt.JT_F32, max_cases=1)
    jt.jt_init_from_cpts(h, fams, vals)
    ms = min(jt.jt_init_from_cpts(h, fams, vals) for _ in range(3))
    h.free()
    cpt_entries = int(sum(v.size for v in vals))
    alg = 4 * (tree.entries() + cpt_entries)
    ach = alg / (ms * 1e-3) / 1e9
    return {"kernel": "k_init_cliques", "kernel_ms": ms, "n_cpts": len(fams), "cpt_entries": cpt_entries,
            "alg_bytes": alg, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm}


def separator_sweep():
    """Analogues of Fig. 6 and Fig. 7 on trees that differ only in separator
    size (32 cliques of 4^8 entries, separators of 4^1 .. 4^7 entries), one
    case without evidence, FP32 on the GPU:

    * speedup over the sequential FP64 oracle (one core) of the fused
      propagation (propagation kernel + finalisation, device time) and of
      the paper's per-message propagation (naive mapping tables), against
      the average separator table size (Fig. 6);
    * the launch-overhead share of the per-message propagation (Fig. 7),
      with the paper's model of a constant cost tau per launch (Eq. 5-6):
      tau is the per-launch time of the per-message propagation of a floor
      tree (cliques of two binary variables, one shared), where every
      kernel has almost nothing to do; a tree's share is
      launches x tau / its per-message time.  A per-message propagation
      without evidence issues 4(n-1) + 8 stream operations: 2 kernels per
      message, 2 for the root's normalisation, 1 for the totals, 1 for the
      finalisation, 2 memsets and 2 device copies (the tables and the
      separators' start values).
    Device times are best of three after a first run."""
    from oracle import hugin
    from paper_1202_3777_gb300 import jt
    configs = [("floor", dict(sep_vars=1, k=2, card=2))] + \
        [(f"sep4^{s}", dict(sep_vars=s, k=8)) for s in range(1, 8)]
    rows = []
    for name, kw in configs:
        tree = synth.separator_sweep_tree(**kw)
        n = tree.n_cliques
        seps = [int(np.prod([int(tree.card[v]) for v in
                             set(tree.cliques[c].tolist()) & set(tree.cliques[int(tree.parent[c])].tolist())]))
                for c in range(1, n)]
        t32 = tree.as_dtype(np.float32)
        cpu = []
        for _ in range(3):
            t0 = time.perf_counter()
            hugin.propagate_tree(t32, {})
            cpu.append(1e3 * (time.perf_counter() - t0))
        h = jt.jt_load_synth(t32, compute=jt.JT_F32, max_cases=1, flags=jt.JT_MATERIALIZE_CLIQUES)
        jt.jt_profile_propagate(h, 0, 1)
        fused = min(float(np.sum(jt.jt_profile_propagate(h, 0, 1))) for _ in range(3))
        jt.jt_propagate_per_message(h, 0, 0)
        pm = min(jt.jt_propagate_per_message(h, 0, 0) for _ in range(3))
        assert jt.jt_get_status(h, 0, 1)[0] == jt.JT_OK
        h.free()
        rows.append({"tree": tree.name, "avg_separator_entries": float(np.mean(seps)),
                     "clique_entries": int(tree.entries()), "cpu_oracle_ms": min(cpu), "fused_ms": fused,
                     "per_message_ms": pm, "launches_per_message_path": 4 * (n - 1) + 8,
                     "speedup_fused": min(cpu) / fused, "speedup_per_message": min(cpu) / pm})
    tau = rows[0]["per_message_ms"] / rows[0]["launches_per_message_path"]
    for r in rows:
        r["launch_overhead_share"] = min(1.0, r["launches_per_message_path"] * tau / r["per_message_ms"])
    return {"sweep": "separator_size", "tau_us": 1e3 * tau, "cpu": "FP64 numpy oracle, one core",
            "rows": rows}


def merging_sweep():
    """Merging small separators (the remedy of Sec. 5) on the latency-bound
    trees: the fused propagation (kernel + finalisation, device time, one
    case without evidence, FP32, best of three after a first run) of the
    original tree against merged trees at a few separator thresholds (the
    merged table capped at 3^8 entries for the small tree, 2^10 for the
    binary one)."""
    from paper_1202_3777_gb300 import jt
    from paper_1202_3777_gb300.merge import load_merged
    rows = []
    for tree, thresholds, cap in ((synth.small_tree(), (10,), 3 ** 8),
                                  (synth.binary_serving_tree(), (4, 8, 16), 1 << 10)):
        t32 = tree.as_dtype(np.float32)
        pot = t32.pot.astype(np.float64)

        def fused(h):
            jt.jt_profile_propagate(h, 0, 1)
            ms = min(float(np.sum(jt.jt_profile_propagate(h, 0, 1))) for _ in range(3))
            assert jt.jt_get_status(h, 0, 1)[0] == jt.JT_OK
            return ms

        h = jt.jt_load_synth(t32, compute=jt.JT_F32, max_cases=1)
        rows.append({"tree": tree.name, "min_separator_entries": 0, "cliques": tree.n_cliques,
                     "depth": int(h.info.depth), "fused_ms": fused(h)})
        h.free()
        for th in thresholds:
            h, m = load_merged(tree.card, tree.cliques, tree.parent, pot, th, cap, compute=jt.JT_F32)
            rows.append({"tree": tree.name, "min_separator_entries": th, "max_clique_entries": cap,
                         "cliques": len(m.cliques), "depth": int(h.info.depth), "fused_ms": fused(h)})
            h.free()
    return {"sweep": "merging", "rows": rows}


def measure_serving(rank):
    """Continuous batching over the four resident trees (small, large-clique,
    high-cardinality, 1024-clique binary): a burst of queries gives the
    sustained rate, then Poisson arrivals at a quarter and at half of it give
    p50/p99 latency."""
    from paper_1202_3777_gb300 import serve
    trees = {
        "small": synth.small_tree().as_dtype(np.float32),
        "large_clique": synth.large_clique_tree().as_dtype(np.float32),
        "high_card": synth.high_card_tree().as_dtype(np.float32),
        "binary": synth.binary_serving_tree().as_dtype(np.float32),
    }
    srv = serve.Server(trees, budget_bytes=60 << 30, max_batch=64)
    srv.warm_up()
    work = {n: r.work for n, r in srv.trees.items()}
    names = list(trees)
    rng = np.random.default_rng(20000 + rank)

    def queries(n, base):
        out = []
        for i in range(n):
            name = names[rng.integers(len(names))]
            ev = synth.evidence_matrix(trees[name], 1, (0.01, 0.20), base + i)[0]
            out.append(serve.Query(base + i, name, ev))
        return out

    burst = queries(512, 30000)
    srv.completed = []
    done = srv.run_arrivals([(0.0, q) for q in burst])
    burst_s = max(q.done for q in done) - min(q.arrival for q in done)
    rate = len(done) / burst_s
    # Poisson arrivals for 1.5 s at a quarter and at half of the burst rate;
    # the headline p50/p99 are the quarter-load ones (each propagation fills
    # every SM, so the trees' batches take turns on the GPU and small batches
    # cost nearly as much as large ones: at half load the queues grow)
    loads = []
    for li, load in enumerate((0.25, 0.5)):
        srv.completed = []
        qs = queries(int(load * rate * 1.5) + 1, 40000 + 10000 * li)
        t, arr = 0.0, []
        for q in qs:
            t += rng.exponential(1.0 / (load * rate))
            arr.append((t, q))
        done = srv.run_arrivals(arr)
        loads.append({"load": load, "offered_queries_per_s": load * rate, **serve.latency_summary(done, work)})
    srv.free()
    return {"trees": names, "budget_gb": 60, "max_batch": 64, "burst_queries_per_s": rate,
            "burst_clique_entries_per_s": sum(work[q.tree] for q in burst) / burst_s,
            "offered_queries_per_s": loads[0]["offered_queries_per_s"], "p50_ms": loads[0]["p50_ms"],
            "p99_ms": loads[0]["p99_ms"], "loads": loads}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--impl", default="cuda", choices=["cuda", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ablation", action="store_true")
    ap.add_argument("--sweep-separators", action="store_true",
                    help="print the separator-size sweep (Fig. 6 / Fig. 7 analogues) instead of the bench line")
    ap.add_argument("--sweep-merging", action="store_true",
                    help="print original against merged-tree propagation times instead of the bench line")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_1202_3777_gb300 import build
    build.build()
    from paper_1202_3777_gb300 import jt

    if args.sweep_separators or args.sweep_merging:
        if rank == 0:
            out = separator_sweep() if args.sweep_separators else merging_sweep()
            print(json.dumps(out, default=_json_default), flush=True)
        return 0

    B = args.batch
    tree = synth.WORKLOADS[WORKLOAD]["build"]().as_dtype(np.float32)
    W = tree.work_per_case()
    ev = synth.evidence_matrix(tree, B, 0.05, evidence_seed(rank))
    h = jt.jt_load_synth(tree, compute=jt.JT_F32, max_cases=B)
    jt.jt_set_evidence_dense(h, 0, ev)
    stream = torch.cuda.current_stream()
    sync = torch.cuda.synchronize

    def barrier():
        if world > 1:
            dist.barrier()

    def timed(first, n, steps):
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        barrier()
        sync()
        s0.record(stream)
        for _ in range(steps):
            jt.jt_propagate(h, first, n, stream)
        s1.record(stream)
        sync()
        barrier()
        return s0.elapsed_time(s1) / steps   # ms per step

    def max_over(x):
        return max_over_ranks(x, world, "cuda")

    # plain: one case per jt_propagate call
    for _ in range(args.warmup):
        jt.jt_propagate(h, 0, 1, stream)
    plain_ms = max_over(timed(0, 1, args.steps))

    # batched (the timed step)
    for _ in range(args.warmup):
        jt.jt_propagate(h, 0, B, stream)
    gi = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local]) \
        if os.environ.get("CUDA_VISIBLE_DEVICES") else local
    with Clocks(gi) as clk:
        step_ms = max_over(timed(0, B, args.steps))
    clocks = clk.summary()

    # correctness guard on the timed results
    st = jt.jt_get_status(h, 0, B)
    assert np.all(st == jt.JT_OK), st

    # device time of the dominant kernel (the persistent propagation kernel),
    # CUDA events on the launching stream, same schedule as the timed steps
    prof_b = np.mean([jt.jt_profile_propagate(h, 0, B, stream) for _ in range(3)], axis=0)
    prof_1 = np.mean([jt.jt_profile_propagate(h, 0, 1, stream) for _ in range(3)], axis=0)
    hbm, src = peaks()
    w = 4
    entries = tree.entries()
    info = h.info

    root_entries = int(tree.table_sizes()[0])
    streamed = 2 * entries - root_entries   # collect reads every non-root table, distribute every table

    def alg_bytes(cases):
        # per case: every clique table read once per pass (the root's collect
        # total comes from its distribute pass), messages written and read in
        # each pass; a batch of cases counts each case's bytes (the kernel
        # shares each table read among a block of 8 cases)
        return cases * (w * streamed + w * (4 * msg_total(tree) + info.marginal_len))

    ach_b = alg_bytes(B) / (prof_b[0] * 1e-3) / 1e9
    ach_1 = alg_bytes(1) / (prof_1[0] * 1e-3) / 1e9

    # end to end through the public API with host buffers
    md = np.empty((B, h.marginal_len))
    lzh = np.empty(B)
    sync()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        jt.jt_set_evidence_dense(h, 0, ev)
        jt.jt_propagate(h, 0, B, stream)
        md = jt.jt_get_marginals(h, 0, B, stream=stream)
        lzh = jt.jt_get_log_evidence(h, 0, B, stream=stream)
    sync()
    barrier()
    e2e_ms = max_over(1e3 * (time.perf_counter() - t0) / args.steps)

    total_cases = B * world
    value = job_rate(W, B, world, step_ms)
    plain_value = job_rate(W, 1, world, plain_ms)
    h.free()
    per_message = None
    if not args.no_ablation:
        per_message = measure_per_message(tree, ev[0])
        per_message["fused_kernel_ms"] = float(prof_1[0])
        per_message["fused_with_finalisation_ms"] = float(prof_1[0] + prof_1[1])
    cpt_init = measure_cpt_init(tree, hbm)
    serving = None
    if not args.no_serving:
        serving = measure_serving(rank)
    if rank != 0:
        return 0
    cpu = None
    if not args.no_cpu_baseline:
        cases = [synth.case_from_row(r) for r in ev[: min(B, 4)]]
        rate, done, dt = oracle_rate(tree.as_dtype(np.float32), cases)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{done} of the {B} evidence cases of one step, FP64 numpy oracle ({dt:.1f} s)",
               "host_cores": host_cores()}
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": tree.name, "cases_per_step": B, "cases_per_gpu": B,
                   "observed_frac": 0.05, "entries_per_case": entries, "work_per_case": W,
                   "l2": "inputs larger than L2 (268 MB of FP32 clique tables)",
                   "parallelism": f"replicas x{world}"},
        "plain": {"value": plain_value, "unit": UNIT, "ms_per_case": plain_ms},
        "batched_over_plain": value / plain_value,
        "roofline": {"bound": "hbm", "achieved": ach_b, "peak": hbm, "unit": "GB/s",
                     "frac": ach_b / hbm, "traffic": measured_traffic(B), "kernel": "k_propagate",
                     "kernel_ms": float(prof_b[0]), "alg_bytes": int(alg_bytes(B)),
                     "peak_source": src + " (MEASURED_PEAKS.json hbm_gbs)"},
        "roofline_plain": {"bound": "hbm", "achieved": ach_1, "peak": hbm, "unit": "GB/s", "frac": ach_1 / hbm,
                           "traffic": measured_traffic(1), "kernel_ms": float(prof_1[0]),
                           "alg_bytes": int(alg_bytes(1))},
        "finalize_ms": {"batched": float(prof_b[1]), "plain": float(prof_1[1])},
        "e2e": {"value": job_rate(W, B, world, e2e_ms), "unit": UNIT, "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": int(ev.nbytes), "d2h_bytes_per_step": int(md.nbytes + lzh.nbytes)},
        "serving": serving,
        "per_message": per_message,
        "cpt_init": cpt_init,
        "gpu_launches": int(2 * args.steps),   # k_propagate + k_finalize per step
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    print(json.dumps(out, default=_json_default), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
