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


# DRAM traffic of the propagation kernel from an ncu capture of the
# large-clique workload (dram__bytes_read.sum + dram__bytes_write.sum, in
# profiles/), valid only while the kernel and planner sources are the ones it
# was taken on.  Per kind of schedule: a one-case launch; a block of 4 or 8
# cases; a slab of 32 cases on the lanes.  Every case block or slab streams
# the tables again, so a launch's traffic grows with their number.
TRAFFIC = {
    "sources_sha256": "af87dea2809168b62fe89e9711b586c8290ed1b775998ccf465cf617f7312821",
    "plain": 471.5e6,
    "per_case_block": {4: 496.4e6, 8: 524.4e6},
    "per_slab": 565.2e6,
}
TRAFFIC_SOURCES = ["paper_1202_3777_gb300/csrc/jt_kernels.cu", "paper_1202_3777_gb300/csrc/jt_caselanes.cu",
                   "paper_1202_3777_gb300/csrc/jt_device.cuh", "paper_1202_3777_gb300/csrc/jt_kernels.h",
                   "paper_1202_3777_gb300/csrc/jt_internal.h", "paper_1202_3777_gb300/csrc/jt_plan.cpp"]


def sources_sha256():
    import hashlib
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(schedule, cases):
    """ncu DRAM bytes per launch of the schedule over `cases` cases, or None
    once the kernel or planner sources differ from the profiled ones."""
    try:
        if TRAFFIC["sources_sha256"] is None or sources_sha256() != TRAFFIC["sources_sha256"]:
            return None
    except OSError:
        return None
    cb = schedule["case_block"]
    if cb == 1:
        per, units = TRAFFIC["plain"], cases
    elif cb == 32:
        per, units = TRAFFIC["per_slab"], (cases + 31) // 32
    else:
        per, units = (TRAFFIC["per_case_block"] or {}).get(cb), (cases + cb - 1) // cb
    return None if per is None else int(per * units)


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


def kernel_tour():
    """One small invocation of every kernel family, for profiling each on its
    own: case lanes (large-clique tree, one slab of 32 cases), padded case
    lanes with their table padding (256-clique tree, 64 cases), one case per
    item (large-clique tree), 4-case blocks (high-cardinality tree, 16
    cases), the whole tree per CTA (32-clique tree, FP32 and FP64), the
    paper's per-message propagation (32-clique tree), CPT initialisation and
    the calibrated-table read-out (large-clique tree).  Schedules are fixed
    (no width timing, no block tuning), every result is checked for its
    status, and the device time of each propagation's two kernels is
    printed (CUDA events; the kernels are the ones a capture of this run
    sees)."""
    from paper_1202_3777_gb300 import jt
    os.environ["JT_BLOCK_TUNE"] = "0"
    out = {}

    def run(name, tree, n, cb, compute=jt.JT_F32, flags=0, seed=50):
        os.environ["JT_CASE_BLOCK"] = str(cb)
        h = jt.jt_load_synth(tree, compute=compute, max_cases=n, flags=flags)
        jt.jt_set_evidence_dense(h, 0, synth.evidence_matrix(tree, n, 0.05, seed))
        jt.jt_propagate(h, 0, n)
        ms = [float(x) for x in jt.jt_profile_propagate(h, 0, n)]
        assert np.all(jt.jt_get_status(h, 0, n) == jt.JT_OK), name
        sch = jt.jt_get_schedule(h, 0, n)
        out[name] = {"cases": n, "case_block": sch["case_block"], "padded": sch["padded"],
                     "propagation_ms": ms[0], "finalisation_ms": ms[1]}
        return h

    large = synth.large_clique_tree().as_dtype(np.float32)
    run("case_lanes", large, 32, 32).free()
    run("padded_lanes", synth.batched_tree().as_dtype(np.float32), 64, 32).free()
    run("one_case", large, 1, 1).free()
    run("case_blocks", synth.high_card_tree().as_dtype(np.float32), 16, 4).free()
    small = synth.small_tree()
    run("whole_tree_f32", small.as_dtype(np.float32), 1, 0).free()
    run("whole_tree_f64", small, 1, 0, compute=jt.JT_F64).free()
    h = run("per_message_tree", small.as_dtype(np.float32), 1, 1, flags=jt.JT_MATERIALIZE_CLIQUES)
    out["per_message"] = {"naive_ms": jt.jt_propagate_per_message(h, 0, 0),
                          "interleaved_ms": jt.jt_propagate_per_message(h, 0, 1)}
    h.free()
    fams, vals = synth.bn_for_tree(large, 7, max_parents=3)
    h = jt.jt_load_tree(large.card, large.cliques, large.parent, None, compute=jt.JT_F32, max_cases=1,
                        flags=jt.JT_MATERIALIZE_CLIQUES)
    out["cpt_init_ms"] = jt.jt_init_from_cpts(h, fams, vals)
    os.environ["JT_CASE_BLOCK"] = "1"
    jt.jt_propagate(h, 0, 1)
    sizes = large.table_sizes()
    tab = jt.jt_get_clique(h, 0, 3, int(sizes[3]))
    assert np.isfinite(tab).all() and abs(float(tab.sum()) - 1.0) < 1e-6
    h.free()
    for k in ("JT_CASE_BLOCK", "JT_BLOCK_TUNE"):
        os.environ.pop(k, None)
    return out


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
    sustained rate; Poisson arrivals at 0.5, 0.8 and 0.95 of it give p50/p99
    latency.  Batches of different trees share the SMs and overlap on the
    device (counted from the kernels' spans on the global timer).  Per tree,
    the batched rate (a full batch of its slots) against the plain one (one
    case per call), and a sample of served queries for the error against the
    oracle."""
    import torch
    from paper_1202_3777_gb300 import jt, serve
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
    srv.completed, srv.spans = [], []
    done = srv.run_arrivals([(0.0, q) for q in burst])
    burst_s = max(q.done for q in done) - min(q.arrival for q in done)
    rate = len(done) / burst_s
    burst_overlap = serve.overlapping_pairs(srv.spans)
    sample = [(q.tree, q.states.copy(), q.marginals.copy(), q.log_z) for q in sorted(done, key=lambda q: q.qid)[:12]]
    loads = []
    for li, load in enumerate((0.5, 0.8, 0.95)):
        srv.completed, srv.spans = [], []
        qs = queries(int(load * rate * 1.5) + 1, 40000 + 10000 * li)
        t, arr = 0.0, []
        for q in qs:
            t += rng.exponential(1.0 / (load * rate))
            arr.append((t, q))
        done = srv.run_arrivals(arr)
        loads.append({"load": load, "offered_queries_per_s": load * rate, **serve.latency_summary(done, work),
                      "batches": len(srv.spans), "mean_batch": float(np.mean([sp[3] for sp in srv.spans])),
                      "overlapping_batch_pairs": serve.overlapping_pairs(srv.spans)})
    # per tree: a full batch of its slots against one case per call
    per_tree = {}
    for name, r in srv.trees.items():
        n = r.slots
        jt.jt_set_evidence_dense(r.handle, 0, synth.evidence_matrix(trees[name], n, (0.01, 0.20), 90000),
                                 stream=r.stream)
        ms = {}
        for k in (n, 1):
            for _ in range(3):
                jt.jt_propagate(r.handle, 0, k, r.stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(r.stream)
            reps = 10
            for _ in range(reps):
                jt.jt_propagate(r.handle, 0, k, r.stream)
            e1.record(r.stream)
            e1.synchronize()
            ms[k] = e0.elapsed_time(e1) / reps
        per_tree[name] = {"slots": n, "batched_clique_entries_per_s": work[name] * n / (ms[n] * 1e-3),
                          "plain_clique_entries_per_s": work[name] / (ms[1] * 1e-3),
                          "batched_over_plain": (work[name] * n / ms[n]) / (work[name] / ms[1]),
                          "case_block": jt.jt_get_schedule(r.handle, 0, n)["case_block"]}
    srv.free()
    return {"trees": names, "budget_gb": 60, "max_batch": 64, "burst_queries_per_s": rate,
            "burst_clique_entries_per_s": sum(work[q.tree] for q in burst) / burst_s,
            "burst_overlapping_batch_pairs": burst_overlap,
            "offered_queries_per_s": loads[0]["offered_queries_per_s"], "p50_ms": loads[0]["p50_ms"],
            "p99_ms": loads[0]["p99_ms"], "loads": loads, "per_tree": per_tree, "_sample": (trees, sample)}


def serving_errors(sample):
    """Error against the oracle of a sample of served queries."""
    from oracle import hugin
    trees, rows = sample
    worst, worst_lz = 0.0, 0.0
    for name, states, marg, lz in rows:
        t = trees[name]
        ref = hugin.propagate_tree(t, hugin.evidence_dict(*synth.case_from_row(states)))
        e = rel_errors(t, [ref], [lz], [marg])
        worst, worst_lz = max(worst, e["max_rel_err"]), max(worst_lz, e["logz_rel_err"])
    return {"cases": len(rows), "max_rel_err": worst, "logz_rel_err": worst_lz, "tolerance": 1e-5,
            "oracle": "FP64 numpy oracle (oracle/hugin.py)"}


def workload_rows(name, tree, n, seed):
    """Dense evidence rows of n cases of a named workload (its own recipe:
    a fraction of the variables, or a fixed number of observed variables)."""
    w = synth.WORKLOADS[name]
    if "n_obs" in w:
        out = np.full((n, tree.n_vars), -1, np.int16)
        for i in range(n):
            v, st = synth.random_evidence(tree, w["n_obs"], seed + i)
            out[i, v] = st
        return out
    return synth.evidence_matrix(tree, n, w["frac"], seed)


def alg_bytes_of(tree, info, cases, w=4):
    """Algorithmic bytes of a propagation launch over `cases` cases: per
    case every clique table read once per pass (the root's collect total
    comes from its distribute pass) plus the messages written and read in
    each pass and the marginal sources; a batch counts each case's bytes (a
    block of cases shares each table read)."""
    streamed = 2 * tree.entries() - int(tree.table_sizes()[0])
    return cases * (w * streamed + w * (4 * msg_total(tree) + info.marginal_len))


def measure_workload(jt, torch, name, tree, B, steps, warmup, seed, world, clocks_index=None, e2e=False,
                     plain=True, keep=4):
    """One workload: B cases per jt_propagate (timed steps, CUDA events on the
    launching stream, max over ranks), the plain one-case path, the device
    time of the propagation and finalisation kernels (jt_profile_propagate),
    the roofline of the propagation kernel, and the results of the first
    `keep` cases for the error against the oracle."""
    import torch.distributed as dist
    W = tree.work_per_case()
    ev = workload_rows(name, tree, B, seed)
    h = jt.jt_load_synth(tree, compute=jt.JT_F32, max_cases=B)
    jt.jt_set_evidence_dense(h, 0, ev)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()

    def timed(first, n, k):
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        s0.record(stream)
        for _ in range(k):
            jt.jt_propagate(h, first, n, stream)
        s1.record(stream)
        torch.cuda.synchronize()
        barrier()
        return max_over_ranks(s0.elapsed_time(s1) / k, world, "cuda")

    out = {"workload": tree.name, "cases": B}
    if plain:
        for _ in range(warmup):
            jt.jt_propagate(h, 0, 1, stream)
        out["plain_ms"] = timed(0, 1, steps)
    for _ in range(warmup):
        jt.jt_propagate(h, 0, B, stream)
    if clocks_index is not None:
        with Clocks(clocks_index) as clk:
            out["step_ms"] = timed(0, B, steps)
        out["clocks"] = clk.summary()
    else:
        out["step_ms"] = timed(0, B, steps)
    st = jt.jt_get_status(h, 0, B)
    assert np.all(st == jt.JT_OK), st
    out["schedule"] = jt.jt_get_schedule(h, 0, B)
    prof_b = np.mean([jt.jt_profile_propagate(h, 0, B, stream) for _ in range(3)], axis=0)
    out["kernel_ms"], out["finalize_ms"] = float(prof_b[0]), float(prof_b[1])
    if plain:
        prof_1 = np.mean([jt.jt_profile_propagate(h, 0, 1, stream) for _ in range(3)], axis=0)
        out["plain_kernel_ms"], out["plain_finalize_ms"] = float(prof_1[0]), float(prof_1[1])
    info = h.info
    out["alg_bytes"] = int(alg_bytes_of(tree, info, B))
    out["alg_bytes_plain"] = int(alg_bytes_of(tree, info, 1))
    out["work_per_case"] = W
    out["value"] = job_rate(W, B, world, out["step_ms"])
    if plain:
        out["plain_value"] = job_rate(W, 1, world, out["plain_ms"])
    if e2e:
        md = lzh = None
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(steps):
            jt.jt_set_evidence_dense(h, 0, ev)
            jt.jt_propagate(h, 0, B, stream)
            md = jt.jt_get_marginals(h, 0, B, stream=stream)
            lzh = jt.jt_get_log_evidence(h, 0, B, stream=stream)
        torch.cuda.synchronize()
        barrier()
        out["e2e_ms"] = max_over_ranks(1e3 * (time.perf_counter() - t0) / steps, world, "cuda")
        out["h2d_bytes"] = int(ev.nbytes)
        out["d2h_bytes"] = int(md.nbytes + lzh.nbytes)
    lz = jt.jt_get_log_evidence(h, 0, B)
    m = jt.jt_get_marginals(h, 0, B)
    out["_sample"] = (ev[:keep].copy(), lz[:keep].copy(), m[:keep].copy())
    h.free()
    return out


def roofline_of(kernel, alg_bytes, kernel_ms, hbm, src, traffic=None):
    ach = alg_bytes / (kernel_ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm, "traffic": traffic,
            "kernel": kernel, "kernel_ms": kernel_ms, "alg_bytes": int(alg_bytes),
            "peak_source": src + " (MEASURED_PEAKS.json hbm_gbs)"}


def prop_kernel_name(schedule):
    if schedule["case_block"] == 32:
        return "k_propagate_cl<true>" if schedule.get("padded") else "k_propagate_cl<false>"
    return f"k_propagate<float, {schedule['case_block']}>"


def measure_latency(jt, torch, steps=50):
    """Device time per propagation (propagation + finalisation kernels, one
    case, CUDA events over back-to-back launches on one stream) of the small
    trees: the 32-clique tree of ternary variables (FP64 potentials, also
    run in FP32) and the 1024-clique binary tree (FP32)."""
    stream = torch.cuda.current_stream()
    out = {}
    for key, tree, comp in (("small_f64", synth.small_tree(), jt.JT_F64),
                            ("small_f32", synth.small_tree().as_dtype(np.float32), jt.JT_F32),
                            ("binary_f32", synth.binary_serving_tree().as_dtype(np.float32), jt.JT_F32)):
        h = jt.jt_load_synth(tree, compute=comp, max_cases=1)
        jt.jt_set_evidence_dense(h, 0, synth.evidence_matrix(tree, 1, 0.10, 77))
        for _ in range(5):
            jt.jt_propagate(h, 0, 1, stream)
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        s0.record(stream)
        for _ in range(steps):
            jt.jt_propagate(h, 0, 1, stream)
        s1.record(stream)
        torch.cuda.synchronize()
        assert jt.jt_get_status(h, 0, 1)[0] == jt.JT_OK
        out[key] = {"workload": tree.name, "us_per_propagation": 1e3 * s0.elapsed_time(s1) / steps,
                    "cliques": tree.n_cliques, "depth": int(h.info.depth), "schedule": jt.jt_get_schedule(h, 0, 1)}
        h.free()
    return out


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
    ap.add_argument("--no-extra", action="store_true",
                    help="only the headline workload (no high-cardinality, 4096-case or latency keys)")
    ap.add_argument("--sweep-separators", action="store_true",
                    help="print the separator-size sweep (Fig. 6 / Fig. 7 analogues) instead of the bench line")
    ap.add_argument("--sweep-merging", action="store_true",
                    help="print original against merged-tree propagation times instead of the bench line")
    ap.add_argument("--kernel-tour", action="store_true",
                    help="run one small case of every kernel family (for profiling) instead of the bench line")
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

    if args.sweep_separators or args.sweep_merging or args.kernel_tour:
        if rank == 0:
            out = separator_sweep() if args.sweep_separators else merging_sweep() if args.sweep_merging \
                else kernel_tour()
            print(json.dumps(out, default=_json_default), flush=True)
        return 0

    B = args.batch
    hbm, src = peaks()
    gi = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local]) \
        if os.environ.get("CUDA_VISIBLE_DEVICES") else local
    tree = synth.WORKLOADS[WORKLOAD]["build"]().as_dtype(np.float32)
    head = measure_workload(jt, torch, WORKLOAD, tree, B, args.steps, args.warmup, evidence_seed(rank), world,
                            clocks_index=gi, e2e=True)
    extra = {}
    if not args.no_extra:
        hc_tree = synth.WORKLOADS["high_card"]["build"]().as_dtype(np.float32)
        extra["high_card"] = measure_workload(jt, torch, "high_card", hc_tree, B, args.steps, args.warmup,
                                              evidence_seed(rank) + 500, world)
        c4_tree = synth.WORKLOADS["batched"]["build"]().as_dtype(np.float32)
        extra["batched_4096"] = measure_workload(jt, torch, "batched", c4_tree, synth.WORKLOADS["batched"]["n_cases"],
                                                 min(args.steps, 3), args.warmup, 4000 + 100000 * rank, world,
                                                 plain=True)
    latency = None if args.no_extra else measure_latency(jt, torch)
    per_message = None
    if not args.no_ablation:
        per_message = measure_per_message(tree, workload_rows(WORKLOAD, tree, 1, evidence_seed(rank))[0])
        per_message["fused_kernel_ms"] = head["plain_kernel_ms"]
        per_message["fused_with_finalisation_ms"] = head["plain_kernel_ms"] + head["plain_finalize_ms"]
    cpt_init = measure_cpt_init(tree, hbm)
    serving = None
    if not args.no_serving:
        serving = measure_serving(rank)
    if rank != 0:
        return 0

    # CPU leg: the oracle on a bounded sample of every workload's cases (its
    # rate is the CPU baseline of the headline workload), and the GPU's error
    # against it on the same cases
    cpu = None
    errors = {}
    if not args.no_cpu_baseline:
        ev, lz, m = head["_sample"]
        cases = [synth.case_from_row(r) for r in ev]
        rate, done, dt, err = oracle_rate(tree, cases, 20.0, gpu=(lz, m))
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{done} of the {B} evidence cases of one step, FP64 numpy oracle ({dt:.1f} s)",
               "host_cores": host_cores()}
        errors[WORKLOAD] = err
        for key, res in extra.items():
            t = hc_tree if key == "high_card" else c4_tree
            ev, lz, m = res["_sample"]
            _, _, _, errors[key] = oracle_rate(t, [synth.case_from_row(r) for r in ev], 10.0, gpu=(lz, m))
        if serving is not None:
            errors["serving"] = serving_errors(serving.pop("_sample"))
    if serving is not None:
        serving.pop("_sample", None)

    def strip(d):
        return {k: v for k, v in d.items() if not k.startswith("_")}

    value = head["value"]
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["step_ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": tree.name, "cases_per_step": B, "cases_per_gpu": B,
                   "observed_frac": 0.05, "entries_per_case": tree.entries(), "work_per_case": head["work_per_case"],
                   "l2": "inputs larger than L2 (268 MB of FP32 clique tables)",
                   "parallelism": f"replicas x{world}"},
        "schedule": head["schedule"],
        "plain": {"value": head["plain_value"], "unit": UNIT, "ms_per_case": head["plain_ms"]},
        "batched_over_plain": value / head["plain_value"],
        "roofline": roofline_of(prop_kernel_name(head["schedule"]), head["alg_bytes"], head["kernel_ms"], hbm, src,
                                measured_traffic(head["schedule"], B)),
        "roofline_plain": roofline_of("k_propagate<float, 1>", head["alg_bytes_plain"], head["plain_kernel_ms"], hbm,
                                      src, measured_traffic({"case_block": 1}, 1)),
        "finalize_ms": {"batched": head["finalize_ms"], "plain": head["plain_finalize_ms"]},
        "e2e": {"value": job_rate(head["work_per_case"], B, world, head["e2e_ms"]), "unit": UNIT,
                "ms_per_step": head["e2e_ms"], "h2d_bytes_per_step": head["h2d_bytes"],
                "d2h_bytes_per_step": head["d2h_bytes"]},
        "oracle_error": errors or None,
        "serving": serving,
        "per_message": per_message,
        "cpt_init": cpt_init,
        "gpu_launches": int(2 * args.steps),   # propagation + finalisation kernel per step
        "clocks": head["clocks"],
        "cpu_baseline": cpu,
    }
    for key, res in extra.items():
        r = strip(res)
        r["roofline"] = roofline_of(prop_kernel_name(res["schedule"]), res["alg_bytes"], res["kernel_ms"], hbm, src)
        r["unit"] = UNIT
        if "plain_value" in res:
            r["batched_over_plain"] = res["value"] / res["plain_value"]
        out[key] = r
    if latency is not None:
        out["latency"] = latency
    print(json.dumps(out, default=_json_default), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
