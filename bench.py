#!/usr/bin/env python3
"""Throughput of the volume-potential box FMM on one GB300 (target points per second).

One step = one call of the box code (S2M, M2M, M2L/S2L/L2L, near-field tables,
L2T, M2T) over the whole tree of the adaptive 20-Gaussian workload (k = 16,
p = 40, tol 1e-10, depth <= 16), with tree, operators and f resident in HBM.
Prints one JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload adaptive_gauss20|uniform_gauss3|kinked] [--precision fp64|mixed]

--impl reference times the CPU oracle (plain numpy FP64 box code) on bounded
samples of the same workload on the host cores. Under torchrun every rank runs an
independent replica of the workload (the path is not sharded: replicas only).
"""
from __future__ import annotations

import os

# the CPU oracle legs run single-threaded BLAS; the GPU path does not use host BLAS
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse  # noqa: E402
import dataclasses  # noqa: E402
import json  # noqa: E402
import math  # noqa: E402
import statistics  # noqa: E402
import subprocess  # noqa: E402
import sys  # noqa: E402
import time  # noqa: E402

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "volume-FMM target pts/s at 1e-10 rel err: mixed/batched vs plain FP64, 1 GB300"
UNIT = "target points/s"
FP64_OVER_BF16 = 1.25 / 2250.0  # nominal dense FP64 / BF16 tensor ratio of GB300


def workload(name):
    if name == "adaptive_gauss20":
        return W.adaptive_gauss20()
    if name == "uniform_gauss3":
        return W.uniform_gauss3()
    if name == "kinked":
        return W.kinked()
    if name == "shared_rhs64":  # 64 right-hand sides sharing the uniform depth-3, k = 8 tree
        base = W.uniform_gauss3()
        return dataclasses.replace(base, name="shared_tree_rhs64_" + base.name, sources=W.shared_tree_rhs(64))
    if name.startswith("uniform_d") and "_k" in name:  # uniform_d<depth>_k<k>: 3 Gaussians, p = 2.5 k
        d, k = name[len("uniform_d"):].split("_k")
        return W.uniform_gauss3(depth=int(d), k=int(k), p=int(2.5 * int(k)))
    raise SystemExit("unknown workload " + name)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def start(self):
        return self.__enter__()

    def stop(self):
        self.__exit__(None, None, None)

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "samples": len(sm),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------- CPU oracle
def oracle_setup(wl, rule="tail"):
    from oracle import tables
    from oracle import tree as T
    src = wl.sources[0]
    if wl.uniform_depth >= 0:
        ot = T.build_uniform(wl.cx, wl.cy, wl.width, wl.k, wl.uniform_depth)
    else:
        ot = T.build_adaptive(wl.cx, wl.cy, wl.width, wl.k, src, wl.tol, wl.max_depth, wl.min_depth, rule=rule)
    return ot, T.build_lists(ot), tables.Ops(wl.k, wl.p), ot.sample(src)


def oracle_sample_step(ot, L, ops, F, leaves):
    """One oracle step on a bounded sample: the full upward pass plus the leaf pass for `leaves`."""
    from oracle import fmm
    t0 = time.perf_counter()
    out = fmm.solve(ot, L, ops, F, leaves=leaves)
    return time.perf_counter() - t0, out


def pick_sample(ot, L, ops, F, budget_s, rng):
    """Leaves for one step of about budget_s seconds (calibrated on a short run)."""
    n_leaves = ot.n_leaves
    probe = rng.choice(n_leaves, size=min(8, n_leaves), replace=False)
    dt, _ = oracle_sample_step(ot, L, ops, F, probe)
    per = dt / len(probe)
    m = int(max(1, min(n_leaves, budget_s / max(per, 1e-6))))
    return np.sort(rng.choice(n_leaves, size=m, replace=False))


# The oracle over all host cores: a pool of spawned worker processes (spawned, since the GPU may
# already be in use by this process), each building the oracle's tree, lists and tables once; one
# step hands every worker an equal share of the sampled leaves, and each worker runs the full upward
# pass plus the leaf pass of its share (the oracle as it stands, one process per core).
_POOL_ORACLE = None


def _pool_init(wl, rule):
    global _POOL_ORACLE
    _POOL_ORACLE = oracle_setup(wl, rule)


def _pool_step(leaves):
    ot, L, ops, F = _POOL_ORACLE
    return oracle_sample_step(ot, L, ops, F, leaves)[0]


class OraclePool:
    def __init__(self, wl, rule, cores=None):
        import multiprocessing as mp
        self.cores = int(cores or os.cpu_count() or 1)
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_pool_init, initargs=(wl, rule))

    def step(self, leaves):
        """Wall time of one pass over `leaves`, split evenly over the workers."""
        chunks = [c for c in np.array_split(np.asarray(leaves), self.cores) if len(c)]
        t0 = time.perf_counter()
        self.pool.map(_pool_step, chunks, chunksize=1)
        return time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def run_reference(args, wl):
    ot, L, ops, F = oracle_setup(wl, args.refine)
    pool = OraclePool(wl, args.refine)
    rng = np.random.default_rng(7)
    # a step of about 120 s / (steps + warmup) on one core, spread over all cores
    leaves = pick_sample(ot, L, ops, F, budget_s=max(2.0, 120.0 / max(1, args.steps + args.warmup)), rng=rng)
    kk = wl.k * wl.k
    times = []
    for i in range(args.warmup + args.steps):
        dt = pool.step(leaves)
        if i >= args.warmup:
            times.append(dt)
    pool.close()
    ms = 1e3 * statistics.mean(times)
    value = len(leaves) * kk / (ms / 1e3)
    sample = ("%d of %d leaves (%d targets) per step split over %d worker processes, each with the full "
              "upward pass" % (len(leaves), ot.n_leaves, len(leaves) * kk, pool.cores))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "n_leaves": ot.n_leaves, "n_targets": ot.n_leaves * kk, "k": wl.k,
                       "p": wl.p, "parallelism": "replicas" if args.gpus > 1 else "single GPU",
                       "refine": args.refine},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(wl, gpu_u, budget_s=15.0, rule="tail"):
    """Oracle on a bounded sample of the same workload; also the sampled error of each GPU result
    (gpu_u: {form: (u, u_x, u_y)})."""
    t0 = time.perf_counter()
    ot, L, ops, F = oracle_setup(wl, rule)
    setup_s = time.perf_counter() - t0
    rng = np.random.default_rng(11)
    leaves = pick_sample(ot, L, ops, F, budget_s, rng)
    dt, ref = oracle_sample_step(ot, L, ops, F, leaves)
    # when the sample is the whole workload and quick, repeat it up to about 10 s and take the mean
    runs = [dt]
    while sum(runs) < min(10.0, budget_s) and len(runs) < 20:
        runs.append(oracle_sample_step(ot, L, ops, F, leaves)[0])
    dt = statistics.mean(runs)
    kk = wl.k * wl.k
    # the same sample over all host cores, repeated up to about 10 s
    pool = OraclePool(wl, rule)
    pool.step(leaves)  # warm-up: every worker has built its oracle
    pruns = []
    while sum(pruns) < 10.0 and len(pruns) < 20:
        pruns.append(pool.step(leaves))
    pool.close()
    pdt = statistics.mean(pruns)
    errs = None
    if gpu_u:
        errs = {}
        for form, res in gpu_u.items():
            if res[0].shape[0] != ot.n_leaves * kk:
                continue
            errs[form] = {}
            for q, nm in enumerate(("u", "u_x", "u_y")):
                got = res[q].reshape(ot.n_leaves, kk)[leaves]
                errs[form][nm] = float(np.max(np.abs(got - ref[q])) / np.max(np.abs(ref[q])))
    one = {"value": len(leaves) * kk / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": "%d of %d leaves (%d targets), full upward pass included, %.1f s per run, mean of %d runs; "
                     "oracle setup %.1f s untimed" % (len(leaves), ot.n_leaves, len(leaves) * kk, dt, len(runs),
                                                        setup_s)}
    allc = {"value": len(leaves) * kk / pdt, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
            "sample": "the same %d leaves split over %d worker processes (one per host core), each with the full "
                      "upward pass, %.2f s per run, mean of %d runs" % (len(leaves), pool.cores, pdt, len(pruns))}
    return allc, one, errs


# ----------------------------------------------------------------------------- batched problems
def batch_workloads(n):
    """Member i of the uneven batch: 3 Gaussians, leaf target N_i, k_i (workloads.batch_members),
    tree by the greedy leaf-count rule on the unit box, max depth 16."""
    out = []
    for m in W.batch_members(n):
        wl = W.Workload("batch_member_k%d_n%d" % (m["k"], m["n_leaves_target"]), 0.0, 0.0, 1.0, m["k"], m["p"],
                        0.0, 16, 0, -1, [m["source"]])
        out.append((wl, m["n_leaves_target"]))
    return out


def run_batch(args):
    """Config 'batchN': N independent uneven problems in one CUDA graph (mixed form), the same batch in
    the FP64 form beside it. The reference arm times the oracle on the smallest members."""
    n_members = int(args.workload[len("batch"):] or 256)
    members = batch_workloads(n_members)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    name = "batch%d_uneven_gauss3" % n_members
    if args.impl == "reference":
        if rank == 0:
            from oracle import fmm, tables
            from oracle import tree as T
            wl, n_t = min(members, key=lambda x: x[1])
            src = wl.sources[0]
            ot = T.build_greedy(0.0, 0.0, 1.0, wl.k, src, n_t, 16)
            L, ops, F = T.build_lists(ot), tables.Ops(wl.k, wl.p), ot.sample(src)
            times = []
            for i in range(args.warmup + args.steps):
                t0 = time.perf_counter()
                fmm.solve(ot, L, ops, F)
                if i >= args.warmup:
                    times.append(time.perf_counter() - t0)
            ms = 1e3 * statistics.mean(times)
            value = ot.n_leaves * wl.k * wl.k / (ms / 1e3)
            sample = "the smallest member (%d leaves, k = %d) solved whole per step" % (ot.n_leaves, wl.k)
            print(json.dumps({"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                              "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                              "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                              "data": "synthetic",
                              "config": {"workload": name, "parallelism": "replicas" if world > 1 else "single GPU"},
                              "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                                               "sample": sample},
                              "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                                      "d2h_bytes_per_step": 0}}), flush=True)
        return
    import torch
    torch.cuda.set_device(local)
    from paper_1610_00823_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_1610_00823_gb300 import build as b
        b.build()
    import paper_1610_00823_gb300 as v
    from paper_1610_00823_gb300.api import Batch, tune, volume_potential_profiled, workspace
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    t0 = time.perf_counter()
    # every member's tree in one native call (host threads, a stream each), then its f
    trees = v.tree_build_many([dict(cx=0.0, cy=0.0, width=1.0, k=wl.k, source=wl.sources[0], n_leaves=n_t,
                                    max_depth=16) for wl, n_t in members])
    fs = [v.source_sample(tree, wl.sources[0]) for (wl, _), tree in zip(members, trees)]
    torch.cuda.synchronize()
    t_tree = time.perf_counter() - t0
    n_targets = sum(f.numel() for f in fs)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def make_items(precision):
        ops = {k: v.ops_create(k, 20 if k == 8 else 40, precision) for k in sorted({wl.k for wl, _ in members})}
        items = []
        for (wl, _), tree, f in zip(members, trees, fs):
            out = tuple(torch.empty_like(f) for _ in range(3))
            ws = workspace(tree, ops[wl.k], 1)
            if precision == v.MIXED and not args.no_tune:
                tune(tree, ops[wl.k], f, out, ws, stream)  # split-K autotuner, per member
            items.append((tree, ops[wl.k], f, out, ws))
        return ops, items

    def time_graph(items, steps, clk=None, streams=None):
        b = Batch(16)
        if streams is None:
            tuned = b.tune(items, stream)  # schedule autotuner: side-stream count by timed graph replays
        else:
            b = Batch(streams)
            tuned = (streams, None)
        g = b.graph(items, stream)
        for _ in range(args.warmup):
            g.launch(stream)
        torch.cuda.synchronize()
        times = []
        if clk is not None:
            clk.start()
        for _ in range(steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.launch(stream)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        if clk is not None:
            clk.stop()
        return statistics.mean(times), tuned, b, g

    t0 = time.perf_counter()
    ops_mx, items_mx = make_items(v.MIXED)
    torch.cuda.synchronize()
    t_ops = time.perf_counter() - t0
    clk = ClockSampler(local)
    ms, tuned, b, g = time_graph(items_mx, args.steps, clk)
    value = n_targets / (ms / 1e3)
    # near-field roofline: executed tensor flops over every member's near stage (profiled solves)
    tc, near_ms, launches = 0.0, 0.0, 0
    for tree, ops, f, out, ws in items_mx:
        stages, nl = volume_potential_profiled(tree, ops, f, out, ws, stream=stream)
        kk_m = tree.k * tree.k
        sn = ops.slices["near"]
        tc += sn * (sn + 1) / 2 * 2.0 * 3 * kk_m * kk_m * tree.list_len[0]  # algorithmic slice-product flops
        near_ms += stages.get("near_tc") or stages["near"]
        launches += nl
    peaks, peak_kind = measured_peaks()
    achieved = tc / (near_ms / 1e3) / 1e12
    roof = {"kernel": "split_gemm_kernel (near field, split-BF16 tcgen05), summed over members",
            "flops": "algorithmic: S(S+1)/2 slice products (S = the near field's slices) x 2 x 3k^2 x k^2 "
                     "per U-list entry",
            "bound": "tensor", "achieved": achieved, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
            "frac": achieved / peaks["bf16_tflops"], "traffic": None, "peak_source": "%s bf16 burst" % peak_kind,
            "flops_per_launch": tc / n_members, "ms_per_launch": near_ms / n_members,
            "note": "members profiled one at a time, outside the batch graph"}
    # end to end: pinned host f in, u/u_x/u_y out, the batch graph between (copies on the same stream)
    hosts = [(f.cpu().pin_memory(), tuple(torch.empty(f.shape, dtype=f.dtype).pin_memory() for _ in range(3)))
             for f in fs]
    e2e = []
    for _ in range(max(3, args.steps // 2)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for (fh, _), (tree, ops, f, out, ws) in zip(hosts, items_mx):
            f.copy_(fh, non_blocking=True)
        g.launch(stream)
        for (_, oh), (tree, ops, f, out, ws) in zip(hosts, items_mx):
            for q in range(3):
                oh[q].copy_(out[q], non_blocking=True)
        stream.synchronize()
        e2e.append(1e3 * (time.perf_counter() - t0))
    res_mx = [tuple(o.clone() for o in it[3]) for it in items_mx]
    del g, b
    fp64 = None
    if not args.no_fp64_compare:
        ops64, items64 = make_items(v.FP64)
        ms64, tuned64, b64, g64 = time_graph(items64, 3, streams=tuned[0])
        err = [0.0, 0.0, 0.0]
        for rm, it in zip(res_mx, items64):
            for q in range(3):
                d = torch.max(torch.abs(rm[q] - it[3][q])).item() / max(torch.max(torch.abs(it[3][q])).item(), 1e-300)
                err[q] = max(err[q], d)
        fp64 = {"value": n_targets / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64, "streams": tuned64[0],
                "mixed_over_fp64_speedup": ms64 / ms, "max_member_rel_diff_mixed_vs_fp64": err}
        del g64, b64, items64
    cpu = None
    if not args.no_cpu_baseline:
        from oracle import fmm, tables
        from oracle import tree as T
        i_small = min(range(n_members), key=lambda i: members[i][1])
        wl, n_t = members[i_small]
        ot = T.build_greedy(0.0, 0.0, 1.0, wl.k, wl.sources[0], n_t, 16)
        L, ops_o, F = T.build_lists(ot), tables.Ops(wl.k, wl.p), ot.sample(wl.sources[0])
        t0 = time.perf_counter()
        ref = fmm.solve(ot, L, ops_o, F)
        dt = time.perf_counter() - t0
        got = [res_mx[i_small][q].cpu().numpy().reshape(ref[q].shape) for q in range(3)]
        cpu = {"value": ot.n_leaves * wl.k * wl.k / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "member %d (%d leaves, k = %d) solved whole, %.1f s" % (i_small, ot.n_leaves, wl.k, dt),
               "rel_err_member_vs_oracle": [float(np.max(np.abs(got[q] - ref[q])) / np.max(np.abs(ref[q])))
                                            for q in range(3)]}
    if rank == 0:
        n_leaves = sum(t.n_leaves for t in trees)
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16x6+f64", "data": "synthetic",
            "config": {"workload": name, "members": n_members, "n_leaves": n_leaves, "n_targets": n_targets,
                       "k_mix": {str(k): sum(1 for wl, _ in members if wl.k == k) for k in (8, 16)},
                       "leaf_targets": [min(n for _, n in members), max(n for _, n in members)],
                       "streams": tuned[0], "tune_ms": tuned[1], "launch": "one CUDA graph (all members)",
                       "l2": "flushed between timed steps (256 MB write outside the events)",
                       "parallelism": "single GPU", "tree_build_s": t_tree, "ops_create_s": t_ops},
            "roofline": roof, "cpu_baseline": cpu, "fp64_form": fp64,
            "e2e": {"value": n_targets / (statistics.mean(e2e) / 1e3), "unit": UNIT,
                    "h2d_bytes_per_step": n_targets * 8, "d2h_bytes_per_step": 3 * n_targets * 8,
                    "ms_per_step": statistics.mean(e2e)},
            "gpu_launches": launches, "clocks": clk.summary()}), flush=True)


# ----------------------------------------------------------------------------- other workloads
def _sub_bench(argv, timeout_s):
    """One bench.py run in a child process (same GPU); its JSON line, or the reason it has none."""
    cmd = [sys.executable, os.path.abspath(__file__)] + argv
    t0 = time.perf_counter()
    try:
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=timeout_s)
    except subprocess.TimeoutExpired:
        return None, "timed out after %d s" % timeout_s
    wall = time.perf_counter() - t0
    for ln in reversed(r.stdout.splitlines()):
        if ln.startswith("{"):
            d = json.loads(ln)
            d["_wall_s"] = wall
            return d, None
    return None, "exit %d: %s" % (r.returncode, (r.stderr or "").strip().splitlines()[-1:] or "")


def _pick(d, keys):
    return {k: d.get(k) for k in keys if k in d}


def run_extras(args):
    """The other workloads of the metric, each run as its own bench.py process and reported beside
    the headline: the kinked source (mixed and FP64 forms), 256 uneven problems in one CUDA graph
    (mixed and FP64 batches), and 64 right-hand sides sharing one tree (folded mixed solve, FP64 loop)."""
    common = ["--steps", "3", "--warmup", "3", "--no-cpu-baseline", "--no-extras"]
    out = {}
    jobs = [("kinked", ["--workload", "kinked"] + common, 900),
            ("batch256", ["--workload", "batch256"] + common, 900),
            ("shared_rhs64", ["--workload", "shared_rhs64"] + common, 600)]
    for key, argv, tmo in jobs:
        d, why = _sub_bench(argv, tmo)
        if d is None:
            out[key] = {"unavailable": why}
            continue
        rec = _pick(d, ("value", "unit", "ms_per_step", "dtype", "config", "fp64_form", "e2e", "clocks",
                        "gpu_launches", "_wall_s"))
        roof = d.get("roofline") or {}
        rec["roofline"] = _pick(roof, ("kernel", "bound", "achieved", "peak", "unit", "frac", "traffic",
                                       "peak_source"))
        if "contractions" in roof:
            rec["roofline"]["contractions"] = {n: _pick(c, ("frac_of_bf16_peak", "useful_fraction", "ms", "form"))
                                               for n, c in roof["contractions"].items()}
        if key == "kinked":
            rec["oracle_check"] = ("the oracle's tree and lists for this workload take over a minute on the host, "
                                   "so the sampled comparison with the oracle runs in the full-size GPU parity "
                                   "test instead; rel. difference of the mixed form from the FP64 form on every "
                                   "target is in fp64_form")
        out[key] = rec
    return out


# ----------------------------------------------------------------------------- GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="adaptive_gauss20")
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--no-fp64-compare", action="store_true",
                    help="with --precision mixed, skip timing the plain FP64 form on the same tree")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="time plain calls instead of CUDA-graph replays")
    ap.add_argument("--no-tune", action="store_true", help="keep the default split-K factors (no autotuner run)")
    ap.add_argument("--refine", default="tail", choices=["tail", "interp", "interp_area", "interp_mixed"],
                    help="refinement rule of the adaptive tree (Section 6.1 alternatives to the tail test)")
    ap.add_argument("--no-extras", action="store_true",
                    help="on the default workload, skip the kinked, batch256 and shared_rhs64 runs that are "
                         "reported beside the headline")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.workload.startswith("batch"):
        return run_batch(args)
    wl = workload(args.workload)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank == 0:
            run_reference(args, wl)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1610_00823_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_1610_00823_gb300 import build as b
        b.build()
    import paper_1610_00823_gb300 as v
    from paper_1610_00823_gb300.api import (SolveGraph, set_schedule, solve_work, tune, volume_potential_profiled,
                                             workspace)
    from paper_1610_00823_gb300.replicas import barrier, max_over_ranks, whole_job_rate

    src = wl.sources[0]

    def build_tree():
        if wl.uniform_depth >= 0:
            return v.tree_build_uniform(wl.cx, wl.cy, wl.width, wl.k, wl.uniform_depth)
        return v.tree_build(wl.cx, wl.cy, wl.width, wl.k, src, wl.tol, wl.max_depth, wl.min_depth, rule=args.refine)

    # the first build in a process also loads the tree kernels and sets up the build pool; the
    # second is the steady cost of building a tree (both reported)
    t0 = time.perf_counter()
    tree = build_tree()
    torch.cuda.synchronize()
    t_tree_first = time.perf_counter() - t0
    del tree
    t0 = time.perf_counter()
    torch.cuda.nvtx.range_push("tree_build")  # NVTX ranges name what an ncu capture filters on
    tree = build_tree()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    t_tree = time.perf_counter() - t0
    t0 = time.perf_counter()
    prec = v.MIXED if args.precision == "mixed" else v.FP64
    ops = v.ops_create(wl.k, wl.p, prec)
    torch.cuda.synchronize()
    t_ops = time.perf_counter() - t0
    nrhs = len(wl.sources)
    if nrhs == 1:
        f = v.source_sample(tree, src)
    else:  # right-hand sides sharing the tree: [nrhs][n_leaves * k^2], one call solves them all
        f = torch.stack([v.source_sample(tree, s) for s in wl.sources]).contiguous()
    kk = wl.k * wl.k
    n_targets = tree.n_leaves * kk * nrhs
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # 256 MB > 129 MB L2
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)

    tuned_ = [None]

    def time_form(ops_, steps, clk=None):
        """Warm-up, then `steps` timed solves (CUDA-graph replays unless --no-graph), L2 flushed between."""
        out_ = tuple(torch.empty_like(f) for _ in range(3))
        ws_ = workspace(tree, ops_, nrhs)
        tuned_[0] = tune(tree, ops_, f, out_, ws_, stream) if not args.no_tune else None  # split-K autotuner
        # the solve is captured once into a CUDA graph; every timed step replays it
        graph_ = SolveGraph(tree, ops_, f, out_, ws_, stream) if not args.no_graph else None

        def step():
            if graph_ is not None:
                graph_.launch(stream)
            else:
                v.volume_potential(tree, ops_, f, out=out_, ws=ws_, stream=stream)

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        barrier(dist)
        torch.cuda.synchronize()
        times = []
        if clk is not None:
            clk.start()
        for _ in range(steps):
            flush.fill_(1.0)  # evict L2 between timed steps (outside the events)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
        if clk is not None:
            clk.stop()
        barrier(dist)
        torch.cuda.synchronize()
        return times, out_, ws_, graph_

    clk = ClockSampler(local)
    step_ms, out, ws, graph = time_form(ops, args.steps, clk)
    split_k = tuned_[0]
    # stage times (CUDA events between stages on the same stream) from separate profiled solves
    stage_acc, launches, n_prof = {}, 0, 3
    for i_prof in range(n_prof):
        flush.fill_(1.0)
        if i_prof == 0:
            torch.cuda.nvtx.range_push("stage_profile")
        stages, launches = volume_potential_profiled(tree, ops, f, out, ws, stream=stream)
        if i_prof == 0:
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()
        for kname, val in stages.items():
            stage_acc[kname] = stage_acc.get(kname, 0.0) + val
    ms = max_over_ranks(statistics.mean(step_ms), dist)
    value = whole_job_rate(n_targets, ms, world)
    stage_ms = {kname: val / n_prof for kname, val in stage_acc.items()}

    # end to end through the host entry point (pinned buffers, copies inside the timed region)
    f_host = f.cpu().pin_memory()
    outs_host = tuple(torch.empty_like(f_host).pin_memory() for _ in range(3))
    ws_io = workspace(tree, ops, nrhs, with_io=True)
    for _ in range(2):
        v.volume_potential_host(tree, ops, f_host, out_host=outs_host, ws=ws_io, stream=stream)
    e2e_ms = []
    for _ in range(max(3, args.steps // 2)):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        v.volume_potential_host(tree, ops, f_host, out_host=outs_host, ws=ws_io, stream=stream)
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_value = whole_job_rate(n_targets, max_over_ranks(statistics.mean(e2e_ms), dist), world)
    del ws_io

    peaks, peak_kind = measured_peaks()
    offnode = None
    if nrhs == 1:
        # v~ (vfmm_leaf_interpolate): the solve's u, u_x, u_y at 2^22 seeded uniform random points of
        # the root box; L2 flushed between the timed calls
        gen = torch.Generator(device="cuda").manual_seed(20161003)
        n_pts = 1 << 22
        px = (wl.cx - wl.width / 2) + wl.width * torch.rand(n_pts, dtype=torch.float64, device="cuda", generator=gen)
        py = (wl.cy - wl.width / 2) + wl.width * torch.rand(n_pts, dtype=torch.float64, device="cuda", generator=gen)
        fields = [o.reshape(-1) for o in out]
        for _ in range(2):
            v.leaf_interpolate(tree, fields, px, py, stream=stream)
        its = []
        for _ in range(5):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            v.leaf_interpolate(tree, fields, px, py, stream=stream)
            e1.record(stream)
            e1.synchronize()
            its.append(e0.elapsed_time(e1))
        ims = statistics.mean(its)
        iflops = n_pts * 3 * 2.0 * kk  # the tensor contraction r_j = sum_i l_i V_ji, sum_j l_j r_j per field
        ipeak = peaks["bf16_tflops"] * FP64_OVER_BF16
        iach = iflops / (ims / 1e3) / 1e12
        offnode = {"kernel": "leaf_interp_kernel", "points": n_pts, "fields": 3, "ms": ims,
                   "pts_per_s": n_pts / (ims / 1e3), "sample": "uniform random in the root box, seed 20161003",
                   "roofline": {"bound": "fp64", "achieved": iach, "peak": ipeak, "unit": "TFLOP/s",
                                "frac": iach / ipeak, "flops": "3 fields x 2 k^2 per point",
                                "peak_source": "%s bf16 x nominal FP64/BF16 ratio (1.25/2250)" % peak_kind}}
        # V f~ itself at arbitrary points from the solve's stored expansions (vfmm_evaluate_points):
        # the first 1024 of the same points; far part O(p), near part by on-the-fly quadrature (FP64)
        n_ev = 1024
        ex, ey = px[:n_ev].contiguous(), py[:n_ev].contiguous()
        v.evaluate_points(tree, ops, f, ws, ex, ey, stream=stream)
        ets = []
        for _ in range(3):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            v.evaluate_points(tree, ops, f, ws, ex, ey, stream=stream)
            e1.record(stream)
            e1.synchronize()
            ets.append(e0.elapsed_time(e1))
        ems = statistics.mean(ets)
        offnode["stored_expansions"] = {"kernel": "offnode_kernel", "points": n_ev, "ms": ems,
                                        "pts_per_s": n_ev / (ems / 1e3),
                                        "sample": "the first 1024 of the points above"}
    co_schedule = None
    if args.precision == "fp64":
        flops = 2.0 * 3 * kk * kk * tree.list_len[0] * nrhs  # near-field table applies per step
        achieved = flops / (stage_ms["near"] / 1e3) / 1e12
        peak = peaks["bf16_tflops"] * FP64_OVER_BF16
        roof = {"kernel": "near_gemm_kernel", "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "peak_source": "%s bf16 x nominal FP64/BF16 ratio (1.25/2250)" % peak_kind,
                "flops_per_launch": flops, "ms_per_launch": stage_ms["near"]}
    else:
        work = solve_work(tree, ops, nrhs)
        # the tuner's co-schedule of the forked step (near-field CTA cap, tree-pass grid cap; 0 = none)
        co_schedule = {"near_field_ctas": int(work["near_ctas"]), "tree_pass_ctas": int(work["pass_ctas"])}
        peak = peaks["bf16_tflops"]
        # algorithmic work of each split contraction: the S(S+1)/2 BF16 slice products (S = its slices) of every real
        # multiply-add the method needs (list entries x rows x K, no zero rows, no padding); the
        # kernels also execute zero rows of targets lacking a table in their group and padded tiles
        # ("executed")
        P2 = 2 * (wl.p + 1)
        n_u, n_v, n_w, n_x = tree.list_len
        alg_fp64eq = {"near": 2.0 * 3 * kk * kk * n_u, "s2m": 2.0 * 2 * wl.p * kk * tree.n_leaves,
                      "m2l": 2.0 * 2 * wl.p * P2 * n_v, "s2l": 2.0 * 2 * wl.p * kk * n_x,
                      "far": 2.0 * 3 * kk * (P2 - 2) * tree.n_leaves + 2.0 * 3 * kk * P2 * n_w}
        contractions = {}
        ENTRY_BIT = {"near": 1, "m2l": 2, "far": 4, "s2l": 8}  # vfmm_solve_work out[7]
        for name in ("near", "s2m", "m2l", "s2l", "far"):
            ms_c = stage_ms.get(name + "_tc", 0.0)
            ex = work[name + "_tc_flops"]
            S = ops.slices[name]
            alg = S * (S + 1) / 2 * alg_fp64eq[name] * nrhs
            if ms_c > 0 and ex > 0:
                contractions[name] = {"tflop_algorithmic": alg / 1e12, "tflop_executed": ex / 1e12, "ms": ms_c,
                                      "tflops": alg / (ms_c / 1e3) / 1e12,
                                      "frac_of_bf16_peak": alg / (ms_c / 1e3) / 1e12 / peak,
                                      "executed_tflops": ex / (ms_c / 1e3) / 1e12, "useful_fraction": alg / ex,
                                      "form": "entry-major" if int(work["entry_major_mask"]) & ENTRY_BIT.get(name, 0)
                                      else "grouped"}
        sn = ops.slices["near"]
        alg_near = sn * (sn + 1) / 2 * alg_fp64eq["near"] * nrhs
        near_ms = stage_ms.get("near_tc") or stage_ms["near"]
        # When the tuner caps the near field's CTAs so that it runs beside the main chain, the kernel's own
        # roofline is taken with the cap lifted to one persistent CTA per SM (one-stream profiled solves);
        # the capped launch the step uses is reported beside it
        in_step = None
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        if 0 < co_schedule["near_field_ctas"] < sms:
            set_schedule(tree, sms, co_schedule["tree_pass_ctas"], nrhs)
            full = []
            for _ in range(3):
                flush.fill_(1.0)
                st_full, _ = volume_potential_profiled(tree, ops, f, out, ws, stream=stream)
                full.append(st_full.get("near_tc") or st_full["near"])
            set_schedule(tree, co_schedule["near_field_ctas"], co_schedule["tree_pass_ctas"], nrhs)
            in_step = {"near_field_ctas": co_schedule["near_field_ctas"], "ms_per_launch": near_ms,
                       "achieved": alg_near / (near_ms / 1e3) / 1e12,
                       "frac": alg_near / (near_ms / 1e3) / 1e12 / peak,
                       "note": "the capped launch of the timed step, alone on one stream"}
            near_ms = statistics.mean(full)
        achieved = alg_near / (near_ms / 1e3) / 1e12
        # DRAM bytes read + written by this launch (tuned schedule, entry-major near field, 6 slices) in
        # one ncu capture (--set full, the NVTX range stage_profile) of this command on this workload;
        # null elsewhere and for other slice counts
        traffic = None
        if (wl.name == "adaptive_gauss20_k16_p40" and args.refine == "tail" and nrhs == 1 and not args.no_tune
                and int(work["entry_major_mask"]) & 1 and ops.slices["near"] == 6):
            traffic = 83487744 + 39357696
        roof = {"kernel": "split_gemm_kernel (near field, split-BF16 tcgen05)", "bound": "tensor",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                "peak_source": "%s bf16 burst" % peak_kind, "flops_per_launch": alg_near, "ms_per_launch": near_ms,
                "flops": "algorithmic: S(S+1)/2 slice products (S = the near field's slices) x 2 x 3k^2 x k^2 "
                         "per U-list entry", "slices": ops.slices,
                "executed_tflops": work["near_tc_flops"] / (near_ms / 1e3) / 1e12,
                "in_step": in_step,
                "fp64_equivalent_tflops": work["near_fp64eq_flops"] / (near_ms / 1e3) / 1e12,
                "contractions": contractions}

    # the plain FP64 form on the same tree and source, timed the same way (the metric's denominator)
    fp64_form, out64 = None, None
    if args.precision == "mixed" and not args.no_fp64_compare:
        t0 = time.perf_counter()
        ops64 = v.ops_create(wl.k, wl.p, v.FP64)
        torch.cuda.synchronize()
        t_ops64 = time.perf_counter() - t0
        ms64_list, out64, ws64, _g64 = time_form(ops64, max(3, min(args.steps, 10)))
        ms64 = max_over_ranks(statistics.mean(ms64_list), dist)
        d = [torch.max(torch.abs(out[q] - out64[q])).item() / torch.max(torch.abs(out64[q])).item()
             for q in range(3)]
        fp64_form = {"value": whole_job_rate(n_targets, ms64, world), "unit": UNIT, "ms_per_step": ms64,
                     "steps": len(ms64_list), "ops_create_s": t_ops64,
                     "mixed_over_fp64_speedup": ms64 / ms, "rel_diff_mixed_vs_fp64_all_targets": d}
        # the same FP64 form with the plane-wave (diagonalised) M2L of Section 3.1 in place of the dense
        # per-entry translation; the downward stage (M2L + S2L + L2L) of one profiled solve of each form
        # and the mixed form's split-BF16 M2L contraction beside it
        flush.fill_(1.0)
        st_dense, _ = volume_potential_profiled(tree, ops64, f, out64, ws64, stream=stream)
        del ws64, _g64
        ops64.set_m2l(v.M2L_PLANEWAVE)
        mspw_list, outpw, wspw, _gpw = time_form(ops64, max(3, min(args.steps, 10)))
        mspw = max_over_ranks(statistics.mean(mspw_list), dist)
        flush.fill_(1.0)
        st_pw, _ = volume_potential_profiled(tree, ops64, f, outpw, wspw, stream=stream)
        dpw = [torch.max(torch.abs(outpw[q] - out64[q])).item() / torch.max(torch.abs(out64[q])).item()
               for q in range(3)]
        fp64_form["planewave_m2l"] = {
            "value": whole_job_rate(n_targets, mspw, world), "unit": UNIT, "ms_per_step": mspw,
            "waves_per_side": ops64.m2l[1], "rel_diff_vs_dense_fp64_all_targets": dpw,
            "down_stage_ms": {"fp64_dense_m2l": st_dense["down"], "fp64_planewave_m2l": st_pw["down"]},
            "mixed_split_bf16_m2l_ms": stage_ms.get("m2l_tc"),
            "note": "down stage = M2L + S2L + L2L + per-box sums (profiled solve, one stream)"}
        del wspw, _gpw, outpw

    cpu, cpu1 = None, None
    errs = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n1 = tree.n_leaves * kk  # the oracle checks the first right-hand side
        got = {args.precision: [o.reshape(-1)[:n1].cpu().numpy() for o in out]}
        if out64 is not None:
            got["fp64"] = [o.reshape(-1)[:n1].cpu().numpy() for o in out64]
        cpu, cpu1, errs = cpu_baseline(wl, got, rule=args.refine)

    extras = None
    if (rank == 0 and world == 1 and args.workload == "adaptive_gauss20" and args.precision == "mixed"
            and not args.no_extras):
        extras = run_extras(args)

    if rank == 0:
        clocks = clk.summary()
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "bf16x6+f64",
                "data": "synthetic",
                "config": {"workload": wl.name, "precision": args.precision, "n_leaves": tree.n_leaves,
                           "n_boxes": tree.n_boxes, "depth": tree.depth, "n_targets": n_targets, "nrhs": nrhs,
                           "k": wl.k,
                           "p": wl.p, "tol": wl.tol, "u_list_len": tree.list_len[0],
                           "l2": "flushed between timed steps (256 MB write outside the events)",
                           "parallelism": "replicas" if world > 1 else "single GPU",
                           "launch": "CUDA graph replay" if graph is not None else "direct calls",
                           "split_k": split_k, "co_schedule": co_schedule,
                           "refine": args.refine, "tree_build_s": t_tree, "tree_build_first_s": t_tree_first,
                           "ops_create_s": t_ops},
                "stage_ms": stage_ms,
                "roofline": roof,
                "cpu_baseline": cpu,
                "cpu_baseline_1core": cpu1,
                "sampled_rel_err_vs_oracle": errs,
                "fp64_form": fp64_form,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": n_targets * 8,
                        "d2h_bytes_per_step": 3 * n_targets * 8, "ms_per_step": statistics.mean(e2e_ms)},
                "gpu_launches": launches,
                "offnode": offnode,
                "clocks": clocks}
        if extras:
            line.update(extras)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
