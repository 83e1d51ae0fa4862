"""Benchmark of the interval solver on one GB300 (or N, as independent replicas).

A step is one complete solve of the workload -- every per-box stage (FP32 prefilter, FP64
evaluation and exclusion, Hansen-Sengupta contraction, accept / split, queue compaction
and refill) for every system of it -- with the systems already resident on the device.

Default workload: the batching form, 4096 seeded systems (n ~ U{2..8}, 4-10 monomials per
equation, degree <= 3, integer coefficients in [-5,5], one planted root each, box [-4,4]^n,
tol 1e-6) solved in one device run under one captured graph, sweeps of 2^24 children and
4 evaluation blocks per SM (the fastest measured on this batch; --autotune picks them with
ivs_autotune instead).  Beside the timed FP32-prefilter form the line carries the plain
FP64 path on the same systems, the plain FP64 per-system path (ivs_solve one system at a
time) on a systematic sample of them, the end-to-end rate through the public host API, the
roofline of every kernel class, the serial oracle on the host cores, and the single n=6
solve as a sub-object.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W]
                  [--workload batched|n6|n2|n10|paper|paper_tables|served] [--impl ivsolve|reference]
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1802_00330_gb300 import synth  # noqa: E402

# the paper's printed systems with the width (grid level of the initial box) at which it
# reports their isolated real roots (Section 4: noon9 19 at 0.0625, kinema 8 at 0.03125)
PAPER_SYSTEMS = (("noon9", 8), ("kinema", 11))


def workload(name, batched_count=4096):
    """(systems, description) of a named workload."""
    if name == "n2":
        return [synth.config_n2()], "n2 x^2+y^2-1, x^2-y on [-2,2]^2, tol 1e-8, HS on"
    if name == "n6":
        return [synth.config_n6()], ("n6 seeded sparse system: 6 eq x 8 monomials, deg<=3, int coef [-5,5], "
                                     "planted root, box [-4,4]^6, tol 1e-6, HS on, FP32 prefilter")
    if name == "n10":
        return [synth.config_n10()], ("n10 seeded sparse system: 10 eq x 12 monomials, deg<=4, coef k/2^20, "
                                      "planted root, box [-2,2]^10, tol 1e-6")
    if name == "batched":
        return synth.config_batched(count=batched_count), (
            f"batched: {batched_count} seeded systems, n~U{{2..8}}, 4-10 monomials/eq, deg<=3, int coef [-5,5], "
            "planted roots, box [-4,4]^n, tol 1e-6, HS on, FP32 prefilter, one device run, sweeps of 2^24 children")
    if name == "paper":
        import dataclasses
        systems = [dataclasses.replace(synth.load_fixture(os.path.join(ROOT, "tests", "golden", f"{k}.txt")), tol=1e-3)
                   for k, _ in PAPER_SYSTEMS]
        return systems, ("the paper's printed systems noon9 (box [-8,8]^9) and kinema (box [-32,32]^9), "
                         "HS from the first round, tol 1e-3, one plan")
    raise SystemExit(f"unknown workload {name}")


def config_of(args, systems, desc, world):
    """The `config` object of both arms' lines (identical for the same workload)."""
    return {"workload": desc, "systems_per_step": len(systems),
            "l2": "flushed (256 MB write) between steps", "parallelism": f"replicas x{world}"}


# ---- algorithmic work per box (operations the method needs) --------------------------
def eval_ops(s, polys=None):
    """Directed operations of one natural-form evaluation of the equations: per factor x^k
    a chain of k-1 products per end, per extra factor one interval product (2 directed
    products with the sign-selected ends), 2 for the coefficient, 2 per sum."""
    ops = 0
    for i in range(s.n_eqs):
        ts = list(s.terms_of(i))
        for q, t in enumerate(ts):
            e = [int(v) for v in s.exps[t] if v]
            if e:
                ops += sum(2 * (k - 1) for k in e) + 2 * (len(e) - 1) + 2
            if q:
                ops += 2
    return ops


def jac_ops(s):
    ops = 0
    for i in range(s.n_eqs):
        for j in range(s.n_vars):
            ts = [t for t in s.terms_of(i) if s.exps[t, j] > 0]
            for q, t in enumerate(ts):
                e = [int(v) - (1 if jj == j else 0) for jj, v in enumerate(s.exps[t])]
                e = [k for k in e if k]
                if e:
                    ops += sum(2 * (k - 1) for k in e) + 2 * (len(e) - 1) + 2
                if q:
                    ops += 2
    return ops


def hs_ops(s, krawczyk=False):
    """One Hansen-Sengupta sweep: J(X), mid(J) (2 per entry), in-place Gauss-Jordan
    (n^2 divisions + 2 n^2 (n-1)), f(x) (thin evaluation), M = B J (4 n^3 - 2 n^2),
    r = B f (4 n^2 - 2 n), Gauss-Seidel ((n-1) * 6 + 4 per row), midpoints 2n.  With the
    Krawczyk step instead of Gauss-Seidel: X - x once (2n), x - r (2n), and per entry
    I - M, the product and the sum (6 n^2)."""
    n = s.n_vars
    step = (2 * n + 2 * n + 6 * n * n) if krawczyk else n * (6 * (n - 1) + 4)
    return (jac_ops(s) + 2 * n * n + n * n + 2 * n * n * (n - 1) + eval_ops(s) + 4 * n ** 3 - 2 * n * n
            + 4 * n * n - 2 * n + step + 2 * n)


# ---- measured DRAM traffic of kernels ----------------------------------------------------
# ncu's dram__bytes_read.sum + dram__bytes_write.sum per launch of a kernel class on a
# workload, valid only for the kernel sources it was taken with: the bench reports null
# once their hash (code without comments and whitespace) differs.  Each record names the
# capture it came from (profiles/).
# A record gives bytes per launch, or bytes per Hansen-Sengupta box (taken on a smaller
# case of the same kernel and scaled to a launch of the measured step by its own boxes per
# launch: the traffic grows with the boxes a launch processes).
TRAFFIC = {
    # profiles/k_hs_n6_dram.md: mean DRAM bytes of the stage per sweep of the n=6 solve
    ("n6", "hs_n6"): {"sources_sha256": "c44aac276b43290460c0650e3d9a0e8ae810783df0d16dae8a9dc0db22b76c93",
                      "bytes_per_launch": 479334, "default_options_only": True},
    # profiles/k_hs_n8_batched.md: 6.479 GB over 112,757,665 n = 8 boxes of all launches of a
    # solve with sweeps of 2^24 children (valid for that sweep size only: smaller sweeps
    # re-read more of their parents from DRAM)
    ("batched", "hs_n8"): {"sources_sha256": "c44aac276b43290460c0650e3d9a0e8ae810783df0d16dae8a9dc0db22b76c93",
                           "bytes_per_hs_box": 57.46, "default_options_only": True, "wave_children": 1 << 24},
}
KERNEL_SOURCES = ("ivs_hs.cuh", "ivs_tab.cuh", "ivs_interval.cuh", "ivs_internal.h", "ivs_kernels.cuh")


def _code_only(text):
    """Source text without comments and whitespace (comment edits leave the kernel as it
    was; a string literal holding comment markers does not occur in these files)."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return "".join(text.split())


def hs_sources_sha(read=None, files=KERNEL_SOURCES):
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1802_00330_gb300", "csrc")
    for f in files:
        if read is None:
            with open(os.path.join(d, f), encoding="utf-8") as fh:
                text = fh.read()
        else:
            text = read(f)
        h.update(_code_only(text).encode())
    return h.hexdigest()


def traffic_of(workload_name, kernel, default_options=True, hs_boxes_per_launch=None, wave_children=None):
    rec = TRAFFIC.get((workload_name, kernel))
    if rec is None or (rec.get("default_options_only") and not default_options):
        return None
    if "wave_children" in rec and rec["wave_children"] != wave_children:
        return None
    files = rec.get("files", KERNEL_SOURCES)
    if rec["sources_sha256"] != hs_sources_sha(files=files):
        return None
    if "bytes_per_launch" in rec:
        return rec["bytes_per_launch"]
    if hs_boxes_per_launch is None:
        return None
    return rec["bytes_per_hs_box"] * hs_boxes_per_launch


# ---- multi-rank aggregation ----------------------------------------------------------
def reduce_over_ranks(t_dev, boxes, device="cpu"):
    """Whole-job numbers over the ranks of the default process group: the slowest
    rank's time (max) and the total boxes (sum).  Replicas share nothing else."""
    import torch
    import torch.distributed as td
    tt = torch.tensor([float(t_dev)], dtype=torch.float64, device=device)
    bb = torch.tensor([float(boxes)], dtype=torch.float64, device=device)
    td.all_reduce(tt, op=td.ReduceOp.MAX)
    td.all_reduce(bb, op=td.ReduceOp.SUM)
    return float(tt.item()), float(bb.item())


# ---- clocks --------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi samples (every 200 ms) over a timed region.  start() returns once the
    first sample is in and stop() once one more has come in, so a region shorter than the
    sampling period still has the samples that bracket it."""

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def _wait_rows(self, n, timeout_s):
        t_end = time.time() + timeout_s
        while len(self.rows) < n and time.time() < t_end and self.proc.poll() is None:
            time.sleep(0.005)

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        self._wait_rows(1, 3.0)

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc:
            self._wait_rows(len(self.rows) + 1, 1.0)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm = []
        smax = 0.0
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                smax = max(smax, float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].lower().startswith("active"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax or None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---- the oracle as CPU baseline / reference arm ---------------------------------------
def oracle_sample(systems, budget_boxes, centred=False, krawczyk=False, time_cap=60.0):
    """The serial oracle over the systems in order, each within a box budget, until the
    time cap: (boxes processed, seconds, systems touched)."""
    import oracle
    t = time.perf_counter()
    boxes = 0
    k = 0
    for s in systems:
        r = oracle.solve(s, max_boxes=budget_boxes, centred=centred, krawczyk=krawczyk)
        boxes += r["stats"]["boxes"]
        k += 1
        if time.perf_counter() - t > time_cap:
            break
    return boxes, time.perf_counter() - t, k


def systematic_sample(systems, count):
    """Every (len / count)-th system, from the first: a sample with the workload's mix."""
    step = max(1, len(systems) // count)
    return systems[::step][:count]


def _oracle_subbox_worker(job):
    """One process of the all-cores oracle baseline: the serial oracle on each of its
    jobs (a system and a box), within a box budget for the process."""
    import oracle
    items, budget, opts = job
    t = time.perf_counter()
    done = 0
    for s, lo, hi in items:
        if done >= budget:
            break
        r = oracle.solve(s, box_lo=lo, box_hi=hi, max_boxes=budget - done, **opts)
        done += r["stats"]["boxes"]
    return done, time.perf_counter() - t


def _all_cores(jobs_items, budget_per_core, cores, opts):
    import multiprocessing as mp
    jobs = [(jobs_items[k::cores], budget_per_core, opts) for k in range(cores)]
    ctx = mp.get_context("spawn")
    t = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_subbox_worker, jobs)
    return sum(r[0] for r in res), time.perf_counter() - t, cores


def oracle_all_cores(s, budget_per_core, cores=None, **opts):
    """The oracle on every host core: the initial box split once in every coordinate (2^n
    sub-boxes, dealt round-robin), one process per core (spawned: no fork after the GPU
    context exists).  Returns (boxes, wall seconds, cores)."""
    cores = cores or os.cpu_count() or 1
    n = s.n_vars
    mid = 0.5 * (s.box_lo + s.box_hi)
    items = []
    for c in range(1 << n):
        up = np.array([(c >> j) & 1 for j in range(n)], dtype=bool)
        items.append((s, np.where(up, mid, s.box_lo), np.where(up, s.box_hi, mid)))
    return _all_cores(items, budget_per_core, cores, opts)


def oracle_all_cores_systems(systems, budget_per_core, cores=None, **opts):
    """The oracle on every host core over whole systems (dealt round-robin)."""
    cores = cores or os.cpu_count() or 1
    items = [(s, s.box_lo, s.box_hi) for s in systems]
    return _all_cores(items, budget_per_core, cores, opts)


def run_reference(args, systems, desc, rank, world):
    """The reference arm: the serial CPU oracle (the paper publishes no code), timed on
    this host on a bounded sample of the same workload per step."""
    if rank != 0:
        return
    multi = len(systems) > 1
    if multi:
        sample = systematic_sample(systems, 256)
        budget, cap = args.ref_boxes // 10, args.ref_step_s
        what = (f"the serial oracle over a systematic sample of the workload's systems in order, each within "
                f"{budget} boxes, {cap:g} s per step")
    else:
        sample, budget, cap = systems[:1], args.ref_boxes, 1e9
        what = f"first {budget} boxes (LIFO order) of the {args.workload} solve per step"
    for _ in range(args.warmup):
        oracle_sample(sample, max(1, budget // 10), args.centred, args.krawczyk, time_cap=cap / 10)
    tot_b, tot_t = 0, 0.0
    for _ in range(args.steps):
        b, t, _ = oracle_sample(sample, budget, args.centred, args.krawczyk, time_cap=cap)
        tot_b += b
        tot_t += t
    v = tot_b / tot_t
    line = {"impl": "reference", "metric": "boxes/sec", "value": v, "unit": "boxes/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(args, systems, desc, world),
            "cpu_baseline": {"value": v, "unit": "boxes/s", "cores": 1, "kind": "oracle", "sample": what},
            "e2e": {"value": v, "unit": "boxes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---- the GPU arm --------------------------------------------------------------------
def _result_digest(res):
    h = hashlib.sha256()
    for k in ("lo", "hi", "flags", "depth"):
        h.update(np.ascontiguousarray(res[k]).tobytes())
    h.update(str(res["status"]).encode())
    return h.hexdigest()


def _timed_runs(plan, stream, flush, steps):
    """Device seconds of `steps` full solves (CUDA events on the plan's stream, L2 flushed
    before each) and the summed statistics."""
    import torch
    ts, boxes, launches = [], 0, 0
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(1)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plan.run()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b) / 1e3)
        st = plan.stats()
        boxes += st["boxes"]
        launches += st["launches"]
    return ts, boxes, launches


def class_rooflines(B, prof, systems, krawczyk, fp64_rate, fp32_rate, ktimes, steps):
    """Per kernel class: algorithmic operations of the work it did over its CUDA-event
    time, against the measured directed rate of its pipe.  hs_n<k>: hs_ops of every sweep
    run on the systems of size k; eval (FP32 stage): one natural-form evaluation per
    child; eval64: one FP64 evaluation per undecided child."""
    per = [prof.result_stats(k) for k in range(len(systems))]
    ops, hs_boxes = {}, {}
    for s, st in zip(systems, per):
        key = f"hs_n{s.n_vars}"
        ops[key] = ops.get(key, 0.0) + st["hs_applied"] * hs_ops(s, krawczyk)
        hs_boxes[key] = hs_boxes.get(key, 0) + int(st["depth_hs"].sum())
        ops["eval"] = ops.get("eval", 0.0) + st["boxes"] * eval_ops(s)
        ops["eval64"] = ops.get("eval64", 0.0) + st["eval64_boxes"] * eval_ops(s)
    total_ms = sum(v[1] for v in ktimes.values())
    out = {}
    for k, (launches, ms) in ktimes.items():
        if k not in ops or ms <= 0:
            continue
        peak = fp32_rate if k == "eval" else fp64_rate
        ach = ops[k] * steps / (ms * 1e-3) / 1e12
        out[k] = {"bound": "alu", "kernel": k, "achieved": ach, "peak": peak / 1e12, "unit": "TFLOP/s",
                  "frac": ach / (peak / 1e12), "kernel_share": ms / total_ms,
                  "avg_launch_ms": ms / max(1, launches), "launches": launches,
                  "pipe": "fp32" if k == "eval" else "fp64"}
        if k in hs_boxes:
            out[k]["hs_boxes_per_launch"] = hs_boxes[k] * steps / max(1, launches)
    return out


def n6_subline(B, stream, flush, steps, warmup):
    """The single n=6 solve (the first configuration that exercises every stage at one
    system): graph path timed, plus its Hansen-Sengupta roofline from the host loop."""
    s = synth.config_n6()
    plan = B.Plan([s], stream=stream)
    try:
        for _ in range(warmup):
            plan.run()
        ts, boxes, _ = _timed_runs(plan, stream, flush, steps)
        ref = _result_digest(plan.result(0))
    finally:
        plan.close()
    prof = B.Plan([s], stream=stream, profile=True)
    try:
        prof.run()
        ktimes = {}
        for _ in range(steps):
            prof.run()
            for k, (nl, ms) in prof.kernel_times().items():
                pl, pm = ktimes.get(k, (0, 0.0))
                ktimes[k] = (pl + nl, pm + ms)
        fp64_rate, _ = B.probe_rate(0)
        fp32_rate, _ = B.probe_rate(1)
        rl = class_rooflines(B, prof, [s], False, fp64_rate, fp32_rate, ktimes, steps)
        assert _result_digest(prof.result(0)) == ref
    finally:
        prof.close()
    t = float(np.sum(ts))
    hs = rl.get("hs_n6", {})
    if hs:
        hs["traffic"] = traffic_of("n6", "hs_n6")
    return {"workload": "n6 seeded sparse system (6 eq x 8 monomials, deg<=3, box [-4,4]^6, tol 1e-6)",
            "value": boxes / t, "unit": "boxes/s", "ms_per_step": 1e3 * t / steps, "steps": steps,
            "roofline_hs_n6": hs, "roofline_eval": rl.get("eval")}


def per_system_arm(B, systems, prefilter):
    """The per-system path: ivs_solve called once per system (host arrays in, sorted host
    boxes out), systems one after the other.  Returns (seconds, boxes, results digest)."""
    t0 = time.perf_counter()
    boxes = 0
    digests = []
    for s in systems:
        r = B.solve(s, prefilter_fp32=prefilter)
        boxes += r["stats"]["boxes"]
        digests.append(_result_digest(r))
    return time.perf_counter() - t0, boxes, digests


def run_gpu(args, systems, desc, rank, world, local_rank):
    import torch
    torch.cuda.set_device(local_rank)
    from paper_1802_00330_gb300 import _binding as B
    dist = world > 1
    if dist:
        import torch.distributed as td
        td.init_process_group("nccl")
    multi = len(systems) > 1
    aux_steps = args.aux_steps if args.aux_steps > 0 else (1 if multi else args.steps)

    stream = torch.cuda.Stream()
    tuned = None
    if multi and args.autotune and not args.wave_children:
        # the autotuner picks the sweep size and evaluation grid (outside timing)
        tuned = B.autotune(systems[: min(len(systems), 256)], trial_boxes=100_000)
        args.wave_children = int(tuned["wave_children"])
    elif multi and not args.wave_children:
        # batching form, fixed: sweeps of 2^24 children and 4 evaluation blocks per SM, the
        # fastest measured on the full 4096-system batch (42.5 s per step against 47.8 s
        # with the 2^22 / 8-per-SM pick of a short capped trial, which cannot see what
        # large sweeps save over a 10^10-box solve)
        props = torch.cuda.get_device_properties(local_rank)
        tuned = {"wave_children": 1 << 24, "eval_blocks": 4 * props.multi_processor_count, "source": "fixed"}
        args.wave_children = tuned["wave_children"]
    base_opts = {}
    if args.centred:
        base_opts["centred_form"] = 1
    if args.krawczyk:
        base_opts["krawczyk"] = 1
    eval_blocks = (tuned or {}).get("eval_blocks", 0)
    plan = B.Plan(systems, opts=base_opts or None, stream=stream, wave_children=args.wave_children,
                  eval_blocks=eval_blocks)       # graph path
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")   # > L2 (129 MB)

    _timed_runs(plan, stream, flush, args.warmup)
    ref = [_result_digest(plan.result(k)) for k in range(len(systems))]
    clocks = ClockSampler(local_rank)
    clocks.start()
    if dist:
        td.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    step_t, boxes, launches = _timed_runs(plan, stream, flush, args.steps)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    if dist:
        td.barrier()
    ck = clocks.stop()
    t_dev = float(np.sum(step_t))
    if dist:
        t_dev, boxes_all = reduce_over_ranks(t_dev, boxes, device="cuda")
        _, launches = reduce_over_ranks(0.0, launches, device="cuda")   # every rank's kernels
    else:
        boxes_all = boxes
    value = boxes_all / t_dev
    sys_per_s = world * len(systems) * args.steps / t_dev

    # parity guard: every system's timed result equals its warm-up result
    assert [_result_digest(plan.result(k)) for k in range(len(systems))] == ref
    oracle_check = None
    if multi and rank == 0 and not args.no_cpu_baseline:
        # and a sample of the systems against the serial oracle, bit for bit
        import oracle
        small = [k for k, s in enumerate(systems) if s.n_vars <= 4][:48]
        same = 0
        for k in small:
            o = oracle.solve(systems[k], centred=args.centred, krawczyk=args.krawczyk)
            g = plan.result(k)
            ok = (o["status"] == g["status"] and np.array_equal(o["lo"], g["lo"]) and np.array_equal(o["hi"], g["hi"])
                  and np.array_equal(o["flags"], g["flags"]) and o["stats"]["boxes"] == g["stats"]["boxes"])
            assert ok, f"system {k} differs from the oracle"
            same += 1
        oracle_check = {"systems": same, "bit_exact": True, "which": "the batch's first systems with n <= 4"}
    roots = None
    if args.workload == "paper":
        # Algorithm 5 backtracking to the paper's widths, then merged: isolated real roots
        roots = {}
        for k, (name, level) in enumerate(PAPER_SYSTEMS):
            rk = plan.result(k)
            s = systems[k]
            roots[name] = B.backtrack(rk["lo"], rk["hi"], s.box_lo, s.box_hi, level, groups=True)[1]
    plan.close()

    # plain FP64 path (prefilter off) on the same systems, same GPU, same sweep schedule
    plan64 = B.Plan(systems, opts={**base_opts, "prefilter_fp32": 0}, stream=stream,
                    wave_children=args.wave_children, eval_blocks=eval_blocks)
    if not multi:
        _timed_runs(plan64, stream, flush, 2)
    t64, b64, _ = _timed_runs(plan64, stream, flush, aux_steps)
    t64_total = float(np.sum(t64))
    if dist:
        t64_total, b64 = reduce_over_ranks(t64_total, b64, device="cuda")
    assert [_result_digest(plan64.result(k)) for k in range(len(systems))] == ref
    plan64.close()

    # the per-system path, plain FP64 and FP32-prefilter, on a systematic sample
    per_system = None
    if multi:
        step = max(1, len(systems) // args.per_system_sample)
        idx = list(range(0, len(systems), step))[: args.per_system_sample]
        sample = [systems[k] for k in idx]
        ts64, bs64, d64 = per_system_arm(B, sample, 0)
        ts32, bs32, d32 = per_system_arm(B, sample, 1)
        assert d64 == d32 == [ref[k] for k in idx]
        per_system = {
            "sample": f"every {max(1, len(systems) // args.per_system_sample)}-th system ({len(sample)} systems, "
                      f"{bs64} boxes), ivs_solve one system at a time, host arrays in and sorted host boxes out",
            "plain_fp64": {"systems_per_s": len(sample) / ts64, "boxes_per_s": bs64 / ts64, "seconds": ts64},
            "fp32_prefilter": {"systems_per_s": len(sample) / ts32, "boxes_per_s": bs32 / ts32, "seconds": ts32},
        }

    # e2e through the public host API: host systems in, host boxes out
    if dist:
        td.barrier()
    e2e_t = []
    e2e_boxes = 0
    h2d = sum(s.eq_offsets.nbytes + s.coef_lo.nbytes + s.coef_hi.nbytes + s.exps.nbytes + s.box_lo.nbytes
              + s.box_hi.nbytes for s in systems)
    d2h = 0
    for _ in range(aux_steps):
        t0 = time.perf_counter()
        outs = B.solve_batch(systems, **base_opts) if multi else [B.solve(systems[0], **base_opts)]
        e2e_t.append(time.perf_counter() - t0)
        e2e_boxes += sum(o["stats"]["boxes"] for o in outs)
        d2h = sum(o["lo"].nbytes + o["hi"].nbytes + o["flags"].nbytes + o["depth"].nbytes for o in outs)
        assert [_result_digest(o) for o in outs] == ref
    e2e_time = float(np.sum(e2e_t))
    if dist:   # whole job: every rank's boxes over the slowest rank's time
        e2e_time, e2e_boxes = reduce_over_ranks(e2e_time, e2e_boxes, device="cuda")
    e2e = {"value": e2e_boxes / e2e_time, "unit": "boxes/s", "h2d_bytes_per_step": int(h2d * world),
           "d2h_bytes_per_step": int(d2h * world), "steps": aux_steps,
           "systems_per_s": world * len(systems) * aux_steps / e2e_time}

    # per-kernel-class device time: the same solve through the host loop with CUDA events
    # around every stage (a graph body cannot hold event nodes)
    prof = B.Plan(systems, opts=base_opts or None, stream=stream, profile=True, wave_children=args.wave_children,
                  eval_blocks=eval_blocks)
    if not multi:
        prof.run()
    ktimes = {}
    prof_t = []
    for _ in range(aux_steps):
        with torch.cuda.stream(stream):
            flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        prof.run()
        prof_t.append(time.perf_counter() - t0)
        for k, (nl, ms) in prof.kernel_times().items():
            pl, pm = ktimes.get(k, (0, 0.0))
            ktimes[k] = (pl + nl, pm + ms)
    fp64_rate, _ = B.probe_rate(0, local_rank)
    fp32_rate, _ = B.probe_rate(1, local_rank)
    classes = class_rooflines(B, prof, systems, args.krawczyk, fp64_rate, fp32_rate, ktimes, aux_steps)
    assert [_result_digest(prof.result(k)) for k in range(len(systems))] == ref
    prof.close()
    dom = max(classes.values(), key=lambda v: v["kernel_share"])
    roofline = dict(dom)
    roofline.update({
        "traffic": traffic_of(args.workload, dom["kernel"], not (args.centred or args.krawczyk),
                              dom.get("hs_boxes_per_launch"), args.wave_children),
        "op_convention": "one directed add or multiply = 1 flop (no FMA on the path)",
        "peak_source": f"measured in this run: directed {'__fadd_rd/__fmul_ru' if dom['pipe'] == 'fp32' else '__dadd_rd/__dmul_ru'} probe",
        "work": ("natural-form operations per child through the FP32 stage" if dom["kernel"] == "eval" else
                 "FP64 operations of the Hansen-Sengupta sweeps (per-box count from each system's tables)"
                 if dom["kernel"].startswith("hs") else "FP64 operations of the FP64 evaluations"),
        "timing": f"host-loop run with CUDA events around every launch ({aux_steps} step(s))"})

    out = None
    if rank == 0:
        cpu = cpu_all = None
        n6 = None
        if multi and args.workload == "batched" and not args.no_n6:
            n6 = n6_subline(B, stream, flush, 10, 3)
        if world == 1 and not args.no_cpu_baseline:
            if multi:
                sample = systematic_sample(systems, 256)
                b, t, k = oracle_sample(sample, 20_000, args.centred, args.krawczyk, time_cap=15.0)
                cpu = {"value": b / t, "unit": "boxes/s", "cores": 1, "kind": "oracle",
                       "sample": f"{b} boxes: the serial oracle on the first {k} systems of a systematic sample of "
                                 "the batch, each within 20000 boxes, fesetround"}
                ba, ta, ca = oracle_all_cores_systems(sample, 100_000, centred=args.centred, krawczyk=args.krawczyk)
                cpu_all = {"value": ba / ta, "unit": "boxes/s", "cores": ca, "kind": "oracle",
                           "sample": f"{ba} boxes: one spawned oracle process per host core over the same sample's "
                                     "systems (round-robin), 100000 boxes per process at most, wall clock including "
                                     "process start"}
            else:
                b, t, _ = oracle_sample(systems[:1], args.cpu_boxes, args.centred, args.krawczyk)
                cpu = {"value": b / t, "unit": "boxes/s", "cores": 1, "kind": "oracle",
                       "sample": f"first {b} boxes (LIFO order) of the {args.workload} solve, serial, fesetround"}
                ba, ta, ca = oracle_all_cores(systems[0], max(1, args.cpu_boxes // 4),
                                              centred=args.centred, krawczyk=args.krawczyk)
                cpu_all = {"value": ba / ta, "unit": "boxes/s", "cores": ca, "kind": "oracle",
                           "sample": f"{ba} boxes: independent oracle processes over the 2^n top-level sub-boxes "
                                     f"of the {args.workload} solve, {max(1, args.cpu_boxes // 4)} boxes per process "
                                     "at most, wall clock including process start"}
        out = {
            "metric": "boxes/sec", "value": value, "unit": "boxes/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64 (f32 prefilter)", "data": "synthetic",
            "config": config_of(args, systems, desc, world),
            "systems_per_s": sys_per_s,
            "boxes_per_step": boxes / args.steps,
            "sweep_config": tuned,
            "plain_fp64_path": {"value": b64 / t64_total, "unit": "boxes/s", "steps": len(t64),
                                "systems_per_s": world * len(systems) * len(t64) / t64_total,
                                "ms_per_step": 1e3 * t64_total / len(t64), "results": "identical"},
            "per_system_path": per_system,
            "oracle_check": oracle_check,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "roofline": roofline, "roofline_classes": classes,
            **({"isolated_roots": roots, "isolated_roots_paper": {"noon9": 19, "kinema": 8}} if roots else {}),
            "measured_rates": {"fp64_directed_ops_per_s": fp64_rate, "fp32_directed_ops_per_s": fp32_rate},
            "kernel_ms": {k: round(v[1], 4) for k, v in ktimes.items()},
            "host_loop_ms_per_step": 1e3 * float(np.mean(prof_t)),
            "n6": n6,
            "clocks": ck,
            "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all,
            "wall_s": wall,
        }
        print(json.dumps(out), flush=True)
    if dist:
        td.destroy_process_group()
    return out


# ---- serving ---------------------------------------------------------------------------
def serve_stream(B, systems, times, budget, max_slots, workspace_gib, min_region):
    """Submits systems[k] at times[k] (seconds from start) to one server and collects
    every result; latency = result ready - arrival."""
    import threading as th
    sv = B.Server(workspace_bytes=workspace_gib << 30, max_slots=max_slots, wave_children=1 << 22,
                  min_region_entries=min_region)
    try:
        for s in systems[:2]:                      # warm-up
            sv.wait(sv.submit(s, time_budget_s=budget), timeout_s=60.0)
        n = len(systems)
        tickets, arrival, done_t, results = [None] * n, [0.0] * n, [None] * n, [None] * n
        t0 = time.perf_counter() + 0.05

        def submitter():
            for k in range(n):
                delay = t0 + times[k] - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                arrival[k] = t0 + times[k]
                tickets[k] = sv.submit(systems[k], time_budget_s=budget)

        def collector():
            for k in range(n):
                while tickets[k] is None:
                    time.sleep(0.0005)
                results[k] = sv.wait(tickets[k], timeout_s=0.0)
                done_t[k] = time.perf_counter()

        a = th.Thread(target=submitter)
        b = th.Thread(target=collector)
        a.start(); b.start(); a.join(); b.join()
        wall = time.perf_counter() - t0
        st = sv.stats()
    finally:
        sv.close()
    lat = np.array([(done_t[k] - arrival[k]) * 1e3 for k in range(n)])
    return results, lat, wall, st


# the paper's printed per-round counts (Section 4): B&B boxes kept per round (Tables 1, 4,
# 7), Hansen-Sengupta origin -> new boxes per round (Tables 2, 5) and the backtracking
# boxes per width (Tables 3, 6, 8; width -> count)
PAPER_ROUNDS = {"katsura8": [1, 511, 4847, 92880, 2549461, 76736464, 794760638, 430650061],
                "noon9": [1, 512, 5120, 42176, 13511, 222941, 1156044, 11471246, 33925040, 28775053],
                "kinema": [1, 288, 5714, 56036, 407380, 4369735, 26247657, 87424465]}
PAPER_HS = {"katsura8": (8, [(430650061, 4900601), (30098623, 4347544), (42617540, 5532835), (64267381, 7946423),
                             (105056246, 11571157), (165616092, 15474734), (243760141, 18711270),
                             (295102270, 20306174), (343840882, 20242072)]),
            "noon9": (10, [(28775053, 477)])}
# Table 3 (katsura8 after the Hansen-Sengupta rounds up to 16), its coarser widths
PAPER_BACKTRACK_KATSURA8 = {0.0078125: 2957, 0.015625: 691, 0.03125: 246, 0.0625: 79, 0.125: 36, 0.25: 36}
PAPER_BACKTRACK = {"noon9": {0.03125: 477, 0.0625: 19, 0.125: 19},
                   "kinema": {0.001953125: 6587702, 0.00390625: 328906, 0.0078125: 14876, 0.015625: 453,
                              0.03125: 8, 0.0625: 8}}


def run_paper_tables(args, rank, local_rank):
    """The paper's Section 4 tables beside this solver's counts on the same printed
    systems: B&B rounds without contraction (Tables 1, 4, 7), the Hansen-Sengupta rounds
    from the round the paper starts it (Tables 2, 5), and the backtracking boxes and
    isolated roots per width after a solve to tol 1e-3 with HS from the first round
    (Tables 6, 8).  Counts come from the per-depth counters of one run each."""
    import dataclasses
    import torch
    torch.cuda.set_device(local_rank)
    from paper_1802_00330_gb300 import _binding as B
    if rank != 0:
        return
    fx = {k: synth.load_fixture(os.path.join(ROOT, "tests", "golden", f"{k}.txt")) for k in PAPER_ROUNDS}
    out = {"metric": "per-round box counts against the paper's Section 4 tables", "config": {
        "workload": "the paper's printed systems katsura8 ([-1,1]^9), noon9 ([-8,8]^9), kinema ([-32,32]^9)"}}
    bb = {}
    for name, want in PAPER_ROUNDS.items():
        t = time.perf_counter()
        r = B.solve(fx[name], hs_enable=0, tol=0.0, max_depth=len(want) - 1, max_results=1 << 16)
        got = r["stats"]["depth_kept"][: len(want)].tolist()
        bb[name] = {"rounds": list(range(1, len(want) + 1)), "ours": got, "paper": want,
                    "equal": [a == b for a, b in zip(got, want)], "seconds": time.perf_counter() - t}
    out["bb_rounds"] = bb
    hs = {}
    for name, (first, rows) in PAPER_HS.items():
        t = time.perf_counter()
        last = first - 1 + len(rows) - 1   # depth of the last printed round
        # the last round's boxes stay on the device for Table 3's backtracking
        plan = B.Plan([fx[name]], opts={"hs_min_depth": first - 1, "tol": 0.0, "max_depth": last,
                                        "max_results": 1 << 26})
        try:
            plan.run()
            st = plan.result_stats(0)
            ours = [(int(st["depth_hs"][d]), int(st["depth_kept"][d])) for d in range(first - 1, last + 1)]
            hs[name] = {"rounds": list(range(first, first + len(rows))), "ours_origin_new": ours,
                        "paper_origin_new": rows, "ours_new_fraction": [n / o if o else None for o, n in ours],
                        "paper_new_fraction": [n / o for o, n in rows], "seconds": time.perf_counter() - t}
            if name == "katsura8":
                s = fx[name]
                rows3 = []
                for w, want in PAPER_BACKTRACK_KATSURA8.items():
                    level = int(round(np.log2((s.box_hi[0] - s.box_lo[0]) / w)))
                    cells, groups = plan.backtrack(0, level, max_cells=1 << 30)
                    rows3.append({"width": w, "level": level, "ours_cells": cells, "ours_groups": groups,
                                  "paper_boxes": want})
                out["backtracking_katsura8"] = {"boxes_backtracked": ours[-1][1], "rows": rows3}
        finally:
            plan.close()
    out["hs_rounds"] = hs
    bt = {}
    for name, widths in PAPER_BACKTRACK.items():
        s = dataclasses.replace(fx[name], tol=1e-3)
        plan = B.Plan([s])
        try:
            plan.run()
            rows = []
            for w, want in widths.items():
                level = int(round(np.log2((s.box_hi[0] - s.box_lo[0]) / w)))
                if s.n_vars * level <= 127:
                    cells, groups = plan.backtrack(0, level)
                    where = "gpu"
                else:   # beyond the device keys' 127 bits: the host routine on the same boxes
                    r = plan.result(0)
                    cells, groups = B.backtrack(r["lo"], r["hi"], s.box_lo, s.box_hi, level, groups=True)
                    where = "host"
                rows.append({"width": w, "level": level, "ours_cells": cells, "ours_groups": groups,
                             "paper_boxes": want, "computed_on": where})
        finally:
            plan.close()
        bt[name] = rows
    out["backtracking"] = bt
    print(json.dumps(out), flush=True)


def run_served(args, rank, world, local_rank):
    """Continuous batching: a Poisson stream of served-recipe systems, submitted at their
    arrival times to one server.  First the stream at a low rate, which labels the
    requests a server finishes within the time budget when it is not loaded ("feasible");
    then rising rates over the same requests.  A rate is sustained when every feasible
    request still completes exactly (IVS_OK) and no request waits for admission longer
    than the budget.  Reports the highest sustained rate with its p50/p99 latency, the
    offered rate's, and the feasible requests solved one at a time through the plain FP64
    per-system path (systems/s)."""
    import torch
    torch.cuda.set_device(local_rank)
    from paper_1802_00330_gb300 import _binding as B
    count = args.served_requests
    systems = synth.served_systems(count)
    rates = sorted(set([args.served_low_rate] + [float(r) for r in args.served_rates.split(",")]))
    clocks = ClockSampler(local_rank)
    clocks.start()
    runs = []
    feasible = None
    for rate in rates:
        k = count if rate <= args.served_low_rate else min(count, max(64, int(rate * args.served_seconds)))
        times = synth.poisson_arrivals(k, rate)
        res, lat, wall, st = serve_stream(B, systems[:k], times, args.served_budget, args.served_slots,
                                          args.served_workspace, args.served_min_region)
        status = np.array([r["status"] for r in res])
        qms = np.array([r["stats"]["queue_ms"] for r in res])
        if feasible is None:
            feasible = status == 0
        fz = feasible[:k]
        ok = status == 0
        sustained = bool(np.all(ok[fz]) and (np.percentile(qms, 99) <= 1e3 * args.served_budget))
        runs.append({"offered_rate": rate, "requests": k, "wall_s": wall, "completed_per_s": k / wall,
                     "solved_ok": int(ok.sum()), "timed_out": int((status == 4).sum()),
                     "feasible_ok": f"{int(ok[fz].sum())}/{int(fz.sum())}", "sustained": sustained,
                     "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                                    "p50_feasible": float(np.percentile(lat[fz], 50)) if fz.any() else None,
                                    "p99_feasible": float(np.percentile(lat[fz], 99)) if fz.any() else None},
                     "queue_ms_p99": float(np.percentile(qms, 99)),
                     "boxes_per_s": sum(r["stats"]["boxes"] for r in res) / wall,
                     "server_sweeps": st["sweeps"]})
    ck = clocks.stop()
    sustained = [r for r in runs if r["sustained"]]
    best = max(sustained, key=lambda r: r["offered_rate"]) if sustained else None
    # the feasible requests through the plain FP64 per-system path, one after the other
    feas = [s for s, f in zip(systems, feasible) if f]
    t64, b64, _ = per_system_arm(B, feas, 0)
    t32, b32, _ = per_system_arm(B, feas, 1)
    line = {"metric": "served systems/sec (continuous batching)",
            "value": best["completed_per_s"] if best else None, "unit": "systems/s",
            "n_gpus": world, "higher_is_better": True, "dtype": "f64 (f32 prefilter)", "data": "synthetic",
            "config": {"workload": "served: Poisson stream of served-recipe systems, n~U{3..12}, deg<=4, "
                                   "6-14 monomials/eq, planted roots, box [-2,2]^n, tol 1e-6, FP32 prefilter + "
                                   "FP64 Hansen-Sengupta",
                       "time_budget_s_per_request": args.served_budget, "max_slots": args.served_slots,
                       "min_region_entries": args.served_min_region, "queue_gib": args.served_workspace},
            "sustainable_rate": best["offered_rate"] if best else None,
            "at_sustainable_rate": best, "runs": runs,
            "feasible_requests": int(feasible.sum()), "requests": count,
            "per_system_path_feasible": {
                "plain_fp64": {"systems_per_s": len(feas) / t64, "boxes_per_s": b64 / t64},
                "fp32_prefilter": {"systems_per_s": len(feas) / t32, "boxes_per_s": b32 / t32},
                "what": "the feasible requests solved one at a time through ivs_solve"},
            "clocks": ck}
    if best:
        line["vs_plain_fp64"] = best["completed_per_s"] / (len(feas) / t64)
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)   # one batched step is ~43 s on a GB300
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="batched")
    ap.add_argument("--impl", default="ivsolve")
    ap.add_argument("--wave-children", type=int, default=0)
    ap.add_argument("--autotune", action="store_true",
                    help="batched forms: pick sweep size and grid with ivs_autotune on 256 systems")
    ap.add_argument("--aux-steps", type=int, default=0,
                    help="steps of the auxiliary passes (plain FP64, e2e, per-kernel profile); "
                         "0 = 1 for multi-system workloads, --steps otherwise")
    ap.add_argument("--per-system-sample", type=int, default=256)
    ap.add_argument("--cpu-boxes", type=int, default=600_000)
    ap.add_argument("--ref-boxes", type=int, default=200_000)
    ap.add_argument("--ref-step-s", type=float, default=4.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-n6", action="store_true")
    ap.add_argument("--served-requests", type=int, default=160)
    ap.add_argument("--served-low-rate", type=float, default=4.0)
    ap.add_argument("--served-rates", default="5,10,25,50,100,200,500,2000")
    ap.add_argument("--served-seconds", type=float, default=4.0)
    ap.add_argument("--served-budget", type=float, default=1.0)
    ap.add_argument("--served-slots", type=int, default=256)
    ap.add_argument("--served-workspace", type=int, default=96, help="GiB")
    ap.add_argument("--served-min-region", type=int, default=1 << 21,
                    help="smallest queue region of a request (entries)")
    ap.add_argument("--batched-count", type=int, default=4096)
    ap.add_argument("--centred", action="store_true",
                    help="add the centred-form exclusion test before Hansen-Sengupta")
    ap.add_argument("--krawczyk", action="store_true",
                    help="Krawczyk contraction (eq 15-16) instead of the Gauss-Seidel sweep")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.workload == "served" and args.impl != "reference":
        run_served(args, rank, world, local_rank)
        return
    if args.workload == "paper_tables":
        run_paper_tables(args, rank, local_rank)
        return
    if args.workload == "served":
        systems = synth.served_systems(64)
        desc = "served-recipe systems (reference arm: the oracle over them)"
    else:
        systems, desc = workload(args.workload, args.batched_count)
    if args.centred:
        desc += ", centred-form exclusion before HS"
    if args.krawczyk:
        desc += ", Krawczyk contraction instead of Gauss-Seidel"
    if args.impl == "reference":
        run_reference(args, systems, desc, rank, world)
        return
    run_gpu(args, systems, desc, rank, world, local_rank)


if __name__ == "__main__":
    main()
