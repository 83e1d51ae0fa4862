"""Benchmark of the interval solver on one GB300 (or N, as independent replicas).

A step is one complete solve of the workload (every per-box stage: FP32 prefilter, FP64
evaluation and exclusion, Hansen-Sengupta contraction, accept / split, queue compaction
and refill) with the system already resident on the device.  Default workload: the
seeded n=6 sparse system (6 equations x 8 monomials, degree <= 3, integer coefficients,
planted root, box [-4,4]^6, tol 1e-6).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload n6|n2|n10|batched]
                  [--impl ivsolve|reference]
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

from paper_1802_00330_gb300 import synth  # noqa: E402

PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")


def workload(name):
    if name == "n2":
        return [synth.config_n2()], "n2 x^2+y^2-1, x^2-y on [-2,2]^2, tol 1e-8, HS on"
    if name == "n6":
        return [synth.config_n6()], ("n6 seeded sparse system: 6 eq x 8 monomials, deg<=3, int coef [-5,5], "
                                     "planted root, box [-4,4]^6, tol 1e-6, HS on, FP32 prefilter")
    if name == "n10":
        return [synth.config_n10()], ("n10 seeded sparse system: 10 eq x 12 monomials, deg<=4, coef k/2^20, "
                                      "planted root, box [-2,2]^10, tol 1e-6")
    if name == "batched":
        return synth.config_batched(), ("batched: 4096 seeded systems, n~U{2..8}, 4-10 monomials/eq, deg<=3, "
                                         "int coef [-5,5], planted roots, box [-4,4]^n, tol 1e-6")
    if name == "paper":
        import dataclasses
        here = os.path.dirname(os.path.abspath(__file__))
        systems = [dataclasses.replace(synth.load_fixture(os.path.join(here, "tests", "golden", f"{k}.txt")), tol=1e-3)
                   for k, _ in PAPER_SYSTEMS]
        return systems, ("the paper's printed systems noon9 (box [-8,8]^9) and kinema (box [-32,32]^9), "
                         "HS from the first round, tol 1e-3, one plan")
    raise SystemExit(f"unknown workload {name}")


# the paper's printed systems with the width (grid level of the initial box) at which it
# reports their isolated real roots (Section 4: noon9 19 at 0.0625, kinema 8 at 0.03125)
PAPER_SYSTEMS = (("noon9", 8), ("kinema", 11))


# ---- algorithmic work per box (FP64 operations the method needs) --------------------
def eval_ops(s, polys=None):
    """Directed FP64 operations of one natural-form evaluation of the given polynomials:
    per factor x^k a chain of k-1 products per end, per extra factor one interval product
    (2 directed products with the sign-selected ends), 2 for the coefficient, 2 per sum."""
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


# ---- measured DRAM traffic of the dominant kernel ----------------------------------------
# ncu's dram__bytes_read.sum + dram__bytes_write.sum of the Hansen-Sengupta stage per sweep
# (k_hs<6> and k_hs_coop<6>), averaged over the 10 sweeps of one n=6 solve (an ncu
# capture of this workload).  Valid only for the kernel sources
# it was taken with: the bench reports null once their hash (code without comments and
# whitespace) differs.
HS_TRAFFIC_N6 = {"sources_sha256": "62891eeae8663b1de6d2d8d6266de4e64e29152cb3868fb6bbab36a76f7ec840",
                 "bytes_per_launch": 485350}
HS_SOURCES = ("ivs_hs.cuh", "ivs_tab.cuh", "ivs_interval.cuh", "ivs_internal.h", "ivs_kernels.cuh")


def _code_only(text):
    """Source text without comments and whitespace (comment edits leave the kernel as it
    was; a string literal holding comment markers does not occur in these files)."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return "".join(text.split())


def hs_sources_sha(read=None):
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_1802_00330_gb300", "csrc")
    for f in HS_SOURCES:
        if read is None:
            with open(os.path.join(d, f), encoding="utf-8") as fh:
                text = fh.read()
        else:
            text = read(f)
        h.update(_code_only(text).encode())
    return h.hexdigest()


def hs_traffic(workload, kernel, default_options=True):
    if (workload != "n6" or kernel != "hs_n6" or not default_options
            or HS_TRAFFIC_N6["sources_sha256"] != hs_sources_sha()):
        return None
    return HS_TRAFFIC_N6["bytes_per_launch"]


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
def oracle_sample(systems, budget_boxes, centred=False, krawczyk=False):
    import oracle
    t = time.perf_counter()
    boxes = 0
    for s in systems:
        r = oracle.solve(s, max_boxes=budget_boxes, centred=centred, krawczyk=krawczyk)
        boxes += r["stats"]["boxes"]
        if time.perf_counter() - t > 60:
            break
    dt = time.perf_counter() - t
    return boxes, dt


def _oracle_subbox_worker(job):
    """One process of the all-cores oracle baseline: the serial oracle on each of its
    top-level sub-boxes, within a box budget."""
    import oracle
    s, boxes, budget, opts = job
    t = time.perf_counter()
    done = 0
    for lo, hi in boxes:
        if done >= budget:
            break
        r = oracle.solve(s, box_lo=lo, box_hi=hi, max_boxes=budget - done, **opts)
        done += r["stats"]["boxes"]
    return done, time.perf_counter() - t


def oracle_all_cores(s, budget_per_core, cores=None, **opts):
    """The oracle on every host core: the initial box split once in every coordinate (2^n
    sub-boxes, dealt round-robin), one process per core (spawned: no fork after the GPU
    context exists).  Returns (boxes, wall seconds, cores)."""
    import multiprocessing as mp
    cores = cores or os.cpu_count() or 1
    n = s.n_vars
    mid = 0.5 * (s.box_lo + s.box_hi)
    subs = []
    for c in range(1 << n):
        up = np.array([(c >> j) & 1 for j in range(n)], dtype=bool)
        subs.append((np.where(up, mid, s.box_lo), np.where(up, s.box_hi, mid)))
    jobs = [(s, subs[k::cores], budget_per_core, opts) for k in range(cores)]
    ctx = mp.get_context("spawn")
    t = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_subbox_worker, jobs)
    return sum(r[0] for r in res), time.perf_counter() - t, cores


def run_reference(args, systems, desc, rank, world):
    if rank != 0:
        return
    budget = args.ref_boxes
    for _ in range(args.warmup):
        oracle_sample(systems[:1], budget // 10, args.centred, args.krawczyk)
    tot_b, tot_t = 0, 0.0
    for _ in range(args.steps):
        b, t = oracle_sample(systems[:1], budget, args.centred, args.krawczyk)
        tot_b += b
        tot_t += t
    v = tot_b / tot_t
    line = {"impl": "reference", "metric": "boxes/sec", "value": v, "unit": "boxes/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": desc},
            "cpu_baseline": {"value": v, "unit": "boxes/s", "cores": 1, "kind": "oracle",
                             "sample": f"first {budget} boxes (LIFO order) of the {args.workload} solve per step"},
            "e2e": {"value": v, "unit": "boxes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---- the GPU arm --------------------------------------------------------------------
def run_gpu(args, systems, desc, rank, world, local_rank):
    import torch
    torch.cuda.set_device(local_rank)
    from paper_1802_00330_gb300 import _binding as B
    dist = world > 1
    if dist:
        import torch.distributed as td
        td.init_process_group("nccl")

    stream = torch.cuda.Stream()
    tuned = None
    if args.workload == "batched" and not args.wave_children:
        # batching form: the autotuner picks the sweep size and evaluation grid (outside timing)
        tuned = B.autotune(systems[: min(len(systems), 256)], trial_boxes=100_000)
        args.wave_children = int(tuned["wave_children"])
    base_opts = {}
    if args.centred:
        base_opts["centred_form"] = 1
    if args.krawczyk:
        base_opts["krawczyk"] = 1
    plan = B.Plan(systems, opts=base_opts or None, stream=stream, wave_children=args.wave_children,
                  eval_blocks=(tuned or {}).get("eval_blocks", 0))       # graph path
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")   # > L2 (129 MB)

    def one_step():
        with torch.cuda.stream(stream):
            flush.fill_(1)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plan.run()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / 1e3

    for _ in range(args.warmup):
        one_step()
    ref = plan.result(0)
    clocks = ClockSampler(local_rank)
    clocks.start()
    if dist:
        td.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    step_t = []
    boxes = 0
    launches = 0
    ktimes = {}
    for _ in range(args.steps):
        step_t.append(one_step())
        st = plan.stats()
        boxes += st["boxes"]
        launches += st["launches"]
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

    if args.only_timed:
        if rank == 0:
            print(json.dumps({"metric": "boxes/sec", "value": boxes_all / t_dev, "unit": "boxes/s",
                              "systems_per_s": world * len(systems) * args.steps / t_dev,
                              "ms_per_step": 1e3 * t_dev / args.steps, "only_timed": True, "autotuned": tuned,
                              "config": {"workload": desc}}), flush=True)
        plan.close()
        return None
    # parity guard: the timed solve's result equals the warm-up solve's
    res = plan.result(0)
    assert np.array_equal(res["lo"], ref["lo"]) and np.array_equal(res["hi"], ref["hi"])
    roots = None
    if args.workload == "paper":
        # Algorithm 5 backtracking to the paper's widths, then merged: isolated real roots
        roots = {}
        for k, (name, level) in enumerate(PAPER_SYSTEMS):
            rk = plan.result(k)
            s = systems[k]
            roots[name] = B.backtrack(rk["lo"], rk["hi"], s.box_lo, s.box_hi, level, groups=True)[1]

    # plain FP64 path (prefilter off) on the same workload, same GPU
    plan64 = B.Plan(systems, opts={**base_opts, "prefilter_fp32": 0}, stream=stream,
                    wave_children=args.wave_children)
    for _ in range(2):
        plan64.run()
    t64 = []
    b64 = 0
    for _ in range(max(1, args.steps // 2)):
        with torch.cuda.stream(stream):
            flush.fill_(1)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plan64.run()
        b.record(stream)
        b.synchronize()
        t64.append(a.elapsed_time(b) / 1e3)
        b64 += plan64.stats()["boxes"]
    t64_total = float(np.sum(t64))
    if dist:
        t64_total, b64 = reduce_over_ranks(t64_total, b64, device="cuda")
    r64 = plan64.result(0)
    assert np.array_equal(r64["lo"], ref["lo"]) and np.array_equal(r64["hi"], ref["hi"])
    plan64.close()

    # e2e through the public host API: host system in, host boxes out
    if dist:
        td.barrier()
    s0 = systems[0]
    e2e_t = []
    e2e_boxes = 0
    h2d = sum(s.eq_offsets.nbytes + s.coef_lo.nbytes + s.coef_hi.nbytes + s.exps.nbytes + s.box_lo.nbytes
              + s.box_hi.nbytes for s in systems)
    d2h = 0
    if len(systems) == 1:
        for _ in range(args.steps):
            t0 = time.perf_counter()
            r = B.solve(s0, **base_opts)
            e2e_t.append(time.perf_counter() - t0)
            e2e_boxes += r["stats"]["boxes"]
            d2h = r["lo"].nbytes + r["hi"].nbytes + r["flags"].nbytes + r["depth"].nbytes
    else:
        for _ in range(max(1, args.steps // 2)):
            t0 = time.perf_counter()
            outs = B.solve_batch(systems, **base_opts)
            e2e_t.append(time.perf_counter() - t0)
            e2e_boxes += sum(o["stats"]["boxes"] for o in outs)
            d2h = sum(o["lo"].nbytes + o["hi"].nbytes + o["flags"].nbytes + o["depth"].nbytes for o in outs)
    e2e_time = float(np.sum(e2e_t))
    if dist:   # whole job: every rank's boxes over the slowest rank's time
        e2e_time, e2e_boxes = reduce_over_ranks(e2e_time, e2e_boxes, device="cuda")
    e2e = {"value": e2e_boxes / e2e_time, "unit": "boxes/s", "h2d_bytes_per_step": int(h2d * world),
           "d2h_bytes_per_step": int(d2h * world)}

    # per-kernel device time: the same solve through the host loop with CUDA events
    # around every stage (a graph body cannot hold event nodes), over the same K steps
    prof = B.Plan(systems, opts=base_opts or None, stream=stream, profile=True, wave_children=args.wave_children)
    prof.run()
    ktimes = {}
    prof_boxes = 0
    prof_t = []
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        prof.run()
        prof_t.append(time.perf_counter() - t0)
        prof_boxes += prof.stats()["boxes"]
        for k, (nl, ms) in prof.kernel_times().items():
            pl, pm = ktimes.get(k, (0, 0.0))
            ktimes[k] = (pl + nl, pm + ms)
    pst = prof.stats()
    prof.close()

    # roofline of the dominant kernel class
    fp64_rate, _ = B.probe_rate(0, local_rank)
    fp32_rate, _ = B.probe_rate(1, local_rank)
    dom = max(ktimes.items(), key=lambda kv: kv[1][1])
    n_steps = args.steps
    if dom[0].startswith("hs"):
        ops = pst["hs_applied"] * np.mean([hs_ops(s, args.krawczyk) for s in systems]) * n_steps
        work = "FP64 ops of the Hansen-Sengupta sweeps (per-box count from the system tables)"
    elif dom[0] in ("eval", "eval64"):
        ops = pst["eval64_boxes"] * np.mean([eval_ops(s) for s in systems]) * n_steps
        work = "FP64 ops of the FP64 evaluations"
    else:
        ops = 0
        work = "control kernels"
    achieved = ops / (dom[1][1] * 1e-3) / 1e12
    roofline = {"bound": "alu", "kernel": dom[0], "achieved": achieved, "peak": fp64_rate / 1e12,
                "unit": "TFLOP/s", "frac": achieved / (fp64_rate / 1e12),
                "traffic": hs_traffic(args.workload, dom[0], not (args.centred or args.krawczyk)),
                "op_convention": "one directed FP64 add or multiply = 1 flop (no FMA on the path)",
                "peak_source": "measured in this run: directed __dadd_rd/__dmul_ru probe",
                "work": work, "kernel_share": dom[1][1] / sum(v[1] for v in ktimes.values()),
                "avg_launch_ms": dom[1][1] / max(1, dom[1][0])}

    # the FP32 stage (evaluation kernel): natural-form operations of every child it
    # evaluates, against the measured directed FP32 rate
    ev_ms = ktimes.get("eval", (0, 0.0))[1]
    ev_ops = pst["boxes"] * np.mean([eval_ops(s) for s in systems]) * n_steps
    prefilter_roofline = None
    if ev_ms > 0:
        ach32 = ev_ops / (ev_ms * 1e-3) / 1e12
        prefilter_roofline = {"bound": "alu", "kernel": "eval", "achieved": ach32, "peak": fp32_rate / 1e12,
                              "unit": "TFLOP/s", "frac": ach32 / (fp32_rate / 1e12),
                              "work": "FP32 natural-form ops per child (the FP64 count of one evaluation) x "
                                      "children through the FP32 stage",
                              "peak_source": "measured in this run: directed __fadd_rd/__fmul_ru probe"}

    out = None
    if rank == 0:
        cpu = cpu_all = None
        if world == 1 and not args.no_cpu_baseline:
            b, t = oracle_sample(systems[:1], args.cpu_boxes, args.centred, args.krawczyk)
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
            "config": {"workload": desc, "systems_per_step": len(systems), "l2": "flushed (256 MB write) between steps",
                       "parallelism": f"replicas x{world}"},
            "systems_per_s": sys_per_s,
            "boxes_per_step": boxes / args.steps,
            "plain_fp64_path": {"value": b64 / t64_total, "unit": "boxes/s",
                                "ms_per_step": 1e3 * t64_total / len(t64)},
            "e2e": e2e,
            "gpu_launches": int(launches),
            "roofline": roofline, "prefilter_roofline": prefilter_roofline,
            **({"isolated_roots": roots, "isolated_roots_paper": {"noon9": 19, "kinema": 8}} if roots else {}),
            "measured_rates": {"fp64_directed_ops_per_s": fp64_rate, "fp32_directed_ops_per_s": fp32_rate},
            "kernel_ms": {k: round(v[1], 4) for k, v in ktimes.items()},
            "host_loop_ms_per_step": 1e3 * float(np.mean(prof_t)),
            "clocks": ck,
            "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all,
            "wall_s": wall,
        }
        print(json.dumps(out), flush=True)
    plan.close()
    if dist:
        td.destroy_process_group()
    return out


def run_served(args, rank, world, local_rank):
    """Continuous batching: Poisson arrivals of served-config systems, submitted at their
    arrival times to one server; latency = result ready - arrival."""
    import threading as th
    import torch
    torch.cuda.set_device(local_rank)
    from paper_1802_00330_gb300 import _binding as B
    times, systems = synth.config_served(duration_s=args.served_seconds, rate=args.served_rate)
    sv = B.Server(workspace_bytes=args.served_workspace << 30, max_slots=1024, wave_children=1 << 22)
    # warm-up: a few small requests
    for s in systems[:3]:
        sv.wait(sv.submit(s, time_budget_s=args.served_budget), timeout_s=60.0)
    tickets = [None] * len(systems)
    arrival = [0.0] * len(systems)
    done_t = [None] * len(systems)
    results = [None] * len(systems)
    t0 = time.perf_counter() + 0.05

    def submitter():
        for k, (ta, s) in enumerate(zip(times, systems)):
            delay = t0 + ta - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            arrival[k] = t0 + ta
            tickets[k] = sv.submit(s, time_budget_s=args.served_budget)

    def collector():
        for k in range(len(systems)):
            while tickets[k] is None:
                time.sleep(0.0005)
            r = sv.wait(tickets[k], timeout_s=0.0)
            done_t[k] = time.perf_counter()
            results[k] = r

    clocks = ClockSampler(local_rank)
    clocks.start()
    a = th.Thread(target=submitter)
    b = th.Thread(target=collector)
    a.start(); b.start(); a.join(); b.join()
    wall = time.perf_counter() - t0
    ck = clocks.stop()
    lat = np.array([(done_t[k] - arrival[k]) * 1e3 for k in range(len(systems))])
    status = np.array([r["status"] for r in results])
    boxes = sum(r["stats"]["boxes"] for r in results)
    st = sv.stats()
    sv.close()
    ok = status == 0
    line = {"metric": "served systems/sec (continuous batching)", "value": len(systems) / wall, "unit": "systems/s",
            "n_gpus": world, "higher_is_better": True, "dtype": "f64 (f32 prefilter)", "data": "synthetic",
            "config": {"workload": f"served: Poisson {args.served_rate} req/s for {args.served_seconds} s, n~U{{3..12}}, "
                                   "deg<=4, 6-14 monomials/eq, planted roots, box [-2,2]^n, tol 1e-6",
                       "time_budget_s_per_request": args.served_budget},
            "offered_rate": args.served_rate, "requests": len(systems), "wall_s": wall,
            "completed_ok": int(ok.sum()), "timed_out": int((status == 4).sum()),
            "status_counts": {int(k): int(v) for k, v in zip(*np.unique(status, return_counts=True))},
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "p50_ok": float(np.percentile(lat[ok], 50)) if ok.any() else None,
                           "p99_ok": float(np.percentile(lat[ok], 99)) if ok.any() else None},
            "boxes_per_s": boxes / wall, "server": st, "clocks": ck}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="n6")
    ap.add_argument("--impl", default="ivsolve")
    ap.add_argument("--wave-children", type=int, default=0)
    ap.add_argument("--cpu-boxes", type=int, default=600_000)
    ap.add_argument("--ref-boxes", type=int, default=200_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--served-rate", type=float, default=2000.0)
    ap.add_argument("--served-seconds", type=float, default=2.0)
    ap.add_argument("--served-budget", type=float, default=2.0)
    ap.add_argument("--served-workspace", type=int, default=16, help="GiB")
    ap.add_argument("--batched-count", type=int, default=4096)
    ap.add_argument("--centred", action="store_true",
                    help="add the centred-form exclusion test before Hansen-Sengupta")
    ap.add_argument("--krawczyk", action="store_true",
                    help="Krawczyk contraction (eq 15-16) instead of the Gauss-Seidel sweep")
    ap.add_argument("--only-timed", action="store_true",
                    help="time the device-resident solve only (for profiler runs)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.workload == "served" and args.impl != "reference":
        run_served(args, rank, world, local_rank)
        return
    if args.workload == "batched":
        systems, desc = synth.config_batched(count=args.batched_count), (
            f"batched: {args.batched_count} seeded systems, n~U{{2..8}}, 4-10 monomials/eq, deg<=3, "
            "int coef [-5,5], planted roots, box [-4,4]^n, tol 1e-6")
    else:
        systems, desc = workload(args.workload)
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
