#!/usr/bin/env python
"""Benchmark: modular 2mnk GOP/s vs prime bitsize, INT8-word vs FP64 form.

Workload (one "step"): the bitsize sweep m = n = k = 4096, one product
C = A B mod p for each b in {20, 23, 26, 32, 40, 48, 52}, p the largest prime
below 2^b, entries uniform in [0, p) (seeded, synthetic).  The headline value
runs the library's default form (INT8-word digits on the tcgen05 tensor
pipe); the FP64 form (the paper's method, (1,1) / (1,2) / (2,2) chosen by the
block-size bound) is timed on the same inputs and reported per bitsize.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun each rank runs the sweep on its own GPU with its own seeds
(independent problems, weak scaling); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2601_07508_b300 import inputs  # noqa: E402

METRIC = "modular 2mnk GOP/s vs prime bitsize, INT8-word vs FP64 form; serve p50/p99"
FP64_NOMINAL_GFLOPS = 1250.0  # B300 FP64 (DFMA) nominal, 148 SMs at 2032 MHz (only if the measurement fails)
FALLBACK_PEAKS = {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mwmm", choices=["mwmm", "reference"])
    ap.add_argument("--size", type=int, default=4096, help="m = n = k")
    ap.add_argument("--bits", default=",".join(str(b) for b in inputs.SWEEP_BITS))
    ap.add_argument("--no-fp64", action="store_true", help="skip the per-bitsize FP64-form timing")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-crt", action="store_true", help="skip the per-bitsize CRT (multimodular) comparison form")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle sample")
    ap.add_argument("--no-batched", action="store_true", help="skip the 512-instance multi-prime batch")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving run")
    ap.add_argument("--no-shapes", action="store_true", help="skip the 50-bit shape study")
    ap.add_argument("--no-unbalanced", action="store_true", help="skip the block-Wiedemann shape")
    ap.add_argument("--variant-sweep", action="store_true",
                    help="time every FP64 variant at every bitsize 20..52, square and unbalanced (Table 4; minutes)")
    ap.add_argument("--no-variant-grid", action="store_true",
                    help="skip the default coarse Table 4 grid (FP64 variants, 2048^3, every 2 bits from 20 to 52)")
    ap.add_argument("--no-pipe-peaks", action="store_true", help="skip the FP64 pipe-rate measurement")
    ap.add_argument("--tc-fused", action="store_true",
                    help="profiling aid: the sweep's INT8 products with the recombination fused (tc_fused = 2)")
    ap.add_argument("--batched-only", action="store_true",
                    help="profiling aid: run only the batched workload and print its results as the JSON line")
    ap.add_argument("--batch-instances", type=int, default=512, help="first N instances of the batched workload")
    ap.add_argument("--batch-forms", default="int8,auto,fp64", help="forms of the batched workload")
    ap.add_argument("--no-batch-autotune", action="store_true", help="batched workload without the autotuner")
    ap.add_argument("--serve-requests", type=int, default=20000)
    ap.add_argument("--serve-pool", type=int, default=256, help="distinct operand sets the requests cycle through")
    return ap.parse_args()


# ----------------------------------------------------------------------------- helpers
def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return dict(FALLBACK_PEAKS), "fallback"


def fp64_bound_rule(p: int):
    """(1,1) where its block size is >= 1, else (1,2), else (2,2)."""
    from paper_2601_07508_b300 import mwmm
    for uv in ((1, 1), (1, 2), (2, 2)):
        try:
            h = mwmm.mwmm_plan(8, 8, 8, p, uv[0], uv[1], "fp64")
        except mwmm.MwmmError:
            continue
        mwmm.mwmm_plan_destroy(h)
        return uv
    raise RuntimeError("no FP64 variant for p=%d" % p)


def profile_traffic():
    """DRAM bytes per launch of the tcgen05 kernel from the committed ncu
    summary, or None when the kernel source changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "gemm_tc_sweep4096.md")
    src = os.path.join(ROOT, "paper_2601_07508_b300", "csrc", "gemm_tc.cu")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        text = f.read()
    m = re.search(r"source_sha256:\s*([0-9a-f]{64})", text)
    t = re.search(r"traffic_bytes_per_launch:\s*(\{[^}]*\})", text)
    if not m or not t:
        return None
    with open(src, "rb") as f:
        if hashlib.sha256(f.read()).hexdigest() != m.group(1):
            return None
    return {int(k): float(v) for k, v in json.loads(t.group(1)).items()}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 7:
                    continue
                try:
                    sm.append(float(parts[0]))
                    smax.append(float(parts[1]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[3:7]):
                    if val.lower() == "active":
                        reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_index(local_rank: int) -> int:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [x.strip() for x in vis.split(",") if x.strip()]
    if ids and ids[local_rank if local_rank < len(ids) else 0].isdigit():
        return int(ids[local_rank if local_rank < len(ids) else 0])
    return local_rank


# ----------------------------------------------------------------------------- CPU oracle
def oracle_sample(bits, size, seconds, rank_seed=0):
    """Time the oracle on the first R rows of C per bitsize (same inputs as the
    GPU run); R is calibrated so that the whole sample takes about `seconds`."""
    from oracle import oracle as O
    O.lib()
    probs = {}
    for b in bits:
        p = inputs.largest_prime_below_pow2(b)
        probs[b] = (p, inputs.matrix(b + rank_seed, inputs.STREAM_A, 64, size, p),
                    inputs.matrix(b + rank_seed, inputs.STREAM_B, size, size, p))
    # calibrate on 4 rows of the widest prime
    b0 = max(bits)
    p, A, B = probs[b0]
    t0 = time.perf_counter()
    O.matmul_mod_rows(A, B, p, 0, 4)
    rate = 4 / max(time.perf_counter() - t0, 1e-6)  # rows per second
    rows = int(max(1, min(64, rate * seconds / len(bits))))
    ops, t = 0.0, 0.0
    for b in bits:
        p, A, B = probs[b]
        t0 = time.perf_counter()
        O.matmul_mod_rows(A, B, p, 0, rows)
        t += time.perf_counter() - t0
        ops += 2.0 * rows * size * size
    return {"value": ops / t / 1e9, "unit": "GOP/s", "cores": O.num_threads(), "kind": "oracle",
            "sample": "first %d rows of C (x %d cols, k = %d) per bitsize b in %s; 128-bit integer "
                      "accumulation, one %% p per entry" % (rows, size, size, list(bits)),
            "seconds": t}, rows


# ----------------------------------------------------------------------------- ranks
# The path shards by independent problems: every rank runs the whole sweep on
# its own GPU with its own seeds; the only collectives are the timing
# barrier and the maximum of the elapsed times (harness, not data path).

def rank_seed(rank: int) -> int:
    """Seed offset of a rank's problems (independent problems per rank)."""
    return 1000 * rank


def max_over_ranks(x: float, dist, device) -> float:
    """The largest of the ranks' values (the job's elapsed time)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, dist, device) -> float:
    """The sum of the ranks' values (e.g. the work of every shard)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def batch_shard(count: int, rank: int, world: int):
    """Instances of the batched workload that a rank runs: i mod world ==
    rank (the instances are independent, so ranks share no data)."""
    return [i for i in range(count) if i % world == rank]


def job_rate(ops_per_rank_step: float, steps: int, world: int, seconds: float) -> float:
    """Whole-job rate in G-units per second: every rank did `steps` steps of
    `ops_per_rank_step` units within `seconds` (the slowest rank's time)."""
    return ops_per_rank_step * steps * world / seconds / 1e9


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    bits = [int(x) for x in args.bits.split(",")]
    cb, rows = oracle_sample(bits, args.size, max(1.0, min(args.cpu_seconds, 10.0)))
    from oracle import oracle as O
    probs = {}
    for b in bits:
        p = inputs.largest_prime_below_pow2(b)
        probs[b] = (p, inputs.matrix(b, inputs.STREAM_A, rows, args.size, p),
                    inputs.matrix(b, inputs.STREAM_B, args.size, args.size, p))
    wrows = max(1, rows // 8)
    for _ in range(args.warmup):
        for b in bits:
            p, A, B = probs[b]
            O.matmul_mod_rows(A, B, p, 0, wrows)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for b in bits:
            p, A, B = probs[b]
            O.matmul_mod_rows(A, B, p, 0, rows)
    dt = time.perf_counter() - t0
    ops = 2.0 * rows * args.size * args.size * len(bits) * args.steps
    value = ops / dt / 1e9
    sample = cb["sample"]
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int128",
            "data": "synthetic (seeded, entries uniform in [0,p))",
            "config": workload_config(args, bits),
            "cpu_baseline": {"value": value, "unit": "GOP/s", "cores": cb["cores"], "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "GOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def workload_config(args, bits):
    return {"workload": "bitsize sweep: m = n = k = %d, one product C = A B mod p per b in %s, p the largest "
                        "prime below 2^b; headline form: INT8-word digits on the tcgen05 tensor pipe (library "
                        "default); FP64 form ((1,1)/(1,2)/(2,2) by the block-size bound) timed per bitsize"
                        % (args.size, bits),
            "m": args.size, "n": args.size, "k": args.size, "bits": bits,
            "l2": "no flush: each product reads %d MB of fresh A, B (> 126 MB L2)"
                  % (2 * args.size * args.size * 8 // 2 ** 20),
            "parallelism": "independent problems per GPU (no collective in the data path)"}


# ----------------------------------------------------------------------------- batched and serving workloads
def run_batched(dev, runs=5, count=512, forms=("int8", "auto", "fp64"), autotune=True, rank=0, world=1, dist=None):
    """512 instances over the 64 largest primes below 2^50, m, n, k log-uniform
    in [128, 2048] (seed 4), INT8 and FP64 forms and the autotuner's tensor
    form (INT8 or CRT per instance), one graph replay per run.  Under
    torchrun each rank runs its shard of the instances (batch_shard) as one
    batch; the time of a run is the slowest rank's."""
    import torch
    from paper_2601_07508_b300 import mwmm
    full = inputs.batch_instances()[:count]
    mine = batch_shard(len(full), rank, world)
    spec = [full[i] for i in mine]
    items = []
    for i, (m, n, k, p) in zip(mine, spec):
        A, B = inputs.problem(4000 + i, m, n, k, p)
        items.append((torch.from_numpy(A.view(np.int64)).to(dev), torch.from_numpy(B.view(np.int64)).to(dev),
                      torch.empty((m, n), dtype=torch.int64, device=dev), p))
    out = {"workload": "512 instances, 64 largest primes below 2^50 (instance i uses prime i mod 64), m, n, k "
                       "log-uniform in [128, 2048], seed 4; one CUDA-graph replay per run; (u,v) and K-range "
                       "per bitsize group chosen by the autotuner (timed at batch creation); 'auto': each "
                       "instance's tensor form (INT8 digits or CRT) from the planner's cost model, the "
                       "autotuner's configuration per (bitsize, form) group"}
    ref = None
    for form in forms:
        fitems = items if ref is None else [(a, b, torch.empty_like(c), p) for (a, b, c, p) in items]
        bt = mwmm.Batch(fitems, form=form, autotune=autotune)
        bt.run()
        torch.cuda.synchronize()
        nrun = 1 if form == "fp64" else runs
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(nrun):
            bt.run()
        e1.record()
        torch.cuda.synchronize()
        assert bt.check() == 0
        ms = max_over_ranks(e0.elapsed_time(e1) / nrun, dist, dev)
        info = bt.info
        d0 = bt.problem_info(0)
        flops_all = sum(2.0 * m * n * k for (m, n, k, _) in full)  # every rank's shard
        out[form] = {"ms_per_run": ms, "gops": flops_all / ms / 1e6,
                     "word_tflops": sum_over_ranks(info["word_flops"], dist, dev) / ms / 1e9,
                     "launches_per_run": info["launches"],
                     "instances_this_rank": len(spec),
                     "tc_items": info["items"], "ctas": info["ctas"],
                     "autotuned": {"groups": info["tuned_groups"], "probe_ms": info["tuned_ms"],
                                   "uv": [d0["u"], d0["v"]], "kc": d0["kc"], "f64_concat": d0["f64_concat"]}}
        if form == "auto":
            fc = [bt.problem_info(i)["form"] for i in range(len(fitems))]
            out[form]["forms"] = {"int8": fc.count(2), "crt8": fc.count(3)}
        if ref is None:
            ref, ref_form = [c.clone() for (_, _, c, _) in fitems], form
        else:
            out[form + "_equals_" + ref_form] = all(torch.equal(c, r) for (_, _, c, _), r in zip(fitems, ref))
        del bt
    out["flops_2mnk_per_run"] = sum(2.0 * m * n * k for (m, n, k, _) in full)
    out["ranks"] = world
    return out


def run_shapes(dev):
    """p = largest prime below 2^50: rank update (8192, 8192, 512), tall-skinny
    (8192, 64, 8192) and cube (8192, 8192, 8192); INT8-word form vs FP64 (2,2)
    (and FP64 (2,3), the form the cost model picks at 50 bits)."""
    import torch
    from paper_2601_07508_b300 import mwmm
    p = inputs.largest_prime_below_pow2(50)
    out = {}
    for (m, n, k), seed, name in (((8192, 8192, 512), 1, "rank_update"), ((8192, 64, 8192), 2, "tall_skinny"),
                                  ((8192, 8192, 8192), 3, "cube")):
        A, B = inputs.problem(seed, m, n, k, p)
        dA = torch.from_numpy(A.view(np.int64)).to(dev)
        dB = torch.from_numpy(B.view(np.int64)).to(dev)
        res = {"m": m, "n": n, "k": k}
        ref = None
        for form, uv in (("int8", (0, 0)), ("fp64", (2, 2)), ("fp64", (2, 3))):
            pl = mwmm.Plan(m, n, k, p, uv[0], uv[1], form=form)
            pl.alloc_workspace(dev)
            C = pl.matmul(dA, dB)
            torch.cuda.synchronize()
            mwmm.mwmm_plan_set_timing(pl.handle, True)
            reps = 5 if form == "int8" else 1
            for _ in range(reps):
                pl.matmul(dA, dB, C)
            t = mwmm.mwmm_plan_timing(pl.handle)
            assert pl.check() == 0
            ms = t["total_ms"] / t["calls"]
            key = form if form == "int8" else "fp64_%d%d" % uv
            d = pl.info
            res[key] = {"ms": ms, "gops": 2.0 * m * n * k / ms / 1e6, "uv": [d["u"], d["v"]],
                        "word_product_ms": t["gemm_ms"] / t["calls"]}
            if ref is None:
                ref = C
            else:
                res[key]["equals_int8"] = bool(torch.equal(C, ref))
            del pl, C
            torch.cuda.empty_cache()
        res["int8_over_fp64_22"] = res["fp64_22"]["ms"] / res["int8"]["ms"]
        out[name] = res
    return out


def _ceil_root(p: int, u: int) -> int:
    lo, hi = 1, 1
    while hi ** u < p:
        hi *= 2
    lo = hi // 2
    while lo < hi:
        mid = (lo + hi) // 2
        if mid ** u >= p:
            hi = mid
        else:
            lo = mid + 1
    return lo


def product_counts(k: int = 4096, lams=(1, 512), t: int = 53):
    """Fig. 7 of the paper recomputed exactly for FP64 words: per bitsize, the
    fewest word products of a multiword variant (u, v <= 8) whose block size
    lambda satisfies lambda max|A_i| max|B_j| + p - 1 <= 2^t (Prop. 3.3, Sec.
    2.2), against the fewest products of the multimodular approach: distinct
    primes m_i with lambda (m_i - 1)^2 <= 2^t whose product exceeds k (p-1)^2
    (eqs. CRT1, CRT2), largest primes first."""
    out = {}
    for b in range(20, 53):
        p = inputs.largest_prime_below_pow2(b)
        row = {}
        for lam in lams:
            best = None
            for u in range(1, 9):
                for v in range(u, 9):
                    amax = p - 1 if u == 1 else _ceil_root(p, u)
                    bmax = p - 1 if v == 1 else _ceil_root(p, v)
                    if lam * amax * bmax + p - 1 <= 2 ** t and (best is None or u * v < best[0]):
                        best = (u * v, u, v)
            bound = math.isqrt((2 ** t) // lam) + 1  # (m - 1)^2 <= 2^t / lambda
            target, prod, s, q = k * (p - 1) ** 2, 1, 0, bound + 1
            while prod <= target:
                q = inputs.prev_prime(q)
                prod *= q
                s += 1
            row[str(lam)] = {"multiword": best[0], "uv": [best[1], best[2]], "multimodular": s}
        out[str(b)] = row
    return out


UNBALANCED = (10923, 32, 32768)  # m, n, k of the block-Wiedemann products (Sec. 4.1)

# One bitsize per FP64 variant inside the range where its block size covers
# the whole k (one reduction per product): the variant's rate plateau.
PLATEAU_BITS = {(1, 2): 20, (1, 3): 26, (1, 4): 26, (2, 2): 32, (2, 3): 40}


_A52 = {}


def _unbalanced_operands(dev, b):
    """A (m x k) and B (k x n) of the unbalanced shape for the largest prime
    below 2^b; A is the 52-bit matrix of seed 7 (drawn once) reduced mod p."""
    import torch
    m, n, k = UNBALANCED
    p = inputs.largest_prime_below_pow2(b)
    if dev not in _A52:
        A52, _ = inputs.problem(7, m, 1, k, inputs.largest_prime_below_pow2(52))
        _A52[dev] = torch.from_numpy(A52.view(np.int64)).to(dev)
    dA = torch.remainder(_A52[dev], p)
    B = inputs.matrix(b, inputs.STREAM_B, k, n, p)
    return p, dA, torch.from_numpy(B.view(np.int64)).to(dev)


def _time_reuse_a(pl, dA, dB, reps):
    """Split A once, then time `reps` products that split B, multiply and
    recombine (the paper excludes A's decomposition in this scenario)."""
    import torch
    from paper_2601_07508_b300 import mwmm
    C = pl.matmul(dA, dB)
    torch.cuda.synchronize()
    mwmm.mwmm_plan_set_timing(pl.handle, True)
    for _ in range(reps):
        pl.matmul_reuse_a(dB, C)
    t = mwmm.mwmm_plan_timing(pl.handle)
    assert pl.check() == 0
    return t["total_ms"] / t["calls"], C


def run_unbalanced(dev, reps=5):
    """The paper's unbalanced scenario (Sec. 4.1): m = 10923, k = 32768, n = 32,
    A decomposed once and reused.  INT8-word form per bitsize, and the FP64
    variants without and with concatenation of B's words (Alg. 6) at their
    plateau bitsizes (the layout of Table 3)."""
    import torch
    from paper_2601_07508_b300 import mwmm
    m, n, k = UNBALANCED
    flops = 2.0 * m * n * k
    out = {"workload": "m = 10923, k = 32768, n = 32 (block-Wiedemann shape); A split once and reused, time "
                       "= split of B + word products + recombination; A = (52-bit uniform matrix) mod p"}
    int8_ref = {}
    for b in (20, 26, 32, 40, 48, 52):
        p, dA, dB = _unbalanced_operands(dev, b)
        pl = mwmm.Plan(m, n, k, p, form="int8")
        ms, C = _time_reuse_a(pl, dA, dB, reps)
        out[str(b)] = {"int8": {"ms": ms, "gops": flops / ms / 1e6, "uv": [pl.info["u"], pl.info["v"]]}}
        int8_ref[b] = C
        del pl, dA, dB
    table = {}
    for uv, b in PLATEAU_BITS.items():
        p, dA, dB = _unbalanced_operands(dev, b)
        row = {"bits": b}
        for name, cat in (("plain", 1), ("concat", 2)):
            pl = mwmm.Plan(m, n, k, p, uv[0], uv[1], form="fp64", f64_concat=cat)
            ms, C = _time_reuse_a(pl, dA, dB, 1)
            row[name] = {"ms": ms, "gops": flops / ms / 1e6, "ksplit": pl.info["ksplit"],
                         "equals_int8": bool(torch.equal(C, int8_ref[b]))}
            del pl, C
        row["increase_pct"] = 100.0 * (row["plain"]["ms"] / row["concat"]["ms"] - 1.0)
        table["%d,%d" % uv] = row
        del dA, dB
        torch.cuda.empty_cache()
    out["fp64_concat_table"] = table
    return out


def run_variant_sweep(dev, size=2048, bits=range(20, 53), unbalanced=True):
    """Every FP64 variant the block-size bound allows at every bitsize in
    `bits`, on a size^3 square product and (unbalanced=True) on the
    unbalanced shape (concatenated variant, A reused): the best variant per
    bitsize gives the crossover ranges of Table 4 measured on this GPU."""
    import torch
    from paper_2601_07508_b300 import mwmm
    variants = [(1, 1), (1, 2), (1, 3), (1, 4), (2, 2), (2, 3)]
    out = {"square": {"m": size, "n": size, "k": size, "bits": list(bits)}}
    sq = {}
    for b in bits:
        p = inputs.largest_prime_below_pow2(b)
        A, B = inputs.problem(b, size, size, size, p)
        dA = torch.from_numpy(A.view(np.int64)).to(dev)
        dB = torch.from_numpy(B.view(np.int64)).to(dev)
        row = {}
        for uv in variants:
            try:
                pl = mwmm.Plan(size, size, size, p, uv[0], uv[1], form="fp64")
            except mwmm.MwmmError:
                continue
            C = pl.matmul(dA, dB)
            torch.cuda.synchronize()
            mwmm.mwmm_plan_set_timing(pl.handle, True)
            pl.matmul(dA, dB, C)
            t = mwmm.mwmm_plan_timing(pl.handle)
            assert pl.check() == 0
            row["%d,%d" % uv] = 2.0 * size ** 3 / (t["total_ms"] / t["calls"]) / 1e6
            del pl, C
        sq[str(b)] = row
    out["square"]["gops"] = sq

    def ranges(tab):
        best = {b: max(r, key=r.get) for b, r in tab.items() if r}
        res = {}
        for b in sorted(best, key=int):
            res.setdefault(best[b], []).append(int(b))
        return {v: [min(bs), max(bs)] for v, bs in res.items()}
    out["square"]["best_ranges"] = ranges(sq)
    if not unbalanced:
        return out
    out["unbalanced_concat"] = {}
    m, n, k = UNBALANCED
    ub = {}
    for b in bits:
        p, dA, dB = _unbalanced_operands(dev, b)
        row = {}
        for uv in variants:
            try:
                pl = mwmm.Plan(m, n, k, p, uv[0], uv[1], form="fp64")
            except mwmm.MwmmError:
                continue
            ms, C = _time_reuse_a(pl, dA, dB, 1)
            row["%d,%d" % uv] = 2.0 * m * n * k / ms / 1e6
            del pl, C
        ub[str(b)] = row
        del dA, dB
    out["unbalanced_concat"]["gops"] = ub
    out["unbalanced_concat"]["best_ranges"] = ranges(ub)
    return out


def run_serve(dev, nreq, pool, budget=40 << 30, ring=4):
    """Poisson stream of requests (m, n, k log-uniform in [64, 4096], bitsize
    uniform in [20, 52], seed 5) against a 40 GB budget, at 0.8 x and 0.5 x the
    closed-loop saturation throughput measured first.  Requests cycle through
    `pool` operand sets; each set has `ring` output buffers, so a request waits
    for an earlier one only when it reuses that output buffer."""
    import torch
    from paper_2601_07508_b300 import mwmm
    spec = inputs.serve_requests(count=pool)
    ents = []
    for i, (m, n, k, p) in enumerate(spec):
        A, B = inputs.problem(5000 + i, m, n, k, p)
        tA = torch.from_numpy(A.view(np.int64)).to(dev)
        tB = torch.from_numpy(B.view(np.int64)).to(dev)
        outs = [torch.empty((m, n), dtype=torch.int64, device=dev) for _ in range(ring)]
        ents.append((tA, tB, outs, [mwmm._problems([(tA, tB, c, p)])[0] for c in outs]))
    torch.cuda.synchronize()
    crt_share = sum(mwmm.mwmm_tensor_form(m, n, k, p) == "crt8" for (m, n, k, p) in spec) / len(spec)
    srv = mwmm.Server(budget, max_inflight=3, max_batch=64, form="int8")
    last = {}

    def stream(count, arrivals):
        t0 = srv.now()
        tickets = []
        for i in range(count):
            e, slot = i % pool, (i // pool) % ring
            if last.get((e, slot)):
                mwmm.mwmm_serve_wait(srv.handle, last[(e, slot)], 120000)
            if arrivals is not None:
                target = t0 + arrivals[i]
                # sleep until shortly before the arrival, then spin: a client
                # that spins all the time takes a core from the server's
                # worker thread on a busy host
                ahead = target - srv.now()
                if ahead > 4e-4:
                    time.sleep(ahead - 3e-4)
                while srv.now() < target:
                    pass
                ta = target
            else:
                ta = -1.0
            st, tk = mwmm.mwmm_serve_submit_ptr(srv.handle, ents[e][3][slot], ta)
            assert st == 0, st
            last[(e, slot)] = tk
            tickets.append(tk)
        for tk in tickets:
            assert mwmm.mwmm_serve_wait(srv.handle, tk, 300000) == 0
        return srv.stats()

    # closed loop: everything submitted at once -> saturation throughput; first
    # with the INT8 form for every request (for comparison), then the served
    # configuration: each request's tensor form from the planner's cost model
    # 16 passes over the operand pool: with 4 output buffers per set, later
    # submissions wait for earlier uses to finish, so the loop reaches a
    # steady state and the run's tail (the largest requests, last under
    # shortest-work-first) is a small part of it
    nsat = min(nreq, 16 * pool)
    sat8 = stream(nsat, None)  # returns after every ticket finished
    srv.close()
    last.clear()
    srv = mwmm.Server(budget, max_inflight=3, max_batch=64, form="auto")
    sat = stream(nsat, None)
    sat_rps = sat["completed"] / sat["busy_s"]
    out = {"workload": "%d requests per rate, Poisson arrivals at 0.8 x and 0.5 x saturation, m, n, k log-uniform "
                       "in [64, 4096], p a random prime of bitsize uniform in [20, 52], seed 5; operands cycle "
                       "through %d device-resident sets with %d output buffers each; 40 GB budget; form per "
                       "request: INT8 digits or CRT, whichever the planner's cost model (mwmm_tensor_form) "
                       "finds faster; 3 streams, <= 64 requests per batch" % (nreq, pool, ring),
           "crt_share_of_requests": crt_share,
           "saturation_requests_per_s": sat_rps, "saturation_gops": sat["gops"],
           "saturation_int8_only": {"requests_per_s": sat8["completed"] / sat8["busy_s"], "gops": sat8["gops"],
                                    "p50_ms": sat8["p50_ms"], "p99_ms": sat8["p99_ms"]}}
    for frac, key in ((0.8, "at_0.8"), (0.5, "at_0.5")):
        srv.reset_stats()
        rate = frac * sat_rps
        arrivals = inputs.poisson_arrivals(5 if frac == 0.8 else 6, nreq, rate)
        rep = stream(nreq, arrivals)
        out[key] = {"rate_requests_per_s": rate, "p50_ms": rep["p50_ms"], "p99_ms": rep["p99_ms"],
                    "mean_ms": rep["mean_ms"], "max_ms": rep["max_ms"], "gops": rep["gops"],
                    "completed": rep["completed"], "rejected": rep["rejected"], "batches": rep["batches"],
                    "mean_batch": rep["mean_batch"], "peak_inflight_batches": rep["peak_inflight"],
                    "peak_queue": rep["peak_queue"], "peak_workspace_gb": rep["peak_bytes"] / 1e9,
                    "budget_gb": rep["budget_bytes"] / 1e9}
    srv.close()
    # the headline serve figures: the 0.8 x rate
    out.update({k: out["at_0.8"][k] for k in ("p50_ms", "p99_ms", "gops", "rate_requests_per_s")})
    return out


# ----------------------------------------------------------------------------- main arm
def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    from paper_2601_07508_b300 import mwmm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    bits = [int(x) for x in args.bits.split(",")]
    n = args.size
    seed_off = rank_seed(rank)
    if args.batched_only:  # profiling aid: the batched workload alone
        mwmm.lib()
        forms = tuple(f for f in args.batch_forms.split(",") if f)
        b = run_batched(dev, count=args.batch_instances, forms=forms, autotune=not args.no_batch_autotune)
        if rank == 0:
            print(json.dumps({"metric": "batched modular 2mnk GOP/s", "value": b[forms[0]]["gops"], "unit": "GOP/s",
                              "higher_is_better": True, "batched_multi_prime": b}))
        return 0

    # CPU baseline first (before any GPU work; rank 0 at N = 1 only)
    cpu_baseline = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu_baseline, _ = oracle_sample(bits, n, args.cpu_seconds)
        cpu_baseline.pop("seconds", None)

    mwmm.lib()
    probs = []
    for b in bits:
        p = inputs.largest_prime_below_pow2(b)
        A, B = inputs.problem(b + seed_off, n, n, n, p)
        probs.append((b, p, A, B))

    def to_dev(x):
        return torch.from_numpy(x.view(np.int64)).to(dev)

    dA = [to_dev(A) for (_, _, A, _) in probs]
    dB = [to_dev(B) for (_, _, _, B) in probs]
    dC = [torch.empty((n, n), dtype=torch.int64, device=dev) for _ in probs]
    plans = [mwmm.Plan(n, n, n, p, form="int8", tc_fused=2 if args.tc_fused else 0) for (_, p, _, _) in probs]
    for pl in plans:
        pl.alloc_workspace(dev)
        mwmm.mwmm_plan_set_timing(pl.handle, True)

    def step():
        for i, pl in enumerate(plans):
            pl.matmul(dA[i], dB[i], dC[i])

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    for pl in plans:
        assert pl.check() == 0, "device-side error during warm-up"
        mwmm.mwmm_plan_timing(pl.handle)  # discard warm-up timings

    sampler = ClockSampler(gpu_index(local))
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    for pl in plans:
        assert pl.check() == 0, "device-side error in the timed region"

    flop_per_step = 2.0 * n * n * n * len(bits)
    value = job_rate(flop_per_step, args.steps, world, ms / 1e3)

    # per-bitsize phases of the INT8 form (CUDA events on the launching stream)
    per_bits, launches = {}, 0
    gemm_flops, gemm_ms = 0.0, 0.0
    for (b, p, _, _), pl in zip(probs, plans):
        t = mwmm.mwmm_plan_timing(pl.handle)
        launches += t["launches"]
        d = pl.info
        calls = max(t["calls"], 1)
        words = d["u"] * d["v"]
        gemm_flops += 2.0 * words * n ** 3 * calls
        gemm_ms += t["gemm_ms"]
        per_bits[str(b)] = {
            "p": p, "int8_words": [d["u"], d["v"]], "int8_digit_bits": d["tc_digit_bits"],
            "int8_kernel": "gemm_tc_pair_kernel" if d["tc_pair"] else "gemm_tc_kernel",
            "int8_gops": 2.0 * n ** 3 / (t["total_ms"] / calls) / 1e6,
            "int8_ms": t["total_ms"] / calls,
            "int8_phase_ms": {"split_a": t["split_a_ms"] / calls, "split_b": t["split_b_ms"] / calls,
                              "word_products": t["gemm_ms"] / calls, "recombine": t["recombine_ms"] / calls},
            "int8_tensor_tflops": 2.0 * words * n ** 3 / (t["gemm_ms"] / calls) / 1e9,
        }

    peaks, peak_kind = load_peaks()
    achieved = gemm_flops / (gemm_ms / 1e3) / 1e12
    traffic = profile_traffic()
    if traffic is not None:
        tr = [traffic.get(b) for b in bits]
        traffic_per_launch = None if any(x is None for x in tr) else sum(tr) / len(tr)
    else:
        traffic_per_launch = None
    try:  # SMs, one-CTA kernel CTAs and pair clusters the device holds at once
        residency = mwmm.mwmm_tc_residency()
    except mwmm.MwmmError:
        residency = None
    kernels = sorted({v["int8_kernel"] for v in per_bits.values()})
    roofline = {"bound": "tensor",
                "kernel": " + ".join(kernels) + " (tcgen05.mma kind::f16; the planner's tile kernel per bitsize: "
                          "gemm_tc_pair_kernel = 256 x 256 tiles on SM pairs, cta_group::2, 8-bit digits in bf16; "
                          "gemm_tc_kernel = 128 x 256 tiles, one CTA, 9-bit digits in fp16)",
                "achieved": achieved, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                "frac": achieved / peaks["bf16_tflops"], "traffic": traffic_per_launch,
                "peak_kind": "%s bf16 dense burst (cuBLAS); sustained %.1f -> frac %.3f" % (
                    peak_kind, peaks.get("bf16_tflops_sustained", 0.0),
                    achieved / peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])),
                "algorithmic": "2 u v m n k word-product flops per launch (u, v digits per side)"}

    # FP64 pipe rate, measured here on the hot GPU (after the timed region):
    # the denominator of the FP64 form's pipe fraction
    fp64_peak, fp64_peak_kind = FP64_NOMINAL_GFLOPS, "nominal (measurement skipped or failed)"
    if not args.no_pipe_peaks and not args.no_fp64 and rank == 0:
        try:
            mwmm.mwmm_measure_fp64_rate(1 << 16)  # warm-up
            fp64_peak = max(mwmm.mwmm_measure_fp64_rate(1 << 17) for _ in range(3))
            fp64_peak_kind = "measured (DFMA loop, mwmm_measure_fp64_rate, best of 3)"
        except mwmm.MwmmError:
            pass

    # FP64 form per bitsize (same inputs), rank 0 only
    if not args.no_fp64 and rank == 0:
        for i, (b, p, _, _) in enumerate(probs):
            uv = fp64_bound_rule(p)
            pl = mwmm.Plan(n, n, n, p, uv[0], uv[1], form="fp64")
            pl.alloc_workspace(dev)
            Cf = torch.empty((n, n), dtype=torch.int64, device=dev)
            pl.matmul(dA[i], dB[i], Cf)  # warm-up
            torch.cuda.synchronize()
            mwmm.mwmm_plan_set_timing(pl.handle, True)
            pl.matmul(dA[i], dB[i], Cf)
            t = mwmm.mwmm_plan_timing(pl.handle)
            assert pl.check() == 0
            same = bool(torch.equal(Cf, dC[i]))
            d = pl.info
            fl = 2.0 * uv[0] * uv[1] * n ** 3
            e = per_bits[str(b)]
            e.update({"fp64_uv": list(uv), "fp64_lambda": d["lambda"], "fp64_ms": t["total_ms"],
                      "fp64_gops": 2.0 * n ** 3 / t["total_ms"] / 1e6,
                      "fp64_pipe_gflops": fl / t["gemm_ms"] / 1e6,
                      "fp64_pipe_frac": fl / t["gemm_ms"] / 1e6 / fp64_peak,
                      "int8_over_fp64": t["total_ms"] / e["int8_ms"],
                      "fp64_equals_int8": same})
            del pl, Cf
            torch.cuda.empty_cache()

    # CRT (multimodular) comparison form per bitsize (Sec. 5.2), rank 0 only:
    # residues modulo s primes below 256, s tcgen05 products, reconstruction
    if not args.no_crt and rank == 0:
        for i, (b, p, _, _) in enumerate(probs):
            pl = mwmm.Plan(n, n, n, p, form="crt8")
            pl.alloc_workspace(dev)
            Cc = torch.empty((n, n), dtype=torch.int64, device=dev)
            pl.matmul(dA[i], dB[i], Cc)  # warm-up
            torch.cuda.synchronize()
            mwmm.mwmm_plan_set_timing(pl.handle, True)
            for _ in range(3):
                pl.matmul(dA[i], dB[i], Cc)
            t = mwmm.mwmm_plan_timing(pl.handle)
            assert pl.check() == 0
            d = pl.info
            calls = max(t["calls"], 1)
            e = per_bits[str(b)]
            lg = math.log2(p)
            e.update({"crt8_moduli": d["u"], "crt8_ms": t["total_ms"] / calls,
                      "crt8_gops": 2.0 * n ** 3 / (t["total_ms"] / calls) / 1e6,
                      "crt8_phase_ms": {"split_a": t["split_a_ms"] / calls, "split_b": t["split_b_ms"] / calls,
                                        "word_products": t["gemm_ms"] / calls,
                                        "reconstruct": t["recombine_ms"] / calls},
                      "crt8_tensor_tflops": 2.0 * d["u"] * n ** 3 / (t["gemm_ms"] / calls) / 1e9,
                      "crt8_equals_int8": bool(torch.equal(Cc, dC[i])),
                      # products per result: multiword u v vs multimodular s, and the
                      # paper's counts (numprodMW, numprodMM) for t - log2(lambda) = 24 - 10
                      # bits per exact FP32 chunk of 1024 products; numprodMW at the
                      # paper's own word count, unsigned words below 2^7 (u = v =
                      # ceil(log2 p / 7)), where the balanced digits here carry 8 bits
                      "products": {"multiword_int8": e["int8_words"][0] * e["int8_words"][1], "crt8": d["u"],
                                   "paper_multiword": math.ceil(2 * math.ceil(lg / 7) * lg / 14),
                                   "paper_multimodular": math.ceil((4 * lg + 2 * math.log2(n)) / 14)}})
            del pl, Cc
            torch.cuda.empty_cache()

    # end to end through the host entry point (pinned buffers, copies timed)
    e2e = None
    if not args.no_e2e:
        hA = [torch.from_numpy(A.view(np.int64)).pin_memory() for (_, _, A, _) in probs]
        hB = [torch.from_numpy(B.view(np.int64)).pin_memory() for (_, _, _, B) in probs]
        hC = [torch.empty((n, n), dtype=torch.int64).pin_memory() for _ in probs]
        for pl in plans:
            mwmm.mwmm_plan_set_timing(pl.handle, False)

        # one stream per product: the copies of one product overlap the
        # compute of the others (each product's own row blocks also overlap)
        streams = [torch.cuda.Stream(device=dev) for _ in plans]

        def host_step():
            for i, pl in enumerate(plans):
                mwmm.mwmm_matmul_host_async_ptr(pl.handle, hA[i].data_ptr(), n, hB[i].data_ptr(), n,
                                                hC[i].data_ptr(), n, stream=streams[i])
            for i, pl in enumerate(plans):
                if pl.check(streams[i]) != 0:
                    raise RuntimeError("device-side error in the host-buffer product")

        host_step()
        esteps = max(1, min(args.steps, 3))
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(esteps):
            host_step()
        dt = max_over_ranks(time.perf_counter() - t0, dist, dev)
        e2e = {"value": job_rate(flop_per_step, esteps, world, dt), "unit": "GOP/s",
               "h2d_bytes_per_step": 2 * n * n * 8 * len(bits), "d2h_bytes_per_step": n * n * 8 * len(bits),
               "steps": esteps,
               "api": "mwmm_matmul_host_async on one stream per product, then mwmm_plan_check (pinned host buffers)"}
        same = all(torch.equal(hC[i], dC[i].cpu()) for i in range(len(plans)))
        e2e["matches_device_result"] = same

    batched = run_batched(dev, rank=rank, world=world, dist=dist) if not args.no_batched else None
    shapes = run_shapes(dev) if (rank == 0 and not args.no_shapes) else None
    unbalanced = run_unbalanced(dev) if (rank == 0 and not args.no_unbalanced) else None
    if rank == 0 and args.variant_sweep:
        sweep = run_variant_sweep(dev)
    elif rank == 0 and not args.no_variant_grid:
        sweep = run_variant_sweep(dev, size=2048, bits=range(20, 53, 2), unbalanced=False)
    else:
        sweep = None
    serve = run_serve(dev, args.serve_requests, args.serve_pool) if (rank == 0 and not args.no_serve) else None

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GOP/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int8-in-bf16",
                "dtype_detail": "exact integer arithmetic throughout: 8-bit digits carried exactly in bf16 (9-bit "
                                "digits in fp16 where they save a digit) -> FP32 tensor memory (exact, every "
                                "partial sum <= 2^24) -> INT32 sums -> 64-bit integer recombination mod p; results "
                                "bit-exact mod p",
                "data": "synthetic (seeded, entries uniform in [0,p))",
                "config": workload_config(args, bits),
                "roofline": roofline, "cpu_baseline": cpu_baseline, "e2e": e2e,
                "gpu_launches": launches * world, "clocks": clocks, "per_bitsize": per_bits,
                "batched_multi_prime": batched, "shapes_50bit": shapes, "unbalanced_block_wiedemann": unbalanced,
                "variant_sweep": sweep,
                "fp64_pipe_peak_gflops": fp64_peak, "fp64_pipe_peak_kind": fp64_peak_kind,
                "tc_residency": residency,
                "product_counts_fp64_words": product_counts(n),
                "serve": serve}
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
