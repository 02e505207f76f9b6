"""Benchmark: exact products of 2^20-bit integers per second on GB300.

Workload (one "step"): a batch of P balanced products of two 2^20-bit
operands (32768 uint32 limbs each, limbs uniform from a seed) through the
whole Toom-Cook path (evaluation, recursive pointwise products, schoolbook
base case, interpolation, recomposition) in one library call.  P = 2432 per
GPU (16 x 152 SMs), so the operands alone (638 MB) exceed the 129 MB L2 and
no L2 flush is needed between steps.  The last timed step's products are
checked (every row modulo three primes, sampled rows exactly) before any
number is printed.

Prints one JSON line (rank 0).  `value` is whole-job products per second
(Mults/s); `e2e` is the same metric through the pipelined host-buffer
entry point (tc_pipe_submit: every step copies its operands in from pinned
host memory and its products out, two steps in flight), with the blocking
host-buffer call (tc_mul_uniform_host) beside it; `roofline` is the dominant
kernel by share of the step and `rooflines` every kernel of the step, the base
case against the integer ceiling measured live by tc_peak_madc, the linear
passes against the measured HBM copy bandwidth; `cpu_baseline` is the
oracle's C Toom-Cook on this machine's host cores (bounded sample).  Also
measured by default: the B sweep, Toom-3 at 1024 limbs, all-ones and sparse
operands, single products of 2^24, 2^26 and 2^27 bits (top-level B = 16 and
32, products and squares), the plain schoolbook on the GPU at 2^20 and 2^24
bits, the mixed-size batch and the serving stream.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
  python bench.py --case interp|leaf|eval [--count N] [--limbs L] [--B B]   (one kernel call)
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import signal
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

LIMBS = 32768            # 2^20 bits
PER_GPU = 2432           # 16 x 152 SMs
METRIC = "exact 2^20-bit products per second (Mults/s)"
PLAN_TABLE = os.path.join(ROOT, "paper_1602_02740_gb300", "plans_gb300.txt")
# three distinct primes (two Mersenne primes and the largest prime below 2^64)
CHECK_PRIMES = ((1 << 61) - 1, (1 << 64) - 59, (1 << 89) - 1)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="tc", choices=["tc", "reference"])
    p.add_argument("--limbs", type=int, default=LIMBS)
    p.add_argument("--batch", type=int, default=PER_GPU)
    p.add_argument("--plan", default="auto", help="comma-separated B per level, or auto")
    p.add_argument("--no-sweep", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--mixed", type=int, default=4096,
                   help="products in the mixed-size batch measurement (0 = skip)")
    p.add_argument("--serve", type=int, default=20000,
                   help="requests per serving run (0 = skip)")
    p.add_argument("--no-configs", action="store_true",
                   help="skip the Toom-3 at 1024 limbs and the all-ones / sparse 2^20-bit lines")
    p.add_argument("--no-large", action="store_true",
                   help="skip the single products of 2^24, 2^26 and 2^27 bits")
    p.add_argument("--case", choices=["interp", "leaf", "eval", "ntt"], default=None,
                   help="time one kernel call for a profiler capture instead of the benchmark")
    p.add_argument("--count", type=int, default=None, help="--case: products or rows")
    p.add_argument("--B", type=int, default=12, help="--case interp/eval: blocks")
    p.add_argument("--reps", type=int, default=3, help="--case: timed repetitions")
    p.add_argument("--method", choices=["newton", "matrix"], default="newton",
                   help="--case interp: even-odd Newton route or inverse-Vandermonde matrix")
    p.add_argument("--leaf", choices=["karatsuba", "schoolbook"], default="schoolbook",
                   help="--case leaf: base-case variant of the lane-pair kernel (karatsuba: "
                        "the in-kernel Karatsuba level from 49 limbs on)")
    return p.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def table_plan(limbs: int):
    """The plan the library's table gives for `limbs` (first row with max >= limbs)."""
    with open(PLAN_TABLE) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            words = line.split()
            parts = [int(x) for x in words[:2 + int(words[1])]]
            if limbs <= parts[0]:
                return parts[2:] + (["ntt"] if words[-1] == "ntt" else [])
    return None


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        fields = dict(l.split(":", 1) for l in out.splitlines() if ":" in l)
        name = fields.get("Model name", "").strip()
        vendor = fields.get("Vendor ID", "").strip()
        if name:
            return f"{vendor} {name}".strip()
    except (OSError, subprocess.SubprocessError, ValueError):
        pass
    return platform.processor() or platform.machine()


# ----------------------------------------------------------------- result checks

def _int(row) -> int:
    return int.from_bytes(np.ascontiguousarray(row, dtype=np.uint32).tobytes(), "little")


def check_products(A, B, O, exact_rows=(), square=False):
    """Every row k: O[k] = A[k] B[k] modulo three primes; rows in `exact_rows`:
    O[k] = A[k] B[k] exactly (CPython's integer product).  Host uint32 arrays.
    Returns a summary dict whose "ok" is False at the first row that differs."""
    bad = None
    for k in range(len(A)):
        a = _int(A[k])
        b = a if square else _int(B[k])
        w = _int(O[k])
        if any((a % p) * (b % p) % p != w % p for p in CHECK_PRIMES):
            bad = k
            break
    exact = []
    if bad is None:
        for k in exact_rows:
            a = _int(A[k])
            b = a if square else _int(B[k])
            want = (a * b).to_bytes(4 * len(O[k]), "little")
            exact.append(int(k))
            if np.ascontiguousarray(O[k], dtype=np.uint32).tobytes() != want:
                bad = k
                break
    return {"ok": bad is None, "rows": int(len(A)), "residue_primes": 3,
            "exact_rows": exact, "first_bad_row": bad}


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL, start_new_session=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        try:
            os.killpg(self.proc.pid, signal.SIGTERM)
        except OSError:
            pass
        self.proc.wait(timeout=5)
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------- CPU oracle legs

def cpu_baselines(limbs: int, plan, seconds: float = 6.0):
    """The oracle's C recursive Toom-Cook (oracle/toom.c, same plan as the GPU)
    on this host, bounded samples of about `seconds` each: one thread and one
    product at a time; whole products on every core (the batch workload's CPU
    rate); one product with its top-level products on every core (the paper's
    scheme, Section 2)."""
    from oracle import native
    from paper_1602_02740_gb300 import inputs
    cores = os.cpu_count() or 1
    model = cpu_model()
    a = inputs.uniform(limbs, 101)
    b = inputs.uniform(limbs, 102)
    native.toom_mul(a, b, plan)                       # warm: builds and pages in
    t0 = time.perf_counter()
    native.toom_mul(a, b, plan)
    one = time.perf_counter() - t0
    n1 = max(1, int(seconds / max(one, 1e-6)))
    t0 = time.perf_counter()
    for _ in range(n1):
        native.toom_mul(a, b, plan)
    single = n1 / (time.perf_counter() - t0)
    count = cores * max(1, int(seconds / max(one, 1e-6)))
    A = np.stack([inputs.uniform(limbs, 200 + k) for k in range(min(count, 64))])
    Bm = np.stack([inputs.uniform(limbs, 300 + k) for k in range(min(count, 64))])
    A = np.resize(A, (count, limbs))
    Bm = np.resize(Bm, (count, limbs))
    t0 = time.perf_counter()
    native.toom_mul_batch(A, Bm, plan, threads=cores)
    wall = time.perf_counter() - t0
    batch = count / wall
    t0 = time.perf_counter()
    native.toom_mul(a, b, plan, threads=cores)
    one_t = time.perf_counter() - t0
    n3 = max(1, int(seconds / max(one_t, 1e-6)))
    t0 = time.perf_counter()
    for _ in range(n3):
        native.toom_mul(a, b, plan, threads=cores)
    toplevel = n3 / (time.perf_counter() - t0)
    common = {"unit": "mults/s", "kind": "oracle", "cpu": model, "nproc": cores,
              "oracle": f"C recursive Toom-Cook, plan {list(plan)}, schoolbook leaves"}
    main = dict(common, value=batch, cores=cores,
                sample=f"{count} products of {limbs}x{limbs} limbs, whole products on "
                       f"{cores} threads, {wall:.1f} s wall")
    return main, {
        "batch_all_cores": main,
        "single_thread": dict(common, value=single, cores=1,
                              sample=f"{n1} products one after another on one thread"),
        "top_level_threads": dict(common, value=toplevel, cores=cores,
                                  sample=f"{n3} products, each with its 2B-1 = {2 * plan[0] - 1} "
                                         f"top-level products on {cores} threads (Section 2)"),
    }


def headline_config(P, L, plan):
    """The workload description both arms print (the reference arm times a
    bounded sample of it, stated in its cpu_baseline)."""
    return {"workload": f"batch of {P} balanced {L * 32}-bit products per GPU, "
                        "uniform random limbs (B sweep at 2^20 bits)",
            "limbs": L, "batch_per_gpu": P, "plan": plan,
            "l2": f"operands ({2 * P * L * 4 / 1e6:.0f} MB) exceed the 129 MB L2; no flush"}


def run_reference(args, rank, world):
    """The reference arm: the oracle's C Toom-Cook (the same method, plain C,
    no GPU) on the host cores, whole products per thread, on the bench's
    workload; each step is a bounded sample of 4 products per core."""
    if rank != 0:
        return
    from oracle import native
    from paper_1602_02740_gb300 import inputs
    limbs = args.limbs
    plan = table_plan(limbs) or [12, 6, 4]
    cores = os.cpu_count() or 1
    count = 4 * cores
    A = np.stack([inputs.uniform(limbs, 2 * k) for k in range(count)])
    Bm = np.stack([inputs.uniform(limbs, 2 * k + 1) for k in range(count)])
    rates = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        native.toom_mul_batch(A, Bm, plan, threads=cores)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            rates.append(count / dt)
    value = statistics.median(rates)
    cpu = {"value": value, "unit": "mults/s", "cores": cores, "kind": "oracle", "cpu": cpu_model(),
           "sample": f"{args.steps} steps of {count} products of {limbs}x{limbs} limbs "
                     f"(C recursive Toom-Cook, plan {plan}, whole products on {cores} threads)"}
    line = {"impl": "reference", "metric": METRIC,
            "value": value, "unit": "mults/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": count / value * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": headline_config(args.batch, limbs, plan),
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": "mults/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- GPU helpers

def _rand_dev(torch, shape, seed):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    return torch.randint(-2 ** 31, 2 ** 31 - 1, shape, dtype=torch.int32, device="cuda", generator=g)


def _timed(torch, stream, fn, reps):
    """Mean ms of `reps` calls after one untimed call (CUDA events on `stream`)."""
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def madc_ceiling(torch, tc, stream):
    """The base case's integer ceiling measured live (tc_peak_madc): best of
    five launches of 4 CTAs per SM, T limb products per second."""
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    blocks, iters = 4 * sms, 2048
    sink = torch.empty(blocks * 256, dtype=torch.int32, device="cuda")
    best, n = None, 0.0
    for _ in range(6):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        n = tc.tc_peak_madc(blocks, iters, sink, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    return {"value": n / (best / 1e3) / 1e12, "unit": "T limb-products/s",
            "how": f"tc_peak_madc: {blocks} CTAs x 256 threads x {iters} iterations of 64 "
                   "register-only limb products (mad.lo.cc, madc.hi.cc, addc), best of 5 launches"}


def kernel_rooflines(phases, steps, ceiling, pk, pk_src):
    """Group the timed phases by kernel; each kernel's achieved rate against its bound."""
    total = sum(p["ms"] for p in phases) or 1.0
    by = {}
    for p in phases:
        k = by.setdefault(p["kernel"] or p["kind"], {"kind": p["kind"], "levels": [], "ms": 0.0,
                                                     "bytes": 0.0, "lp": 0.0, "launches": 0})
        k["levels"].append(p["level"])
        k["ms"] += p["ms"]
        k["bytes"] += p["bytes"]
        k["lp"] += p["limb_products"]
        k["launches"] += p["launches"]
    out = []
    for name, k in by.items():
        share = k["ms"] / total
        if k["kind"] == "base_case":
            ach = k["lp"] / (k["ms"] / 1e3) / 1e12
            r = {"kernel": name, "levels": k["levels"], "share": share, "bound": "alu",
                 "achieved": ach, "peak": ceiling["value"], "unit": "T limb-products/s",
                 "frac": ach / ceiling["value"], "peak_source": "measured live: " + ceiling["how"]}
        else:
            ach = k["bytes"] / (k["ms"] / 1e3) / 1e9
            r = {"kernel": name, "levels": k["levels"], "share": share, "bound": "hbm",
                 "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                 "frac": ach / pk["hbm_gbs"],
                 "peak_source": f"{pk_src} hbm_gbs (MEASURED_PEAKS.json)"}
        r["ms_per_step"] = k["ms"] / steps
        r["launches_per_step"] = k["launches"] / steps
        r["traffic"] = None   # DRAM bytes come from ncu captures, not from a live run
        out.append(r)
    out.sort(key=lambda r: -r["share"])
    return out


def large_products(ctx, tc, torch, stream):
    """Single products of 2^24, 2^26 and 2^27 bits: top-level B = 16 and 32
    (lower levels the cost model's best), products and squares, 5 timed calls
    each; the library's own plan; the transform base product alone and the best
    top-level B over it (Section 5); the plain schoolbook at 2^24 bits.  Every
    result is checked modulo three primes."""
    from paper_1602_02740_gb300 import autotune
    out = {}
    for L in (1 << 19, 1 << 21, 1 << 22):
        ga, gb = _rand_dev(torch, (L,), L), _rand_dev(torch, (L,), L + 1)
        go = torch.empty(2 * L, dtype=torch.int32, device="cuda")
        ha, hb = tc.to_numpy(ga)[None], tc.to_numpy(gb)[None]
        entry = {"limbs": L}
        plans = {"table": tc.tc_plan_for(ctx, L)}
        allc = autotune.candidates(L)
        for Btop in (16, 32):
            mine = [list(p) for p in allc if p and p[0] == Btop]
            plans[f"B{Btop}"] = min(mine, key=lambda p: autotune.model_seconds(L, p, 1))
        plans["ntt"] = ["ntt"]
        # Toom-Cook as the wrapper around the transform product (Section 5): best top B
        best = None
        for Btop in (2, 3, 4, 8, 16):
            ms = _timed(torch, stream, lambda: tc.tc_mul(ctx, ga, gb, go, plan=[Btop, "ntt"]), 3)
            if best is None or ms < best[0]:
                best = (ms, [Btop, "ntt"])
        plans["toom_over_ntt"] = best[1]
        for key, pl in plans.items():
            ms_m = _timed(torch, stream, lambda: tc.tc_mul(ctx, ga, gb, go, plan=pl), 5)
            ok_m = check_products(ha, hb, tc.to_numpy(go)[None])["ok"]
            ms_s = _timed(torch, stream, lambda: tc.tc_sqr(ctx, ga, go, plan=pl), 5)
            ok_s = check_products(ha, ha, tc.to_numpy(go)[None], square=True)["ok"]
            entry[key] = {"plan": pl, "ms_mul": ms_m, "ms_sqr": ms_s, "reps": 5,
                          "verified": bool(ok_m and ok_s)}
        if L == 1 << 19:
            ms_p = _timed(torch, stream, lambda: tc.tc_mul(ctx, ga, gb, go, plan=[]), 3)
            entry["plain_schoolbook_gpu"] = {
                "plan": [], "ms_mul": ms_p, "reps": 3,
                "verified": check_products(ha, hb, tc.to_numpy(go)[None])["ok"]}
        out[f"2^{(L * 32).bit_length() - 1}_bits"] = entry
        del ga, gb, go
    return out


def ntt_batch_2e20(ctx, tc, torch, stream, dA, dB, dO, A, B, toom_value):
    """The benchmark's batch through the transform base product alone and with
    Toom-12 over it (Section 5), beside the Toom-Cook path's rate."""
    P = dA.shape[0]
    out = {}
    for key, plan in (("ntt", ["ntt"]), ("toom12_over_ntt", [12, "ntt"])):
        ms = _timed(torch, stream, lambda: tc.tc_mul_uniform(ctx, dA, dB, dO, plan=plan), 3)
        rows = [0, P // 2, P - 1]
        chk = check_products(A[rows], B[rows], tc.to_numpy(dO[rows]), exact_rows=(0,))
        out[key] = {"plan": plan, "mults_per_s": P / (ms / 1e3), "ms_per_call": ms,
                    "vs_toom_schoolbook": P / (ms / 1e3) / toom_value, "verified": chk["ok"]}
    return out


def schoolbook_batch_2e20(ctx, tc, torch, stream, limbs, toom_value):
    """The plain batched schoolbook on the GPU (plan with no Toom level) on
    2^20-bit products, beside the Toom path's rate on the same size."""
    P = 608
    A, B = _rand_dev(torch, (P, limbs), 31), _rand_dev(torch, (P, limbs), 32)
    O = torch.empty((P, 2 * limbs), dtype=torch.int32, device="cuda")
    ms = _timed(torch, stream, lambda: tc.tc_mul_uniform(ctx, A, B, O, plan=[]), 3)
    rows = [0, P - 1]
    chk = check_products(tc.to_numpy(A[rows]), tc.to_numpy(B[rows]), tc.to_numpy(O[rows]))
    rate = P / (ms / 1e3)
    return {"workload": f"batch of {P} products of {limbs}x{limbs} limbs, plan [] "
                        "(bigmul column kernels)", "mults_per_s": rate, "ms_per_call": ms,
            "toom_over_schoolbook": toom_value / rate, "verified": chk["ok"]}


# ----------------------------------------------------------------- mixed batch

def mixed_batch(ctx, tc, count, rank, steps=3):
    """4096 independent products, lengths log-uniform 64..65536 limbs, 25 %
    unbalanced (ratio uniform 1..4), all in one tc_mul_batch call per step."""
    import torch
    from paper_1602_02740_gb300 import inputs
    la, lb = inputs.batch_lengths(count, seed=7 + rank)
    a_off = np.concatenate([[0], np.cumsum(la)[:-1]]).astype(np.int64)
    b_off = np.concatenate([[0], np.cumsum(lb)[:-1]]).astype(np.int64)
    o_off = np.concatenate([[0], np.cumsum(la + lb)[:-1]]).astype(np.int64)
    g = torch.Generator(device="cuda")
    g.manual_seed(11 + rank)
    A = torch.randint(-2 ** 31, 2 ** 31 - 1, (int(la.sum()),), dtype=torch.int32, device="cuda", generator=g)
    B = torch.randint(-2 ** 31, 2 ** 31 - 1, (int(lb.sum()),), dtype=torch.int32, device="cuda", generator=g)
    O = torch.empty(int((la + lb).sum()), dtype=torch.int32, device="cuda")
    tc.tc_mul_batch(ctx, A, a_off, la, B, b_off, lb, O, o_off)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        tc.tc_mul_batch(ctx, A, a_off, la, B, b_off, lb, O, o_off)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    bits = 32.0 * float((la + lb).sum())
    # the same batch prepared once (tc_batch_prepare) and its run captured into a
    # CUDA graph: each step is one graph replay (device time by CUDA events)
    bt = tc.tc_batch_prepare(ctx, a_off, la, b_off, lb, o_off)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    tc.tc_batch_run(ctx, bt, A, B, O, stream=s)
    s.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        tc.tc_batch_run(ctx, bt, A, B, O, stream=s)
    graph.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        graph.replay()
    e1.record()
    torch.cuda.synchronize()
    tc.tc_batch_check(ctx, bt)
    gdt = e0.elapsed_time(e1) / 1e3 / steps
    del graph
    bt.close()
    # every product of the last replay, modulo three primes
    hA, hB, hO = tc.to_numpy(A), tc.to_numpy(B), tc.to_numpy(O)
    bad = None
    for k in range(count):
        a = hA[a_off[k]:a_off[k] + la[k]][None]
        b = hB[b_off[k]:b_off[k] + lb[k]][None]
        o = hO[o_off[k]:o_off[k] + la[k] + lb[k]][None]
        if not check_products(a, b, o)["ok"]:
            bad = k
            break
    return {"workload": f"{count} products, lengths log-uniform 64..65536 limbs, 25% unbalanced "
                        "(ratio 1..4), one tc_mul_batch call", "mults_per_s": count / dt,
            "ms_per_call": dt * 1e3, "product_bits_per_s": bits / dt, "steps": steps,
            "graph_replay": {"mults_per_s": count / gdt, "ms_per_call": gdt * 1e3,
                             "product_bits_per_s": bits / gdt,
                             "how": "tc_batch_prepare once, tc_batch_run captured in one CUDA graph"},
            "verified": {"ok": bad is None, "rows": count, "residue_primes": 3,
                         "first_bad_row": bad}}


# ----------------------------------------------------------------- serving

def serving(ctx, tc, count, rank, warm=2000):
    """Poisson stream of multiply requests, lengths log-uniform 256..2^20 limbs,
    admitted by a 40 GB scratch budget; first the saturated rate (all submitted
    at once), then arrivals at 0.5x and 0.8x of it.  Latency = submit -> done."""
    import torch
    from paper_1602_02740_gb300 import inputs
    sctx = tc.tc_create(torch.cuda.current_device(), budget_bytes=40 << 30,
                        table=PLAN_TABLE if os.path.exists(PLAN_TABLE) else None)
    _, lens = inputs.poisson_stream(count, seed=5 + rank, rate_per_s=1.0)
    lens = lens.astype(np.int64)
    g = inputs.rng(9 + rank)
    pool_len = 1 << 21
    gen = torch.Generator(device="cuda")
    gen.manual_seed(13 + rank)
    poolA = torch.randint(-2 ** 31, 2 ** 31 - 1, (pool_len,), dtype=torch.int32, device="cuda", generator=gen)
    poolB = torch.randint(-2 ** 31, 2 ** 31 - 1, (pool_len,), dtype=torch.int32, device="cuda", generator=gen)
    offs_a = (g.random(count) * (pool_len - lens)).astype(np.int64)
    offs_b = (g.random(count) * (pool_len - lens)).astype(np.int64)
    out_off = np.concatenate([[0], np.cumsum(2 * lens)[:-1]]).astype(np.int64)
    OUT = torch.empty(int(2 * lens.sum()), dtype=torch.int32, device="cuda")
    views = [(poolA[offs_a[i]:offs_a[i] + lens[i]], poolB[offs_b[i]:offs_b[i] + lens[i]],
              OUT[out_off[i]:out_off[i] + 2 * lens[i]]) for i in range(count)]

    def run(rate, n=count):
        arrivals = None
        if rate:
            arrivals = np.cumsum(inputs.rng(17 + rank).exponential(1.0 / rate, size=count))
        pending = []
        t0 = time.perf_counter()
        for i, (a, b, o) in enumerate(views[:n]):
            if arrivals is not None:
                while time.perf_counter() - t0 < arrivals[i]:
                    pending = [k for k in pending if not tc.tc_serve_poll(sctx, k)]
            while True:
                k = tc.tc_serve_submit(sctx, a, b, o)
                if k >= 0:
                    break
                pending = [k2 for k2 in pending if not tc.tc_serve_poll(sctx, k2)]
            pending.append(k)
        while pending:
            pending = [k for k in pending if not tc.tc_serve_poll(sctx, k)]
        wall = time.perf_counter() - t0
        st = tc.tc_serve_stats(sctx)
        tc.tc_serve_stop(sctx)
        return {"requests": n, "rate_per_s": rate, "wall_s": wall,
                "completed_per_s": n / wall, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
                "product_bits_per_s": st["bits_per_s"]}

    run(None, min(count, warm))                  # warm-up (plans, pool)
    sat = run(None)
    sat_rate = sat["completed_per_s"]
    loads = [run(f * sat_rate) for f in (0.5, 0.8)]
    sctx.close()
    return {"workload": "Poisson stream, balanced lengths log-uniform 256..2^20 limbs, uniform limbs, "
                        "40 GB scratch budget", "requests_per_run": count,
            "saturated": sat, "load_0.5": loads[0], "load_0.8": loads[1]}


# ----------------------------------------------------------------- ranks

def combine_ranks(value, dist, device=None):
    """Max over ranks of a per-rank duration (every rank gets the max).
    Products are sharded, not exchanged: this is the only collective."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_seed(rank: int, k: int) -> int:
    """Seed of operand k on a rank: every rank multiplies its own products."""
    return 1_000_000 * rank + k


# ----------------------------------------------------------------- single-kernel cases

def _time_case(torch, fn, reps):
    # the calls under study run inside the NVTX range "measure", so a capture can
    # select them with: ncu --nvtx --nvtx-include "measure/" ...
    torch.cuda.nvtx.range_push("measure")
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    return e0.elapsed_time(e1) / reps


def run_case(args):
    """One library call under study (for ncu captures and kernel timing).

    interp: one Toom level's interpolation (tc_toom_interpolate, or with
            --method matrix tc_toom_interpolate_matrix) of `count` products of
            `limbs`-limb operands split into B blocks; its inputs are the true
            pointwise products (evaluation, then products of the evaluations).
    leaf:   the batched schoolbook (tc_schoolbook) of `count` products.
    eval:   one level's evaluation (tc_toom_evaluate) of `count` operands.
    ntt:    the transform base product (tc_ntt_mul) of `count` products.
    Prints one JSON line with the mean time of `reps` calls after one untimed call.
    """
    import torch
    from paper_1602_02740_gb300 import tc
    torch.cuda.set_device(0)
    res = {"case": args.case, "B": args.B, "reps": args.reps}
    if args.case == "leaf":
        count, L = args.count or 157320, args.limbs if args.limbs != LIMBS else 184
        A, B = _rand_dev(torch, (count, L), 1), _rand_dev(torch, (count, L), 2)
        OUT = torch.empty((count, 2 * L), dtype=torch.int32, device="cuda")
        tc.tc_set_leaf_karatsuba(49 if args.leaf == "karatsuba" else 0)
        ms = _time_case(torch, lambda: tc.tc_schoolbook(A, B, OUT), args.reps)
        tc.tc_set_leaf_karatsuba(tc.TC_LEAF_KARATSUBA_DEFAULT)
        res["leaf"] = args.leaf
    elif args.case == "ntt":
        count, L = args.count or 1, args.limbs
        A, B = _rand_dev(torch, (count, L), 1), _rand_dev(torch, (count, L), 2)
        OUT = torch.empty((count, 2 * L), dtype=torch.int32, device="cuda")
        work = torch.empty(tc.tc_ntt_work_bytes(count, L), dtype=torch.uint8, device="cuda")
        ms = _time_case(torch, lambda: tc.tc_ntt_mul(A, B, OUT, work), args.reps)
    elif args.case == "eval":
        count, L = args.count or 2432, args.limbs
        U = _rand_dev(torch, (count, L), 1)
        _, e, estride, _ = tc.level_sizes(L, args.B)
        E = torch.empty((count, 2 * args.B - 1, estride), dtype=torch.int32, device="cuda")
        S = torch.empty((count, 2 * args.B - 1), dtype=torch.uint8, device="cuda")
        ms = _time_case(torch, lambda: tc.tc_toom_evaluate(U, args.B, E, S), args.reps)
    else:
        count, L = args.count or 2048, args.limbs
        npts = 2 * args.B - 1
        _, e, estride, ystride = tc.level_sizes(L, args.B)
        ctx = tc.tc_create(0)
        U, V = _rand_dev(torch, (count, L), 1), _rand_dev(torch, (count, L), 2)
        EU, SU = tc.tc_toom_evaluate(U, args.B)
        EV, SV = tc.tc_toom_evaluate(V, args.B)
        del U, V
        Y = torch.zeros((count, npts, ystride), dtype=torch.int32, device="cuda")
        rows = count * npts
        tc.tc_mul_uniform(ctx, EU.view(rows, estride)[:, :e], EV.view(rows, estride)[:, :e],
                          Y.view(rows, ystride)[:, :2 * e])
        del EU, EV
        OUT = torch.empty((count, 2 * L), dtype=torch.int32, device="cuda")
        wb = tc.tc_toom_interpolate_work_bytes(count, L, args.B)
        work = torch.empty(max(wb, 1), dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        ctx.close()
        if args.method == "matrix":
            ms = _time_case(torch, lambda: tc.tc_toom_interpolate_matrix(Y, L, args.B, SU, SV, OUT),
                            args.reps)
        else:
            ms = _time_case(torch, lambda: tc.tc_toom_interpolate(Y, L, args.B, SU, SV, OUT, work),
                            args.reps)
        res["method"] = args.method
    res.update(count=count, limbs=L, ms_per_call=ms)
    print(json.dumps(res), flush=True)


# ----------------------------------------------------------------- GPU leg

def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.case:
        return run_case(args)

    import torch
    from paper_1602_02740_gb300 import inputs, tc

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    L, P = args.limbs, args.batch
    ctx = tc.tc_create(local, table=PLAN_TABLE if os.path.exists(PLAN_TABLE) else None)
    plan = None if args.plan == "auto" else [int(x) for x in args.plan.split(",") if x]
    used_plan = plan if plan is not None else tc.tc_plan_for(ctx, L)

    # seeded operands (host generation, one upload)
    A = np.empty((P, L), dtype=np.uint32)
    B = np.empty((P, L), dtype=np.uint32)
    for k in range(P):
        A[k] = inputs.uniform(L, rank_seed(rank, 2 * k))
        B[k] = inputs.uniform(L, rank_seed(rank, 2 * k + 1))
    dA, dB = tc.to_device(A), tc.to_device(B)
    dO = torch.empty((P, 2 * L), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    for _ in range(max(3, args.warmup)):
        tc.tc_mul_uniform(ctx, dA, dB, dO, plan=used_plan)
    torch.cuda.synchronize()
    dO.fill_(-1)                                  # the check below sees only the timed steps' output

    clocks = ClockSampler(local).start()
    time.sleep(0.3)
    tc.tc_profile_enable(ctx, True)
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        tc.tc_mul_uniform(ctx, dA, dB, dO, plan=used_plan)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_total = ev0.elapsed_time(ev1)
    phases = tc.tc_profile_read(ctx)
    tc.tc_profile_enable(ctx, False)
    clk = clocks.stop()
    ms_total = combine_ranks(ms_total, dist, device="cuda")
    ms_step = ms_total / args.steps
    value = world * P / (ms_step / 1e3)
    launches = sum(p["launches"] for p in phases)

    # ---- the last timed step's products: every row modulo three primes, some exactly ----
    verified = check_products(A, B, tc.to_numpy(dO), exact_rows=(0, P // 2, P - 1))

    # ---- the base case's integer ceiling, measured live ----
    ceiling = madc_ceiling(torch, tc, stream)

    # ---- end to end through the host-buffer entry points (pinned memory) ----
    hA = torch.from_numpy(A.view(np.int32)).pin_memory()
    hB = torch.from_numpy(B.view(np.int32)).pin_memory()
    hO = torch.empty((P, 2 * L), dtype=torch.int32).pin_memory()
    e2e_steps = max(3, min(args.steps, 20))
    # pipelined entry point: each step copies its inputs in and its products out,
    # two steps in flight (copies overlap the kernels of the neighbouring step)
    pipe = tc.tc_pipe_create(ctx, P, L, plan=used_plan)
    pipe.submit(hA, hB, hO)
    pipe.wait()
    hO.fill_(-1)
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        pipe.submit(hA, hB, hO)
    pipe.wait()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_s = combine_ranks(e2e_s, dist, device="cuda")
    pipe.close()
    e2e_verified = check_products(A, B, hO.numpy().view(np.uint32))
    # blocking entry point: copy in, multiply, copy out, wait -- one step at a time
    tc.tc_mul_uniform_host(ctx, hA, hB, hO, plan=used_plan)
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        tc.tc_mul_uniform_host(ctx, hA, hB, hO, plan=used_plan)
    blk_s = (time.perf_counter() - t0) / e2e_steps
    blk_s = combine_ranks(blk_s, dist, device="cuda")
    e2e = {"value": world * P / e2e_s, "unit": "mults/s",
           "h2d_bytes_per_step": 2 * P * L * 4, "d2h_bytes_per_step": P * 2 * L * 4,
           "api": "tc_pipe_submit x %d + tc_pipe_wait (pinned host buffers)" % e2e_steps,
           "pinned": bool(hA.is_pinned() and hB.is_pinned() and hO.is_pinned()),
           "verified": e2e_verified,
           "blocking": {"api": "tc_mul_uniform_host", "value": world * P / blk_s}}
    del hA, hB, hO

    # ---- B sweep: top-level B in {2,3,4,8,16}; lower levels = the cost model's 3 best ----
    sweep = None
    if not args.no_sweep:
        from paper_1602_02740_gb300 import autotune
        allc = autotune.candidates(L)
        sweep = {}
        for Btop in (2, 3, 4, 8, 16):
            mine = sorted((list(p) for p in allc if p and p[0] == Btop),
                          key=lambda p: autotune.model_seconds(L, p, P))[:3]
            best = None
            for pl in mine:
                try:
                    ms = _timed(torch, stream, lambda: tc.tc_mul_uniform(ctx, dA, dB, dO, plan=pl), 3)
                except tc.TCError:
                    continue
                if best is None or ms < best[0]:
                    best = (ms, pl)
            if best:
                sweep[str(Btop)] = {"plan": best[1], "mults_per_s": P / (best[0] / 1e3),
                                    "ns_per_product": best[0] * 1e6 / P}

    # ---- Toom-3 at 1024 limbs; all-ones and sparse limbs at 2^20 bits ----
    other = None
    if not args.no_configs:
        other = {}
        n3 = 16384
        a3, b3 = _rand_dev(torch, (n3, 1024), 41), _rand_dev(torch, (n3, 1024), 42)
        o3 = torch.empty((n3, 2048), dtype=torch.int32, device="cuda")
        ms_b = _timed(torch, stream, lambda: tc.tc_mul_uniform(ctx, a3, b3, o3, plan=[3]), 10)
        rows = [0, 1, n3 - 1]
        ok3 = check_products(tc.to_numpy(a3[rows]), tc.to_numpy(b3[rows]), tc.to_numpy(o3[rows]),
                             exact_rows=(0,))["ok"]
        ms_1 = _timed(torch, stream, lambda: tc.tc_mul(ctx, a3[0], b3[0], o3[0], plan=[3]), 1000)
        ones = torch.full((1024,), -1, dtype=torch.int32, device="cuda")
        tc.tc_mul(ctx, ones, ones, o3[1], plan=[3])
        w1 = tc.to_numpy(o3[1])
        want1 = ((1 << 32768) - 1) ** 2
        ok1 = _int(w1) == want1
        other["toom3_1024_limbs"] = {"plan": [3], "batch": n3,
                                     "ns_per_product_batched": ms_b * 1e6 / n3,
                                     "ns_per_product_single": ms_1 * 1e6, "reps_single": 1000,
                                     "verified": bool(ok3 and ok1),
                                     "all_ones_closed_form": bool(ok1)}
        del a3, b3, o3
        for kind in ("all_ones", "sparse"):
            rows = np.stack([inputs.operand(kind, L, 500 + k) for k in range(8)])
            reps_rows = np.tile(rows, (P // 8 + 1, 1))[:P]
            dA2 = tc.to_device(reps_rows)
            dB2 = dA2 if kind == "all_ones" else dB
            ms_k = _timed(torch, stream,
                          lambda: tc.tc_mul_uniform(ctx, dA2, dB2, dO, plan=used_plan), 3)
            chk = check_products(reps_rows[:16], (reps_rows if kind == "all_ones" else B)[:16],
                                 tc.to_numpy(dO[:16]), exact_rows=(0,))
            other[f"{kind}_2e20"] = {"mults_per_s": P / (ms_k / 1e3), "plan": used_plan,
                                     "operands": "all-ones squared" if kind == "all_ones"
                                     else "sparse (1 % nonzero limbs) x uniform",
                                     "verified": chk["ok"]}
            del dA2
        other["plain_schoolbook_gpu_2e20"] = schoolbook_batch_2e20(ctx, tc, torch, stream, L, value)
        other["ntt_2e20"] = ntt_batch_2e20(ctx, tc, torch, stream, dA, dB, dO, A, B, value)

    large = None
    if not args.no_large:
        lclk = ClockSampler(local).start()
        large = large_products(ctx, tc, torch, stream)
        large["clocks"] = lclk.stop()

    mixed = mixed_batch(ctx, tc, args.mixed, rank) if args.mixed else None
    serve = serving(ctx, tc, args.serve, rank) if args.serve else None

    # ---- rooflines: every kernel of the timed step, the dominant one by share ----
    pk, pk_src = peaks()
    roofs = kernel_rooflines(phases, args.steps, ceiling, pk, pk_src)
    roof = dict(roofs[0]) if roofs else None

    cpu, cpus = None, None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu, cpus = cpu_baselines(L, used_plan)

    if rank == 0:
        ok = verified["ok"] and e2e_verified["ok"]
        line = {
            "metric": METRIC,
            "value": value if ok else None, "unit": "mults/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "ns_per_product": ms_step * 1e6 / P,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": headline_config(P, L, used_plan),
            "verified": verified,
            "roofline": roof, "rooflines": roofs, "int_ceiling": ceiling,
            "phases": [{"kind": p["kind"], "level": p["level"], "kernel": p["kernel"],
                        "ms_per_step": p["ms"] / args.steps} for p in phases],
            "sweep": sweep, "mixed_batch": mixed, "serving": serve, "configs": other,
            "large": large, "cpu_baseline": cpu, "cpu_baselines": cpus, "e2e": e2e,
            "gpu_launches": launches, "clocks": clk,
        }
        if not ok:
            line["error"] = "products of the timed run differ from a * b: no value reported"
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
