"""Benchmark: exact products of 2^20-bit integers per second on GB300.

Workload (one "step"): a batch of P balanced products of two 2^20-bit
operands (32768 uint32 limbs each, limbs uniform from a seed) through the
whole Toom-Cook path (evaluation, recursive pointwise products, schoolbook
base case, interpolation, recomposition) in one library call.  P = 2432 per
GPU (16 x 152 SMs), so the operands alone (608 MB) exceed the 129 MB L2 and
no L2 flush is needed between steps.

Prints one JSON line (rank 0).  `value` is whole-job products per second
(Mults/s); `e2e` is the same metric through the pipelined host-buffer
entry point (tc_pipe_submit: every step copies its operands in from pinned
host memory and its products out, two steps in flight), with the blocking
host-buffer call (tc_mul_uniform_host) beside it; `roofline` describes
the dominant kernel; `cpu_baseline` is the CPU oracle (plain schoolbook) on
a bounded sample on this machine's host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import signal
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

LIMBS = 32768            # 2^20 bits
PER_GPU = 2432           # 16 x 152 SMs
SM_COUNT = 152
IMAD_PER_CLK_SM = 64     # 32-bit integer multiply(-add) results per clock per SM
IMAD_PER_LIMB_PRODUCT = 2  # low and high halves of a 32 x 32 -> 64-bit product

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
    p.add_argument("--serve", type=int, default=2000,
                   help="requests per serving run (the full serving workload is 20000; 0 = skip)")
    p.add_argument("--no-configs", action="store_true",
                   help="skip the Toom-3 at 1024 limbs and the all-ones / sparse 2^20-bit lines")
    p.add_argument("--large", action="store_true",
                   help="also time single products of 2^24, 2^26 and 2^27 bits (and squares)")
    p.add_argument("--case", choices=["interp", "leaf", "eval"], default=None,
                   help="time one kernel call for a profiler capture instead of the benchmark")
    p.add_argument("--count", type=int, default=None, help="--case: products or rows")
    p.add_argument("--B", type=int, default=12, help="--case interp/eval: blocks")
    p.add_argument("--reps", type=int, default=3, help="--case: timed repetitions")
    p.add_argument("--method", choices=["newton", "matrix"], default="newton",
                   help="--case interp: even-odd Newton route or inverse-Vandermonde matrix")
    return p.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


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


# ----------------------------------------------------------------- CPU oracle leg

def cpu_oracle_rate(limbs: int, seconds_budget: float = 20.0):
    """Products/s of the oracle's C schoolbook on this host's cores (bounded sample)."""
    from concurrent.futures import ThreadPoolExecutor
    from oracle import native
    from paper_1602_02740_gb300 import inputs
    cores = os.cpu_count() or 1
    a = inputs.uniform(limbs, 101)
    b = inputs.uniform(limbs, 102)
    t0 = time.perf_counter()
    native.schoolbook(a, b)                      # one product: calibrates the sample size
    one = time.perf_counter() - t0
    per_thread = max(1, int(seconds_budget / max(one, 1e-6) / cores))
    n = per_thread * cores
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=cores) as ex:
        list(ex.map(lambda _: native.schoolbook(a, b), range(n)))
    wall = time.perf_counter() - t0
    return {"value": n / wall, "unit": "mults/s", "cores": cores, "kind": "oracle",
            "sample": f"{n} products of {limbs}x{limbs} limbs by the plain C schoolbook, "
                      f"{cores} threads, {wall:.1f} s wall"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    limbs = args.limbs
    rates = []
    cpu = None
    for i in range(args.warmup + args.steps):
        r = cpu_oracle_rate(limbs, seconds_budget=4.0 if i >= args.warmup else 1.0)
        if i >= args.warmup:
            rates.append(r["value"])
            cpu = r
    value = statistics.median(rates)
    cpu["value"] = value
    line = {"impl": "reference", "metric": "exact 2^20-bit products per second (Mults/s)",
            "value": value, "unit": "mults/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"balanced {limbs * 32}-bit products, uniform limbs",
                       "limbs": limbs},
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": "mults/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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
    return {"workload": f"{count} products, lengths log-uniform 64..65536 limbs, 25% unbalanced "
                        "(ratio 1..4), one tc_mul_batch call", "mults_per_s": count / dt,
            "ms_per_call": dt * 1e3, "product_bits_per_s": bits / dt, "steps": steps,
            "graph_replay": {"mults_per_s": count / gdt, "ms_per_call": gdt * 1e3,
                             "product_bits_per_s": bits / gdt,
                             "how": "tc_batch_prepare once, tc_batch_run captured in one CUDA graph"}}


# ----------------------------------------------------------------- serving

def serving(ctx, tc, count, rank):
    """Poisson stream of multiply requests, lengths log-uniform 256..2^20 limbs,
    admitted by a 40 GB scratch budget; first the saturated rate (all submitted
    at once), then arrivals at 0.5x and 0.8x of it.  Latency = submit -> done."""
    import torch
    from paper_1602_02740_gb300 import inputs
    sctx = tc.tc_create(torch.cuda.current_device(), budget_bytes=40 << 30)
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

    def run(rate):
        arrivals = None
        if rate:
            arrivals = np.cumsum(inputs.rng(17 + rank).exponential(1.0 / rate, size=count))
        pending = []
        t0 = time.perf_counter()
        for i, (a, b, o) in enumerate(views):
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
        return {"requests": count, "rate_per_s": rate, "wall_s": wall,
                "completed_per_s": count / wall, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
                "product_bits_per_s": st["bits_per_s"]}

    run(None)                                    # warm-up (plans, pool)
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

def _rand_dev(torch, shape, seed):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    return torch.randint(-2 ** 31, 2 ** 31 - 1, shape, dtype=torch.int32, device="cuda", generator=g)


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
        ms = _time_case(torch, lambda: tc.tc_schoolbook(A, B, OUT), args.reps)
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
    table = os.path.join(ROOT, "paper_1602_02740_gb300", "plans_gb300.txt")
    ctx = tc.tc_create(local, table=table if os.path.exists(table) else None)
    plan = None if args.plan == "auto" else [int(x) for x in args.plan.split(",")]
    used_plan = plan or tc.tc_plan_for(ctx, L)

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

    clocks = ClockSampler(local)
    clocks.start()
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

    # ---- end to end through the host-buffer entry point (pinned memory) ----
    hA = torch.from_numpy(A.view(np.int32)).pin_memory()
    hB = torch.from_numpy(B.view(np.int32)).pin_memory()
    hO = torch.empty((P, 2 * L), dtype=torch.int32).pin_memory()
    e2e_steps = max(3, min(args.steps, 10))
    # pipelined entry point: each step copies its inputs in and its products out,
    # two steps in flight (copies overlap the kernels of the neighbouring step)
    pipe = tc.tc_pipe_create(ctx, P, L, plan=used_plan)
    pipe.submit(hA, hB, hO)
    pipe.wait()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        pipe.submit(hA, hB, hO)
    pipe.wait()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_s = combine_ranks(e2e_s, dist, device="cuda")
    pipe.close()
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
           "blocking": {"api": "tc_mul_uniform_host", "value": world * P / blk_s}}

    # ---- B sweep: top-level B in {2,3,4,8,16}; lower levels = the cost model's 3 best ----
    sweep = None
    if not args.no_sweep:
        from paper_1602_02740_gb300 import autotune
        allc = autotune.candidates(L)
        cands = {}
        for Btop in (2, 3, 4, 8, 16):
            mine = [list(p) for p in allc if p and p[0] == Btop]
            mine.sort(key=lambda p: autotune.model_seconds(L, p, P))
            cands[Btop] = mine[:3]
        sweep = {}
        for Btop, plans in cands.items():
            best = None
            for pl in plans:
                try:
                    tc.tc_mul_uniform(ctx, dA, dB, dO, plan=pl)
                except tc.TCError:
                    continue
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(3):
                    tc.tc_mul_uniform(ctx, dA, dB, dO, plan=pl)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / 3
                if best is None or ms < best[0]:
                    best = (ms, pl)
            if best:
                sweep[str(Btop)] = {"plan": best[1], "mults_per_s": P / (best[0] / 1e3),
                                    "ns_per_product": best[0] * 1e6 / P}

    # ---- the other configurations: Toom-3 at 1024 limbs; all-ones and sparse limbs ----
    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    other = None
    if not args.no_configs:
        other = {}
        # one Toom-3 level over a batch of 1024-limb products, and one product alone
        n3 = 16384
        a3 = torch.randint(-2 ** 31, 2 ** 31 - 1, (n3, 1024), dtype=torch.int32, device="cuda")
        b3 = torch.randint(-2 ** 31, 2 ** 31 - 1, (n3, 1024), dtype=torch.int32, device="cuda")
        o3 = torch.empty((n3, 2048), dtype=torch.int32, device="cuda")

        ms_b = timed(lambda: tc.tc_mul_uniform(ctx, a3, b3, o3, plan=[3]), 10)
        ms_1 = timed(lambda: tc.tc_mul(ctx, a3[0], b3[0], o3[0], plan=[3]), 1000)
        other["toom3_1024_limbs"] = {"plan": [3], "batch": n3,
                                       "ns_per_product_batched": ms_b * 1e6 / n3,
                                       "ns_per_product_single": ms_1 * 1e6, "reps_single": 1000}
        del a3, b3, o3
        # the headline batch with all-ones and with sparse limbs (1 % nonzero)
        from paper_1602_02740_gb300 import inputs as _inputs
        for kind in ("all_ones", "sparse"):
            rows = np.stack([_inputs.operand(kind, L, 500 + k) for k in range(8)])
            reps_rows = np.tile(rows, (P // 8 + 1, 1))[:P]
            dA2 = torch.from_numpy(reps_rows.view(np.int32)).to("cuda")
            ms_k = timed(lambda: tc.tc_mul_uniform(ctx, dA2, dA2 if kind == "all_ones" else dB, dO,
                                                   plan=used_plan), 3)
            other[f"{kind}_2e20"] = {"mults_per_s": P / (ms_k / 1e3), "plan": used_plan,
                                       "operands": "all-ones squared" if kind == "all_ones"
                                       else "sparse (1 % nonzero limbs) x uniform"}
            del dA2
    large = None
    if args.large:
        large = {}
        for Lg in (1 << 19, 1 << 21, 1 << 22):
            ga = torch.randint(-2 ** 31, 2 ** 31 - 1, (Lg,), dtype=torch.int32, device="cuda")
            gb = torch.randint(-2 ** 31, 2 ** 31 - 1, (Lg,), dtype=torch.int32, device="cuda")
            go = torch.empty(2 * Lg, dtype=torch.int32, device="cuda")
            ms_m = timed(lambda: tc.tc_mul(ctx, ga, gb, go), 3)
            ms_s = timed(lambda: tc.tc_sqr(ctx, ga, go), 3)
            large[f"2^{(Lg * 32).bit_length() - 1}_bits"] = {
                "plan": tc.tc_plan_for(ctx, Lg), "ms_mul": ms_m, "ms_sqr": ms_s}
            del ga, gb, go

    mixed = mixed_batch(ctx, tc, args.mixed, rank) if args.mixed else None
    serve = serving(ctx, tc, args.serve, rank) if args.serve else None

    # ---- roofline of the dominant phase ----
    pk, pk_src = peaks()
    top = max(phases, key=lambda p: p["ms"])
    avg_ms = top["ms"] / top["launches"]
    if top["kind"] == "base_case":
        mhz = pk.get("sm_max_mhz", 2070.0)
        peak = SM_COUNT * IMAD_PER_CLK_SM / IMAD_PER_LIMB_PRODUCT * mhz * 1e6 / 1e12
        achieved = top["limb_products"] / top["launches"] / (avg_ms / 1e3) / 1e12
        # per launch: bytes = 16 s N and limb products = s^2 N for N products of s limbs
        leaf_s = int(round(top["limb_products"] / (top["bytes"] / 16.0))) if top["bytes"] else 0
        n_leaf = top["limb_products"] / top["launches"] / max(1, leaf_s) ** 2 if leaf_s else 0
        # the library's base-case choice: tile kernel below 4096 products, else a
        # lane pair per product while a block's rows (256 x stride bytes) fit 200 KB
        sp = -(-leaf_s // 8) * 8
        sp += 8 if sp % 32 in (0, 16) else 0
        kname = ("leaf_kernel" if n_leaf < 4096 else
                 "leaf_pair_kernel<false>" if 256 * sp <= 200 * 1024 else "leaf_lane_kernel<false>")
        traffic = (n_leaf * LEAF_TRAFFIC["bytes_per_product"]
                   if leaf_s == LEAF_TRAFFIC["limbs"] and kname == LEAF_TRAFFIC["kernel"] else None)
        roof = {"kernel": kname, "bound": "alu", "achieved": achieved, "peak": peak,
                "unit": "T limb-products/s", "frac": achieved / peak, "traffic": traffic,
                "traffic_source": "profiles/leaf_pair_2e20.md (scaled by leaf products)",
                "peak_source": f"derived: {SM_COUNT} SMs x {IMAD_PER_CLK_SM} IMAD/clk / "
                               f"{IMAD_PER_LIMB_PRODUCT} x {mhz:.0f} MHz"}
    else:
        peak = pk["hbm_gbs"]
        achieved = top["bytes"] / top["launches"] / (avg_ms / 1e3) / 1e9
        name = "interp_kernel" if top["kind"] == "interpolate" else "eval_kernel"
        roof = {"kernel": name, "level": top["level"], "bound": "hbm", "achieved": achieved,
                "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                "peak_source": f"{pk_src} hbm_gbs (MEASURED_PEAKS.json)"}
    phase_summary = [{"kind": p["kind"], "level": p["level"],
                      "ms_per_step": p["ms"] / args.steps,
                      "share": p["ms"] / sum(q["ms"] for q in phases)} for p in phases]

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_oracle_rate(L)

    if rank == 0:
        line = {
            "metric": "exact 2^20-bit products per second (Mults/s)",
            "value": value, "unit": "mults/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "ns_per_product": ms_step * 1e6 / P,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": f"batch of {P} balanced {L * 32}-bit products per GPU, "
                                   "uniform random limbs (B sweep at 2^20 bits)",
                       "limbs": L, "batch_per_gpu": P, "plan": used_plan,
                       "l2": f"operands ({2 * P * L * 4 / 1e6:.0f} MB) exceed the 129 MB L2; no flush"},
            "roofline": roof, "phases": phase_summary, "sweep": sweep,
            "mixed_batch": mixed, "serving": serve, "configs": other, "large": large,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
