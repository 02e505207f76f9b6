"""Autotuner: choose the recursion plan (B per level, hence the Toom-to-schoolbook
threshold) per operand size class, by timing candidate plans on the GPU.

Candidates are all B sequences over {2, 3, 4, 5, 6, 8, 12, 16, 32} up to five
levels whose base-case length falls in [LEAF_MIN, LEAF_MAX] limbs; a cost model
(base-case limb products, interpolation work n^2 * values, evaluation work)
ranks them and the best few are timed through the C ABI with CUDA events.
From NTT_MIN limbs on, the transform base product alone and one or two Toom
levels over it (Section 5) are timed as well.  The winners are written as a
plan table (one line per size class: "<max_limbs> <levels> <B0> <B1> ...
[ntt]") that tc_create loads.

    python -m paper_1602_02740_gb300.autotune --out paper_1602_02740_gb300/plans_gb300.txt
"""
from __future__ import annotations

import argparse
import itertools
import math
import os
import sys
import time

BS = (2, 3, 4, 5, 6, 8, 12, 16, 32)
LEAF_MIN, LEAF_MAX = 24, 224

# cost-model rates (per second), measured on GB300 with the current kernels on
# the 2^20-bit batch (2432 products, plan [12, 6, 4]): base case 6.9 T limb
# products/s; interpolation 3.1-4.3e11 n^2 Y product-limbs/s (levels 0, 1, 2:
# 3.4, 3.1, 4.3e11); evaluation 1.0-1.5e12 B n e row-limbs/s (1.4, 1.5, 1.0e12)
LEAF_RATE = 6.9e12        # base-case limb products
INTERP_RATE = 3.5e11      # n^2 x interpolation-value limbs
EVAL_RATE = 1.3e12        # B x n x evaluation limbs
LAUNCH_S = 6e-6           # per kernel launch
NTT_MIN = 1024            # smallest size class at which transform-based plans are timed


def level(s: int, B: int):
    n = B - 1
    b = -(-s // B)
    e = b + -(-(n * (n - 1) + 1) // 32)
    return b, e


def plan_leaf(s: int, plan) -> int:
    for B in plan:
        s = level(s, B)[1]
    return s


def model_seconds(s: int, plan, count: int) -> float:
    P = count
    t = 0.0
    for B in plan:
        n = B - 1
        b, e = level(s, B)
        Y = 2 * e + 2
        t += INTERP_RATE ** -1 * n * n * Y * P
        t += EVAL_RATE ** -1 * 2 * B * n * e * P
        t += 4 * LAUNCH_S
        P *= 2 * B - 1
        s = e
    t += s * s * P / LEAF_RATE
    return t


def candidates(s: int, max_levels: int = 5):
    out = []
    if s <= LEAF_MAX * 2:
        out.append(())
    for depth in range(1, max_levels + 1):
        for plan in itertools.product(BS, repeat=depth):
            ok = True
            L = s
            for B in plan:
                if B > L:
                    ok = False
                    break
                L = level(L, B)[1]
            if ok and LEAF_MIN <= L <= LEAF_MAX and L < s:
                out.append(plan)
    return out


def ntt_candidates(s: int):
    """Transform-based plans: the transform product alone, and one or two Toom
    levels over it (Section 5)."""
    if s < NTT_MIN:
        return []
    out = [("ntt",)]
    for B in (2, 3, 4, 8, 16):
        if B <= s:
            out.append((B, "ntt"))
    for B1, B2 in ((3, 3), (4, 4), (16, 4)):
        if B1 * B2 <= s:
            out.append((B1, B2, "ntt"))
    return out


def tune_size(ctx, s: int, count: int, top: int = 10, reps: int = 3, verbose=False, ntt=True):
    import torch
    from . import tc
    cands = sorted(candidates(s), key=lambda p: model_seconds(s, p, count))[:top]
    if ntt:
        cands += ntt_candidates(s)
    g = torch.Generator(device="cuda")
    g.manual_seed(s)
    A = torch.randint(-2 ** 31, 2 ** 31 - 1, (count, s), dtype=torch.int32, device="cuda", generator=g)
    B = torch.randint(-2 ** 31, 2 ** 31 - 1, (count, s), dtype=torch.int32, device="cuda", generator=g)
    O = torch.empty((count, 2 * s), dtype=torch.int32, device="cuda")
    best = None
    for plan in cands:
        try:
            tc.tc_mul_uniform(ctx, A, B, O, plan=list(plan))
        except tc.TCError:
            continue
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            tc.tc_mul_uniform(ctx, A, B, O, plan=list(plan))
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        if verbose:
            model = ("" if plan and plan[-1] == "ntt"
                     else f" (model {model_seconds(s, plan, count) * 1e3:.3f})")
            print(f"  s={s} count={count} plan={list(plan)} {ms:.3f} ms{model}", flush=True)
        if best is None or ms < best[0]:
            best = (ms, list(plan))
    del A, B, O
    return best


def size_classes(lo: int = 32, hi: int = 1 << 21):
    c = lo
    while c <= hi:
        yield c
        if c + c // 2 <= hi:
            yield c + c // 2
        c *= 2


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(os.path.dirname(__file__), "plans_gb300.txt"))
    ap.add_argument("--max-limbs", type=int, default=1 << 21)
    ap.add_argument("--work", type=float, default=2 ** 26, help="limbs per timed batch")
    ap.add_argument("--top", type=int, default=10)
    ap.add_argument("-v", action="store_true")
    ap.add_argument("--no-ntt", action="store_true", help="schoolbook-base plans only")
    args = ap.parse_args()
    import torch
    from . import tc
    torch.cuda.set_device(0)
    ctx = tc.tc_create(0)
    rows = []
    t0 = time.time()
    for s in size_classes(32, args.max_limbs):
        count = max(1, int(args.work // s))
        best = tune_size(ctx, s, count, top=args.top, verbose=args.v, ntt=not args.no_ntt)
        if best is None:
            continue
        rows.append((s, best[1], best[0], count))
        print(f"{s:8d} limbs x {count:6d}: plan {best[1]}  {best[0]:.3f} ms", flush=True)
    with open(args.out, "w") as f:
        f.write("# plan table written by paper_1602_02740_gb300.autotune on "
                f"{torch.cuda.get_device_name(0)}\n")
        f.write("# <max_limbs> <levels> <B0> <B1> ... [ntt]  (first row with max_limbs >= size wins;\n"
                "# ntt: the transform base product below the levels)\n")
        for s, plan, ms, count in rows:
            Bs = [B for B in plan if B != "ntt"]
            tail = " ntt" if plan and plan[-1] == "ntt" else ""
            f.write(f"{s} {len(Bs)} {' '.join(map(str, Bs))}{tail}\n".replace("  ", " "))
    print(f"wrote {args.out} ({len(rows)} classes) in {time.time() - t0:.0f} s")
    ctx.close()


if __name__ == "__main__":
    sys.exit(main())
