"""Single-kernel workloads for profiler captures and kernel timing.

Each case prepares valid inputs with the library's own calls, synchronises,
then, inside the NVTX range "measure", runs the call under study once and
`--reps` more times and prints the mean time of the latter (CUDA events on
the current stream).  Default sizes keep device memory
to a few GB, so a full `ncu` capture of one launch ends quickly.

  python -m paper_1602_02740_gb300.profile_cases interp --count 2048 --limbs 32768 --B 12
  python -m paper_1602_02740_gb300.profile_cases leaf --count 157320 --limbs 184
  python -m paper_1602_02740_gb300.profile_cases eval --count 2432 --limbs 32768 --B 12

interp: one Toom level's interpolation (tc_toom_interpolate, or with
        --method matrix tc_toom_interpolate_matrix) of `count` products of
        `limbs`-limb operands split into B blocks; its inputs are the true
        pointwise products (evaluation, then products of the evaluations
        through tc_mul_uniform).
leaf:   the batched schoolbook (tc_schoolbook) of `count` products.
eval:   one level's evaluation (tc_toom_evaluate) of `count` operands.
"""
from __future__ import annotations

import argparse
import json


def _rand(torch, shape, seed):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    return torch.randint(-2 ** 31, 2 ** 31 - 1, shape, dtype=torch.int32, device="cuda", generator=g)


def _time(torch, fn, reps):
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


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["interp", "leaf", "eval"])
    ap.add_argument("--count", type=int, default=None)
    ap.add_argument("--limbs", type=int, default=None)
    ap.add_argument("--B", type=int, default=12)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--method", choices=["newton", "matrix"], default="newton",
                    help="interp: even-odd Newton route or inverse-Vandermonde matrix")
    args = ap.parse_args(argv)
    import torch
    from . import tc
    torch.cuda.set_device(0)
    res = {"case": args.case, "B": args.B, "reps": args.reps}
    if args.case == "leaf":
        count, L = args.count or 157320, args.limbs or 184
        A, B = _rand(torch, (count, L), 1), _rand(torch, (count, L), 2)
        OUT = torch.empty((count, 2 * L), dtype=torch.int32, device="cuda")
        ms = _time(torch, lambda: tc.tc_schoolbook(A, B, OUT), args.reps)
    elif args.case == "eval":
        count, L = args.count or 2432, args.limbs or 32768
        U = _rand(torch, (count, L), 1)
        _, e, estride, _ = tc.level_sizes(L, args.B)
        E = torch.empty((count, 2 * args.B - 1, estride), dtype=torch.int32, device="cuda")
        S = torch.empty((count, 2 * args.B - 1), dtype=torch.uint8, device="cuda")
        ms = _time(torch, lambda: tc.tc_toom_evaluate(U, args.B, E, S), args.reps)
    else:
        count, L = args.count or 2048, args.limbs or 32768
        npts = 2 * args.B - 1
        _, e, estride, ystride = tc.level_sizes(L, args.B)
        ctx = tc.tc_create(0)
        U, V = _rand(torch, (count, L), 1), _rand(torch, (count, L), 2)
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
            ms = _time(torch, lambda: tc.tc_toom_interpolate_matrix(Y, L, args.B, SU, SV, OUT),
                       args.reps)
        else:
            ms = _time(torch, lambda: tc.tc_toom_interpolate(Y, L, args.B, SU, SV, OUT, work),
                       args.reps)
        res["method"] = args.method
    res.update(count=count, limbs=L, ms_per_call=ms)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
