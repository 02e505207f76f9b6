"""Serving loop: every result is the same alone and in a concurrent mix.

Requests of uneven sizes (including an unbalanced pair and empty operands)
are submitted together in a shuffled order while earlier ones run; each
output must equal, bit for bit, the product computed alone by tc_mul, and
the small ones the oracle as well.
"""
import time

import numpy as np
import pytest

from oracle import native
from oracle.limbs import to_int
from paper_1602_02740_gb300 import inputs

pytestmark = pytest.mark.gpu

SIZES = [(1, 1), (5, 5), (64, 64), (300, 300), (1000, 1000), (4096, 4096), (20000, 20000),
         (3000, 9000), (70000, 70000), (0, 7), (129, 129), (2055, 2055)]


def _wait_all(t, ctx, tickets, timeout=120.0):
    t0 = time.time()
    pending = set(tickets)
    while pending:
        pending = {k for k in pending if not t.tc_serve_poll(ctx, k)}
        assert time.time() - t0 < timeout, "serving loop did not finish"
        time.sleep(0.001)


def test_results_same_alone_and_in_the_mix(tc):
    import torch
    t = tc.tc
    ctx = t.tc_create(0, budget_bytes=8 << 30)
    try:
        reqs = []
        for i, (na, nb) in enumerate(SIZES * 3):
            a = inputs.uniform(na, 10 * i) if na else np.zeros(0, np.uint32)
            b = inputs.all_ones(nb) if i % 5 == 0 and nb else (inputs.uniform(nb, 10 * i + 1)
                                                                 if nb else np.zeros(0, np.uint32))
            da = t.to_device(a) if na else torch.empty(0, dtype=torch.int32, device="cuda")
            db = t.to_device(b) if nb else torch.empty(0, dtype=torch.int32, device="cuda")
            alone = t.to_numpy(t.tc_mul(ctx, da, db))
            reqs.append((a, b, da, db, alone))
        torch.cuda.synchronize()
        for rnd in range(2):
            order = inputs.rng(rnd).permutation(len(reqs))
            outs, tickets = {}, []
            for idx in order:
                a, b, da, db, alone = reqs[idx]
                out = torch.full((len(a) + len(b),), -1, dtype=torch.int32, device="cuda")
                while True:
                    k = t.tc_serve_submit(ctx, da, db, out)
                    if k >= 0:
                        break
                    time.sleep(0.001)       # not admitted now: budget or slots full
                outs[idx] = out
                tickets.append(k)
            _wait_all(t, ctx, tickets)
            for idx, out in outs.items():
                a, b, _, _, alone = reqs[idx]
                got = t.to_numpy(out)
                assert np.array_equal(got, alone), (rnd, idx, len(a), len(b))
                if len(a) * len(b) <= 5000 * 5000:
                    assert np.array_equal(got, native.schoolbook(a, b))
            st = t.tc_serve_stats(ctx)
            assert st["completed"] == len(reqs)
            assert 0 < st["p50_ms"] <= st["p99_ms"]
            assert st["bits_per_s"] > 0
            t.tc_serve_stop(ctx)            # next round starts a fresh loop
    finally:
        ctx.close()


def test_admission_by_budget(tc):
    import torch
    t = tc.tc
    ctx = t.tc_create(0, budget_bytes=64 << 20)
    try:
        big = torch.zeros(1 << 20, dtype=torch.int32, device="cuda")   # 2^25-bit operands
        out = torch.empty(2 << 20, dtype=torch.int32, device="cuda")
        with pytest.raises(t.TCError) as ei:                            # can never fit 64 MB
            t.tc_serve_submit(ctx, big, big, out)
        assert ei.value.status == t.TC_ENOMEM
        a = t.to_device(inputs.uniform(4000, 1))
        b = t.to_device(inputs.uniform(4000, 2))
        outs, tickets, busy = [], [], 0
        for _ in range(400):
            o = torch.empty(8000, dtype=torch.int32, device="cuda")
            k = t.tc_serve_submit(ctx, a, b, o)
            if k < 0:
                busy += 1
                continue
            outs.append(o)
            tickets.append(k)
        _wait_all(t, ctx, tickets)
        want = to_int(t.to_numpy(a)) * to_int(t.to_numpy(b))
        for o in outs:
            assert to_int(t.to_numpy(o)) == want
        assert busy > 0   # the 64 MB budget cannot hold 400 of these at once
    finally:
        ctx.close()


def test_ticket_released_after_final_poll(tc):
    t = tc.tc
    ctx = t.tc_create(0, budget_bytes=1 << 30)
    try:
        a = t.to_device(inputs.uniform(500, 3))
        b = t.to_device(inputs.uniform(500, 4))
        import torch
        out = torch.empty(1000, dtype=torch.int32, device="cuda")
        k = t.tc_serve_submit(ctx, a, b, out)
        assert k >= 0
        _wait_all(t, ctx, [k])
        with pytest.raises(t.TCError) as ei:   # the final poll released the ticket
            t.tc_serve_poll(ctx, k)
        assert ei.value.status == t.TC_EINVAL
        assert to_int(t.to_numpy(out)) == to_int(t.to_numpy(a)) * to_int(t.to_numpy(b))
    finally:
        ctx.close()
