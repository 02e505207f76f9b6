"""Asynchronous calls and bounded device waits.

- A product whose levels run segment-parallel (few huge products, bounded
  look-back waits between segments) is made to give up its waits: the test
  hook shortens every wait to a few thousand polls and withholds the first
  segment's carry of every add/subtract chain.  The call must come back
  (no hang), tc_check must report TC_ETIMEOUT, and the same context must then
  compute the product exactly.  Nothing faults: the kernels only read a
  status word that nobody sets.
- Multiply calls no longer wait for the device, so once a shape has run, the
  call can be captured into a CUDA graph and replayed.
"""
import numpy as np
import pytest

from oracle import native
from oracle.limbs import from_int, to_int
from paper_1602_02740_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture
def ctx(tc):
    c = tc.tc.tc_create(0)
    yield c
    c.close()


def test_bounded_wait_gives_up_and_the_context_survives(ctx, tc):
    t = tc.tc
    L = 1 << 16                   # one product: top-level evaluation and interpolation segment-parallel
    a, b = inputs.uniform(L, 61), inputs.uniform(L, 62)
    da, db = t.to_device(a), t.to_device(b)
    want = from_int(to_int(a) * to_int(b), 2 * L)
    plan = [3, 8, 6, 4]
    out = t.tc_mul(ctx, da, db, plan=plan)
    t.tc_check(ctx)
    assert np.array_equal(t.to_numpy(out), want)
    t.tc_test_bounded_waits(2000, True)
    try:
        t.tc_mul(ctx, da, db, out, plan=plan)
        with pytest.raises(t.TCError) as ei:
            t.tc_check(ctx)
        assert ei.value.status == t.TC_ETIMEOUT
    finally:
        t.tc_test_bounded_waits(0, False)
    t.tc_check(ctx)               # the sticky word was cleared by the report
    out.fill_(-1)
    t.tc_mul(ctx, da, db, out, plan=plan)
    t.tc_check(ctx)
    assert np.array_equal(t.to_numpy(out), want)


def test_prepared_batch_reports_a_wait_that_gave_up(ctx, tc):
    import torch
    t = tc.tc
    L = 40000
    la = np.array([L, 300], dtype=np.int64)
    lb = np.array([L, 300], dtype=np.int64)
    a_off = np.array([0, L], dtype=np.int64)
    o_off = np.array([0, 2 * L], dtype=np.int64)
    A = np.concatenate([inputs.uniform(L, 1), inputs.uniform(300, 2)])
    B = np.concatenate([inputs.uniform(L, 3), inputs.uniform(300, 4)])
    dA, dB = t.to_device(A), t.to_device(B)
    O = torch.empty(2 * L + 600, dtype=torch.int32, device="cuda")
    bt = t.tc_batch_prepare(ctx, a_off, la, a_off, lb, o_off, plan=[3, 8, 6, 4])
    try:
        t.tc_test_bounded_waits(2000, True)
        try:
            t.tc_batch_run(ctx, bt, dA, dB, O)
            with pytest.raises(t.TCError) as ei:
                t.tc_batch_check(ctx, bt)
            assert ei.value.status == t.TC_ETIMEOUT
        finally:
            t.tc_test_bounded_waits(0, False)
        t.tc_batch_run(ctx, bt, dA, dB, O)
        t.tc_batch_check(ctx, bt)
        got = t.to_numpy(O)
        assert to_int(got[:2 * L]) == to_int(A[:L]) * to_int(B[:L])
        assert np.array_equal(got[2 * L:], native.schoolbook(A[L:], B[L:]))
    finally:
        bt.close()


def test_large_product_captured_in_a_cuda_graph(ctx, tc):
    import torch
    t = tc.tc
    L = 1 << 17
    a, b = inputs.uniform(L, 71), inputs.uniform(L, 72)
    da, db = t.to_device(a), t.to_device(b)
    out = torch.empty(2 * L, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    t.tc_mul(ctx, da, db, out, stream=s)         # sizes the context's scratch outside the capture
    s.synchronize()
    out.fill_(-1)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        t.tc_mul(ctx, da, db, out, stream=s)
    g.replay()
    torch.cuda.synchronize()
    t.tc_check(ctx)
    want = native.toom_mul(a, b, t.tc_plan_for(ctx, L), threads=8)
    assert np.array_equal(t.to_numpy(out), want)


def test_mixed_batch_calls_back_to_back(ctx, tc):
    """tc_mul_batch stages its index tables in two pinned buffers used in turn:
    several calls in a row with different tables must all be right."""
    import torch
    t = tc.tc
    outs, wants = [], []
    for rep in range(4):
        la, lb = inputs.batch_lengths(40, seed=90 + rep, hi=3000)
        a_off = np.concatenate([[0], np.cumsum(la)[:-1]]).astype(np.int64)
        b_off = np.concatenate([[0], np.cumsum(lb)[:-1]]).astype(np.int64)
        o_off = np.concatenate([[0], np.cumsum(la + lb)[:-1]]).astype(np.int64)
        A = inputs.uniform(int(la.sum()), 100 + rep)
        B = inputs.uniform(int(lb.sum()), 200 + rep)
        O = torch.empty(int((la + lb).sum()), dtype=torch.int32, device="cuda")
        t.tc_mul_batch(ctx, t.to_device(A), a_off, la, t.to_device(B), b_off, lb, O, o_off)
        outs.append(O)
        wants.append((A, B, la, lb, a_off, b_off, o_off))
    t.tc_check(ctx)
    for O, (A, B, la, lb, a_off, b_off, o_off) in zip(outs, wants):
        got = t.to_numpy(O)
        for k in range(len(la)):
            a = A[a_off[k]:a_off[k] + la[k]]
            b = B[b_off[k]:b_off[k] + lb[k]]
            assert np.array_equal(got[o_off[k]:o_off[k] + la[k] + lb[k]], native.schoolbook(a, b))


def _packed(count, seed, hi):
    la, lb = inputs.batch_lengths(count, seed=seed, hi=hi)
    a_off = np.concatenate([[0], np.cumsum(la)[:-1]]).astype(np.int64)
    b_off = np.concatenate([[0], np.cumsum(lb)[:-1]]).astype(np.int64)
    o_off = np.concatenate([[0], np.cumsum(la + lb)[:-1]]).astype(np.int64)
    A = inputs.uniform(int(la.sum()), seed + 1)
    B = inputs.uniform(int(lb.sum()), seed + 2)
    return la, lb, a_off, b_off, o_off, A, B


def test_batch_with_device_tables_equals_host_tables(ctx, tc):
    """tc_mul_batch_dev (device offset/length tables, one padded size class) gives
    the same products as tc_mul_batch (host tables, size classes), and the
    oracle's on every product."""
    import torch
    t = tc.tc
    la, lb, a_off, b_off, o_off, A, B = _packed(60, 300, 2500)
    la[3], lb[3] = 0, 17                         # an empty operand: 17 zero limbs
    o_off = np.concatenate([[0], np.cumsum(la + lb)[:-1]]).astype(np.int64)
    dA, dB = t.to_device(A), t.to_device(B)
    total = int((la + lb).sum())
    O1 = torch.full((total,), -1, dtype=torch.int32, device="cuda")
    O2 = torch.full((total,), -1, dtype=torch.int32, device="cuda")
    t.tc_mul_batch(ctx, dA, a_off, la, dB, b_off, lb, O1, o_off)
    dev = [torch.from_numpy(x).cuda() for x in (a_off, la, b_off, lb, o_off)]
    t.tc_mul_batch_dev(ctx, dA, dev[0], dev[1], dB, dev[2], dev[3], O2, dev[4],
                       max_limbs=int(max(la.max(), lb.max())))
    t.tc_check(ctx)
    g1, g2 = t.to_numpy(O1), t.to_numpy(O2)
    assert np.array_equal(g1, g2)
    for k in range(len(la)):
        a = A[a_off[k]:a_off[k] + la[k]]
        b = B[b_off[k]:b_off[k] + lb[k]]
        assert np.array_equal(g2[o_off[k]:o_off[k] + la[k] + lb[k]], native.schoolbook(a, b)), k


def test_batch_with_device_tables_rejects_bad_entries_on_the_device(ctx, tc):
    import torch
    t = tc.tc
    la, lb, a_off, b_off, o_off, A, B = _packed(8, 400, 900)
    bad_len = la.copy()
    bad_len[2] = int(max(la.max(), lb.max())) + 5   # above max_limbs
    dev = [torch.from_numpy(x).cuda() for x in (a_off, bad_len, b_off, lb, o_off)]
    O = torch.full((int((la + lb).sum()) + 16,), -1, dtype=torch.int32, device="cuda")
    t.tc_mul_batch_dev(ctx, t.to_device(A), dev[0], dev[1], t.to_device(B), dev[2], dev[3], O, dev[4],
                       max_limbs=int(max(la.max(), lb.max())))
    with pytest.raises(t.TCError) as ei:
        t.tc_check(ctx)
    assert ei.value.status == t.TC_EINVAL
    got = t.to_numpy(O)
    assert (got[o_off[2]:o_off[2] + la[2] + lb[2]] == 0xFFFFFFFF).all()   # skipped, not written
    for k in (0, 1, 3):
        a = A[a_off[k]:a_off[k] + la[k]]
        b = B[b_off[k]:b_off[k] + lb[k]]
        assert np.array_equal(got[o_off[k]:o_off[k] + la[k] + lb[k]], native.schoolbook(a, b))
    t.tc_check(ctx)                               # the report cleared the word


def test_batch_with_device_tables_in_a_cuda_graph(ctx, tc):
    import torch
    t = tc.tc
    la, lb, a_off, b_off, o_off, A, B = _packed(40, 500, 4000)
    dA, dB = t.to_device(A), t.to_device(B)
    dev = [torch.from_numpy(x).cuda() for x in (a_off, la, b_off, lb, o_off)]
    O = torch.empty(int((la + lb).sum()), dtype=torch.int32, device="cuda")
    mx = int(max(la.max(), lb.max()))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    t.tc_mul_batch_dev(ctx, dA, dev[0], dev[1], dB, dev[2], dev[3], O, dev[4], max_limbs=mx, stream=s)
    s.synchronize()
    O.fill_(-1)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        t.tc_mul_batch_dev(ctx, dA, dev[0], dev[1], dB, dev[2], dev[3], O, dev[4], max_limbs=mx,
                           stream=s)
    g.replay()
    torch.cuda.synchronize()
    t.tc_check(ctx)
    got = t.to_numpy(O)
    for k in range(len(la)):
        a = A[a_off[k]:a_off[k] + la[k]]
        b = B[b_off[k]:b_off[k] + lb[k]]
        assert np.array_equal(got[o_off[k]:o_off[k] + la[k] + lb[k]], native.schoolbook(a, b)), k
