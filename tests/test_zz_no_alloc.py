"""tc_toom_interpolate_noalloc against tc_toom_interpolate, through the C ABI.

The no-allocation entry point serves callers that must not allocate device
memory while they run; its scratch is a fixed array inside the library.  Its
results must equal the regular entry point's bit for bit (all arithmetic is
exact), on consecutive calls that reuse the same built-in scratch.  This file
is collected last so a run that stops at the first failure has run every
other test first; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from oracle import toom
from oracle.limbs import from_int, to_int
from paper_1602_02740_gb300 import inputs

pytestmark = pytest.mark.gpu


def _level_inputs(tc, B, L, count, seed):
    import torch
    _, e, _, ystride = tc.level_sizes(L, B)
    Y = np.zeros((count, 2 * B - 1, ystride), dtype=np.uint32)
    S = np.zeros((count, 2 * B - 1), dtype=np.uint8)
    for k in range(count):
        a = inputs.uniform(L, seed + 2 * k)
        b = inputs.uniform(L, seed + 2 * k + 1)
        bsz = toom.ceil_div(L, B)
        ue = toom.evaluate(toom.split(to_int(a), B, bsz))
        ve = toom.evaluate(toom.split(to_int(b), B, bsz))
        for p, (x, y) in enumerate(zip(ue, ve)):
            v = x * y
            Y[k, p, :2 * e] = from_int(abs(v), 2 * e)
            S[k, p] = 1 if v < 0 else 0
    return tc.to_device(Y), torch.from_numpy(S).cuda()


# (B, limbs, count): the first two need built-in scratch (values in global
# memory), the last runs entirely in shared memory (no scratch at all).
CASES = [(16, 32768, 2), (8, 20000, 3), (4, 300, 5)]


@pytest.mark.parametrize("B,L,count", CASES)
def test_noalloc_matches_regular_entry_point_twice(tc, B, L, count):
    import torch
    t = tc.tc
    wb = t.tc_toom_interpolate_work_bytes(count, L, B)
    assert wb <= t.TC_NOALLOC_SCRATCH_BYTES
    if L > 300:
        assert wb > 0, "this case is meant to run through the built-in scratch"
    else:
        assert wb == 0
    Y, S = _level_inputs(t, B, L, count, seed=100 * B + L)
    want = t.to_numpy(t.tc_toom_interpolate(Y, L, B, SGN_U=S))
    for call in range(2):  # two calls in a row share the built-in scratch
        out = torch.full((count, 2 * L), -1, dtype=torch.int32, device="cuda")
        t.tc_toom_interpolate_noalloc(Y, L, B, SGN_U=S, OUT=out)
        torch.cuda.synchronize()
        assert np.array_equal(t.to_numpy(out), want), (B, L, count, call)


def test_noalloc_rejects_requests_beyond_the_fixed_scratch(tc):
    import torch
    t = tc.tc
    B, L, count = 16, 32768, 20      # about 20 x 1.1 MB of scratch > 16 MiB
    assert t.tc_toom_interpolate_work_bytes(count, L, B) > t.TC_NOALLOC_SCRATCH_BYTES
    _, e, _, ystride = t.level_sizes(L, B)
    Y = torch.zeros((count, 2 * B - 1, ystride), dtype=torch.int32, device="cuda")
    with pytest.raises(t.TCError) as ei:
        t.tc_toom_interpolate_noalloc(Y, L, B)
    assert ei.value.status == t.TC_ENOMEM
