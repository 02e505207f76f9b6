"""Host logic of the plan choice, on CPU: the autotuner's level-size rule, its
candidate plans, its cost model, and the committed plan table that tc_create
loads (format, ordering, every plan valid for its size class)."""
import os

import pytest

from oracle import toom
from paper_1602_02740_gb300 import autotune as at
from paper_1602_02740_gb300 import tc

TABLE = os.path.join(os.path.dirname(at.__file__), "plans_gb300.txt")


def _rows():
    rows = []
    with open(TABLE) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            words = line.split()
            ntt = words[-1] == "ntt"
            nums = [int(x) for x in (words[:-1] if ntt else words)]
            rows.append((nums[0], nums[1], nums[2:] + (["ntt"] if ntt else [])))
    return rows


@pytest.mark.parametrize("L", [1, 7, 64, 116, 457, 2735, 32768, 1 << 19, (1 << 21) + 3])
@pytest.mark.parametrize("B", [2, 3, 4, 5, 6, 8, 12, 16, 32])
def test_level_rule_agrees_with_oracle_and_binding(L, B):
    """b = ceil(L/B), e = b + ceil((n(n-1)+1)/32): the autotuner, the binding's
    layout helper and the oracle use one rule (Section 3 block size, reading P4)."""
    (_, _, b_or, e_or), = toom.level_sizes(L, [B])
    assert at.level(L, B) == (b_or, e_or)
    b, e, estride, ystride = tc.level_sizes(L, B)
    assert (b, e) == (b_or, e_or)
    assert estride % 4 == 0 and estride >= e and estride - e < 4
    assert ystride % 4 == 0 and ystride >= 2 * e and ystride - 2 * e < 4


def test_bench_plan_leaf_sizes():
    # the 2^20-bit workload's plan and its level lengths (2432 x 23 x 11 x 7 leaves of 116)
    assert [e for (_, _, _, e) in toom.level_sizes(32768, [12, 6, 4])] == [2735, 457, 116]
    assert at.plan_leaf(32768, (12, 6, 4)) == 116


@pytest.mark.parametrize("s", [200, 600, 4096, 32768])
def test_candidates_are_valid_plans(s):
    cands = at.candidates(s, max_levels=4)
    assert cands, "no candidate plan"
    for plan in cands:
        L = s
        for B in plan:
            assert B in at.BS and B <= L
            L = at.level(L, B)[1]
        if plan:
            assert at.LEAF_MIN <= L <= at.LEAF_MAX and L < s
    assert len(set(cands)) == len(cands)


def test_cost_model_grows_with_work():
    plan = (12, 6, 4)
    t1 = at.model_seconds(32768, plan, 100)
    t2 = at.model_seconds(32768, plan, 200)
    assert 0 < t1 < t2
    # a deeper split of the same size does less base-case work
    assert at.plan_leaf(32768, (12, 6, 4, 2)) < at.plan_leaf(32768, (12, 6, 4))


def test_size_classes_cover_the_range():
    cl = list(at.size_classes(32, 1 << 21))
    assert cl[0] == 32 and cl[-1] <= 1 << 21
    assert all(a < b for a, b in zip(cl, cl[1:]))
    assert all(b <= 2 * a for a, b in zip(cl, cl[1:]))


def test_plan_table_well_formed():
    rows = _rows()
    assert rows, "empty plan table"
    sizes = [r[0] for r in rows]
    assert sizes == sorted(sizes) and len(set(sizes)) == len(sizes)
    assert sizes[-1] >= 1 << 20  # covers the 2^20-bit workload (32768 limbs)
    for s, levels, plan in rows:
        ntt = bool(plan) and plan[-1] == "ntt"
        Bs = plan[:-1] if ntt else plan
        assert levels == len(Bs) <= 5
        L = s
        for B in Bs:
            assert B in at.BS and B <= L
            L = at.level(L, B)[1]
        if ntt:
            assert s >= at.NTT_MIN and L <= 1 << 24, (s, plan, L)   # transform base product
        elif Bs:
            assert at.LEAF_MIN <= L <= at.LEAF_MAX, (s, plan, L)


def test_plan_table_row_for_the_bench_size():
    # first row with max_limbs >= size wins
    row = next(r for r in _rows() if r[0] >= 32768)
    assert row[2] == [12, 6, 4]


def test_ntt_candidates():
    assert at.ntt_candidates(at.NTT_MIN - 1) == []
    c = at.ntt_candidates(1 << 20)
    assert ("ntt",) in c and all(p[-1] == "ntt" for p in c)
    assert len(set(c)) == len(c)
    for p in c:
        assert all(B in at.BS for B in p[:-1])
