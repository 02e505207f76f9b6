"""Figures the paper prints, read from tests/golden/ (each file cites its source)."""
import os

from oracle import toom

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLD, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_complexity_exponents_section2():
    rows = _rows("complexity_exponents.txt")
    assert len(rows) == 3
    for B, alpha in rows:
        assert round(toom.complexity_exponent(int(B)), 3) == float(alpha)


def test_points_section6():
    kv = {r[0]: r[1:] for r in _rows("section6_nodes.txt")}
    B = int(kv["B"][0])
    assert int(kv["n"][0]) == B - 1
    pts = toom.eval_points(B)
    assert [int(x) for x in kv["points"]] == sorted(p for p in pts if p >= 0)
    assert max(toom.nodes(B)) == int(kv["max_x_squared"][0])
