"""Oracle: plain recursive B-way Toom-Cook on Python integers.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import this module; the library's product
path never does.

It follows the paper step by step, in the paper's notation, with Python
integers (so there are no limbs, carries or overflow to get wrong):

1. Split (Section 1, eq. 1.1-1.3): u = U(2^(32 b)) with B blocks u_0..u_n of
   b limbs, n = B - 1.  Block size b = ceil(L / B) limbs, top block
   zero-padded (the paper only says "about N/B").
2. Evaluate (Section 4, eq. 4.1 and the points of Section 6): with the even
   part E(x) = sum_{i even} u_i x^i and the odd part O(x) = sum_{i odd} u_i x^i,
   U(x) = E + O and U(-x) = E - O at x = 2^j, j = 0..n-1, plus U(0) = u_0.
   That is 2n + 1 = 2B - 1 points (Section 2).  Point order everywhere:
   index 0 -> x = 0, index 2j+1 -> x = +2^j, index 2j+2 -> x = -2^j.
3. Pointwise products y = U(x) V(x) (Section 1), each computed by this
   same procedure on the magnitudes |U(x)|, |V(x)| (child operands of
   e = b + ceil((n(n-1)+1)/32) limbs) until the plan runs out, then by the
   integer product itself (a library primitive).  The sign of y is the
   product of the two signs.
4. Even-odd combine (Section 4, eq. 4.5-4.6): W_e(x^2) = (W(x) + W(-x)) / 2 and
   x^2 W_o(x^2) = x (W(x) - W(-x)) / 2, with W_e(0) = W(0) and, for the odd
   polynomial, the extra point (0, 0).  Both are degree-n polynomials in
   X = x^2 on the nodes X = 0, 1, 4, ..., 4^(n-1).
5. Newton divided differences (Section 3, Theorem 3.2): the table
   alpha_k^(m) = (alpha_(k-1)^(m+1) - alpha_(k-1)^(m)) / (X_(m+k) - X_m), kept
   in one array indexed by m + k as the paper describes, every division exact.
6. Newton basis to monomial basis (Section 3, Theorem 3.3):
   beta_k^(m) = beta_k^(m+1) - X_m beta_(k+1)^(m+1) for k = m..n-1, m = n-1..0.
7. Re-interleave (eq. 4.3): w_(2i) = even coefficient i, w_(2i+1) = odd
   coefficient i + 1 (the odd polynomial's coefficients sit one place higher),
   and recompose w = W(2^(32 b)) = sum_k w_k 2^(32 b k) (Section 1).

Every division asserts a zero remainder, and every interpolation intermediate
is asserted non-negative and below 2^(32 (2e + 1)): with non-negative blocks
the combination W(x) >= |W(-x)| makes both even-odd values non-negative, and
the divided differences and partial conversions on increasing nodes stay
non-negative.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

LIMB = 32


def ceil_div(a: int, b: int) -> int:
    return -(-a // b)


def growth_limbs(B: int) -> int:
    """Extra limbs of an evaluation value over its block size.

    |U(+-2^j)| <= (2^(32b) - 1) * sum_{i=0..n} 2^(j i) < 2^(32b + j n + 1) and
    j <= n - 1, so the value has at most 32b + n(n-1) + 1 bits.
    """
    n = B - 1
    return ceil_div(n * (n - 1) + 1, LIMB)


def eval_points(B: int) -> List[int]:
    """The 2B-1 evaluation points in the library's order: 0, +1, -1, +2, -2, ..."""
    pts = [0]
    for j in range(B - 1):
        pts += [1 << j, -(1 << j)]
    return pts


def nodes(B: int) -> List[int]:
    """Interpolation nodes X = x^2 of the even-odd method: 0, 1, 4, ..., 4^(n-1)."""
    return [0] + [1 << (2 * j) for j in range(B - 1)]


def split(u: int, B: int, b: int) -> List[int]:
    """Blocks u_0..u_(B-1) of b limbs (Section 1)."""
    mask = (1 << (LIMB * b)) - 1
    return [(u >> (LIMB * b * i)) & mask for i in range(B)]


def even_odd_parts(blocks: Sequence[int], x: int) -> Tuple[int, int]:
    """E(x) = sum over even i of u_i x^i and O(x) = sum over odd i of u_i x^i (eq. 4.1)."""
    E = sum(c * x ** i for i, c in enumerate(blocks) if i % 2 == 0)
    O = sum(c * x ** i for i, c in enumerate(blocks) if i % 2 == 1)
    return E, O


def evaluate(blocks: Sequence[int]) -> List[int]:
    """Signed values U(x) at eval_points(B), built from E and O as U(+-x) = E +- O."""
    B = len(blocks)
    vals = [blocks[0]]
    for j in range(B - 1):
        E, O = even_odd_parts(blocks, 1 << j)
        vals += [E + O, E - O]
    return vals


def exact_div(num: int, den: int) -> int:
    q, r = divmod(num, den)
    assert r == 0, f"inexact division: {num} / {den}"
    return q


def even_odd_combine(y: Sequence[int]) -> Tuple[List[int], List[int]]:
    """Values of W_e and of X W_o at the nodes X (eq. 4.5-4.6 with the point (0,0))."""
    n = (len(y) - 1) // 2
    ye = [y[0]]
    yo = [0]
    for k in range(1, n + 1):
        x = 1 << (k - 1)
        wp, wm = y[2 * k - 1], y[2 * k]
        ye.append(exact_div(wp + wm, 2))
        yo.append(x * exact_div(wp - wm, 2))
    return ye, yo


def divided_differences(X: Sequence[int], y: Sequence[int]) -> List[int]:
    """Newton coefficients alpha_0..alpha_n of the polynomial through (X_m, y_m).

    Theorem 3.2: alpha_k^(m) = (alpha_(k-1)^(m+1) - alpha_(k-1)^(m)) / (X_(m+k) - X_m)
    with alpha_0^(m) = y_m and alpha_k = alpha_k^(0).  Column k of the table is
    stored at positions k..n (entry alpha_k^(m) at position m + k), so after
    column k the prefix 0..k holds alpha_0..alpha_k.
    """
    n = len(X) - 1
    col = list(y)                      # column 0: alpha_0^(m) at position m
    for k in range(1, n + 1):
        prev = col
        col = list(prev)
        for pos in range(k, n + 1):    # pos = m + k
            m = pos - k
            col[pos] = exact_div(prev[pos] - prev[pos - 1], X[pos] - X[m])
    return col


def newton_to_monomial(X: Sequence[int], alpha: Sequence[int]) -> List[int]:
    """Monomial coefficients from Newton coefficients (Theorem 3.3).

    beta^(n) = alpha; for m = n-1 down to 0, beta_k^(m) = beta_k^(m+1) -
    X_m beta_(k+1)^(m+1) for k = m..n-1 and beta_k^(m) = beta_k^(m+1) otherwise;
    the result is beta^(0).
    """
    n = len(X) - 1
    beta = list(alpha)
    for m in range(n - 1, -1, -1):
        old = beta
        beta = list(old)
        for k in range(m, n):
            beta[k] = old[k] - X[m] * old[k + 1]
    return beta


def interleave(ce: Sequence[int], co: Sequence[int]) -> List[int]:
    """w_(2i) = ce_i, w_(2i+1) = co_(i+1) (eq. 4.3 with the odd shift of Section 4)."""
    n = len(ce) - 1
    assert co[0] == 0
    w = []
    for i in range(n + 1):
        w.append(ce[i])
        if i < n:
            w.append(co[i + 1])
    return w


def recompose(w: Sequence[int], b: int) -> int:
    """W(2^(32 b)) = sum_k w_k 2^(32 b k) (Section 1)."""
    return sum(c << (LIMB * b * k) for k, c in enumerate(w))


@dataclass
class LevelTrace:
    """Every intermediate of one Toom level of one product."""
    B: int
    L: int                     # operand length in limbs at this level
    b: int                     # block size in limbs
    e: int                     # evaluation value length in limbs
    u_blocks: List[int]
    v_blocks: List[int]
    u_eval: List[int]          # signed U(x) in eval_points order
    v_eval: List[int]
    y: List[int]               # signed W(x) = U(x) V(x)
    ye: List[int]
    yo: List[int]
    alpha_e: List[int]
    alpha_o: List[int]
    ce: List[int]
    co: List[int]
    w: List[int]
    result: int


@dataclass
class Trace:
    """Intermediates keyed by (level, product index in breadth-first order)."""
    levels: Dict[Tuple[int, int], LevelTrace] = field(default_factory=dict)
    leaves: Dict[int, Tuple[int, int, int]] = field(default_factory=dict)  # index -> (u, v, uv)


def _interp_bound_check(vals: Sequence[int], e: int) -> None:
    lim = 1 << (LIMB * (2 * e + 1))
    for v in vals:
        assert 0 <= v < lim, "interpolation intermediate out of the stated range"


def level_sizes(L: int, plan: Sequence[int]) -> List[Tuple[int, int, int, int]]:
    """(B, L, b, e) for each level of a plan: the child operand length is e."""
    out = []
    for B in plan:
        b = ceil_div(L, B)
        e = b + growth_limbs(B)
        out.append((B, L, b, e))
        L = e
    return out


def toom_multiply(u: int, v: int, L: int, plan: Sequence[int],
                  trace: Optional[Trace] = None, level: int = 0, index: int = 0) -> int:
    """u * v for 0 <= u, v < 2^(32 L), by Toom-Cook with B = plan[level] per level.

    Below the last planned level the product is the plain integer product.
    ``trace`` (optional) collects every intermediate.
    """
    assert 0 <= u < (1 << (LIMB * L)) and 0 <= v < (1 << (LIMB * L))
    if level == len(plan):
        r = u * v
        if trace is not None:
            trace.leaves[index] = (u, v, r)
        return r
    B = plan[level]
    assert B >= 2
    n = B - 1
    b = ceil_div(L, B)
    e = b + growth_limbs(B)
    ub, vb = split(u, B, b), split(v, B, b)
    ue, ve = evaluate(ub), evaluate(vb)
    for val in ue + ve:
        assert abs(val) < (1 << (LIMB * e)), "evaluation exceeds e limbs"
    y = []
    for p, (a, c) in enumerate(zip(ue, ve)):
        mag = toom_multiply(abs(a), abs(c), e, plan, trace, level + 1, index * (2 * B - 1) + p)
        y.append(-mag if (a < 0) != (c < 0) and mag else mag)
    X = nodes(B)
    ye, yo = even_odd_combine(y)
    alpha_e = divided_differences(X, ye)
    alpha_o = divided_differences(X, yo)
    ce = newton_to_monomial(X, alpha_e)
    co = newton_to_monomial(X, alpha_o)
    _interp_bound_check(ye + yo + alpha_e + alpha_o + ce + co, e)
    w = interleave(ce, co)
    r = recompose(w, b)
    if trace is not None:
        trace.levels[(level, index)] = LevelTrace(B, L, b, e, ub, vb, ue, ve, y, ye, yo,
                                                  alpha_e, alpha_o, ce, co, w, r)
    assert r < (1 << (2 * LIMB * L))
    return r


def interpolation_intermediates_all(X: Sequence[int], y: Sequence[int]) -> List[List[int]]:
    """Every array state of Theorems 3.2 and 3.3 (columns, then conversions)."""
    n = len(X) - 1
    states = []
    col = list(y)
    states.append(list(col))
    for k in range(1, n + 1):
        prev = col
        col = list(prev)
        for pos in range(k, n + 1):
            col[pos] = exact_div(prev[pos] - prev[pos - 1], X[pos] - X[pos - k])
        states.append(list(col))
    beta = col
    for m in range(n - 1, -1, -1):
        old = beta
        beta = list(old)
        for k in range(m, n):
            beta[k] = old[k] - X[m] * old[k + 1]
        states.append(list(beta))
    return states


def complexity_exponent(B: int) -> float:
    """alpha = log(2B - 1) / log(B): the cost exponent of B-way Toom-Cook (Section 2)."""
    import math
    return math.log(2 * B - 1) / math.log(B)
