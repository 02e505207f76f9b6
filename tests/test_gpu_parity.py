"""GPU parity: every step and the whole product, limb-exact against the oracle.

All arithmetic is exact integer, so the bar is bit-exactness everywhere.
"""
import numpy as np
import pytest

from oracle import native, residues, toom
from oracle.limbs import from_int, to_int
from paper_1602_02740_gb300 import inputs

pytestmark = pytest.mark.gpu


def same_limbs(got, want_int_or_arr, L=None):
    """Bit-exact comparison with a readable failure (first differing limb)."""
    want = want_int_or_arr
    if not isinstance(want, np.ndarray):
        want = from_int(int(want), len(got))
    got = np.asarray(got, dtype=np.uint32)
    if len(got) != len(want) or not np.array_equal(got, want):
        bad = np.nonzero(got != want)[0] if len(got) == len(want) else [-1]
        i = int(bad[0])
        raise AssertionError(f"{len(bad)} limbs differ; first at {i}: got "
                             f"{hex(int(got[i])) if i >= 0 else len(got)} want "
                             f"{hex(int(want[i])) if i >= 0 else len(want)}")
    return True


def dev(x):
    from paper_1602_02740_gb300 import tc
    return tc.to_device(x)


def host(t):
    from paper_1602_02740_gb300 import tc
    return tc.to_numpy(t)


@pytest.fixture(scope="module")
def ctx(tc):
    c = tc.tc.tc_create(0)
    yield c
    c.close()


# ---------------------------------------------------------------- schoolbook

@pytest.mark.parametrize("L", [1, 2, 3, 4, 5, 7, 8, 15, 16, 17, 31, 33, 48, 49, 64, 65, 66, 100,
                               127, 128, 129, 255, 256, 257, 300, 511, 512, 513, 777, 1024])
def test_schoolbook_vs_oracle(tc, L):
    count = 3
    A = np.stack([inputs.uniform(L, 10 * L + k) for k in range(count - 1)] + [inputs.all_ones(L)])
    B = np.stack([inputs.uniform(L, 7 * L + k) for k in range(count - 1)] + [inputs.all_ones(L)])
    out = host(tc.tc.tc_schoolbook(dev(A), dev(B)))
    for k in range(count):
        assert np.array_equal(out[k], native.schoolbook(A[k], B[k])), (L, k)


def test_schoolbook_many_and_strided(tc):
    import torch
    L, count = 70, 1000
    A = np.stack([inputs.uniform(L, k) for k in range(count)])
    B = np.stack([inputs.sparse(L, 5000 + k) for k in range(count)])
    dA = dev(np.pad(A, ((0, 0), (0, 5))))[:, :L]   # row stride 75
    dB = dev(B)
    out = host(tc.tc.tc_schoolbook(dA, dB))
    for k in range(0, count, 37):
        assert np.array_equal(out[k], native.schoolbook(A[k], B[k]))


# ---------------------------------------------------------------- evaluation

EVAL_CASES = [(2, 1), (2, 5), (3, 7), (3, 1024), (4, 9), (5, 33), (8, 100), (8, 129),
              (16, 16), (16, 300), (16, 2055), (32, 32), (32, 999)]


@pytest.mark.parametrize("B,L", EVAL_CASES)
@pytest.mark.parametrize("kind", ["uniform", "all_ones", "sparse"])
def test_evaluate_vs_oracle(tc, B, L, kind):
    count = 2
    U = np.stack([inputs.operand(kind, L, 100 * B + L + k) for k in range(count)])
    OUT, SGN = tc.tc.tc_toom_evaluate(dev(U), B)
    out, sgn = host(OUT), SGN.cpu().numpy()
    b = toom.ceil_div(L, B)
    e = b + toom.growth_limbs(B)
    for k in range(count):
        vals = toom.evaluate(toom.split(to_int(U[k]), B, b))
        for p, v in enumerate(vals):
            assert to_int(out[k, p]) == abs(v), (B, L, kind, k, p)
            assert int(sgn[k, p]) == (1 if v < 0 else 0), (B, L, kind, k, p)
            assert not out[k, p, e:].any()


def test_evaluate_equal_halves_sign(tc):
    # u_0 = u_1 makes U(-1) = 0 exactly; E = O on every limb (full-length sign scan)
    L = 4000
    h = inputs.uniform(L // 2, 3)
    U = np.concatenate([h, h])[None, :]
    OUT, SGN = tc.tc.tc_toom_evaluate(dev(U), 2)
    out = host(OUT)
    assert not out[0, 2].any() and int(SGN.cpu()[0, 2]) == 0
    assert to_int(out[0, 1]) == 2 * to_int(h)


# ---------------------------------------------------------------- interpolation

def _oracle_level(u, v, L, B):
    b = toom.ceil_div(L, B)
    ue = toom.evaluate(toom.split(u, B, b))
    ve = toom.evaluate(toom.split(v, B, b))
    y = [p * q for p, q in zip(ue, ve)]
    return y


INTERP_CASES = [(2, 4), (2, 1000), (3, 9), (3, 1024), (4, 100), (5, 77), (8, 515), (16, 64),
                (16, 2055), (16, 32768), (32, 96), (32, 4000), (8, 40000),
                (2, 2000), (4, 8000), (2, 9000), (32, 65536),
                # few long values: the segment-parallel (look-back) path
                (3, 30000), (16, 150000), (32, 300000)]


@pytest.mark.parametrize("B,L", INTERP_CASES)
@pytest.mark.parametrize("kind", ["uniform", "all_ones"])
def test_interpolate_vs_oracle(tc, B, L, kind):
    import torch
    count = 2
    _, e, _, ystride = tc.tc.level_sizes(L, B)
    Y = np.zeros((count, 2 * B - 1, ystride), dtype=np.uint32)
    S = np.zeros((count, 2 * B - 1), dtype=np.uint8)
    want = []
    for k in range(count):
        a = inputs.operand(kind, L, 31 * L + k)
        b = inputs.operand(kind, L, 17 * L + k + 1)
        y = _oracle_level(to_int(a), to_int(b), L, B)
        for p, val in enumerate(y):
            Y[k, p, :2 * e] = from_int(abs(val), 2 * e)
            S[k, p] = 1 if val < 0 else 0
        want.append(to_int(a) * to_int(b))
    out = host(tc.tc.tc_toom_interpolate(dev(Y), L, B, SGN_U=torch.from_numpy(S).cuda()))
    for k in range(count):
        assert same_limbs(out[k], want[k]), (B, L, kind, k)


MATRIX_CASES = [(2, 4), (2, 100), (2, 250), (3, 9), (3, 150), (3, 300), (3, 378),
                (4, 16), (4, 200), (4, 457), (4, 504),
                # degree 4 and 5, values of up to 8 chunks (the bench's level-1 shape: B = 6, 2735)
                (5, 30), (5, 600), (5, 2400), (6, 12), (6, 700), (6, 2735), (4, 1900), (2, 1000)]


@pytest.mark.parametrize("B,L", MATRIX_CASES)
@pytest.mark.parametrize("kind", ["uniform", "all_ones", "sparse"])
def test_interpolate_matrix_vs_oracle(tc, B, L, kind):
    """Inverse-Vandermonde interpolation (one pass per coefficient) against the
    oracle's product and the Newton route's output, limb for limb."""
    import torch
    count = 3
    _, e, _, ystride = tc.tc.level_sizes(L, B)
    Y = np.zeros((count, 2 * B - 1, ystride), dtype=np.uint32)
    S = np.zeros((count, 2 * B - 1), dtype=np.uint8)
    want = []
    for k in range(count):
        a = inputs.operand(kind, L, 41 * L + k)
        b = inputs.operand(kind, L, 43 * L + k + 1)
        y = _oracle_level(to_int(a), to_int(b), L, B)
        for p, val in enumerate(y):
            Y[k, p, :2 * e] = from_int(abs(val), 2 * e)
            S[k, p] = 1 if val < 0 else 0
        want.append(to_int(a) * to_int(b))
    dY, dS = dev(Y), torch.from_numpy(S).cuda()
    out = host(tc.tc.tc_toom_interpolate_matrix(dY, L, B, SGN_U=dS))
    ref = host(tc.tc.tc_toom_interpolate(dY, L, B, SGN_U=dS))
    for k in range(count):
        assert same_limbs(out[k], want[k]), (B, L, kind, k)
    assert np.array_equal(out, ref)


def test_interpolate_matrix_many_products(tc):
    """The bench's level-2 shape (B = 4, 457-limb operands) over many products and
    several blocks: equal to the Newton route everywhere, to the oracle on samples."""
    import torch
    B, L, count = 4, 457, 3000
    _, e, _, ystride = tc.tc.level_sizes(L, B)
    rng = np.random.default_rng(5)
    Y = np.zeros((count, 2 * B - 1, ystride), dtype=np.uint32)
    S = np.zeros((count, 2 * B - 1), dtype=np.uint8)
    want = {}
    for k in range(count):
        a = inputs.uniform(L, 7000 + k)
        b = inputs.uniform(L, 9000 + k)
        y = _oracle_level(to_int(a), to_int(b), L, B)
        for p, val in enumerate(y):
            Y[k, p, :2 * e] = from_int(abs(val), 2 * e)
            S[k, p] = 1 if val < 0 else 0
        if k % 500 == 0 or k == count - 1:
            want[k] = to_int(a) * to_int(b)
    dY, dS = dev(Y), torch.from_numpy(S).cuda()
    out = host(tc.tc.tc_toom_interpolate_matrix(dY, L, B, SGN_U=dS))
    ref = host(tc.tc.tc_toom_interpolate(dY, L, B, SGN_U=dS))
    assert np.array_equal(out, ref)
    for k, w in want.items():
        assert same_limbs(out[k], w), k


def test_interpolate_matrix_rejects_unsupported(tc):
    import torch
    t = tc.tc
    Y = torch.zeros((1, 13, 64), dtype=torch.int32, device="cuda")
    with pytest.raises(t.TCError):
        t.tc_toom_interpolate_matrix(Y, 100, 7)          # B = 7: not supported
    _, e, _, ystride = t.level_sizes(5000, 4)
    Y = torch.zeros((1, 7, ystride), dtype=torch.int32, device="cuda")
    with pytest.raises(t.TCError):
        t.tc_toom_interpolate_matrix(Y, 5000, 4)         # values longer than 1024 limbs


# ---------------------------------------------------------------- whole product

MUL_CASES = [
    (1, None), (2, None), (5, None), (64, None), (128, None), (129, None), (1024, [3]),
    (1024, None), (1000, [2, 2, 2]), (3000, [16]), (3000, [4, 4]), (5000, [32]),
    (2055, [8, 4]), (32768, None), (32768, [16, 8, 4]), (32768, [2, 2, 2, 2, 2, 2, 2, 2]),
]


@pytest.mark.parametrize("L,plan", MUL_CASES)
@pytest.mark.parametrize("kind", ["uniform", "all_ones", "sparse"])
def test_mul_vs_oracle(ctx, tc, L, plan, kind):
    a = inputs.operand(kind, L, L + 1)
    b = inputs.operand(kind, L, L + 2)
    out = host(tc.tc.tc_mul(ctx, dev(a), dev(b), plan=plan))
    want = native.schoolbook(a, b) if L <= 4096 else from_int(to_int(a) * to_int(b), 2 * L)
    assert same_limbs(out, want)


@pytest.mark.parametrize("L,plan", [(1, None), (100, None), (1024, [3]), (4096, [16]), (10000, None)])
def test_square_vs_oracle(ctx, tc, L, plan):
    a = inputs.uniform(L, 99 + L)
    da = dev(a)
    out = host(tc.tc.tc_mul(ctx, da, da, plan=plan))
    assert same_limbs(out, to_int(a) ** 2)
    out2 = host(tc.tc.tc_sqr(ctx, da, plan=plan))
    assert np.array_equal(out, out2)


def _degenerate(kind, L, seed):
    a = np.zeros(L, np.uint32)
    if kind == "zero":
        pass
    elif kind == "one":
        a[0] = 1
    elif kind == "top_bit":        # 2^(32 L - 1): only the last block is nonzero
        a[-1] = 0x80000000
    elif kind == "top_limb":
        a[-1] = 0xFFFFFFFF
    elif kind == "zero_blocks":    # every other 1/12 of the limbs zero (whole blocks vanish)
        a[:] = inputs.uniform(L, seed)
        step = max(1, L // 12)
        for i in range(0, L, 2 * step):
            a[i:i + step] = 0
    else:
        a[:] = inputs.uniform(L, seed)
    return a


@pytest.mark.parametrize("L,plan", [(3000, [4, 3]), (32768, [12, 6, 4]), (32768, [16, 8, 4])])
@pytest.mark.parametrize("ka,kb", [("zero", "uniform"), ("uniform", "zero"), ("zero", "zero"),
                                   ("one", "uniform"), ("top_bit", "top_bit"),
                                   ("top_limb", "uniform"), ("zero_blocks", "zero_blocks"),
                                   ("zero_blocks", "top_bit")])
def test_degenerate_operands(ctx, tc, L, plan, ka, kb):
    """Zero operands, one, a single top bit, whole zero blocks: the evaluation's
    sign cases (U(-x) = 0, E = O) and empty pointwise products, limb-exact."""
    a = _degenerate(ka, L, 7)
    b = _degenerate(kb, L, 8)
    out = host(tc.tc.tc_mul(ctx, dev(a), dev(b), plan=plan))
    assert same_limbs(out, to_int(a) * to_int(b))
    if ka == kb:
        out2 = host(tc.tc.tc_sqr(ctx, dev(a), plan=plan))
        assert same_limbs(out2, to_int(a) ** 2)


def test_degenerate_rows_in_a_batch(ctx, tc):
    """A batch whose rows mix degenerate and uniform operands (one launch per level)."""
    L = 4096
    kinds = ["zero", "one", "top_bit", "top_limb", "zero_blocks", "uniform"] * 2
    A = np.stack([_degenerate(k, L, 20 + i) for i, k in enumerate(kinds)])
    B = np.stack([_degenerate(kinds[(i + 3) % len(kinds)], L, 40 + i) for i in range(len(kinds))])
    OUT = host(tc.tc.tc_mul_uniform(ctx, dev(A), dev(B), plan=[8, 4]))
    for k in range(len(kinds)):
        assert same_limbs(OUT[k], to_int(A[k]) * to_int(B[k])), k


@pytest.mark.parametrize("na,nb", [(1, 7), (7, 1), (100, 150), (150, 100), (300, 1200),
                                   (5000, 1234), (64, 65536), (1, 1), (3, 0), (0, 5)])
def test_unbalanced_and_empty(ctx, tc, na, nb):
    import torch
    a = inputs.uniform(na, 1) if na else np.zeros(0, np.uint32)
    b = inputs.uniform(nb, 2) if nb else np.zeros(0, np.uint32)
    da = dev(a) if na else torch.empty(0, dtype=torch.int32, device="cuda")
    db = dev(b) if nb else torch.empty(0, dtype=torch.int32, device="cuda")
    out = host(tc.tc.tc_mul(ctx, da, db))
    assert len(out) == na + nb
    assert same_limbs(out, to_int(a) * to_int(b))


def test_uniform_batch_matches_single(ctx, tc):
    L, count = 4096, 12
    A = np.stack([inputs.uniform(L, k) for k in range(count)])
    B = np.stack([inputs.uniform(L, 100 + k) for k in range(count)])
    OUT = host(tc.tc.tc_mul_uniform(ctx, dev(A), dev(B)))
    for k in range(count):
        single = host(tc.tc.tc_mul(ctx, dev(A[k]), dev(B[k])))
        assert np.array_equal(OUT[k], single)
        assert same_limbs(OUT[k], to_int(A[k]) * to_int(B[k]))


def test_host_entry_point(ctx, tc):
    import torch
    L, count = 3000, 5
    A = np.stack([inputs.uniform(L, k) for k in range(count)])
    B = np.stack([inputs.uniform(L, 50 + k) for k in range(count)])
    OUT = np.zeros((count, 2 * L), dtype=np.uint32)
    tc.tc.tc_mul_uniform_host(ctx, A, B, OUT)
    for k in range(count):
        assert same_limbs(OUT[k], to_int(A[k]) * to_int(B[k]))


@pytest.mark.parametrize("square", [False, True])
def test_pipe_batches_in_flight(ctx, tc, square):
    """Five batches submitted back to back (two in flight, copies overlapping
    the kernels): every product exact, each batch in its own output buffer."""
    import torch
    L, count, nb = 2731, 6, 5
    As = [np.stack([inputs.uniform(L, 1000 * i + k) for k in range(count)]) for i in range(nb)]
    Bs = As if square else [np.stack([inputs.uniform(L, 1000 * i + 500 + k) for k in range(count)])
                            for i in range(nb)]
    hA = [torch.from_numpy(a.view(np.int32)).pin_memory() for a in As]
    hB = hA if square else [torch.from_numpy(b.view(np.int32)).pin_memory() for b in Bs]
    hO = [torch.zeros((count, 2 * L), dtype=torch.int32).pin_memory() for _ in range(nb)]
    pipe = tc.tc.tc_pipe_create(ctx, count, L, square=square)
    for i in range(nb):
        pipe.submit(hA[i], hB[i], hO[i])
    pipe.wait()
    # and again into the same buffers: results unchanged
    for i in range(nb):
        pipe.submit(hA[i], hB[i], hO[i])
    pipe.wait()
    pipe.close()
    for i in range(nb):
        out = hO[i].numpy().view(np.uint32)
        for k in range(count):
            assert same_limbs(out[k], to_int(As[i][k]) * to_int(Bs[i][k]))


def test_pipe_rejects_bad_input(ctx, tc):
    t = tc.tc
    with pytest.raises(t.TCError):
        t.tc_pipe_create(ctx, 0, 100)
    with pytest.raises(t.TCError):
        t.tc_pipe_create(ctx, 4, 0)
    pipe = t.tc_pipe_create(ctx, 2, 64)
    with pytest.raises(ValueError):
        pipe.submit(np.zeros((3, 64), np.uint32), np.zeros((2, 64), np.uint32),
                    np.zeros((2, 128), np.uint32))
    pipe.close()


def test_batch_mixed_sizes(ctx, tc):
    la, lb = inputs.batch_lengths(120, seed=4, lo=64, hi=6000)
    a_off = np.concatenate([[0], np.cumsum(la)[:-1]])
    b_off = np.concatenate([[0], np.cumsum(lb)[:-1]])
    o_off = np.concatenate([[0], np.cumsum(la + lb)[:-1]])
    A = inputs.uniform(int(la.sum()), 1)
    B = inputs.uniform(int(lb.sum()), 2)
    import torch
    OUT = torch.zeros(int((la + lb).sum()), dtype=torch.int32, device="cuda")
    tc.tc.tc_mul_batch(ctx, dev(A), a_off, la, dev(B), b_off, lb, OUT, o_off)
    want = native.schoolbook_batch(A, a_off, la, B, b_off, lb, o_off, int((la + lb).sum()))
    assert np.array_equal(host(OUT), want)


def _packed(la, lb, seed):
    a_off = np.concatenate([[0], np.cumsum(la)[:-1]])
    b_off = np.concatenate([[0], np.cumsum(lb)[:-1]])
    o_off = np.concatenate([[0], np.cumsum(la + lb)[:-1]])
    A = inputs.uniform(max(1, int(la.sum())), seed)
    B = inputs.uniform(max(1, int(lb.sum())), seed + 1)
    return A, B, a_off, b_off, o_off


def test_prepared_batch_run_and_graph_replay(ctx, tc):
    """A prepared batch gives the products directly and when its run is captured
    into a CUDA graph and replayed; zero-length products get zero outputs."""
    import torch
    t = tc.tc
    la, lb = inputs.batch_lengths(150, seed=9, lo=64, hi=9000)
    la[3], lb[7] = 0, 0
    A, B, a_off, b_off, o_off = _packed(la, lb, 40)
    n_out = int((la + lb).sum())
    want = native.schoolbook_batch(A, a_off, la, B, b_off, lb, o_off, n_out)
    dA, dB = dev(A), dev(B)
    bt = t.tc_batch_prepare(ctx, a_off, la, b_off, lb, o_off)
    assert t.tc_batch_scratch_bytes(bt) > 0
    OUT = torch.full((n_out,), -1, dtype=torch.int32, device="cuda")
    t.tc_batch_run(ctx, bt, dA, dB, OUT)
    t.tc_batch_check(ctx, bt)
    assert np.array_equal(host(OUT), want)
    # capture one run and replay it into a fresh output
    OUT2 = torch.full((n_out,), -1, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        t.tc_batch_run(ctx, bt, dA, dB, OUT2, stream=s)
    OUT2.fill_(-1)
    graph.replay()
    torch.cuda.synchronize()
    assert np.array_equal(host(OUT2), want)
    # replay on new operand values in the same buffers
    A2 = inputs.uniform(A.size, 77)
    dA.copy_(dev(A2))
    graph.replay()
    torch.cuda.synchronize()
    want2 = native.schoolbook_batch(A2, a_off, la, B, b_off, lb, o_off, n_out)
    assert np.array_equal(host(OUT2), want2)
    bt.close()


def test_prepared_batch_rejects_bad_input(ctx, tc):
    t = tc.tc
    with pytest.raises(t.TCError):
        t.tc_batch_prepare(ctx, [0], [-1], [0], [4], [0])


# ---------------------------------------------------------------- base case, large batches
# 4096 or more products select the lane-per-product kernels: a lane pair per
# product (rows in shared memory) up to 792 limbs, one lane per product from
# global memory beyond.

@pytest.mark.parametrize("L", [1, 3, 7, 8, 9, 31, 63, 64, 65, 88, 100, 128, 137, 184, 200, 224,
                               300, 511, 800])
@pytest.mark.parametrize("layout", ["aligned", "strided"])
def test_schoolbook_lane_kernel(tc, L, layout):
    count = 4100
    g = inputs.rng(L)
    A = g.integers(0, 1 << 32, size=(count, L), dtype=np.uint64).astype(np.uint32)
    B = g.integers(0, 1 << 32, size=(count, L), dtype=np.uint64).astype(np.uint32)
    A[5] = 0xFFFFFFFF
    B[5] = 0xFFFFFFFF
    B[7] = 0
    if layout == "strided":
        dA = dev(np.pad(A, ((0, 0), (0, 3))))[:, :L]
        dB = dev(np.pad(B, ((0, 0), (1, 0))))[:, 1:]
    else:
        dA, dB = dev(A), dev(B)
    out = host(tc.tc.tc_schoolbook(dA, dB))
    for k in list(range(0, count, 97)) + [5, 7, count - 1]:
        assert np.array_equal(out[k], native.schoolbook(A[k], B[k])), (L, k)


@pytest.mark.parametrize("L", [1, 2, 8, 9, 15, 16, 17, 64, 88, 130, 137, 184, 255, 800])
def test_square_lane_kernel(tc, L):
    count = 4200
    g = inputs.rng(1000 + L)
    A = g.integers(0, 1 << 32, size=(count, L), dtype=np.uint64).astype(np.uint32)
    A[3] = 0xFFFFFFFF
    dA = dev(A)
    out = host(tc.tc.tc_schoolbook(dA, dA))
    for k in list(range(0, count, 101)) + [3, count - 1]:
        assert np.array_equal(out[k], native.schoolbook(A[k], A[k])), (L, k)


def _karatsuba_rows(count, L, seed):
    """Operand rows that reach every sign case of the in-kernel Karatsuba level
    (a = a0 + a1 X with a0 the first 8 ceil(T/2) limbs): a0 above, below and
    equal to a1, a zero half, all-ones rows, then uniform rows."""
    k = 8 * (((L + 7) // 8 + 1) // 2)
    g = inputs.rng(seed)
    A = g.integers(0, 1 << 32, size=(count, L), dtype=np.uint64).astype(np.uint32)
    B = g.integers(0, 1 << 32, size=(count, L), dtype=np.uint64).astype(np.uint32)
    n1 = L - k
    A[0] = 0xFFFFFFFF; B[0] = 0xFFFFFFFF              # a0 > a1 (a1 shorter)
    A[1, :k] = 0; B[1, :k] = 0                        # a0 < a1, b0 < b1: P1 subtracted
    A[2, :k] = 0                                      # a0 < a1, b0 > b1 likely: added
    A[3, :n1] = A[3, k:]; A[3, n1:k] = 0              # a0 == a1: zero difference
    B[3, :n1] = B[3, k:]; B[3, n1:k] = 0
    A[4, k:] = 0                                      # a1 = 0
    B[5] = 0                                          # a zero operand
    A[6, :k] = 0xFFFFFFFF; A[6, k:] = 0xFFFFFFFF; B[6, :k] = 1; B[6, k:] = 0xFFFFFFFF
    A[7, n1:k] = 0; A[7, :n1] = A[7, k:]; A[7, 0] ^= 1    # a0, a1 differ in one low bit
    return A, B


@pytest.mark.parametrize("L", [48, 49, 56, 57, 64, 100, 116, 120, 121, 184, 224, 255, 792])
@pytest.mark.parametrize("square", [False, True])
def test_karatsuba_base_case(tc, L, square):
    """The lane-pair base case with its Karatsuba level forced on from 49 limbs
    against the oracle's schoolbook on every row (sampled rows at 792 limbs),
    and the plain variant of the same kernel on the same rows."""
    t = tc.tc
    count = 4100
    A, B = _karatsuba_rows(count, L, 7000 + L)
    if square:
        B = A
    dA = dev(A)
    dB = dA if square else dev(B)
    try:
        t.tc_set_leaf_karatsuba(49)
        got = host(t.tc_schoolbook(dA, dB))
        t.tc_set_leaf_karatsuba(0)
        plain = host(t.tc_schoolbook(dA, dB))
    finally:
        t.tc_set_leaf_karatsuba(t.TC_LEAF_KARATSUBA_DEFAULT)
    rows = range(count) if L <= 256 else list(range(0, count, 41)) + list(range(8)) + [count - 1]
    for r in rows:
        want = native.schoolbook(A[r], B[r])
        assert np.array_equal(got[r], want), (L, r, square)
        assert np.array_equal(plain[r], want), (L, r, square, "plain")


# ---------------------------------------------------------------- many small interpolations
# 2048 or more products with small values select the warp-per-product kernel.

# values over 24 KB per product ((4, 2000) onward) take the streaming kernel; (20, 4000) has
# right shifts of 32 bits or more, (32, 3000) two divisors per Newton step.  Short values of
# small degree ((2, 9), (3, 100), (4, 259), (3, 2) and the last six) take the register-resident
# kernel with 8, 12 or 16 limbs per lane.
@pytest.mark.parametrize("B,L", [(2, 9), (3, 100), (4, 259), (8, 130), (3, 2), (4, 2000), (8, 2055),
                                 (12, 6000), (20, 4000), (32, 3000),
                                 (2, 5000), (3, 4000), (6, 3000), (7, 4000), (10, 3000),
                                 (3, 450), (3, 650), (2, 400), (4, 600), (6, 500), (5, 400),
                                 # two warps per product (degree 8..15, values a multiple of 256 limbs)
                                 (9, 3000), (16, 8000)])
def test_interpolate_many_products(tc, B, L):
    import torch
    count = 2100
    _, e, _, ystride = tc.tc.level_sizes(L, B)
    g = inputs.rng(7 * B + L)
    A = g.integers(0, 1 << 32, size=(count, L), dtype=np.uint64).astype(np.uint32)
    Bm = g.integers(0, 1 << 32, size=(count, L), dtype=np.uint64).astype(np.uint32)
    A[1] = 0xFFFFFFFF
    Bm[1] = 0xFFFFFFFF
    Y = np.zeros((count, 2 * B - 1, ystride), dtype=np.uint32)
    S = np.zeros((count, 2 * B - 1), dtype=np.uint8)
    check = list(range(0, count, 53)) + [1, count - 1]
    for k in range(count):
        y = _oracle_level(to_int(A[k]), to_int(Bm[k]), L, B)
        for p, val in enumerate(y):
            Y[k, p, :2 * e] = from_int(abs(val), 2 * e)
            S[k, p] = 1 if val < 0 else 0
    out = host(tc.tc.tc_toom_interpolate(dev(Y), L, B, SGN_U=torch.from_numpy(S).cuda()))
    for k in check:
        assert same_limbs(out[k], to_int(A[k]) * to_int(Bm[k])), (B, L, k)


# Large batches of low degree, every product checked: 16 400 products (a grid of
# 513 blocks of 32 warps for the warp-per-product kernels); (4, 457) is the 2^20-bit
# benchmark's level-2 shape; ragged top blocks except for (2, 16), (3, 24), (4, 32).
@pytest.mark.parametrize("B,L", [(2, 16), (2, 101), (3, 24), (3, 100), (4, 32), (4, 259),
                                 (4, 457), (4, 1000)])
def test_interpolate_large_batch_low_degree(tc, B, L):
    import torch
    count = 16400
    _, e, _, ystride = tc.tc.level_sizes(L, B)
    g = inputs.rng(11 * B + L)
    A = g.integers(0, 1 << 32, size=(count, L), dtype=np.uint64).astype(np.uint32)
    Bm = g.integers(0, 1 << 32, size=(count, L), dtype=np.uint64).astype(np.uint32)
    b = toom.ceil_div(L, B)
    A[1] = 0xFFFFFFFF; Bm[1] = 0xFFFFFFFF              # largest values
    A[2] = 0                                            # a zero operand
    A[3, :] = 0; A[3, b:min(2 * b, L)] = 0xFFFFFFFF     # odd block only: negative values at -x
    Bm[3, b:] = 0                                       # ... times block 0 alone
    A[4] = inputs.sparse(L, 5)
    Y = np.zeros((count, 2 * B - 1, ystride), dtype=np.uint32)
    S = np.zeros((count, 2 * B - 1), dtype=np.uint8)
    for k in range(count):
        y = _oracle_level(to_int(A[k]), to_int(Bm[k]), L, B)
        for p, val in enumerate(y):
            Y[k, p, :2 * e] = from_int(abs(val), 2 * e)
            S[k, p] = 1 if val < 0 else 0
    assert S[3].any()
    out = host(tc.tc.tc_toom_interpolate(dev(Y), L, B, SGN_U=torch.from_numpy(S).cuda()))
    for k in range(count):
        assert same_limbs(out[k], to_int(A[k]) * to_int(Bm[k])), (B, L, k)


def test_uniform_batch_bench_launch(tc):
    """The timed workload in its own launch configuration: 2432 products of
    2^20-bit operands in one tc_mul_uniform call, with the plan the benchmark
    takes from the plan table ([12, 6, 4]: levels of 2432, 55 936 and 615 296
    products, 4 307 072 base-case products of 116 limbs; the streaming
    interpolation at n = 11 and n = 5, the register-resident one at n = 3 and
    the pair base case).  Every product is checked modulo three 61-bit primes,
    sampled ones limb by limb; rows 5 and 6 are all-ones and sparse."""
    import os
    t = tc.tc
    L, count = 32768, 2432
    table = os.path.join(os.path.dirname(tc.__file__), "plans_gb300.txt")
    ctx = t.tc_create(0, table=table)
    try:
        plan = t.tc_plan_for(ctx, L)
        assert plan == [12, 6, 4], plan     # the plan the benchmark line reports
        A = np.stack([inputs.uniform(L, 1000 + 2 * k) for k in range(count)])
        B = np.stack([inputs.uniform(L, 1001 + 2 * k) for k in range(count)])
        A[5] = 0xFFFFFFFF
        B[5] = 0xFFFFFFFF
        A[6] = inputs.sparse(L, 77)
        OUT = host(t.tc_mul_uniform(ctx, dev(A), dev(B), plan=plan))
    finally:
        ctx.close()
    for k in (0, 5, 6, 1217, count - 1):
        assert same_limbs(OUT[k], to_int(A[k]) * to_int(B[k])), k
    for k in range(count):
        assert residues.product_residues_match(A[k], B[k], OUT[k]), k


@pytest.mark.parametrize("plan", [[16, 8, 3], [16, 4, 4], [8, 8, 4], [32, 8]])
def test_uniform_batch_full_size_2e20(ctx, tc, plan):
    """The benchmark's workload shape (2^20-bit operands) at a reduced batch,
    with every level's kernels in their large-batch variants."""
    L, count = 32768, 72   # 72 x 31 = 2232 level-1 products: the many-product kernels
    A = np.stack([inputs.uniform(L, 2 * k) for k in range(count)])
    B = np.stack([inputs.uniform(L, 2 * k + 1) for k in range(count)])
    A[3] = 0xFFFFFFFF
    B[3] = 0xFFFFFFFF
    OUT = host(tc.tc.tc_mul_uniform(ctx, dev(A), dev(B), plan=plan))
    for k in (0, 3, 17, count - 1):
        assert same_limbs(OUT[k], to_int(A[k]) * to_int(B[k])), (plan, k)
    for k in range(count):
        assert residues.product_residues_match(A[k], B[k], OUT[k]), (plan, k)


# ---------------------------------------------------------------- plain schoolbook, any length

@pytest.mark.parametrize("L", [1025, 2000, 5000, 12345])
def test_plain_schoolbook_plan_any_length(ctx, tc, L):
    a = inputs.uniform(L, 3 * L)
    b = inputs.all_ones(L) if L == 2000 else inputs.uniform(L, 3 * L + 1)
    out = host(tc.tc.tc_mul(ctx, dev(a), dev(b), plan=[]))
    assert same_limbs(out, native.schoolbook(a, b) if L <= 5000 else to_int(a) * to_int(b))


def test_plain_schoolbook_plan_batch(ctx, tc):
    L, count = 3000, 7
    A = np.stack([inputs.uniform(L, 40 + k) for k in range(count)])
    B = np.stack([inputs.uniform(L, 80 + k) for k in range(count)])
    OUT = host(tc.tc.tc_mul_uniform(ctx, dev(A), dev(B), plan=[]))
    for k in range(count):
        assert same_limbs(OUT[k], native.schoolbook(A[k], B[k]))


# ---------------------------------------------------------------- one stage exposed
# The streaming interpolation kernels leave Theorem 3.3's output in their work
# buffer: rows (0, m) hold the even polynomial's monomial coefficients ce_m
# (m = 0..n) and rows (1, m) the odd one's co_m (m = 1..n), each Y limbs, before
# re-interleaving and recomposition.  (12, 6000) and (9, 3000) run the two-warp
# kernel, (6, 3000) and (10, 3000) the one-warp kernel.

@pytest.mark.parametrize("B,L", [(12, 6000), (9, 3000), (6, 3000), (10, 3000)])
def test_interpolation_stage_outputs_vs_oracle(tc, B, L):
    import torch
    t = tc.tc
    count = 2100
    n = B - 1
    _, e, _, ystride = t.level_sizes(L, B)
    K = 8 if 2 * e + 2 > 1536 else 4
    Yl = -(-(2 * e + 2) // (32 * K)) * (32 * K)
    g = inputs.rng(31 * B + L)
    A = g.integers(0, 1 << 32, size=(count, L), dtype=np.uint64).astype(np.uint32)
    Bm = g.integers(0, 1 << 32, size=(count, L), dtype=np.uint64).astype(np.uint32)
    A[4] = 0xFFFFFFFF
    Bm[4] = 0xFFFFFFFF
    Y = np.zeros((count, 2 * B - 1, ystride), dtype=np.uint32)
    S = np.zeros((count, 2 * B - 1), dtype=np.uint8)
    ys = {}
    for k in range(count):
        y = _oracle_level(to_int(A[k]), to_int(Bm[k]), L, B)
        ys[k] = y
        for p, val in enumerate(y):
            Y[k, p, :2 * e] = from_int(abs(val), 2 * e)
            S[k, p] = 1 if val < 0 else 0
    wb = t.tc_toom_interpolate_work_bytes(count, L, B)
    assert wb == count * 2 * (n + 1) * Yl * 4, "not a streaming shape"
    work = torch.zeros(wb, dtype=torch.uint8, device="cuda")
    out = host(t.tc_toom_interpolate(dev(Y), L, B, SGN_U=torch.from_numpy(S).cuda(), work=work))
    W = work.cpu().numpy().view(np.uint32).reshape(count, 2, n + 1, Yl)
    X = toom.nodes(B)
    for k in (0, 4, 1001, count - 1):
        ye, yo = toom.even_odd_combine(ys[k])
        ce = toom.newton_to_monomial(X, toom.divided_differences(X, ye))
        co = toom.newton_to_monomial(X, toom.divided_differences(X, yo))
        for m in range(n + 1):
            assert to_int(W[k, 0, m]) == ce[m], (B, L, k, "ce", m)
        for m in range(1, n + 1):
            assert to_int(W[k, 1, m]) == co[m], (B, L, k, "co", m)
        assert same_limbs(out[k], to_int(A[k]) * to_int(Bm[k])), k
