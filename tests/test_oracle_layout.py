"""Pins of the oracle's layout: the paper's worked slot examples (tests/golden), the
operation counts of Tab. 2 and Tab. 3, and exactness of the cleartext model against X y."""
import json
import os

import numpy as np
import pytest
import sympy

from oracle import layout

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")))


def _sym_matrix(m, n):
    """X[i, j] = symbol '<letter i><j>' as a sympy symbol."""
    return np.array([[sympy.Symbol(f"{chr(65 + i)}{j}") for j in range(n)] for i in range(m)], dtype=object)


def _diag_symbols(plan, X):
    """Same index formula as layout.diagonal_slots, evaluated on symbols (object dtype)."""
    # diagonal_slots works on float arrays; evaluate it on integer codes and map back
    m, n = X.shape
    codes = np.arange(1, m * n + 1, dtype=np.float64).reshape(m, n)
    E = layout.diagonal_slots(codes, plan)
    flat = X.reshape(-1)
    return np.vectorize(lambda c: flat[int(c) - 1] if c else 0, otypes=[object])(E)


def test_worked_example_diagonal_m4_n2():
    ex = GOLD["diagonal_m4_n2"]
    plan = layout.make_plan(ex["m"], ex["n"], ex["slots"])
    X = _sym_matrix(4, 2)
    E = _diag_symbols(plan, X)
    assert [str(v) for v in E[0, 0, 0]] == ex["e0"]
    codes = layout.vector_slots(np.array([1.0, 2.0]), plan)[0]
    assert [f"M{int(c) - 1}" for c in codes] == ex["y_replicated"]


def test_worked_example_input_packing():
    ex = GOLD["input_packing_m4_n4_slots8"]
    plan = layout.make_plan(ex["m"], ex["n"], ex["slots"])
    assert plan.m_prime == 2 and plan.regime == "pack"
    E = _diag_symbols(plan, _sym_matrix(4, 4))
    assert [str(v) for v in E[0, 0, 1]] == ex["e1"]
    codes = layout.vector_slots(np.array([1.0, 2.0, 3.0, 4.0]), plan)[0]
    assert [f"M{int(c) - 1}" for c in codes] == ex["y_replicated"]


def test_worked_example_lazy_ras():
    ex = GOLD["lazy_ras_m4_n4_slots8"]
    plan = layout.make_plan(4, 4, 8)
    X = _sym_matrix(4, 4)
    M = [sympy.Symbol(f"M{j}") for j in range(4)]
    E = _diag_symbols(plan, X)
    yrep = [M[s % 4] for s in range(8)]
    slots = [sum(E[0, 0, i, s] * yrep[(s + i) % 8] for i in range(plan.m_prime)) for s in range(8)]

    def parse(terms):
        return sum(sympy.Symbol(t[:2]) * sympy.Symbol(t[2:]) for t in terms)

    for s, terms in enumerate(ex["slots_first4"]):
        assert sympy.expand(slots[s] - parse(terms)) == 0
    # lazy RaS on symbols: out[b*m' + t] = sum_s slot[b*n + t + s*m']
    out = [sum(slots[b * 4 + t + s * 2] for s in range(2)) for b in range(2) for t in range(2)]
    for row, terms in enumerate(ex["result"]):
        assert sympy.expand(out[row] - parse(terms)) == 0
    # and layout.lazy_ras applies exactly that map
    probe = np.zeros((1, 8))
    probe[0] = np.arange(8) * 10.0 ** np.arange(8)
    got = layout.lazy_ras(probe, plan)
    want = [probe[0, 0] + probe[0, 2], probe[0, 1] + probe[0, 3], probe[0, 4] + probe[0, 6], probe[0, 5] + probe[0, 7]]
    assert np.allclose(got, want)


def test_rotation_direction_examples():
    ex = GOLD["rotl_naive"]
    assert list(layout.rotl(np.array(ex["input"], dtype=object), ex["step"]))[0] == ex["output_slot0"]
    ex = GOLD["rotr_gala"]
    # RotR is the inverse of RotL
    assert list(layout.rotl(np.array(ex["input"], dtype=object), -ex["right_step"])) == ex["output"]


# (m, n, N') and the paper's counts: Tab. 2 PackVFL row (m, n <= N'), Tab. 3 columns
@pytest.mark.parametrize("m,n,slots", [(4, 4, 8), (16, 64, 2048), (256, 1024, 4096), (1024, 256, 4096), (64, 64, 4096),
                                       (8192, 512, 4096), (16384, 64, 4096), (512, 8192, 4096), (64, 16384, 4096),
                                       (8192, 8192, 4096), (16384, 8192, 4096)])
def test_op_counts_match_tables(m, n, slots):
    plan = layout.make_plan(m, n, slots)
    if m <= slots and n <= slots:
        mp = -(-m * n // slots)
        assert (plan.n_add, plan.n_mult, plan.n_rot, plan.n_hstrot) == (mp - 1, mp, 0, mp - 1)
        assert (plan.col_blocks, plan.row_blocks) == (1, 1)
    elif m > slots >= n:
        assert plan.n_add == (m * n - m) // slots
        assert plan.n_mult == m * n // slots
        assert plan.n_hstrot == n - 1
        assert (plan.col_blocks, plan.row_blocks) == (1, m // slots)
    elif m <= slots < n:
        assert plan.n_add == (n * m - slots) // slots
        assert plan.n_mult == m * n // slots
        assert plan.n_hstrot == (m * n - n) // slots
        assert (plan.col_blocks, plan.row_blocks) == (n // slots, 1)
    else:
        assert plan.n_mult == m * n // slots
        assert plan.n_hstrot == (n * slots - n) // slots
        assert (plan.col_blocks, plan.row_blocks) == (n // slots, m // slots)
        # Tab. 3 prints mn/N' - 1 additions; summing each of the m/N' outputs separately takes
        # mn/N' - m/N' (equal when m = N')
        assert plan.n_add == m * n // slots - m // slots
    assert plan.n_rot == 0


@pytest.mark.parametrize("m,n,slots", [(4, 4, 8), (4, 2, 4), (16, 64, 2048), (64, 16, 2048), (256, 1024, 4096), (1024, 256, 4096),
                                       (3, 5, 8), (100, 37, 64), (1, 1, 8), (130, 20, 64), (20, 130, 64), (130, 130, 64),
                                       (64, 64, 64), (8, 1, 16), (1, 8, 16)])
def test_cleartext_model_is_exact(m, n, slots):
    rng = np.random.default_rng(m * 1000 + n)
    X = rng.integers(-9, 10, size=(m, n)).astype(np.float64)
    y = rng.integers(-9, 10, size=n).astype(np.float64)
    plan = layout.make_plan(m, n, slots)
    _, out = layout.cleartext_model(X, y, plan)
    assert np.array_equal(out, X @ y)


def test_plan_rejects_bad_input():
    with pytest.raises(ValueError):
        layout.make_plan(0, 4, 8)
    with pytest.raises(ValueError):
        layout.make_plan(4, 4, 6)


@pytest.mark.parametrize("m,n,slots", [(8, 4, 8), (4, 8, 8), (16, 16, 16), (64, 8, 128), (8, 64, 64), (1, 4, 4)])
def test_cipher_diagonal_model_is_exact(m, n, slots):
    """Alg. 3 with the encrypted matrix in Eq. 2's diagonal order: sum_i e_i (x) RotL(w_k, i)
    gives (A W)[:, k] in slots j < m (m >= n) or after summing the n/m slot groups (m < n)."""
    rng = np.random.default_rng(m + 7 * n)
    A = rng.integers(-9, 10, size=(m, n)).astype(float)
    W = rng.integers(-9, 10, size=(n, 3)).astype(float)
    assert np.array_equal(layout.cipher_diag_model(A, W, slots), A @ W)
    # the diagonal e_0 of the Sec. 4.1 example layout (m = 4, n = 2): [A0, B1, C0, D1]
    codes = np.arange(1, 9, dtype=float).reshape(4, 2)
    assert list(layout.cipher_diagonals(codes, 4)[0]) == [1.0, 4.0, 5.0, 8.0]


@pytest.mark.parametrize("m,n", [(4, 4), (8, 4), (16, 4), (4, 8), (4, 16), (32, 8), (8, 32), (64, 64)])
def test_transposed_diagonal_conversion(m, n):
    """The diagonals of A^T are rotations of A's diagonals (Eq. 5 as read: see transpose_rotations);
    the printed RotR(e_{(min-i) mod min}, max - min + i) fails on these same shapes."""
    slots = 2 * max(m, n)
    A = np.arange(m * n, dtype=float).reshape(m, n) + 1
    E = layout.cipher_diagonals(A, slots)
    Et = layout.cipher_diagonals(A.T.copy(), slots)
    lo, hi = min(m, n), max(m, n)
    for i, (k, r) in enumerate(layout.transpose_rotations(m, n)):
        assert np.array_equal(layout.rotl(E[k], r), Et[i])
    assert not all(np.array_equal(np.roll(E[(lo - i) % lo], hi - lo + i), Et[i]) for i in range(lo))


@pytest.mark.parametrize("m,n,slots", [(4, 4, 8), (16, 64, 2048), (256, 1024, 4096), (1024, 256, 4096), (3, 5, 8), (100, 37, 64),
                                       (64, 64, 64), (8, 1, 16), (1, 8, 16), (130, 20, 64), (20, 130, 64), (130, 130, 64)])
def test_ciphertext_ras_model_equals_lazy_ras(m, n, slots):
    """The rotate-and-sum that Sec. 4.3 makes lazy: log2(nb/m') rounds of x <- x + RotL(x, m' 2^j)
    leave in slot b*nb + t exactly the cleartext sum the lazy RaS takes (brute force on integer
    slot vectors, every regime)."""
    plan = layout.make_plan(m, n, slots)
    steps = layout.ras_steps(plan)
    assert len(steps) == int(np.log2(plan.nb // plan.m_prime))
    rng = np.random.default_rng(m + 3 * n)
    S = rng.integers(-50, 50, size=(plan.row_blocks, slots)).astype(np.float64)
    T = S.copy()
    for r in steps:
        T = T + np.stack([layout.rotl(row, r) for row in T])
    assert np.array_equal(layout.ras_decode(T, plan), layout.lazy_ras(S, plan))


@pytest.mark.parametrize("m,n,slots", [(16, 16, 16), (256, 1024, 4096), (1024, 256, 4096), (64, 64, 64), (130, 130, 64),
                                       (100, 37, 64), (20, 130, 64), (8, 8, 8)])
def test_bsgs_schedule_equals_diagonal_method(m, n, slots):
    """The baby-step giant-step schedule (sum_g RotL(sum_b RotR(e_{gB+b}, gB) (x) RotL(y, b), gB))
    gives the slots of the diagonal method exactly, for every power-of-two split of m'; with the
    pre-rotation left out (or its direction reversed) it does not."""
    rng = np.random.default_rng(m * 31 + n)
    X = rng.integers(-9, 10, size=(m, n)).astype(np.float64)
    y = rng.integers(-9, 10, size=n).astype(np.float64)
    plan = layout.make_plan(m, n, slots)
    want, _ = layout.cleartext_model(X, y, plan)
    B = 1
    while B <= plan.m_prime:
        got, out = layout.bsgs_cleartext_model(X, y, plan, B)
        assert np.array_equal(got, want)
        assert np.array_equal(out, X @ y)
        baby, giant = layout.bsgs_steps(plan, B)
        assert len(baby) + len(giant) == B - 1 + plan.m_prime // B - 1
        B *= 2
    if plan.m_prime >= 4:
        B = plan.m_prime // 4  # G = 4 giant steps: RotR and RotL by g B differ for g = 1
        E = layout.diagonal_slots(X, plan)
        Y = layout.vector_slots(y, plan)
        for sign in (0, -1):  # no pre-rotation; RotL instead of RotR
            acc = np.zeros((plan.row_blocks, plan.slots))
            for r in range(plan.row_blocks):
                for g in range(plan.m_prime // B):
                    inner = sum(np.roll(E[r, c, g * B + b], sign * g * B) * layout.rotl(Y[c], b)
                                for c in range(plan.col_blocks) for b in range(B))
                    acc[r] += layout.rotl(inner, g * B)
            assert not np.array_equal(acc, want)


def test_bsgs_split_rejects_bad_baby():
    plan = layout.make_plan(256, 1024, 4096)
    for bad in (0, 3, 128):
        with pytest.raises(ValueError):
            layout.bsgs_split(plan, bad)
