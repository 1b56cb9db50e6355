"""PackVFL hybrid MatMult layout on cleartext slots (oracle side).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the library.

This module holds the planner, the diagonal plaintext layout, the replicated
vector layout, the lazy rotate-and-sum and an exact cleartext model of the whole
slot computation.  It follows the paper:

* zero padding of m, n to powers of two (Sec. 3, "pad X_A and y_B with zero");
* the generalised diagonal encoding, Eq. 2 (Sec. 4.1), applied "in parts" after
  the input packing transform of Eq. 3 (Sec. 4.2.1);
* input partitioning into N'-sized row and column blocks (Sec. 4.2.2, Tab. 3),
  with one group of hoisted rotations per input ciphertext shared by all row
  blocks and column-block results added before output;
* lazy rotate-and-sum (Sec. 4.3): the slot sums happen after decryption.

RotL(v, i)[s] = v[(s + i) mod N'] (the left rotation of the naive-method example
in Sec. 3.1.1).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def pow2(v: int) -> int:
    """Smallest power of two >= v (v >= 1)."""
    p = 1
    while p < v:
        p *= 2
    return p


@dataclass(frozen=True)
class Plan:
    m: int  # rows of X (outputs)
    n: int  # columns of X (vector length)
    slots: int  # N' = N/2
    mp: int  # padded m
    np_: int  # padded n
    mb: int  # rows of one sub-matrix
    nb: int  # columns of one sub-matrix
    row_blocks: int  # R: output ciphertexts
    col_blocks: int  # C: input ciphertexts
    m_prime: int  # diagonals (plaintexts) per sub-matrix
    blocks: int  # B = N'/nb packed row groups per ciphertext

    @property
    def regime(self) -> str:
        if self.row_blocks == 1 and self.col_blocks == 1:
            return "pack"
        if self.col_blocks == 1:
            return "rows"
        if self.row_blocks == 1:
            return "cols"
        return "both"

    @property
    def rotation_steps(self) -> list[int]:
        """Left-rotation steps applied (hoisted) to every input ciphertext."""
        return list(range(1, self.m_prime))

    # operation counts, Tab. 2 (PackVFL row) and Tab. 3
    @property
    def n_mult(self) -> int:
        return self.row_blocks * self.col_blocks * self.m_prime

    @property
    def n_hstrot(self) -> int:
        return self.col_blocks * (self.m_prime - 1)

    @property
    def n_add(self) -> int:
        return self.row_blocks * (self.col_blocks * self.m_prime - 1)

    @property
    def n_rot(self) -> int:
        return 0


def make_plan(m: int, n: int, slots: int) -> Plan:
    """Planner: padding, regime choice and m' = ceil(m n / N') (Eq. 3)."""
    if m < 1 or n < 1 or slots < 1 or slots & (slots - 1):
        raise ValueError("m, n >= 1 and a power-of-two slot count are required")
    mp, np_ = pow2(m), pow2(n)
    mb, nb = min(mp, slots), min(np_, slots)
    row_blocks, col_blocks = mp // mb, np_ // nb
    m_prime = max(1, (mb * nb) // slots)
    return Plan(m, n, slots, mp, np_, mb, nb, row_blocks, col_blocks, m_prime, slots // nb)


def diagonal_slots(X: np.ndarray, plan: Plan) -> np.ndarray:
    """Diagonal plaintext slots, shape [R][C][m'][N'].

    e_{r,c,i}[b*nb + jj] = X[r*mb + b*m' + (jj mod m'), c*nb + (i + jj) mod nb]
    i.e. Eq. 3's transformed matrix X' (rows b*m'+t of a sub-matrix placed in slot
    block b) diagonally encoded per block as in Eq. 2; zero outside X.
    """
    m, n = X.shape
    assert (m, n) == (plan.m, plan.n)
    Xp = np.zeros((plan.mp, plan.np_), dtype=np.float64)
    Xp[:m, :n] = X
    R, C, mpr, N1, nb, mb = plan.row_blocks, plan.col_blocks, plan.m_prime, plan.slots, plan.nb, plan.mb
    out = np.zeros((R, C, mpr, N1), dtype=np.float64)
    s = np.arange(N1)
    b, jj = s // nb, s % nb
    for r in range(R):
        for c in range(C):
            for i in range(mpr):
                row = r * mb + b * mpr + (jj % mpr)
                col = c * nb + (i + jj) % nb
                ok = row < plan.mp
                out[r, c, i, ok] = Xp[row[ok], col[ok]]
    return out


def vector_slots(y: np.ndarray, plan: Plan) -> np.ndarray:
    """Encrypted-operand slots, shape [C][N']: piece c of y replicated N'/nb times."""
    yp = np.zeros(plan.np_, dtype=np.float64)
    yp[: plan.n] = y
    out = np.zeros((plan.col_blocks, plan.slots), dtype=np.float64)
    s = np.arange(plan.slots)
    for c in range(plan.col_blocks):
        out[c] = yp[c * plan.nb + s % plan.nb]
    return out


def rotl(v: np.ndarray, i: int) -> np.ndarray:
    """RotL(v, i)[s] = v[(s + i) mod len(v)]."""
    return np.roll(v, -i)


def ras_steps(plan: Plan) -> list[int]:
    """Rotation steps of the ciphertext rotate-and-sum (Sec. 3 / Sec. 4.3): m' * 2^j for
    j < log2(nb / m'), applied one after the other as x <- x + RotL(x, step).  Afterwards slot
    b*nb + t holds sum_{s < nb/m'} x[b*nb + t + s*m'] for t < m' (the blocks never mix, since
    t + (nb/m' - 1) m' < nb)."""
    steps, step = [], plan.m_prime
    while step < plan.nb:
        steps.append(step)
        step *= 2
    return steps


def ras_decode(slots: np.ndarray, plan: Plan) -> np.ndarray:
    """After the ciphertext RaS: out[r*mb + b*m' + t] = slot_r[b*nb + t]."""
    out = np.zeros(plan.mp, dtype=np.float64)
    mpr, nb, mb = plan.m_prime, plan.nb, plan.mb
    t = np.arange(mpr)
    for r in range(plan.row_blocks):
        for b in range(plan.blocks):
            row = r * mb + b * mpr + t
            ok = row < plan.mp
            out[row[ok]] = slots[r][b * nb + t][ok]
    return out[: plan.m]


def lazy_ras(slots: np.ndarray, plan: Plan) -> np.ndarray:
    """Lazy rotate-and-sum after decryption (Sec. 4.3), slots shape [R][N'] -> X y (length m).

    out[r*mb + b*m' + t] = sum_{s < nb/m'} slot_r[b*nb + t + s*m'].
    """
    out = np.zeros(plan.mp, dtype=np.float64)
    mpr, nb, mb = plan.m_prime, plan.nb, plan.mb
    t = np.arange(mpr)
    for r in range(plan.row_blocks):
        for b in range(plan.blocks):
            row = r * mb + b * mpr + t
            ok = row < plan.mp
            total = np.zeros(mpr)
            for s in range(nb // mpr):
                total += slots[r][b * nb + t + s * mpr]
            out[row[ok]] = total[ok]
    return out[: plan.m]


def cleartext_model(X: np.ndarray, y: np.ndarray, plan: Plan) -> tuple[np.ndarray, np.ndarray]:
    """Slot-exact cleartext model of the MatMult: sum_c sum_i e_{r,c,i} (x) RotL(y_c, i).

    Returns (slots [R][N'], lazy-RaS result [m]).
    """
    E = diagonal_slots(X, plan)
    Y = vector_slots(y, plan)
    acc = np.zeros((plan.row_blocks, plan.slots))
    for r in range(plan.row_blocks):
        for c in range(plan.col_blocks):
            for i in range(plan.m_prime):
                acc[r] += E[r, c, i] * rotl(Y[c], i)
    return acc, lazy_ras(acc, plan)


# ---- VFL-NN forward: the encrypted operand is the matrix (Sec. 5.3, Alg. 3) ----------------

def cipher_diagonals(A: np.ndarray, slots: int) -> np.ndarray:
    """Eq. 2 applied to the encrypted activation matrix A (m x n, powers of two, max(m, n) | N'):
    e_i[j] = A[j mod m, (i + j) mod n] for i < min(m, n), j < max(m, n), each diagonal repeated
    to fill the N' slots.  Shape [min(m, n)][N']."""
    m, n = A.shape
    lo, hi = min(m, n), max(m, n)
    assert slots % hi == 0
    out = np.zeros((lo, slots))
    j = np.arange(slots) % hi
    for i in range(lo):
        out[i] = A[j % m, (i + j) % n]
    return out


def weight_slots(w: np.ndarray, slots: int) -> np.ndarray:
    """A weight column w (length n) repeated with period n over the N' slots."""
    n = len(w)
    return w[np.arange(slots) % n]


def cipher_diag_model(A: np.ndarray, W: np.ndarray, slots: int) -> np.ndarray:
    """Cleartext model of Alg. 3's MatMult: output column k has slots
    sum_i e_i (x) RotL(w_k, i); with m >= n, slot j < m holds (A W)[j, k] and with m < n the
    n/m groups of m slots are summed after decryption (lazy RaS).  Returns A W (m x K)."""
    m, n = A.shape
    E = cipher_diagonals(A, slots)
    out = np.zeros((m, W.shape[1]))
    for k in range(W.shape[1]):
        acc = np.zeros(slots)
        for i in range(E.shape[0]):
            acc += E[i] * rotl(weight_slots(W[:, k], slots), i)
        out[:, k] = cipher_diag_decode(acc, m, n)
    return out


def cipher_diag_decode(slots_k: np.ndarray, m: int, n: int) -> np.ndarray:
    """Rows of one output column from its decrypted slots: slot j for m >= n; the sum over the
    n/m groups of m slots for m < n (lazy RaS, Sec. 4.3)."""
    if m >= n:
        return slots_k[:m].copy()
    return sum(slots_k[s * m:(s + 1) * m] for s in range(n // m))


def transpose_rotations(m: int, n: int) -> list[tuple[int, int]]:
    """Transposed matrices' diagonal conversion (Sec. 5.3, Eq. 5): the diagonals of A^T are
    rotations of A's diagonals, e'_i = RotL(e_k, r).  Worked out from Eq. 2 for both operands:
    k = (-i) mod min(m, n); r = i when m >= n, r = (-k) mod n when m < n (rotation over the
    period max(m, n) of the repeated diagonals).  The printed form, RotR by max - min + i, does
    not reproduce A^T's diagonals (checked by brute force in the tests).  Returns [(k, r)]."""
    lo = min(m, n)
    out = []
    for i in range(lo):
        k = (-i) % lo
        r = i if m >= n else (-k) % n
        out.append((k, r))
    return out


# ---- baby-step giant-step schedule of the diagonal method (an extension of Tab. 2's row) -----
#
# With m' = B G diagonals, i = g B + b (b < B baby steps, g < G giant steps), and RotL of a
# slot-wise product being the product of the RotLs,
#   sum_i e_i (x) RotL(y, i) = sum_g RotL( sum_b RotR(e_{gB+b}, gB) (x) RotL(y, b), gB ),
# so only the B - 1 baby rotations of y (hoisted, one decomposition) and G - 1 giant rotations of
# the partial sums are needed: about 2 sqrt(m') Galois keys instead of m' - 1.

def bsgs_split(plan: Plan, baby: int) -> tuple[int, int]:
    """(B, G): baby steps B (a power of two dividing m') and giant steps G = m' / B."""
    if baby < 1 or baby & (baby - 1) or plan.m_prime % baby:
        raise ValueError("baby steps: a power of two dividing m'")
    return baby, plan.m_prime // baby


def bsgs_steps(plan: Plan, baby: int) -> tuple[list[int], list[int]]:
    """Left-rotation steps: baby 1..B-1 (of every input ciphertext) and giant g B, g = 1..G-1
    (of the partial sums)."""
    B, G = bsgs_split(plan, baby)
    return list(range(1, B)), [g * B for g in range(1, G)]


def bsgs_diagonal_slots(X: np.ndarray, plan: Plan, baby: int) -> np.ndarray:
    """The plaintext slots of the schedule, shape [R][C][m'][N']: entry i = g B + b holds
    RotR(e_i, g B), RotR(v, r)[s] = v[(s - r) mod N']."""
    B, _ = bsgs_split(plan, baby)
    E = diagonal_slots(X, plan)
    out = np.empty_like(E)
    for i in range(plan.m_prime):
        out[:, :, i] = np.roll(E[:, :, i], (i // B) * B, axis=-1)
    return out


def bsgs_cleartext_model(X: np.ndarray, y: np.ndarray, plan: Plan, baby: int) -> tuple[np.ndarray, np.ndarray]:
    """Slot-exact cleartext model of the schedule: sum_g RotL(sum_c sum_b e'_{gB+b} (x) RotL(y_c, b), gB).
    Returns (slots [R][N'], lazy-RaS result [m])."""
    B, G = bsgs_split(plan, baby)
    E = bsgs_diagonal_slots(X, plan, baby)
    Y = vector_slots(y, plan)
    acc = np.zeros((plan.row_blocks, plan.slots))
    for r in range(plan.row_blocks):
        for g in range(G):
            inner = np.zeros(plan.slots)
            for c in range(plan.col_blocks):
                for b in range(B):
                    inner += E[r, c, g * B + b] * rotl(Y[c], b)
            acc[r] += rotl(inner, g * B)
    return acc, lazy_ras(acc, plan)
