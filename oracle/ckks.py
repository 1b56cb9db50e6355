"""RNS-CKKS scheme and the PackVFL MatMult, composed from the C oracle primitives.

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the library.

Conventions (the scheme is only named by the paper -- CKKS through Lattigo,
Sec. 6 -- so these are readings, each stated where it is used):
  * ciphertexts are symmetric RLWE pairs (c0, c1) = (m - a s + e, a) (Sec. 2.2);
  * rotation by r slots to the left is the automorphism X -> X^(5^r mod 2N);
  * a rotation is always the hoisted form (O4, Sec. 2.2): ModUp of c1 once, then
    per Galois element the key-switch inner product and ModDown;
  * the MatMult plaintexts are encoded at scale q_l (the last prime of the input
    level) so that the rescale after the multiply-accumulate returns scale Delta.
All polynomials are numpy uint64 arrays in the coefficient domain.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

import numpy as np

from . import build as _build
from . import encoding, layout

_u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


class OrParams(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("L", ctypes.c_int32), ("K", ctypes.c_int32), ("dnum", ctypes.c_int32),
                ("primes", ctypes.c_uint64 * 64)]


_lib = None


def lib():
    """Load (building first if needed) the C oracle."""
    global _lib
    if _lib is None:
        L = ctypes.CDLL(_build())
        P = ctypes.POINTER(OrParams)
        u64, i32, i64 = ctypes.c_uint64, ctypes.c_int, ctypes.c_int64
        sig = {
            "or_powmod": (u64, [u64, u64, u64]),
            "or_invmod": (u64, [u64, u64]),
            "or_is_prime": (i32, [u64]),
            "or_gen_primes": (i32, [i32, i32, np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS"), _u64p]),
            "or_negacyclic_schoolbook": (None, [i32, u64, _u64p, _u64p, _u64p]),
            "or_ntt_forward": (None, [i32, u64, _u64p]),
            "or_ntt_inverse": (None, [i32, u64, _u64p]),
            "or_poly_mul": (None, [i32, u64, _u64p, _u64p, _u64p]),
            "or_automorph": (None, [i32, u64, u64, _u64p, _u64p]),
            "or_philox4x64": (None, [_u64p, _u64p, _u64p]),
            "or_sample_ternary": (None, [i32, u64, _i64p]),
            "or_sample_uniform": (None, [i32, u64, u64, u64, i32, u64, _u64p]),
            "or_sample_gauss": (None, [i32, u64, u64, u64, _i64p]),
            "or_cdt_table": (None, [_u64p]),
            "or_keygen_secret": (None, [P, u64, _i64p]),
            "or_galois_key": (None, [P, u64, _i64p, u64, _u64p]),
            "or_encrypt": (None, [P, u64, _i64p, u64, i32, _u64p, _u64p]),
            "or_decrypt": (None, [P, _i64p, i32, _u64p, _u64p]),
            "or_add": (None, [P, i32, _u64p, _u64p, _u64p]),
            "or_add_plain": (None, [P, i32, _u64p, _u64p, _u64p]),
            "or_mul_plain": (None, [P, i32, _u64p, _u64p, _u64p]),
            "or_modup": (None, [P, i32, _u64p, _u64p]),
            "or_moddown": (None, [P, i32, _u64p, _u64p]),
            "or_rotate_hoisted": (None, [P, i32, _u64p, i32, _u64p, _u64p, _u64p]),
            "or_matmult_double": (None, [P, i32, _u64p, i32, _u64p, _u64p, _u64p, _u64p]),
            "or_rescale": (None, [P, i32, _u64p, _u64p]),
            "or_max_threads": (i32, []),
            "or_set_threads": (None, [i32]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


TAG_ENC_A, TAG_ENC_E, TAG_EVK_A, TAG_EVK_E = 2, 3, 4, 5


def gen_primes(log_n: int, bits: list[int]) -> list[int]:
    out = np.zeros(len(bits), dtype=np.uint64)
    rc = lib().or_gen_primes(log_n, len(bits), np.asarray(bits, dtype=np.int32), out)
    if rc != 0:
        raise ValueError(f"no prime chain for log N = {log_n}, bits = {bits}")
    return [int(v) for v in out]


def to_rns(coeffs, primes) -> np.ndarray:
    """Signed integer coefficients -> [limbs][N] residues."""
    c = [int(v) for v in coeffs]
    return np.array([[v % q for v in c] for q in primes], dtype=np.uint64)


def centred(res: np.ndarray, q: int) -> np.ndarray:
    """Residues mod q -> signed representatives in (-q/2, q/2] as Python ints in an object array."""
    r = res.astype(object)
    return np.where(r > q // 2, r - q, r)


@dataclass
class Ciphertext:
    data: np.ndarray  # [2][level+1][N]
    level: int
    scale: float


@dataclass
class OpCounts:
    """Counters of the paper's basic operations (Tab. 2, Tab. 3)."""
    add: int = 0
    mult: int = 0
    rot: int = 0
    hstrot: int = 0


@dataclass
class Oracle:
    log_n: int
    q_bits: list[int]
    p_bits: list[int]
    dnum: int
    seed: int = 0
    primes: list[int] = field(init=False)
    counts: OpCounts = field(default_factory=OpCounts)

    def __post_init__(self):
        self.n = 1 << self.log_n
        self.slots = self.n // 2
        self.L, self.K = len(self.q_bits), len(self.p_bits)
        self.primes = gen_primes(self.log_n, list(self.q_bits) + list(self.p_bits))
        self.q = self.primes[: self.L]
        self.p = self.primes[self.L:]
        self.params = OrParams(self.n, self.L, self.K, self.dnum)
        for i, v in enumerate(self.primes):
            self.params.primes[i] = v
        self.sk = np.zeros(self.n, dtype=np.int64)
        lib().or_keygen_secret(ctypes.byref(self.params), self.seed, self.sk)
        self.keys: dict[int, np.ndarray] = {}

    # ---- parameters --------------------------------------------------------
    @property
    def P(self) -> int:
        out = 1
        for v in self.p:
            out *= v
        return out

    def galois(self, step: int) -> int:
        """Galois element of a left rotation by `step` slots: 5^step mod 2N."""
        return pow(5, step % self.slots, 2 * self.n)

    def level_primes(self, level: int, ext: bool = False) -> list[int]:
        return self.q[: level + 1] + (self.p if ext else [])

    # ---- keys --------------------------------------------------------------
    def gen_rotation_keys(self, steps):
        for r in steps:
            g = self.galois(r)
            if g in self.keys:
                continue
            evk = np.zeros((self.dnum, 2, self.L + self.K, self.n), dtype=np.uint64)
            lib().or_galois_key(ctypes.byref(self.params), self.seed, self.sk, g, evk.reshape(-1))
            self.keys[g] = evk

    # ---- encode / encrypt / decrypt ---------------------------------------
    def encode(self, z, scale: float, level: int, ext: bool = False) -> np.ndarray:
        """Plaintext [limbs][N] of real slots z at `scale` over Q_level (and P if ext)."""
        return to_rns(encoding.encode(z, scale, self.n), self.level_primes(level, ext))

    def encrypt(self, pt: np.ndarray, level: int, scale: float, nonce: int) -> Ciphertext:
        ct = np.zeros((2, level + 1, self.n), dtype=np.uint64)
        lib().or_encrypt(ctypes.byref(self.params), self.seed, self.sk, nonce, level,
                         np.ascontiguousarray(pt[: level + 1]).reshape(-1), ct.reshape(-1))
        return Ciphertext(ct, level, scale)

    def decrypt(self, ct: Ciphertext) -> np.ndarray:
        m = np.zeros((ct.level + 1, self.n), dtype=np.uint64)
        lib().or_decrypt(ctypes.byref(self.params), self.sk, ct.level, np.ascontiguousarray(ct.data).reshape(-1), m.reshape(-1))
        return m

    def decrypt_slots(self, ct: Ciphertext) -> np.ndarray:
        """Decrypt at q_0 alone (the other limbs dropped), centre, decode: real slot values."""
        m = self.decrypt(Ciphertext(ct.data[:, :1].copy(), 0, ct.scale))
        coeffs = centred(m[0], self.q[0]).astype(np.float64)
        return encoding.decode(coeffs, ct.scale, self.n).real

    # ---- O1..O4 -------------------------------------------------------------
    def add(self, x: Ciphertext, y: Ciphertext) -> Ciphertext:
        assert x.level == y.level
        out = np.zeros_like(x.data)
        lib().or_add(ctypes.byref(self.params), x.level, x.data.reshape(-1), y.data.reshape(-1), out.reshape(-1))
        self.counts.add += 1
        return Ciphertext(out, x.level, x.scale)

    def add_plain(self, ct: Ciphertext, pt: np.ndarray) -> Ciphertext:
        """O1 with a plaintext encoded at the ciphertext's scale (Sec. 2.2): (c0 + m, c1)."""
        out = np.zeros_like(ct.data)
        lib().or_add_plain(ctypes.byref(self.params), ct.level, ct.data.reshape(-1),
                           np.ascontiguousarray(pt[: ct.level + 1]).reshape(-1), out.reshape(-1))
        self.counts.add += 1
        return Ciphertext(out, ct.level, ct.scale)

    def ras(self, ct: Ciphertext, plan: layout.Plan) -> Ciphertext:
        """Ciphertext rotate-and-sum, the step the lazy RaS of Sec. 4.3 replaces: for each step
        r of layout.ras_steps, ct <- ct + RotL(ct, r); slot r*... b*nb + t then holds output
        row b*m' + t of its row block."""
        for r in layout.ras_steps(plan):
            ct = self.add(ct, self.rotate(ct, r))
        return ct

    def mul_plain(self, ct: Ciphertext, pt: np.ndarray, pt_scale: float) -> Ciphertext:
        out = np.zeros_like(ct.data)
        lib().or_mul_plain(ctypes.byref(self.params), ct.level, ct.data.reshape(-1),
                           np.ascontiguousarray(pt[: ct.level + 1]).reshape(-1), out.reshape(-1))
        self.counts.mult += 1
        return Ciphertext(out, ct.level, ct.scale * pt_scale)

    def rotate_hoisted(self, ct: Ciphertext, steps: list[int]) -> list[Ciphertext]:
        """HstRotL(ct, r) for every r in steps, sharing one ModUp."""
        if not steps:
            return []
        self.gen_rotation_keys(steps)
        gs = np.array([self.galois(r) for r in steps], dtype=np.uint64)
        evks = np.stack([self.keys[int(g)] for g in gs])
        outs = np.zeros((len(steps), 2, ct.level + 1, self.n), dtype=np.uint64)
        lib().or_rotate_hoisted(ctypes.byref(self.params), ct.level, np.ascontiguousarray(ct.data).reshape(-1), len(steps),
                                gs, evks.reshape(-1), outs.reshape(-1))
        self.counts.hstrot += len(steps)
        return [Ciphertext(outs[i], ct.level, ct.scale) for i in range(len(steps))]

    def rotate(self, ct: Ciphertext, step: int) -> Ciphertext:
        """O3: RotL(ct, step), the hoisted definition with a single element."""
        out = self.rotate_hoisted(ct, [step])[0]
        self.counts.hstrot -= 1
        self.counts.rot += 1
        return out

    def rescale(self, ct: Ciphertext) -> Ciphertext:
        out = np.zeros((2, ct.level, self.n), dtype=np.uint64)
        lib().or_rescale(ctypes.byref(self.params), ct.level, np.ascontiguousarray(ct.data).reshape(-1), out.reshape(-1))
        return Ciphertext(out, ct.level - 1, ct.scale / self.q[ct.level])

    def modup(self, c1: np.ndarray, level: int) -> np.ndarray:
        al = -(-self.L // self.dnum)
        nd = -(-(level + 1) // al)
        D = np.zeros((nd, level + 1 + self.K, self.n), dtype=np.uint64)
        lib().or_modup(ctypes.byref(self.params), level, np.ascontiguousarray(c1).reshape(-1), D.reshape(-1))
        return D

    def moddown(self, x: np.ndarray, level: int) -> np.ndarray:
        out = np.zeros((level + 1, self.n), dtype=np.uint64)
        lib().or_moddown(ctypes.byref(self.params), level, np.ascontiguousarray(x).reshape(-1), out.reshape(-1))
        return out

    # ---- PackVFL MatMult ------------------------------------------------------
    def encrypt_vector(self, y: np.ndarray, plan: layout.Plan, scale: float, nonce0: int = 0) -> list[Ciphertext]:
        """P_B's side: replicate y per the plan (Eq. 3 / Sec. 4.2) and encrypt each piece."""
        Y = layout.vector_slots(y, plan)
        return [self.encrypt(self.encode(Y[c], scale, self.L - 1), self.L - 1, scale, nonce0 + c) for c in range(plan.col_blocks)]

    def encode_matrix(self, X: np.ndarray, plan: layout.Plan, level: int, ext: bool) -> np.ndarray:
        """Diagonal plaintexts [R][C][m'][limbs][N] at scale q_level."""
        E = layout.diagonal_slots(X, plan)
        R, C, M = E.shape[:3]
        nl = level + 1 + (self.K if ext else 0)
        out = np.zeros((R, C, M, nl, self.n), dtype=np.uint64)
        for r in range(R):
            for c in range(C):
                for i in range(M):
                    out[r, c, i] = self.encode(E[r, c, i], float(self.q[level]), level, ext)
        return out

    def matmult(self, pts: np.ndarray, cts: list[Ciphertext], plan: layout.Plan, hoisting: str = "double") -> list[Ciphertext]:
        """X [[y]] in the hybrid layout, then one rescale: one output ciphertext per row block.

        hoisting="single": sum_i pt_i (x) HstRotL(ct, i) with each rotation divided by P (the
        paper's O4 followed by O2 and O1).  hoisting="double": the same sum with the rotations
        left in Q U P and one ModDown per output (or_matmult_double).
        """
        level = cts[0].level
        qp = float(self.q[level])
        steps = plan.rotation_steps
        outs = []
        if hoisting == "single":
            rots = [[c] + self.rotate_hoisted(c, steps) for c in cts]
            for r in range(plan.row_blocks):
                acc = None
                for c in range(plan.col_blocks):
                    for i in range(plan.m_prime):
                        t = self.mul_plain(rots[c][i], pts[r, c, i], qp)
                        acc = t if acc is None else self.add(acc, t)
                outs.append(self.rescale(acc))
            return outs
        self.gen_rotation_keys(steps)
        gs = np.array([self.galois(s) for s in steps], dtype=np.uint64)
        evks = np.stack([self.keys[int(g)] for g in gs]) if steps else np.zeros(1, dtype=np.uint64)
        if not steps:
            gs = np.zeros(1, dtype=np.uint64)
        for r in range(plan.row_blocks):
            acc = None
            for c in range(plan.col_blocks):
                out = np.zeros((2, level + 1, self.n), dtype=np.uint64)
                lib().or_matmult_double(ctypes.byref(self.params), level, np.ascontiguousarray(cts[c].data).reshape(-1),
                                        plan.m_prime, np.ascontiguousarray(pts[r, c]).reshape(-1), gs, evks.reshape(-1),
                                        out.reshape(-1))
                self.counts.mult += plan.m_prime
                self.counts.add += plan.m_prime - 1
                t = Ciphertext(out, level, cts[c].scale * qp)
                acc = t if acc is None else self.add(acc, t)
            outs.append(self.rescale(acc))
        self.counts.hstrot += plan.col_blocks * len(steps)
        return outs

    def encode_matrix_bsgs(self, X: np.ndarray, plan: layout.Plan, level: int, baby: int, ext: bool = False) -> np.ndarray:
        """Plaintexts of the baby-step giant-step schedule, [R][C][m'][limbs][N] at scale q_level:
        entry i = g B + b encodes RotR(e_i, g B) (layout.bsgs_diagonal_slots)."""
        E = layout.bsgs_diagonal_slots(X, plan, baby)
        R, C, M = E.shape[:3]
        nl = level + 1 + (self.K if ext else 0)
        out = np.zeros((R, C, M, nl, self.n), dtype=np.uint64)
        for r in range(R):
            for c in range(C):
                for i in range(M):
                    out[r, c, i] = self.encode(E[r, c, i], float(self.q[level]), level, ext)
        return out

    def matmult_bsgs(self, pts: np.ndarray, cts: list[Ciphertext], plan: layout.Plan, baby: int) -> list[Ciphertext]:
        """X [[y]] by the baby-step giant-step schedule (layout.bsgs_cleartext_model), composed from
        O1-O4: the baby rotations x_{c,b} = HstRotL(ct_c, b) share one decomposition; per row
        block and giant step g the partial sum s_g = sum_c sum_b pt_{gB+b} (x) x_{c,b} (O2, O1), then
        RotL(s_g, gB) (O3) for g >= 1, the sum over g, and one rescale.  Only the Q limbs of pts
        are used."""
        B, G = layout.bsgs_split(plan, baby)
        level = cts[0].level
        qp = float(self.q[level])
        baby_steps, _ = layout.bsgs_steps(plan, baby)
        xs = [[c] + self.rotate_hoisted(c, baby_steps) for c in cts]
        outs = []
        for r in range(plan.row_blocks):
            acc = None
            for g in range(G):
                inner = None
                for c in range(plan.col_blocks):
                    for b in range(B):
                        t = self.mul_plain(xs[c][b], pts[r, c, g * B + b][: level + 1], qp)
                        inner = t if inner is None else self.add(inner, t)
                if g > 0:
                    inner = self.rotate(inner, g * B)
                acc = inner if acc is None else self.add(acc, inner)
            outs.append(self.rescale(acc))
        return outs

    def matmult_decode(self, outs: list[Ciphertext], plan: layout.Plan) -> np.ndarray:
        """P_B's side: decrypt every output and apply the lazy rotate-and-sum (Sec. 4.3)."""
        slots = np.stack([self.decrypt_slots(o) for o in outs])
        return layout.lazy_ras(slots, plan)


def automorph_pt(o: "Oracle", pt: np.ndarray, g: int) -> np.ndarray:
    """X -> X^g on every limb of a plaintext (exact: a signed permutation of coefficients)."""
    out = np.zeros_like(pt)
    for l in range(pt.shape[0]):
        lib().or_automorph(o.n, o.primes[l], g, np.ascontiguousarray(pt[l]), out[l])
    return out


def cipher_diag_matmult(o: "Oracle", cts: list, pts_w: list, pt_scale: float) -> list:
    """Alg. 3, line 3, for every column k: [[z_k]] = Rescale( sum_i phi_{5^i}(p_k) (x) [[e_i]] ),
    the plaintext rotation RotL(w_k, i) realised as the automorphism X -> X^(5^i) of p_k, so no
    key switching is needed (Sec. 5.3: "eliminate all O4")."""
    outs = []
    for p in pts_w:
        acc = None
        for i, ct in enumerate(cts):
            t = o.mul_plain(ct, automorph_pt(o, p, o.galois(i)), pt_scale)
            acc = t if acc is None else o.add(acc, t)
        outs.append(o.rescale(acc))
    return outs


def transpose_diagonals(o: "Oracle", cts: list, m: int, n: int) -> list:
    """[[A^T]]'s diagonal ciphertexts from [[A]]'s (Eq. 5 as read in layout.transpose_rotations)."""
    outs = []
    for k, r in layout.transpose_rotations(m, n):
        outs.append(o.rotate(cts[k], r) if r else Ciphertext(cts[k].data.copy(), cts[k].level, cts[k].scale))
    return outs
