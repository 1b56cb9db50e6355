"""Pins of the oracle's scheme: exact big-integer checks of ModUp, ModDown, rescale and the
Galois-key relation (Python integers, CRT), homomorphism invariants of O1-O4 (Sec. 2.2),
and the MatMult against the FP64 product X y (Eq. 1) within the stated tolerance."""
import numpy as np
import pytest

from oracle import ckks, layout

TOL_2_40 = 1e-4


def crt(limbs, primes):
    """Residues -> the integer in [0, prod primes)."""
    M = 1
    for q in primes:
        M *= q
    x = 0
    for r, q in zip(limbs, primes):
        Mq = M // q
        x += int(r) * Mq * pow(Mq, -1, q)
    return x % M, M


@pytest.fixture(scope="module")
def small():
    # three Q primes, digits of one prime each, plus a two-prime P to exercise alpha > 1 elsewhere
    return ckks.Oracle(log_n=5, q_bits=[60, 40, 40], p_bits=[60], dnum=3, seed=1)


@pytest.fixture(scope="module")
def small_alpha2():
    return ckks.Oracle(log_n=5, q_bits=[50, 40, 40, 40], p_bits=[55, 55], dnum=2, seed=2)


def _rand_limbs(rng, primes, n):
    return np.array([[int(v) % q for v in rng.integers(0, 1 << 62, size=n, dtype=np.int64)] for q in primes], dtype=np.uint64)


@pytest.mark.parametrize("which", ["small", "small_alpha2"])
def test_modup_is_exact_fast_base_conversion(which, request):
    o = request.getfixturevalue(which)
    rng = np.random.default_rng(0)
    level = o.L - 1
    c1 = _rand_limbs(rng, o.q, o.n)
    D = o.modup(c1, level)
    al = -(-o.L // o.dnum)
    ext = o.level_primes(level, True)
    for d in range(D.shape[0]):
        dig = list(range(d * al, min((d + 1) * al, level + 1)))
        Qd = 1
        for i in dig:
            Qd *= o.q[i]
        for k in range(o.n):
            xs = [int(c1[i, k]) for i in dig]
            # sum_i [x_i (Qd/q_i)^-1]_{q_i} (Qd/q_i): an integer congruent to the digit value mod Qd,
            # equal to it plus a multiple u*Qd with 0 <= u < len(digit)
            v = sum((x * pow(Qd // o.q[i], -1, o.q[i]) % o.q[i]) * (Qd // o.q[i]) for x, i in zip(xs, dig))
            exact, _ = crt(xs, [o.q[i] for i in dig])
            assert (v - exact) % Qd == 0 and 0 <= (v - exact) // Qd < len(dig)
            for u, t in enumerate(ext):
                assert int(D[d, u, k]) == v % t


@pytest.mark.parametrize("which", ["small", "small_alpha2"])
def test_moddown_divides_by_p(which, request):
    o = request.getfixturevalue(which)
    rng = np.random.default_rng(1)
    level = o.L - 1
    ext = o.level_primes(level, True)
    x = _rand_limbs(rng, ext, o.n)
    out = o.moddown(x, level)
    P = o.P
    for k in range(o.n):
        X, M = crt(x[:, k], ext)
        for j, q in enumerate(o.q[: level + 1]):
            # (X - (X mod P) - u P) / P = floor(X / P) - u with 0 <= u < K
            ok = any((X // P - u - int(out[j, k])) % q == 0 for u in range(o.K))
            assert ok
    # a multiple of P comes back exactly
    y = _rand_limbs(rng, o.q[: level + 1], o.n)
    Py = np.concatenate([np.array([[(int(v) * P) % q for v in y[j]] for j, q in enumerate(o.q[: level + 1])], dtype=np.uint64),
                         np.zeros((o.K, o.n), dtype=np.uint64)])
    assert np.array_equal(o.moddown(Py, level), y)


def test_rescale_rounds_to_nearest(small):
    o = small
    rng = np.random.default_rng(2)
    level = 2
    ct = ckks.Ciphertext(np.stack([_rand_limbs(rng, o.q, o.n) for _ in range(2)]), level, 2.0**80)
    out = o.rescale(ct)
    ql = o.q[level]
    for c in range(2):
        for k in range(o.n):
            X, M = crt(ct.data[c, :, k], o.q)
            r = X % ql
            if r > ql // 2:
                r -= ql
            want = (X - r) // ql
            for j in range(level):
                assert int(out.data[c, j, k]) == want % o.q[j]


@pytest.mark.parametrize("which", ["small", "small_alpha2"])
def test_galois_key_relation(which, request):
    """b_d + a_d s = e_d + P T_d phi_g(s) (mod QP) with |e_d| <= 19 (key-switching key form)."""
    o = request.getfixturevalue(which)
    g = o.galois(3)
    o.gen_rotation_keys([3])
    evk = o.keys[g]
    s = [int(v) for v in o.sk]
    n, P = o.n, o.P
    # phi_g(s) as integers
    sg = [0] * n
    for k in range(n):
        t = (k * g) % (2 * n)
        if t < n:
            sg[t] += s[k]
        else:
            sg[t - n] -= s[k]
    al = -(-o.L // o.dnum)
    Q = 1
    for q in o.q:
        Q *= q
    for d in range(o.dnum):
        dig = o.q[d * al:(d + 1) * al]
        Qd = 1
        for q in dig:
            Qd *= q
        Td = (Q // Qd) * pow(Q // Qd, -1, Qd)
        for k in range(0, n, 7):
            # (a s)_k negacyclic, as an integer
            vals = []
            for l, q in enumerate(o.primes):
                a = [int(v) for v in evk[d, 1, l]]
                as_k = sum(a[i] * s[(k - i) % n] * (1 if i <= k else -1) for i in range(n))
                vals.append((int(evk[d, 0, l, k]) + as_k - P * Td * sg[k]) % q)
            e, M = crt(vals, o.primes)
            if e > M // 2:
                e -= M
            assert abs(e) <= 19


def test_encrypt_decrypt_round_trip():
    o = ckks.Oracle(log_n=10, q_bits=[60, 40, 40], p_bits=[60], dnum=3, seed=3)
    z = np.random.default_rng(4).uniform(-1, 1, o.slots)
    ct = o.encrypt(o.encode(z, 2.0**40, 2), 2, 2.0**40, nonce=5)
    # |e| <= 19 per coefficient, decode gain <= N: a loose deterministic bound, and a tight typical one
    err = np.abs(o.decrypt_slots(ct) - z).max()
    assert err < 19 * o.n / 2**40
    assert err < 1e-9


def test_homomorphism_add_mult_rotate():
    o = ckks.Oracle(log_n=8, q_bits=[60, 40, 40], p_bits=[60], dnum=3, seed=4)
    rng = np.random.default_rng(5)
    a, b, w = (rng.uniform(-1, 1, o.slots) for _ in range(3))
    D = 2.0**40
    ca = o.encrypt(o.encode(a, D, 2), 2, D, 1)
    cb = o.encrypt(o.encode(b, D, 2), 2, D, 2)
    assert np.abs(o.decrypt_slots(o.add(ca, cb)) - (a + b)).max() < 1e-9
    qs = float(o.q[2])
    prod = o.rescale(o.mul_plain(cb, o.encode(w, qs, 2), qs))
    assert abs(prod.scale - D) < 1e-6 * D
    assert np.abs(o.decrypt_slots(prod) - w * b).max() < 1e-8
    for k in (1, 2, 5, o.slots - 1):
        assert np.abs(o.decrypt_slots(o.rotate(ca, k)) - np.roll(a, -k)).max() < 1e-8
    # hoisted rotations are the same definition: bit-equal to one-at-a-time
    hs = o.rotate_hoisted(ca, [1, 2, 5])
    for k, h in zip([1, 2, 5], hs):
        assert np.array_equal(h.data, o.rotate(ca, k).data)


@pytest.mark.parametrize("m,n", [(4, 4), (16, 8), (8, 16), (100, 3), (3, 100), (256, 16), (16, 256), (256, 256), (1, 1)])
def test_matmult_matches_fp64_product(m, n):
    """Dec(MatMult(X, Enc(y))) with lazy RaS equals X y within the scale-2^40 tolerance, both hoistings."""
    o = ckks.Oracle(log_n=7, q_bits=[60, 40, 40], p_bits=[60], dnum=3, seed=5)
    rng = np.random.default_rng(m * 7 + n)
    X = rng.normal(size=(m, n))
    y = rng.uniform(-1, 1, n)
    plan = layout.make_plan(m, n, o.slots)
    cts = o.encrypt_vector(y, plan, 2.0**40)
    res = {}
    for h in ("single", "double"):
        o.counts = ckks.OpCounts()
        pts = o.encode_matrix(X, plan, 2, ext=(h == "double"))
        outs = o.matmult(pts, cts, plan, hoisting=h)
        assert len(outs) == plan.row_blocks
        assert outs[0].level == 1 and abs(outs[0].scale - 2.0**40) < 1e-3
        res[h] = o.matmult_decode(outs, plan)
        assert np.abs(res[h] - X @ y).max() < TOL_2_40
        assert (o.counts.mult, o.counts.hstrot, o.counts.rot) == (plan.n_mult, plan.n_hstrot, 0)
        assert o.counts.add == plan.n_add
    assert np.abs(res["single"] - res["double"]).max() < TOL_2_40


def test_matmult_worked_example_through_encryption():
    """m = n = 4, N' = 8 (ring degree 16): the Sec. 4.3 example end to end."""
    o = ckks.Oracle(log_n=4, q_bits=[60, 40, 40], p_bits=[60], dnum=3, seed=6)
    X = np.arange(16, dtype=float).reshape(4, 4) / 10
    y = np.array([0.5, -0.25, 0.75, 1.0])
    plan = layout.make_plan(4, 4, 8)
    outs = o.matmult(o.encode_matrix(X, plan, 2, ext=True), o.encrypt_vector(y, plan, 2.0**40), plan)
    slots = o.decrypt_slots(outs[0])
    want_slots, want = layout.cleartext_model(X, y, plan)
    assert np.abs(slots - want_slots[0]).max() < TOL_2_40
    assert np.abs(layout.lazy_ras(slots[None], plan) - X @ y).max() < TOL_2_40


def test_config1_gradient_within_tolerance():
    """N = 4096, Q = [40, 20], P = [40], scale 2^20: X^T r with X 64x16 ~ N(0,1), r ~ U[-1,1]."""
    o = ckks.Oracle(log_n=12, q_bits=[40, 20], p_bits=[40], dnum=2, seed=0)
    rng = np.random.default_rng(0)
    X = rng.normal(size=(64, 16))
    r = rng.uniform(-1, 1, 64)
    plan = layout.make_plan(16, 64, o.slots)
    assert plan.m_prime == 1
    outs = o.matmult(o.encode_matrix(X.T, plan, 1, ext=True), o.encrypt_vector(r, plan, 2.0**20), plan)
    assert np.abs(o.matmult_decode(outs, plan) - X.T @ r).max() < 5e-2


@pytest.mark.parametrize("m,n,K", [(32, 8, 2), (8, 32, 2)])
def test_cipher_diag_matmult_matches_fp64(m, n, K):
    """Alg. 3 through encryption: the plaintext rotations as automorphisms, no key switching."""
    o = ckks.Oracle(log_n=6, q_bits=[60, 40, 40], p_bits=[60], dnum=3, seed=8)
    rng = np.random.default_rng(m * n)
    A = rng.uniform(-1, 1, (m, n))
    W = rng.normal(size=(n, K)) / np.sqrt(n)
    E = layout.cipher_diagonals(A, o.slots)
    cts = [o.encrypt(o.encode(E[i], 2.0**40, 2), 2, 2.0**40, nonce=i) for i in range(E.shape[0])]
    qs = float(o.q[2])
    pts = [o.encode(layout.weight_slots(W[:, k], o.slots), qs, 2) for k in range(K)]
    outs = ckks.cipher_diag_matmult(o, cts, pts, qs)
    res = np.stack([layout.cipher_diag_decode(o.decrypt_slots(c), m, n) for c in outs], 1)
    assert np.abs(res - A @ W).max() < TOL_2_40
    # the automorphism of an encoded plaintext is the encoding of the rotated slots (up to rounding)
    p = pts[0]
    rot = ckks.automorph_pt(o, p, o.galois(3))
    assert np.abs(o.decrypt_slots(o.encrypt(rot, 2, qs, 99)) - np.roll(layout.weight_slots(W[:, 0], o.slots), -3)).max() < 1e-6


@pytest.mark.parametrize("m,n", [(32, 8), (8, 32)])
def test_transpose_then_backward_product(m, n):
    """VFL-NN backward (Alg. 4): diagonals of [[A^T]] by rotation (Eq. 5), then [[A^T]] D^T."""
    o = ckks.Oracle(log_n=6, q_bits=[60, 40, 40], p_bits=[60], dnum=3, seed=9)
    rng = np.random.default_rng(m + n)
    A = rng.uniform(-1, 1, (m, n))
    Dt = rng.normal(size=(m, 2)) / np.sqrt(m)
    E = layout.cipher_diagonals(A, o.slots)
    cts = [o.encrypt(o.encode(E[i], 2.0**40, 2), 2, 2.0**40, nonce=i) for i in range(E.shape[0])]
    o.gen_rotation_keys([r for _, r in layout.transpose_rotations(m, n) if r])
    tcts = ckks.transpose_diagonals(o, cts, m, n)
    Et = layout.cipher_diagonals(A.T.copy(), o.slots)
    for i, c in enumerate(tcts):
        assert np.abs(o.decrypt_slots(c) - Et[i]).max() < 1e-8
    qs = float(o.q[2])
    pts = [o.encode(layout.weight_slots(Dt[:, k], o.slots), qs, 2) for k in range(2)]
    outs = ckks.cipher_diag_matmult(o, tcts, pts, qs)
    res = np.stack([layout.cipher_diag_decode(o.decrypt_slots(c), n, m) for c in outs], 1)
    assert np.abs(res - A.T @ Dt).max() < TOL_2_40


@pytest.mark.parametrize("m,n", [(4, 4), (16, 64), (8, 16), (64, 8)])
def test_add_plain_and_ciphertext_ras(m, n):
    """O1 with a plaintext operand, and the MatMult finished by the ciphertext rotate-and-sum
    instead of the lazy one: both decrypt to the FP64 result; the RaS costs len(ras_steps)
    rotations and additions."""
    o = ckks.Oracle(log_n=7, q_bits=[60, 40, 40], p_bits=[60], dnum=3, seed=11)
    rng = np.random.default_rng(m * n)
    D = 2.0**40
    a, w = rng.uniform(-1, 1, o.slots), rng.uniform(-1, 1, o.slots)
    ca = o.encrypt(o.encode(a, D, 2), 2, D, 1)
    s = o.add_plain(ca, o.encode(w, D, 2))
    assert np.array_equal(s.data[1], ca.data[1])
    assert np.abs(o.decrypt_slots(s) - (a + w)).max() < 1e-9
    X = rng.normal(size=(m, n))
    y = rng.uniform(-1, 1, n)
    plan = layout.make_plan(m, n, o.slots)
    outs = o.matmult(o.encode_matrix(X, plan, 2, ext=True), o.encrypt_vector(y, plan, D), plan)
    o.gen_rotation_keys(layout.ras_steps(plan))
    o.counts = ckks.OpCounts()
    rased = [o.ras(c, plan) for c in outs]
    assert (o.counts.rot, o.counts.add) == (len(layout.ras_steps(plan)) * len(outs),) * 2
    got = layout.ras_decode(np.stack([o.decrypt_slots(c) for c in rased]), plan)
    assert np.abs(got - X @ y).max() < TOL_2_40


def test_vfl_linr_gradient_step():
    """Alg. 1 for one party's gradient: [[d]] = [[u_A]] + (u_B - y) in the replicated layout,
    X_A^T [[d]], a random mask added before decryption and removed after, lazy RaS.  Equals
    X_A^T (u_A + u_B - y); the masked result alone does not."""
    o = ckks.Oracle(log_n=8, q_bits=[60, 40, 40], p_bits=[60], dnum=3, seed=12)
    rng = np.random.default_rng(13)
    b, f = 64, 16
    XA = rng.normal(size=(b, f))
    uA, uB, y = rng.normal(size=b), rng.normal(size=b), rng.uniform(-1, 1, b)
    D = 2.0**40
    plan = layout.make_plan(f, b, o.slots)  # X_A^T: m = features, n = batch
    o.gen_rotation_keys(plan.rotation_steps)
    ct_uA = o.encrypt_vector(uA, plan, D, nonce0=3)
    dv = layout.vector_slots(uB - y, plan)
    ct_d = [o.add_plain(c, o.encode(dv[i], D, o.L - 1)) for i, c in enumerate(ct_uA)]
    outs = o.matmult(o.encode_matrix(XA.T, plan, o.L - 1, ext=True), ct_d, plan)
    mask = rng.uniform(-100, 100, (len(outs), o.slots))
    masked = [o.add_plain(c, o.encode(mask[i], c.scale, c.level)) for i, c in enumerate(outs)]
    slots = np.stack([o.decrypt_slots(c) for c in masked])
    want = XA.T @ (uA + uB - y)
    assert np.abs(layout.lazy_ras(slots, plan) - want).max() > 1.0
    assert np.abs(layout.lazy_ras(slots - mask, plan) - want).max() < TOL_2_40


def test_matmult_same_on_any_thread_count():
    """The oracle's parallel MatMult loop combines per-thread partial sums with exact modular
    additions, so one thread and every host core give the same ciphertext."""
    o = ckks.Oracle(6, [60, 40, 40], [60], 3, seed=5)
    rng = np.random.default_rng(5)
    X = rng.normal(size=(32, 32))
    y = rng.uniform(-1, 1, 32)
    plan = layout.make_plan(32, 32, o.slots)
    cts = o.encrypt_vector(y, plan, 2.0**40)
    pts = o.encode_matrix(X, plan, o.L - 1, ext=True)
    lib = ckks.lib()
    cores = lib.or_max_threads()
    try:
        lib.or_set_threads(1)
        one = o.matmult(pts, cts, plan)
        lib.or_set_threads(max(cores, 4))
        many = o.matmult(pts, cts, plan)
    finally:
        lib.or_set_threads(cores)
    assert plan.m_prime > 8
    for a, b in zip(one, many):
        assert np.array_equal(a.data, b.data)


@pytest.mark.parametrize("m,n,baby", [(256, 256, 4), (256, 16, 2), (16, 256, 8), (128, 512, 16), (256, 256, 64)])
def test_matmult_bsgs_matches_fp64_product(m, n, baby):
    """The baby-step giant-step MatMult (O1-O4 composition) decrypts to X y within the scale-2^40
    tolerance, and agrees with the diagonal method's result within it."""
    o = ckks.Oracle(log_n=7, q_bits=[60, 40, 40], p_bits=[60], dnum=3, seed=9)
    rng = np.random.default_rng(m + 3 * n + baby)
    X = rng.normal(size=(m, n))
    y = rng.uniform(-1, 1, n)
    plan = layout.make_plan(m, n, o.slots)
    if plan.m_prime % baby:
        pytest.skip("baby steps must divide m'")
    cts = o.encrypt_vector(y, plan, 2.0**40)
    pts = o.encode_matrix_bsgs(X, plan, 2, baby)
    outs = o.matmult_bsgs(pts, cts, plan, baby)
    assert outs[0].level == 1 and abs(outs[0].scale - 2.0**40) < 1e-3
    got = o.matmult_decode(outs, plan)
    assert np.abs(got - X @ y).max() < TOL_2_40
    ref = o.matmult_decode(o.matmult(o.encode_matrix(X, plan, 2, ext=True), cts, plan), plan)
    assert np.abs(got - ref).max() < TOL_2_40
