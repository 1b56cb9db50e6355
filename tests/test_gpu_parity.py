"""GPU library vs the CPU oracle, through the C ABI.

Integer work is compared bit-exactly in the canonical coefficient form: NTT round trips,
O1/O2, encryption (same seed and nonce, same Philox-4x64-10 streams), rescale, rotations
(Galois keys drawn by both sides from the same streams) and the MatMult with the oracle's
own plaintexts imported (parity tier 1).  Floating-point work is compared within stated
tolerances: encoding (integers may differ by one only where the exact value sits next to
a rounding boundary), decoding, and the whole path from fp64 inputs (tier 2) against the
FP64 product X y.
"""
import numpy as np
import pytest

from oracle import ckks, encoding, layout

pytestmark = pytest.mark.gpu

TOL = {20: 5e-2, 40: 1e-4}  # absolute tolerance on X y by log2(scale)

PARAM_SETS = {
    "n32": (5, [60, 40, 40], [60], 3),
    "n1024_alpha2": (10, [50, 40, 40, 40], [55, 55], 2),
    "n4096": (12, [40, 20], [40], 2),
    "n8192": (13, [60, 40, 40], [60], 3),
    "n16384": (14, [60] + [40] * 6, [60, 60, 60], 3),
}


@pytest.fixture(scope="module")
def he():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_00482_gb300 import build as b

    b.build()
    from paper_2405_00482_gb300 import he as h

    return h


_CACHE = {}


def pair(he, name, seed=0):
    key = (name, seed)
    if key not in _CACHE:
        log_n, qb, pb, d = PARAM_SETS[name]
        _CACHE[key] = (he.Context(log_n, qb, pb, d, seed), ckks.Oracle(log_n, qb, pb, d, seed))
    return _CACHE[key]


def rand_rns(rng, primes, shape_prefix, n):
    out = np.zeros(tuple(shape_prefix) + (len(primes), n), dtype=np.uint64)
    for idx in np.ndindex(*shape_prefix):
        for l, q in enumerate(primes):
            out[idx + (l,)] = [int(v) % q for v in rng.integers(0, 2**62, size=n, dtype=np.int64)]
    return out


def dev(he, ctx, a):
    return he.from_u64(a, ctx.device)


@pytest.mark.parametrize("name", list(PARAM_SETS))
def test_ntt_round_trip(he, name):
    ctx, o = pair(he, name)
    rng = np.random.default_rng(1)
    for level in range(o.L):
        data = rand_rns(rng, o.q[: level + 1], (2,), o.n)
        ct = ctx.ct_import(dev(he, ctx, data), level, 1.0)
        assert np.array_equal(he.as_u64(ctx.ct_export(ct)), data)


@pytest.mark.parametrize("name", ["n32", "n4096", "n8192"])
def test_add_and_mul_plain(he, name):
    ctx, o = pair(he, name)
    rng = np.random.default_rng(2)
    level = o.L - 1
    a = rand_rns(rng, o.q, (2,), o.n)
    b = rand_rns(rng, o.q, (2,), o.n)
    p = rand_rns(rng, o.q, (), o.n)
    ga, gb = ctx.ct_import(dev(he, ctx, a), level, 1.0), ctx.ct_import(dev(he, ctx, b), level, 1.0)
    gp = ctx.pt_import(dev(he, ctx, p), level, 1.0)
    want = o.add(ckks.Ciphertext(a, level, 1.0), ckks.Ciphertext(b, level, 1.0)).data
    assert np.array_equal(he.as_u64(ctx.ct_export(ctx.add(ga, gb))), want)
    want = o.mul_plain(ckks.Ciphertext(a, level, 1.0), p, 1.0).data
    assert np.array_equal(he.as_u64(ctx.ct_export(ctx.mul_plain(ga, gp))), want)


@pytest.mark.parametrize("name", ["n32", "n1024_alpha2", "n4096", "n8192"])
def test_encrypt_bit_exact_and_decrypt(he, name):
    ctx, o = pair(he, name)
    rng = np.random.default_rng(3)
    level = o.L - 1
    scale = 2.0**20 if name == "n4096" else 2.0**40
    z = rng.uniform(-1, 1, o.slots)
    pt = o.encode(z, scale, level)
    for nonce in (0, 7, 2**40 + 3):
        gct = ctx.encrypt(ctx.pt_import(dev(he, ctx, pt), level, scale), nonce)
        want = o.encrypt(pt, level, scale, nonce)
        assert np.array_equal(he.as_u64(ctx.ct_export(gct)), want.data)
        got = ctx.decrypt(gct).cpu().numpy()
        ref = o.decrypt_slots(want)
        assert np.abs(got - ref).max() < 1e-9
        assert np.abs(got - z).max() < (1e-2 if scale == 2.0**20 else 1e-8)


@pytest.mark.parametrize("name", ["n32", "n1024_alpha2", "n8192"])
def test_rescale_bit_exact(he, name):
    ctx, o = pair(he, name)
    rng = np.random.default_rng(4)
    for level in range(1, o.L):
        data = rand_rns(rng, o.q[: level + 1], (2,), o.n)
        g = ctx.rescale(ctx.ct_import(dev(he, ctx, data), level, 2.0**80))
        want = o.rescale(ckks.Ciphertext(data, level, 2.0**80))
        assert g.level == level - 1
        assert np.array_equal(he.as_u64(ctx.ct_export(g)), want.data)


@pytest.mark.parametrize("name", ["n32", "n1024_alpha2", "n4096", "n8192", "n16384"])
def test_rotation_bit_exact(he, name):
    ctx, o = pair(he, name)
    rng = np.random.default_rng(5)
    level = o.L - 1
    steps = [1, 2, 5, o.slots - 1]
    ctx.keygen(steps)
    data = rand_rns(rng, o.q, (2,), o.n)
    gct = ctx.ct_import(dev(he, ctx, data), level, 1.0)
    ref = ckks.Ciphertext(data, level, 1.0)
    hoisted = ctx.rotate_hoisted(gct, steps)
    want = o.rotate_hoisted(ref, steps)
    for s, g, w in zip(steps, hoisted, want):
        assert np.array_equal(he.as_u64(ctx.ct_export(g)), w.data), s
        assert np.array_equal(he.as_u64(ctx.ct_export(ctx.rotate(gct, s))), w.data), s
    # and at a lower level (fewer digits)
    if level >= 1:
        d1 = rand_rns(rng, o.q[:level], (2,), o.n)
        g = ctx.rotate(ctx.ct_import(dev(he, ctx, d1), level - 1, 1.0), 2)
        assert np.array_equal(he.as_u64(ctx.ct_export(g)), o.rotate(ckks.Ciphertext(d1, level - 1, 1.0), 2).data)


@pytest.mark.parametrize("name", ["n32", "n4096", "n8192"])
def test_encode_within_rounding(he, name):
    """Integer coefficients agree except where the exact value is within 1e-2 of a half-integer.

    The GPU FFT runs in double-float arithmetic (~2^-46 relative per operation), so a coefficient
    near 2^34 carries an absolute error of a few 1e-3 before rounding; only values that close to
    a rounding boundary may round the other way, and then by one."""
    import torch

    ctx, o = pair(he, name)
    rng = np.random.default_rng(6)
    scale = 2.0**40 if name != "n4096" else 2.0**20
    for n_slots in (o.slots, o.slots // 2 + 3, 1):
        z = rng.normal(size=n_slots)
        gpt = ctx.encode(torch.from_numpy(z).cuda(), scale, 0)
        got = he.as_u64(ctx.pt_export(gpt))[0]
        exact = encoding.encode_real(z, scale, o.n)
        want = np.array([int(v) % o.q[0] for v in np.rint(exact).astype(np.int64)], dtype=np.uint64)
        diff = got != want
        frac = np.abs(exact - np.floor(exact) - 0.5)
        assert np.all(frac[diff] < 1e-2), (diff.sum(), frac[diff].max() if diff.any() else 0)
        assert diff.sum() <= max(2, 0.03 * o.n)
        off = (got.astype(object) - want.astype(object)) % o.q[0]
        assert all(v in (1, o.q[0] - 1) for v in off[diff])


def _matmult_case(he, name, m, n, seed):
    ctx, o = pair(he, name)
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(m, n))
    y = rng.uniform(-1, 1, n)
    scale = 2.0**20 if name == "n4096" else 2.0**40
    level = o.L - 1
    plan_o = layout.make_plan(m, n, o.slots)
    plan_g = he.Plan(m, n, o.slots)
    ctx.keygen(plan_o.rotation_steps)
    cts = o.encrypt_vector(y, plan_o, scale, nonce0=100)
    pts = o.encode_matrix(X, plan_o, level, ext=True)
    outs = o.matmult(pts, cts, plan_o, hoisting="double")
    pm = ctx.ptmat_import(plan_g, dev(he, ctx, pts.reshape(-1)), level, float(o.q[level]))
    gcts = [ctx.ct_import(dev(he, ctx, c.data), level, scale) for c in cts]
    gouts = ctx.matmult(plan_g, pm, gcts)
    assert len(gouts) == len(outs)
    for g, w in zip(gouts, outs):
        assert g.level == w.level and abs(g.scale - w.scale) < 1e-6 * w.scale
        assert np.array_equal(he.as_u64(ctx.ct_export(g)), w.data)
    return ctx, o, X, y, plan_g, gouts, scale


@pytest.mark.parametrize("m,n", [(16, 8), (32, 32), (3, 5), (100, 20), (20, 100), (64, 64), (1, 1), (17, 31)])
def test_matmult_bit_exact_small_ring(he, m, n):
    """All four layout regimes of Sec. 4.2 (N' = 16 slots), ragged shapes, tier-1 parity."""
    _matmult_case(he, "n32", m, n, seed=m * 100 + n)


@pytest.mark.parametrize("m,n", [(256, 16), (16, 256), (700, 300)])
def test_matmult_bit_exact_alpha2(he, m, n):
    _matmult_case(he, "n1024_alpha2", m, n, seed=7)


@pytest.mark.parametrize("name,m,n", [("n4096", 16, 64), ("n8192", 256, 1024), ("n16384", 64, 512), ("n16384", 9000, 2)])
def test_matmult_bit_exact_full_size(he, name, m, n):
    """The gradient X^T [[r]] at the benchmark sizes, bit-exact against the oracle."""
    ctx, o, X, y, plan, gouts, scale = _matmult_case(he, name, m, n, seed=11)
    import torch

    slots = torch.stack([ctx.decrypt(g) for g in gouts])
    res = ctx.matmult_decode(plan, slots).cpu().numpy()
    assert np.abs(res - X @ y).max() < TOL[int(np.log2(scale))]


@pytest.mark.parametrize("name,m,n", [("n4096", 16, 64), ("n4096", 64, 16), ("n8192", 256, 1024), ("n8192", 1024, 256),
                                      ("n8192", 300, 5000), ("n8192", 5000, 300)])
def test_matmult_end_to_end_from_fp64(he, name, m, n):
    """Tier 2: GPU encode, encrypt, MatMult, decrypt and lazy RaS from fp64 inputs, within tolerance of X y."""
    import torch

    ctx, o = pair(he, name)
    rng = np.random.default_rng(m + n)
    X = rng.normal(size=(m, n))
    y = rng.uniform(-1, 1, n)
    scale = 2.0**20 if name == "n4096" else 2.0**40
    level = o.L - 1
    plan = he.Plan(m, n, o.slots)
    ctx.keygen(list(range(1, plan.m_prime)))
    pm = ctx.encode_matrix(plan, torch.from_numpy(X).cuda(), level)
    pts = ctx.encode_vector(plan, torch.from_numpy(y).cuda(), scale, level)
    cts = [ctx.encrypt(p, 500 + i) for i, p in enumerate(pts)]
    outs = ctx.matmult(plan, pm, cts)
    slots = torch.stack([ctx.decrypt(c) for c in outs])
    res = ctx.matmult_decode(plan, slots).cpu().numpy()
    assert np.abs(res - X @ y).max() < TOL[int(np.log2(scale))]


def test_missing_key_and_level_errors(he):
    import torch

    ctx, o = pair(he, "n32", seed=9)
    ct = ctx.encrypt(ctx.encode(torch.zeros(4, dtype=torch.float64, device="cuda"), 2.0**40, o.L - 1), 1)
    with pytest.raises(he.HEError) as e:
        ctx.rotate(ct, 3)
    assert e.value.status == he.HE_EKEY
    plan = he.Plan(8, 8, o.slots)
    ctx.keygen(list(range(1, plan.m_prime)))
    pm = ctx.encode_matrix(plan, torch.zeros((8, 8), dtype=torch.float64, device="cuda"), o.L - 1)
    low = ctx.rescale(ct)
    with pytest.raises(he.HEError) as e:
        ctx.matmult(plan, pm, [low])
    assert e.value.status == he.HE_ELEVEL
    with pytest.raises(he.HEError) as e:
        ctx.rescale(ctx.rescale(low))
    assert e.value.status == he.HE_ELEVEL


@pytest.mark.parametrize("name,m,n", [("n8192", 256, 1024), ("n8192", 1024, 256), ("n8192", 300, 5000), ("n4096", 64, 16),
                                      ("n1024_alpha2", 100, 300), ("n32", 17, 31)])
def test_encode_matrix_against_oracle(he, name, m, n):
    """Eq. 2 / Eq. 3 plaintexts from fp64 X (layout, cluster FFT, NTT of every limb): every limb of
    Q_level U P equals the oracle's rounding of the exact encoding, except where the exact value
    is within the double-float window of a half-integer, and there by one."""
    import torch

    ctx, o = pair(he, name)
    rng = np.random.default_rng(m + 3 * n)
    X = rng.normal(size=(m, n))
    level = o.L - 1
    plan_o, plan_g = layout.make_plan(m, n, o.slots), he.Plan(m, n, o.slots)
    pm = ctx.encode_matrix(plan_g, torch.from_numpy(X).cuda(), level)
    got = he.as_u64(pm.export())
    E = layout.diagonal_slots(X, plan_o)
    primes = o.level_primes(level, True)
    scale = float(o.q[level])
    total_diff = total = 0
    idxs = list(np.ndindex(*E.shape[:3]))
    if len(idxs) > 32:  # a fixed sample of the diagonals (first, last, random middle)
        pick = sorted(set([0, len(idxs) - 1] + list(np.random.default_rng(1).choice(len(idxs), 30, replace=False))))
        idxs = [idxs[i] for i in pick]
    for idx in idxs:
        exact = encoding.encode_real(E[idx], scale, o.n)
        ints = np.rint(exact).astype(np.int64)  # |coefficients| < 2^50
        frac = np.abs(exact - np.floor(exact) - 0.5)
        for li, q in enumerate(primes):
            want = np.mod(ints, np.int64(q)).astype(np.uint64)
            g = got[idx + (li,)]
            diff = g != want
            assert np.all(frac[diff] < 1e-2)
            off = (g[diff].astype(object) - want[diff].astype(object)) % q
            assert all(v in (1, q - 1) for v in off)
            total_diff += int(diff.sum())
            total += g.size
    assert total_diff <= 0.03 * total


def test_small_context_does_not_limit_a_large_one(he):
    """Kernel shared-memory limits are per process: creating an N = 32 context after an N = 8192
    one must leave the large context's launches (one-CTA NTTs above 48 KB) working."""
    import torch

    big = he.Context(13, [60, 40, 40], [60], 3, seed=41)
    he.Context(5, [60, 40, 40], [60], 3, seed=42)
    plan = he.Plan(256, 1024, big.slots)
    big.keygen(list(range(1, plan.m_prime)))
    X = torch.randn(256, 1024, dtype=torch.float64, device="cuda")
    y = torch.rand(1024, dtype=torch.float64, device="cuda") * 2 - 1
    pm = big.encode_matrix(plan, X, 2)
    out = big.matmult(plan, pm, [big.encrypt(big.encode_vector(plan, y, 2.0**40, 2)[0], 1)])
    res = big.matmult_decode(plan, torch.stack([big.decrypt(c) for c in out]))
    assert torch.abs(res - X @ y).max().item() < 1e-4


def test_buffer_sizes(he):
    ctx, o = pair(he, "n8192")
    for level in range(o.L):
        assert ctx.ct_bytes(level) == ctx.new_ct(level).data.numel() * 8 == 2 * (level + 1) * o.n * 8
        assert ctx.pt_bytes(level) == ctx.new_pt(level).data.numel() * 8
    assert ctx.ct_bytes(o.L) == 0 and ctx.pt_bytes(-1) == 0


@pytest.mark.parametrize("name,m,n", [("n32", 4, 4), ("n32", 3, 5), ("n32", 1, 8), ("n8192", 256, 1024), ("n8192", 1024, 256),
                                      ("n8192", 300, 5000), ("n8192", 5000, 300)])
def test_encode_matrix_transposed_bit_exact(he, name, m, n):
    """The matrix given as its transpose (he_encode_matrix_transposed, he_ptmat_encode_transposed)
    encodes to the same plaintexts, bit for bit, as the matrix itself."""
    import torch

    ctx, o = pair(he, name)
    rng = np.random.default_rng(7 * m + n)
    X = rng.normal(size=(m, n))
    level = o.L - 1
    plan = he.Plan(m, n, o.slots)
    want = he.as_u64(ctx.encode_matrix(plan, torch.from_numpy(X).cuda(), level).export())
    Xt = torch.from_numpy(np.ascontiguousarray(X.T)).cuda()
    pm = ctx.encode_matrix(plan, Xt, level, transposed=True)
    assert np.array_equal(he.as_u64(pm.export()), want)
    ctx.encode_matrix(plan, torch.zeros_like(Xt), level, out=pm, transposed=True)
    ctx.encode_matrix(plan, Xt, level, out=pm, transposed=True)  # in place
    assert np.array_equal(he.as_u64(pm.export()), want)
    with pytest.raises(ValueError):
        ctx.encode_matrix(plan, Xt, level) if m != n else ctx.encode_matrix(plan, Xt[:, :1], level)
