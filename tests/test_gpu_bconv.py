"""The basis extension of ModUp on the INT8 tensor cores (HE_BCONV_INT8_TC) against the exact
INT64 engine and the oracle's fast base conversion (or_modup), through the C ABI: ModUp digits
bit-equal limb by limb, and rotations and the Eq. 5 transposition bit-identical under either
engine."""
import numpy as np
import pytest

from oracle import ckks

pytestmark = pytest.mark.gpu

PARAMS = {
    "n16384_dnum3": (14, [60] + [40] * 6, [60, 60, 60], 3),
    "n8192": (13, [60, 40, 40], [60], 3),
    "n1024_alpha2": (10, [50, 40, 40, 40], [55, 55], 2),
    "n32_alpha4": (5, [30] * 8, [61, 61], 2),
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


def modup(he, ctx, ct, engine):
    import torch

    ctx.set_basis_extension(engine)
    al = -(-ctx.L // ctx.params.dnum)
    nd = -(-(ct.level + 1) // al)
    out = torch.empty((nd, ct.level + 1 + ctx.K, ctx.n), dtype=torch.int64, device=ctx.device)
    ctx.modup_export(ct, out)
    return he.as_u64(out)


@pytest.mark.parametrize("name", list(PARAMS))
def test_modup_int8_equals_int64_and_oracle(he, name):
    log_n, qb, pb, dnum = PARAMS[name]
    ctx = he.Context(log_n, qb, pb, dnum, seed=2)
    o = ckks.Oracle(log_n, qb, pb, dnum, seed=2)
    rng = np.random.default_rng(3)
    for level in range(len(qb)):
        data = np.zeros((2, level + 1, o.n), dtype=np.uint64)
        for c in range(2):
            for l in range(level + 1):
                data[c, l] = rng.integers(0, o.q[l], size=o.n, dtype=np.uint64)
        data[1, 0, :4] = o.q[0] - 1  # the largest residues
        ct = ctx.ct_import(he.from_u64(data, ctx.device), level, 1.0)
        d64 = modup(he, ctx, ct, he.HE_BCONV_INT64)
        d8 = modup(he, ctx, ct, he.HE_BCONV_INT8_TC)
        want = o.modup(data[1], level)
        assert np.array_equal(d64, want)
        assert np.array_equal(d8, want)
    ctx.set_basis_extension(he.HE_BCONV_INT64)


@pytest.mark.parametrize("name", ["n16384_dnum3", "n8192"])
def test_rotations_identical_under_both_engines(he, name):
    import torch

    log_n, qb, pb, dnum = PARAMS[name]
    ctx = he.Context(log_n, qb, pb, dnum, seed=4)
    o = ckks.Oracle(log_n, qb, pb, dnum, seed=4)
    level = len(qb) - 1
    steps = [1, 5, 77, ctx.slots - 3]
    ctx.keygen(steps)
    o.gen_rotation_keys(steps)
    z = torch.linspace(-1, 1, ctx.slots, dtype=torch.float64).cuda()
    ct = ctx.encrypt(ctx.encode(z, 2.0**40, level), 9)
    cts = [ctx.encrypt(ctx.encode(z * (i + 1), 2.0**40, level), 20 + i) for i in range(len(steps))]
    res = {}
    for eng in (he.HE_BCONV_INT64, he.HE_BCONV_INT8_TC):
        ctx.set_basis_extension(eng)
        hoist = [ctx.ct_export(c) for c in ctx.rotate_hoisted(ct, steps)]
        many = [ctx.ct_export(c) for c in ctx.rotate_many(cts, steps)]
        single = ctx.ct_export(ctx.rotate(ct, steps[1]))
        res[eng] = (hoist, many, single)
    ctx.set_basis_extension(he.HE_BCONV_INT64)
    a, b = res[he.HE_BCONV_INT64], res[he.HE_BCONV_INT8_TC]
    for x, y in zip(a[0] + a[1] + [a[2]], b[0] + b[1] + [b[2]]):
        assert torch.equal(x, y)
    # and the oracle's hoisted rotation of the same ciphertext
    want = o.rotate_hoisted(ckks.Ciphertext(he.as_u64(ctx.ct_export(ct)), level, 2.0**40), steps)
    for g, w in zip(b[0], want):
        assert np.array_equal(he.as_u64(g), w.data)


def test_transposition_identical_under_both_engines(he):
    import torch

    log_n, qb, pb, dnum = PARAMS["n16384_dnum3"]
    ctx = he.Context(log_n, qb, pb, dnum, seed=6)
    m, n = 256, 32
    rng = np.random.default_rng(6)
    A = rng.uniform(-1, 1, size=(m, n))
    level = len(qb) - 1
    cts = [ctx.encrypt(p, 40 + i) for i, p in enumerate(ctx.cdiag_encode_matrix(torch.from_numpy(A).cuda(), 2.0**40, level))]
    ctx.keygen(he.Context.cdiag_transpose_steps(m, n))
    out = {}
    for eng in (he.HE_BCONV_INT64, he.HE_BCONV_INT8_TC):
        ctx.set_basis_extension(eng)
        out[eng] = [ctx.ct_export(c) for c in ctx.cdiag_transpose(cts, m, n)]
    ctx.set_basis_extension(he.HE_BCONV_INT64)
    for x, y in zip(out[he.HE_BCONV_INT64], out[he.HE_BCONV_INT8_TC]):
        assert torch.equal(x, y)
