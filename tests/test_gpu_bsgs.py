"""The baby-step giant-step schedule of the MatMult (he_plan_set_baby_steps) on the GPU, through
the C ABI: with the oracle's own plaintexts and ciphertexts the outputs equal the oracle's BSGS
composition (Oracle.matmult_bsgs) bit for bit (parity tier 1); from fp64 inputs the result
decrypts to X y within the scale-2^40 tolerance and agrees with the diagonal method's."""
import numpy as np
import pytest

from oracle import ckks, layout

pytestmark = pytest.mark.gpu

PARAMS = {"n1024_alpha2": (10, [50, 40, 40, 40], [55, 55], 2), "n8192": (13, [60, 40, 40], [60], 3)}


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


def pair(he, name):
    if name not in _CACHE:
        log_n, qb, pb, d = PARAMS[name]
        _CACHE[name] = (he.Context(log_n, qb, pb, d, seed=11), ckks.Oracle(log_n, qb, pb, d, seed=11))
    return _CACHE[name]


@pytest.mark.parametrize("name,m,n,baby", [("n1024_alpha2", 64, 64, 2), ("n1024_alpha2", 600, 300, 4), ("n1024_alpha2", 300, 600, 1),
                                           ("n1024_alpha2", 512, 512, 512), ("n8192", 256, 1024, 8)])
def test_bsgs_bit_exact_vs_oracle(he, name, m, n, baby):
    ctx, o = pair(he, name)
    rng = np.random.default_rng(m + n + baby)
    X = rng.normal(size=(m, n))
    y = rng.uniform(-1, 1, n)
    level = o.L - 1
    oplan = layout.make_plan(m, n, o.slots)
    plan = he.Plan(m, n, ctx.slots, baby=baby)
    bs, gs = layout.bsgs_steps(oplan, baby)
    ctx.keygen(bs + gs)
    cts = o.encrypt_vector(y, oplan, 2.0**40, nonce0=5)
    pts = o.encode_matrix_bsgs(X, oplan, level, baby, ext=True)
    want = o.matmult_bsgs(pts, cts, oplan, baby)
    pm = ctx.ptmat_import(plan, he.from_u64(pts.reshape(-1), ctx.device), level, float(o.q[level]))
    ins = [ctx.ct_import(he.from_u64(c.data, ctx.device), level, 2.0**40) for c in cts]
    outs = ctx.matmult(plan, pm, ins)
    for g, w in zip(outs, want):
        assert g.level == w.level
        assert np.array_equal(he.as_u64(ctx.ct_export(g)), w.data)


@pytest.mark.parametrize("m,n,baby", [(256, 1024, 8), (1024, 256, 4), (256, 1024, 64), (300, 5000, 16), (16, 64, 1)])
def test_bsgs_fp64_path(he, m, n, baby):
    import torch

    ctx, _ = pair(he, "n8192")
    rng = np.random.default_rng(m * 3 + n + baby)
    X = rng.normal(size=(m, n))
    y = rng.uniform(-1, 1, n)
    plan = he.Plan(m, n, ctx.slots, baby=baby)
    ref_plan = he.Plan(m, n, ctx.slots)
    ctx.keygen(plan.rotation_steps + ref_plan.rotation_steps)
    dX = torch.from_numpy(X).cuda()
    cts = ctx.encrypt_vector(plan, torch.from_numpy(y).cuda(), 2.0**40, 2, 31)
    got = ctx.matmult_decrypt(plan, ctx.matmult(plan, ctx.encode_matrix(plan, dX, 2), cts)).cpu().numpy()
    ref = ctx.matmult_decrypt(ref_plan, ctx.matmult(ref_plan, ctx.encode_matrix(ref_plan, dX, 2), cts)).cpu().numpy()
    assert np.abs(got - X @ y).max() < 1e-4
    assert np.abs(got - ref).max() < 1e-4
