"""Every loop-kernel variant of the double-hoisted MatMult (register prefetch and cp.async
pipelines, 1 or 2 coefficients per thread, 4 or 8 rotation groups) pinned in turn and compared
bit for bit with the oracle, at one, two and three key-switching digits, at the generic digit
count, on a ring smaller than one tile, and in the persistent batch kernel."""
import numpy as np
import pytest

from oracle import ckks, layout

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def he():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2405_00482_gb300 import he as mod

    return mod


def test_variant_table(he):
    shapes = he.loop_variants()
    assert len(shapes) >= 7 and len(shapes) <= he.HE_MM_MAX_VARIANTS
    assert len(set(shapes)) == len(shapes)
    assert {s[2] > 0 for s in shapes} == {False, True}  # register form and cp.async pipelines
    assert {s[3] for s in shapes} == {0, 1}  # with and without staged gathers


# (log N, Q bits, P bits, dnum, level, m, n): digits at that level = ceil((level + 1) / alpha)
CASES = {
    "n8192_l2_3dig": (13, [60, 40, 40], [60], 3, 2, 256, 1024),
    "n8192_l1_2dig": (13, [60, 40, 40], [60], 3, 1, 128, 512),
    "n1024_l3_2dig_alpha2": (10, [50, 40, 40, 40], [55, 55], 2, 3, 100, 300),
    "n1024_l1_1dig_alpha2": (10, [50, 40, 40, 40], [55, 55], 2, 1, 40, 30),
    "n1024_l4_5dig_generic": (10, [40] * 5, [50], 5, 4, 20, 50),
    "n32_ragged": (5, [60, 40, 40], [60], 3, 2, 17, 31),
}


@pytest.mark.parametrize("case", list(CASES))
def test_every_variant_bit_exact(he, case):
    log_n, qb, pb, dnum, level, m, n = CASES[case]
    ctx = he.Context(log_n, qb, pb, dnum, seed=3)
    o = ckks.Oracle(log_n, qb, pb, dnum, seed=3)
    rng = np.random.default_rng(len(case))
    X = rng.normal(size=(m, n))
    y = rng.uniform(-1, 1, n)
    scale = 2.0**30
    plan_o = layout.make_plan(m, n, o.slots)
    plan_g = he.Plan(m, n, o.slots)
    ctx.keygen(plan_o.rotation_steps)
    Y = layout.vector_slots(y, plan_o)
    cts = [o.encrypt(o.encode(Y[c], scale, level), level, scale, 70 + c) for c in range(plan_o.col_blocks)]
    pts = o.encode_matrix(X, plan_o, level, ext=True)
    want = [w.data for w in o.matmult(pts, cts, plan_o, hoisting="double")]
    pm = ctx.ptmat_import(plan_g, he.from_u64(pts.reshape(-1), ctx.device), level, float(o.q[level]))
    gcts = [ctx.ct_import(he.from_u64(c.data, ctx.device), level, scale) for c in cts]
    for v in range(len(he.loop_variants())):
        pm.set_variant(v)
        gouts = ctx.matmult(plan_g, pm, gcts)
        for g, w in zip(gouts, want):
            assert np.array_equal(he.as_u64(ctx.ct_export(g)), w), f"variant {v}"
        assert pm.tuning()["variant"] == v
    # -1 re-enables tuning: the next product times every variant and keeps one
    pm.set_variant(-1)
    gouts = ctx.matmult(plan_g, pm, gcts)
    assert all(np.array_equal(he.as_u64(ctx.ct_export(g)), w) for g, w in zip(gouts, want))
    t = pm.tuning()
    assert 0 <= t["variant"] < len(he.loop_variants()) and all(ms > 0 for ms in t["variant_ms"])


def test_every_variant_in_batch(he):
    log_n, qb, pb, d = 13, [60, 40, 40], [60], 3
    ctx = he.Context(log_n, qb, pb, d, seed=5)
    o = ckks.Oracle(log_n, qb, pb, d, seed=5)
    level, scale = 2, 2.0**40
    rng = np.random.default_rng(8)
    plans, pms, cts, wants = [], [], [], []
    for i, (m, n) in enumerate([(16, 128), (64, 512), (8, 8)]):
        X = rng.normal(size=(m, n))
        y = rng.uniform(-1, 1, n)
        po = layout.make_plan(m, n, o.slots)
        pg = he.Plan(m, n, o.slots)
        ctx.keygen(po.rotation_steps)
        c = o.encrypt_vector(y, po, scale, nonce0=90 + i)
        pts = o.encode_matrix(X, po, level, ext=True)
        wants.append(o.matmult(pts, c, po)[0].data)
        plans.append(pg)
        pms.append(ctx.ptmat_import(pg, he.from_u64(pts.reshape(-1), ctx.device), level, float(o.q[level])))
        cts.append(ctx.ct_import(he.from_u64(c[0].data, ctx.device), level, scale))
    b = he.Batch(ctx, plans, pms)
    for v in range(len(he.loop_variants())):
        b.set_variant(v)
        for _ in range(2):  # the first run captures the graph, the second replays it
            outs = b.run(cts)
            for out, want in zip(outs, wants):
                assert np.array_equal(he.as_u64(ctx.ct_export(out)), want), f"variant {v}"
    with pytest.raises(he.HEError):
        b.set_variant(len(he.loop_variants()))
