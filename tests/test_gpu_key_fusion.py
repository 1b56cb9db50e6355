"""Fused key tables (he_set_key_fusion): the MatMult reading F_i = ksk_i (x) pt_i instead of the
Galois key and the plaintext gives the same residues as the two-level loop, so its outputs are
compared bit for bit with the oracle's double-hoisted MatMult (Sec. 4.2 with O4) and with the
two-level form, for every fused variant, partitioned plans, re-encoding and graph replay."""
import numpy as np
import pytest

from oracle import ckks, layout

pytestmark = pytest.mark.gpu

PARAMS = {
    "n32": (5, [60, 40, 40], [60], 3),
    "n1024_alpha2": (10, [50, 40, 40, 40], [55, 55], 2),
    "n8192": (13, [60, 40, 40], [60], 3),
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


def pair(he, name):
    if name not in _CACHE:
        log_n, qb, pb, d = PARAMS[name]
        _CACHE[name] = (he.Context(log_n, qb, pb, d, 0), ckks.Oracle(log_n, qb, pb, d, 0))
    return _CACHE[name]


def fused_variants(he):
    """variants with cp.async stages: the ones with a fused form (1 to 3 digits)"""
    return [v for v, (vec, grp, st, ga) in enumerate(he.loop_variants()) if st > 0]


def setup(he, name, m, n, seed):
    ctx, o = pair(he, name)
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(m, n))
    y = rng.uniform(-1, 1, n)
    level = o.L - 1
    plan_o = layout.make_plan(m, n, o.slots)
    plan_g = he.Plan(m, n, o.slots)
    ctx.keygen(plan_o.rotation_steps)
    cts = o.encrypt_vector(y, plan_o, 2.0**40, nonce0=300)
    pts = o.encode_matrix(X, plan_o, level, ext=True)
    want = o.matmult(pts, cts, plan_o, hoisting="double")
    gcts = [ctx.ct_import(he.from_u64(c.data, ctx.device), level, 2.0**40) for c in cts]
    return ctx, o, plan_g, pts, gcts, want, level


@pytest.mark.parametrize("name,m,n", [("n32", 16, 8), ("n32", 100, 20), ("n32", 20, 100), ("n32", 17, 31),
                                      ("n1024_alpha2", 700, 300), ("n8192", 256, 1024)])
def test_fused_variants_bit_exact(he, name, m, n):
    """Every fused variant, pinned, on regimes with row and column blocks: bit-equal to the oracle."""
    ctx, o, plan, pts, gcts, want, level = setup(he, name, m, n, seed=m + 7 * n)
    for v in fused_variants(he):
        pm = ctx.ptmat_import(plan, he.from_u64(pts.reshape(-1), ctx.device), level, float(o.q[level]))
        pm.set_key_fusion(True, v)
        outs = ctx.matmult(plan, pm, gcts)
        kf = pm.key_fusion()
        assert kf["state"] == 1 and kf["variant"] == v
        for g, w in zip(outs, want):
            assert np.array_equal(he.as_u64(ctx.ct_export(g)), w.data), f"variant {v}"
        outs2 = ctx.matmult(plan, pm, gcts)  # second call on the built tables
        for g, w in zip(outs2, want):
            assert np.array_equal(he.as_u64(ctx.ct_export(g)), w.data), f"variant {v}, second call"


def test_policy_reuse_reencode_and_graph(he):
    """Mode 1 builds the tables on the second MatMult of an encoding (kept only when timed faster);
    re-encoding rebuilds them in stream order; a graph captured on the fused form replays to the
    same ciphertext; turning fusion off frees them and the two-level form gives the same bits."""
    import torch

    ctx, o = pair(he, "n8192")
    level = o.L - 1
    rng = np.random.default_rng(5)
    X1, X2 = rng.normal(size=(256, 1024)), rng.normal(size=(256, 1024))
    y = rng.uniform(-1, 1, 1024)
    plan = he.Plan(256, 1024, o.slots)
    ctx.keygen(plan.rotation_steps)
    ct = ctx.encrypt_vector(plan, torch.from_numpy(y).cuda(), 2.0**40, level, 77)
    ref = ctx.encode_matrix(plan, torch.from_numpy(X2).cuda(), level)
    ref.set_key_fusion(False)
    want2 = he.as_u64(ctx.ct_export(ctx.matmult(plan, ref, ct)[0]))

    ctx.set_key_fusion(1)
    pm = ctx.encode_matrix(plan, torch.from_numpy(X1).cuda(), level)
    ctx.matmult(plan, pm, ct)
    assert pm.key_fusion()["state"] == 0  # first use of the encoding: two-level form
    first = he.as_u64(ctx.ct_export(ctx.matmult(plan, pm, ct)[0]))
    kf = pm.key_fusion()
    assert kf["state"] in (1, -1) and kf["variant"] in fused_variants(he)
    pm.set_key_fusion(True, kf["variant"])  # pinned: used from the next call whatever the timing
    ctx.matmult(plan, pm, ct)
    assert pm.key_fusion()["state"] == 1
    assert np.array_equal(he.as_u64(ctx.ct_export(ctx.matmult(plan, pm, ct)[0])), first)

    ctx.encode_matrix(plan, torch.from_numpy(X2).cuda(), level, out=pm)  # tables rebuilt
    out = ctx.new_ct(level - 1)
    ctx.matmult(plan, pm, ct, [out])
    assert np.array_equal(he.as_u64(ctx.ct_export(out)), want2)

    fk = ctx.fork()  # graphs are captured on a non-default stream
    torch.cuda.synchronize()
    with torch.cuda.stream(fk.stream):
        g = he.Graph(fk, lambda: fk.matmult(plan, pm, ct, [out]))
        out.data.zero_()
        g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(he.as_u64(ctx.ct_export(out)), want2)

    pm.set_key_fusion(False)
    assert pm.key_fusion()["state"] == -1
    assert np.array_equal(he.as_u64(ctx.ct_export(ctx.matmult(plan, pm, ct)[0])), want2)
    ctx.set_key_fusion(1)
