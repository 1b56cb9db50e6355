"""Alg. 1 around the MatMult on the GPU: O1 with a plaintext operand, the slot mask and its
removal before the lazy rotate-and-sum, and the ciphertext rotate-and-sum that the lazy form
replaces.  Ciphertexts bit-exact against the oracle; decrypted results within tolerance of the
FP64 products."""
import numpy as np
import pytest

from oracle import ckks, layout

pytestmark = pytest.mark.gpu

TOL = 1e-4  # scale 2^40


@pytest.fixture(scope="module")
def he():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2405_00482_gb300 import he as mod

    return mod


def _ctx_pair(he, log_n, seed):
    qb, pb, d = [60, 40, 40], [60], 3
    return he.Context(log_n, qb, pb, d, seed), ckks.Oracle(log_n, qb, pb, d, seed)


@pytest.mark.parametrize("log_n", [5, 13])
def test_add_plain_bit_exact(he, log_n):
    ctx, o = _ctx_pair(he, log_n, 21)
    rng = np.random.default_rng(log_n)
    D, level = 2.0**40, 2
    a, w = rng.uniform(-1, 1, o.slots), rng.uniform(-1, 1, o.slots)
    ct = o.encrypt(o.encode(a, D, level), level, D, 7)
    pt = o.encode(w, D, level)
    want = o.add_plain(ct, pt).data
    gct = ctx.ct_import(he.from_u64(ct.data, ctx.device), level, D)
    gpt = ctx.pt_import(he.from_u64(pt, ctx.device), level, D)
    got = ctx.add_plain(gct, gpt)
    assert np.array_equal(he.as_u64(ctx.ct_export(got)), want)
    ctx.add_plain(gct, gpt, out=gct)  # in place
    assert np.array_equal(he.as_u64(ctx.ct_export(gct)), want)
    with pytest.raises(he.HEError) as e:
        ctx.add_plain(got, ctx.pt_import(he.from_u64(pt, ctx.device), level, 2.0**30))
    assert e.value.status == he.HE_ESCALE


@pytest.mark.parametrize("log_n,m,n", [(5, 4, 4), (5, 3, 5), (5, 1, 8), (5, 64, 4), (13, 256, 1024), (13, 16, 64)])
def test_ciphertext_ras_bit_exact(he, log_n, m, n):
    """MatMult then he_ras: every output ciphertext bit-equal to the oracle's; the gathered
    decryption equals X y."""
    import torch

    ctx, o = _ctx_pair(he, log_n, 22)
    rng = np.random.default_rng(m + n)
    X, y = rng.normal(size=(m, n)), rng.uniform(-1, 1, n)
    D, level = 2.0**40, 2
    po, pg = layout.make_plan(m, n, o.slots), he.Plan(m, n, o.slots)
    assert pg.ras_steps == layout.ras_steps(po)
    cts = o.encrypt_vector(y, po, D, nonce0=30)
    pts = o.encode_matrix(X, po, level, ext=True)
    outs = o.matmult(pts, cts, po)
    o.gen_rotation_keys(layout.ras_steps(po))
    want = [o.ras(c, po) for c in outs]
    ctx.keygen(sorted(set(po.rotation_steps) | set(layout.ras_steps(po))))
    pm = ctx.ptmat_import(pg, he.from_u64(pts.reshape(-1), ctx.device), level, float(o.q[level]))
    gouts = ctx.matmult(pg, pm, [ctx.ct_import(he.from_u64(c.data, ctx.device), level, D) for c in cts])
    got = [ctx.ras(pg, g) for g in gouts]
    for g, w in zip(got, want):
        assert np.array_equal(he.as_u64(ctx.ct_export(g)), w.data)
    slots = torch.stack([ctx.decrypt(g) for g in got])
    res = ctx.ras_decode(pg, slots).cpu().numpy()
    assert np.array_equal(res, layout.ras_decode(slots.cpu().numpy(), po))
    assert np.abs(res - X @ y).max() < TOL


def test_ras_missing_key(he):
    import torch

    ctx, o = _ctx_pair(he, 5, 23)
    plan = he.Plan(4, 4, o.slots)
    ct = ctx.encrypt(ctx.encode(torch.zeros(4, dtype=torch.float64, device="cuda"), 2.0**40, 2), 1)
    with pytest.raises(he.HEError) as e:
        ctx.ras(plan, ct)
    assert e.value.status == he.HE_EKEY


def test_masked_decode_matches_oracle_layout(he):
    import torch

    ctx, o = _ctx_pair(he, 13, 24)
    rng = np.random.default_rng(3)
    for m, n in [(256, 1024), (1024, 256), (300, 5000), (5000, 300)]:
        pg, po = he.Plan(m, n, o.slots), layout.make_plan(m, n, o.slots)
        S = rng.normal(size=(pg.row_blocks, o.slots))
        M = rng.uniform(-100, 100, size=S.shape)
        got = ctx.matmult_decode(pg, torch.from_numpy(S).cuda(), mask=torch.from_numpy(M).cuda()).cpu().numpy()
        assert np.allclose(got, layout.lazy_ras(S - M, po), rtol=0, atol=1e-9)


def test_vfl_linr_gradient_step_n8192(he):
    """Alg. 1 for P_A's gradient at N = 8192: [[d]] = [[u_A]] + (u_B - y), X_A^T [[d]], mask
    added, decrypted, removed, lazy RaS.  The masked ciphertext is bit-equal to the oracle's (same
    imported inputs); the GPU path from fp64 inputs gives X_A^T (u_A + u_B - y)."""
    import torch

    ctx, o = _ctx_pair(he, 13, 25)
    rng = np.random.default_rng(4)
    b, f = 1024, 256
    XA = rng.normal(size=(b, f))
    uA, uB, y = rng.normal(size=b), rng.normal(size=b), rng.uniform(-1, 1, b)
    D, level = 2.0**40, 2
    po, pg = layout.make_plan(f, b, o.slots), he.Plan(f, b, o.slots)
    ctx.keygen(po.rotation_steps)
    # oracle: every stage of the party's computation
    ct_uA = o.encrypt_vector(uA, po, D, nonce0=50)
    dv = layout.vector_slots(uB - y, po)
    pt_d = o.encode(dv[0], D, level)
    ct_d = o.add_plain(ct_uA[0], pt_d)
    pts = o.encode_matrix(XA.T, po, level, ext=True)
    out = o.matmult(pts, [ct_d], po)[0]
    mask = rng.uniform(-100, 100, o.slots)
    pt_mask = o.encode(mask, out.scale, out.level)
    masked = o.add_plain(out, pt_mask)
    # GPU from the same integer inputs: bit-exact
    g_d = ctx.add_plain(ctx.ct_import(he.from_u64(ct_uA[0].data, ctx.device), level, D),
                        ctx.pt_import(he.from_u64(pt_d, ctx.device), level, D))
    pm = ctx.ptmat_import(pg, he.from_u64(pts.reshape(-1), ctx.device), level, float(o.q[level]))
    g_out = ctx.matmult(pg, pm, [g_d])[0]
    g_masked = ctx.add_plain(g_out, ctx.pt_import(he.from_u64(pt_mask, ctx.device), out.level, out.scale))
    assert np.array_equal(he.as_u64(ctx.ct_export(g_masked)), masked.data)
    # GPU from fp64 inputs, every step in the library
    dev = ctx.device
    c_uA = ctx.encrypt(ctx.encode_vector(pg, torch.from_numpy(uA).to(dev), D, level)[0], 60)
    c_d = ctx.add_plain(c_uA, ctx.encode_vector(pg, torch.from_numpy(uB - y).to(dev), D, level)[0])
    pmx = ctx.encode_matrix(pg, torch.from_numpy(XA.T.copy()).to(dev), level)
    c_out = ctx.matmult(pg, pmx, [c_d])[0]
    mk = torch.from_numpy(mask).to(dev)
    c_masked = ctx.add_plain(c_out, ctx.encode(mk, c_out.scale, c_out.level))
    slots = torch.stack([ctx.decrypt(c_masked)])
    grad = ctx.matmult_decode(pg, slots, mask=mk[None]).cpu().numpy()
    want = XA.T @ (uA + uB - y)
    assert np.abs(grad - want).max() < TOL
    assert np.abs(ctx.matmult_decode(pg, slots).cpu().numpy() - want).max() > 1.0


@pytest.mark.parametrize("log_n,m,n", [(5, 4, 4), (5, 40, 8), (13, 256, 1024), (13, 1024, 256), (13, 9000, 64), (13, 300, 5000)])
def test_matmult_decrypt_equals_decrypt_then_decode(he, log_n, m, n):
    """he_matmult_decrypt (decoding and lazy RaS in one launch at N >= 2^10) gives the doubles of
    decrypt on every output then matmult_decode(_masked), bit for bit."""
    import torch

    ctx, o = _ctx_pair(he, log_n, 31)
    rng = np.random.default_rng(m + 7 * n)
    X, y = rng.normal(size=(m, n)), rng.uniform(-1, 1, n)
    D, level = 2.0**40, 2
    plan = he.Plan(m, n, o.slots)
    ctx.keygen(list(range(1, plan.m_prime)))
    pm = ctx.encode_matrix(plan, torch.from_numpy(X).cuda(), level)
    cts = ctx.encrypt_vector(plan, torch.from_numpy(y).cuda(), D, level, 5)
    outs = ctx.matmult(plan, pm, cts)
    slots = torch.stack([ctx.decrypt(c) for c in outs])
    mask = torch.from_numpy(rng.uniform(-10, 10, size=(plan.row_blocks, o.slots))).cuda()
    for mk in (None, mask):
        want = ctx.matmult_decode(plan, slots, mask=mk).cpu().numpy()
        got = ctx.matmult_decrypt(plan, outs, mask=mk).cpu().numpy()
        assert np.array_equal(got, want)
    assert np.abs(ctx.matmult_decrypt(plan, outs).cpu().numpy() - X @ y).max() < TOL
    with pytest.raises(he.HEError):
        ctx.matmult_decrypt(plan, outs[:-1] if len(outs) > 1 else outs + outs)
