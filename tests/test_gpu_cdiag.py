"""VFL-NN forward pass (Alg. 3) with the encrypted activation matrix diagonally encoded: GPU
ciphertexts bit-exact against the oracle (same plaintexts, same encryption streams), and the
decrypted product within tolerance of A W, up to the N = 16384 configuration."""
import numpy as np
import pytest

from oracle import ckks, layout

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def he():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_00482_gb300 import build as b

    b.build()
    from paper_2405_00482_gb300 import he as h

    return h


def _bit_exact_case(he, log_n, qb, pb, dnum, m, n, K, n_ct=None, seed=0):
    import torch

    ctx = he.Context(log_n, qb, pb, dnum, seed=seed)
    o = ckks.Oracle(log_n, qb, pb, dnum, seed=seed)
    rng = np.random.default_rng(m * 31 + n + K)
    A = rng.uniform(-1, 1, (m, n))
    W = rng.normal(size=(n, K)) / np.sqrt(n)
    level, scale = len(qb) - 1, 2.0**40
    qs = float(o.q[level])
    E = layout.cipher_diagonals(A, o.slots)
    n_ct = n_ct or E.shape[0]
    cts = [o.encrypt(o.encode(E[i], scale, level), level, scale, nonce=i) for i in range(n_ct)]
    pts = [o.encode(layout.weight_slots(W[:, k], o.slots), qs, level) for k in range(K)]
    want = ckks.cipher_diag_matmult(o, cts, pts, qs)
    Wm = he.WeightMatrix(ctx, torch.from_numpy(W).cuda(), level)
    gcts = [ctx.ct_import(he.from_u64(c.data, ctx.device), level, scale) for c in cts]
    got = ctx.cdiag_matmult(Wm, gcts)
    for g, w in zip(got, want):
        assert g.level == level - 1
        assert np.array_equal(he.as_u64(ctx.ct_export(g)), w.data)
    return ctx, o, A, W, got


@pytest.mark.parametrize("m,n,K", [(32, 8, 3), (8, 32, 2), (16, 16, 9), (32, 32, 17)])
def test_cdiag_bit_exact_small_ring(he, m, n, K):
    _bit_exact_case(he, 6, [60, 40, 40], [60], 3, m, n, K)


def test_cdiag_bit_exact_n16384_config(he):
    """N = 16384, Q = [60, 40 x 6], P = [60, 60, 60]: 8 of the 256 diagonals, 2 columns."""
    _bit_exact_case(he, 14, [60] + [40] * 6, [60, 60, 60], 3, 4096, 256, 2, n_ct=8)


def test_cdiag_end_to_end_n16384(he):
    """A 4096 x 256 ~ U[-1,1] encrypted as 256 diagonals, W 256 x 128 ~ N(0, 1/256): Z = A W."""
    import torch

    ctx = he.Context(14, [60] + [40] * 6, [60, 60, 60], 3, seed=1)
    rng = np.random.default_rng(3)
    A = rng.uniform(-1, 1, (4096, 256))
    W = rng.normal(scale=1 / 16, size=(256, 128))
    level, scale = 6, 2.0**40
    pts = ctx.cdiag_encode_matrix(torch.from_numpy(A).cuda(), scale, level)
    cts = [ctx.encrypt(p, 10 + i) for i, p in enumerate(pts)]
    Wm = he.WeightMatrix(ctx, torch.from_numpy(W).cuda(), level)
    outs = ctx.cdiag_matmult(Wm, cts)
    slots = torch.stack([ctx.decrypt(c) for c in outs])
    Z = ctx.cdiag_decode(4096, 256, slots).cpu().numpy()
    assert np.abs(Z - A @ W).max() < 1e-4


@pytest.mark.parametrize("log_n,qb,pb,dnum,m,n", [(6, [60, 40, 40], [60], 3, 32, 8), (6, [60, 40, 40], [60], 3, 8, 32),
                                                  (14, [60] + [40] * 6, [60, 60, 60], 3, 16, 8)])
def test_transpose_bit_exact(he, log_n, qb, pb, dnum, m, n):
    """Eq. 5 conversion, bit-exact against the oracle (N = 16384 with dnum = 3 in the last case)."""
    ctx = he.Context(log_n, qb, pb, dnum, seed=2)
    o = ckks.Oracle(log_n, qb, pb, dnum, seed=2)
    rng = np.random.default_rng(m * n)
    A = rng.uniform(-1, 1, (m, n))
    level, scale = len(qb) - 1, 2.0**40
    E = layout.cipher_diagonals(A, o.slots)
    cts = [o.encrypt(o.encode(E[i], scale, level), level, scale, nonce=i) for i in range(E.shape[0])]
    steps = [r for _, r in layout.transpose_rotations(m, n) if r]
    assert sorted(set(steps)) == he.Context.cdiag_transpose_steps(m, n)
    o.gen_rotation_keys(steps)
    ctx.keygen(steps)
    want = ckks.transpose_diagonals(o, cts, m, n)
    got = ctx.cdiag_transpose([ctx.ct_import(he.from_u64(c.data, ctx.device), level, scale) for c in cts], m, n)
    for g, w in zip(got, want):
        assert np.array_equal(he.as_u64(ctx.ct_export(g)), w.data)


def test_backward_pass_n16384(he):
    """Alg. 4 at N = 16384: [[A^T]] by conversion from [[A]]'s 256 diagonals, times D^T (4096 x 128)."""
    import torch

    ctx = he.Context(14, [60] + [40] * 6, [60, 60, 60], 3, seed=4)
    rng = np.random.default_rng(8)
    m, n, K = 4096, 256, 128
    A = rng.uniform(-1, 1, (m, n))
    Dt = rng.normal(scale=1 / 64, size=(m, K))
    level, scale = 6, 2.0**40
    cts = [ctx.encrypt(p, 20 + i) for i, p in enumerate(ctx.cdiag_encode_matrix(torch.from_numpy(A).cuda(), scale, level))]
    ctx.keygen(he.Context.cdiag_transpose_steps(m, n))
    tcts = ctx.cdiag_transpose(cts, m, n)
    Wm = he.WeightMatrix(ctx, torch.from_numpy(Dt).cuda(), level)
    outs = ctx.cdiag_matmult(Wm, tcts)
    slots = torch.stack([ctx.decrypt(c) for c in outs])
    Z = ctx.cdiag_decode(n, m, slots).cpu().numpy()
    assert np.abs(Z - A.T @ Dt).max() < 1e-4
