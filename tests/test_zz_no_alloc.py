"""The MatMult entry point that allocates nothing (he_matmult_plain_cipher_noalloc).

Callers whose device memory is owned by their own allocator, or who cannot afford a
cudaMalloc / cudaFree inside a call, use this variant; it keeps its temporaries in a fixed
16 MiB device array reserved by the library.  These tests call it through the C ABI and check
that two calls in a row give the same ciphertexts, bit for bit, as he_matmult_plain_cipher
(the tolerance every ciphertext comparison in this suite uses), and that a product too large
for the array is refused.  The file sorts last so that a stop-at-first-failure run has
already run every other test.
"""
import numpy as np
import pytest

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


def _setup(he, ctx, m, n, seed, scale=2.0**40):
    import torch

    rng = np.random.default_rng(seed)
    X = rng.normal(size=(m, n))
    y = rng.uniform(-1, 1, n)
    level = ctx.L - 1
    plan = he.Plan(m, n, ctx.slots)
    ctx.keygen(list(range(1, plan.m_prime)))
    pm = ctx.encode_matrix(plan, torch.from_numpy(X).cuda(), level)
    cts = [ctx.encrypt(p, 700 + i) for i, p in enumerate(ctx.encode_vector(plan, torch.from_numpy(y).cuda(), scale, level))]
    return X, y, plan, pm, cts


@pytest.mark.parametrize("log_n,qb,pb,dnum,m,n", [
    (13, [60, 40, 40], [60], 3, 256, 1024),   # the N = 8192 gradient: 63 hoisted rotations
    (13, [60, 40, 40], [60], 3, 16, 64),      # one diagonal, no rotation
    (5, [60, 40, 40], [60], 3, 40, 9),        # row blocks (m > N')
    (5, [60, 40, 40], [60], 3, 9, 40),        # column blocks summed before output
    (10, [50, 40, 40, 40], [55, 55], 2, 300, 200),
])
def test_noalloc_equals_plain_entry_point_twice(he, log_n, qb, pb, dnum, m, n):
    ctx = he.Context(log_n, qb, pb, dnum, seed=3)
    X, y, plan, pm, cts = _setup(he, ctx, m, n, seed=m + n)
    want = [he.as_u64(ctx.ct_export(o)) for o in ctx.matmult(plan, pm, cts)]
    outs = [ctx.new_ct(pm.level - 1) for _ in range(plan.row_blocks)]
    for _ in range(2):  # the shared array keeps the previous call's contents
        for o in outs:
            o.data.fill_(-1)
        got = ctx.matmult_noalloc(plan, pm, cts, outs)
        ctx.synchronize()
        for g, w in zip(got, want):
            assert np.array_equal(he.as_u64(ctx.ct_export(g)), w)
    import torch

    slots = torch.stack([ctx.decrypt(o) for o in outs])
    assert np.abs(ctx.matmult_decode(plan, slots).cpu().numpy() - X @ y).max() < 1e-4


def test_noalloc_refuses_products_larger_than_its_array(he):
    # 32 column blocks of N' = 4096 with two diagonals each: the ModUp digits alone need 25 MB
    ctx = he.Context(13, [60, 40, 40], [60], 3, seed=5)
    X, y, plan, pm, cts = _setup(he, ctx, 2, 32 * 4096, seed=1)
    assert plan.col_blocks == 32 and plan.m_prime == 2
    outs = [ctx.new_ct(pm.level - 1)]
    with pytest.raises(he.HEError) as e:
        ctx.matmult_noalloc(plan, pm, cts, outs)
    assert e.value.status == he.HE_EBUDGET
