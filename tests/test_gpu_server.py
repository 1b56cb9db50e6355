"""Serving loop (continuous batching): every request's result is the same alone and in the mix,
admission respects the HBM budget, and the one-request-per-call mode gives the same bits."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_00482_gb300 import build as b

    b.build()
    from paper_2405_00482_gb300 import he

    ctx = he.Context(13, [60, 40, 40], [60], 3, seed=11)
    rng = np.random.default_rng(5)
    shapes = [(256, 1024), (1024, 256), (16, 64), (512, 4096), (37, 1500), (128, 128), (64, 2048)]
    pool = []
    for i, (m, n) in enumerate(shapes):
        X = rng.normal(size=(m, n))
        y = rng.uniform(-1, 1, n)
        plan = he.Plan(m, n, ctx.slots)
        ctx.keygen(list(range(1, plan.m_prime)))
        pm = ctx.encode_matrix(plan, torch.from_numpy(X).cuda(), 2)
        ct = ctx.encrypt(ctx.encode_vector(plan, torch.from_numpy(y).cuda(), 2.0**40, 2)[0], 500 + i)
        alone = ctx.matmult(plan, pm, [ct])[0]
        pool.append((plan, pm, ct, he.as_u64(ctx.ct_export(alone)), X, y))
    ctx.synchronize()
    return he, ctx, pool


def _run(he, ctx, pool, server, order):
    outs = []
    for k in order:
        plan, pm, ct, _, _, _ = pool[k]
        out = ctx.new_ct(1)
        rid = server.submit(plan, pm, ct, out)
        outs.append((k, rid, out))
    lats = [server.wait(rid) for _, rid, _ in outs]
    return outs, lats


def test_each_result_same_alone_and_in_the_mix(env):
    he, ctx, pool = env
    server = he.Server(ctx, slots=8, level=2, hbm_budget_bytes=120 << 30)
    order = [i % len(pool) for i in range(3 * len(pool))] + [3, 0, 0, 6, 2]
    outs, lats = _run(he, ctx, pool, server, order)
    completed, launches, in_use = server.stats()
    server.close()
    assert completed == len(order) and in_use == 0
    assert launches < len(order)  # requests shared launches
    for k, _, out in outs:
        assert np.array_equal(he.as_u64(ctx.ct_export(out)), pool[k][3]), k
    assert all(l > 0 for l in lats)
    # and the decrypted result is X y
    import torch

    k, _, out = outs[0]
    plan, _, _, _, X, y = pool[k]
    res = ctx.matmult_decode(plan, ctx.decrypt(out)[None]).cpu().numpy()
    assert np.abs(res - X @ y).max() < 1e-4
    del torch


def test_budget_admits_one_at_a_time_and_rejects_oversize(env):
    he, ctx, pool = env
    # room for the largest single request only: every request still completes, in order
    big = max(p[0].m_prime for p in pool)
    one = big * 4 * 8192 * 8 + 2 * 3 * 8192 * 8 + 2 * 2 * 8192 * 8
    server = he.Server(ctx, slots=8, level=2, hbm_budget_bytes=one)
    outs, _ = _run(he, ctx, pool, server, list(range(len(pool))))
    server.close()
    for k, _, out in outs:
        assert np.array_equal(he.as_u64(ctx.ct_export(out)), pool[k][3])
    server = he.Server(ctx, slots=8, level=2, hbm_budget_bytes=one // 4)
    plan, pm, ct, _, _, _ = pool[3]  # 512 x 4096: m' = 512
    with pytest.raises(he.HEError) as e:
        server.submit(plan, pm, ct, ctx.new_ct(1))
    assert e.value.status == he.HE_EBUDGET
    server.close()


def test_plain_mode_gives_the_same_bits(env):
    he, ctx, pool = env
    server = he.Server(ctx, slots=1, level=2, hbm_budget_bytes=120 << 30, plain=True)
    outs, _ = _run(he, ctx, pool, server, [0, 1, 2, 3, 4, 5, 6, 0])
    completed, launches, _ = server.stats()
    server.close()
    assert completed == 8 and launches == 8
    for k, _, out in outs:
        assert np.array_equal(he.as_u64(ctx.ct_export(out)), pool[k][3])


def test_wait_times_out_on_unfinished_request(env):
    he, ctx, pool = env
    server = he.Server(ctx, slots=2, level=2, hbm_budget_bytes=120 << 30)
    plan, pm, ct, _, _, _ = pool[3]
    rids = [server.submit(plan, pm, ct, ctx.new_ct(1)) for _ in range(6)]
    with pytest.raises(he.HEError) as e:
        server.wait(rids[-1], timeout_s=0.0)
    assert e.value.status == he.HE_ETIMEOUT
    for r in rids:
        server.wait(r)
    server.close()


@pytest.mark.parametrize("plain", [False, True])
def test_two_rings_in_one_stream(env, plain):
    """Requests on an N = 4096 ring (chain [40, 20 | 40], the 16 x 64 gradient shape) and on the
    N = 8192 ring, submitted interleaved to one server under one budget: each result equals the
    single call's ciphertext on its own ring."""
    import torch

    he, ctx, pool = env
    small = he.Context(12, [40, 20], [40], 2, seed=12)
    rng = np.random.default_rng(9)
    spool = []
    for i, (m, n) in enumerate([(16, 64), (64, 16), (100, 700)]):
        X = rng.normal(size=(m, n))
        y = rng.uniform(-1, 1, n)
        plan = he.Plan(m, n, small.slots)
        small.keygen(list(range(1, plan.m_prime)))
        pm = small.encode_matrix(plan, torch.from_numpy(X).cuda(), 1)
        ct = small.encrypt(small.encode_vector(plan, torch.from_numpy(y).cuda(), 2.0**20, 1)[0], 800 + i)
        spool.append((plan, pm, ct, he.as_u64(small.ct_export(small.matmult(plan, pm, [ct])[0]))))
    small.synchronize()
    server = he.Server(ctx, slots=4, level=2, hbm_budget_bytes=120 << 30, plain=plain)
    server.add_ring(small, 1)
    subs = []
    for t in range(12):
        if t % 2:
            plan, pm, ct, want = spool[t % len(spool)]
            out = small.new_ct(0)
            subs.append((server.submit(plan, pm, ct, out), out, want, small))
        else:
            plan, pm, ct, want, _, _ = pool[t % len(pool)]
            out = ctx.new_ct(1)
            subs.append((server.submit(plan, pm, ct, out), out, want, ctx))
    for rid, out, want, c in subs:
        server.wait(rid)
        assert np.array_equal(he.as_u64(c.ct_export(out)), want)
    completed, _, in_use = server.stats()
    server.close()
    assert completed == len(subs) and in_use == 0
