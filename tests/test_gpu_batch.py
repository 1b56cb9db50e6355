"""Batched MatMult (one persistent work-queue kernel for all jobs, CUDA graph) against the
single-call path and the oracle: bit-identical ciphertexts, on uneven shapes."""
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


def _jobs(he, ctx, shapes, seed, scale):
    import torch

    rng = np.random.default_rng(seed)
    level = ctx.L - 1
    out = []
    for i, (m, n) in enumerate(shapes):
        X = rng.normal(size=(m, n))
        y = rng.uniform(-1, 1, n)
        plan = he.Plan(m, n, ctx.slots)
        ctx.keygen(list(range(1, plan.m_prime)))
        pm = ctx.encode_matrix(plan, torch.from_numpy(X).cuda(), level)
        ct = ctx.encrypt(ctx.encode_vector(plan, torch.from_numpy(y).cuda(), scale, level)[0], 300 + i)
        out.append((X, y, plan, pm, ct))
    return out


@pytest.mark.parametrize("log_n,qb,pb,dnum", [(5, [60, 40, 40], [60], 3), (10, [50, 40, 40, 40], [55, 55], 2)])
def test_batch_equals_single_calls_small(he, log_n, qb, pb, dnum):
    import torch

    ctx = he.Context(log_n, qb, pb, dnum, seed=4)
    n2 = ctx.slots
    shapes = [(1, 1), (3, 5), (n2, n2), (n2 // 2, 7), (2, n2), (n2, 2), (5, n2 // 4)]
    jobs = _jobs(he, ctx, shapes, 1, 2.0**40)
    b = he.Batch(ctx, [j[2] for j in jobs], [j[3] for j in jobs])
    for rep in range(2):  # first run captures the graph, the second replays it
        outs = b.run([j[4] for j in jobs])
        for (X, y, plan, pm, ct), o in zip(jobs, outs):
            single = ctx.matmult(plan, pm, [ct])[0]
            assert np.array_equal(he.as_u64(ctx.ct_export(o)), he.as_u64(ctx.ct_export(single)))
            res = ctx.matmult_decode(plan, ctx.decrypt(o)[None]).cpu().numpy()
            assert np.abs(res - X @ y).max() < 1e-4
    del torch


def test_batch_matches_oracle_n8192(he):
    """Three uneven jobs at N = 8192, each compared with the oracle bit for bit."""
    log_n, qb, pb, d = 13, [60, 40, 40], [60], 3
    ctx = he.Context(log_n, qb, pb, d, seed=0)
    o = ckks.Oracle(log_n, qb, pb, d, seed=0)
    level, scale = 2, 2.0**40
    shapes = [(16, 128), (32, 512), (64, 256)]
    rng = np.random.default_rng(2)
    plans, pms, cts, wants = [], [], [], []
    for i, (m, n) in enumerate(shapes):
        X = rng.normal(size=(m, n))
        y = rng.uniform(-1, 1, n)
        po = layout.make_plan(m, n, o.slots)
        pg = he.Plan(m, n, o.slots)
        ctx.keygen(po.rotation_steps)
        c = o.encrypt_vector(y, po, scale, nonce0=40 + i)
        pts = o.encode_matrix(X, po, level, ext=True)
        wants.append(o.matmult(pts, c, po)[0].data)
        plans.append(pg)
        pms.append(ctx.ptmat_import(pg, he.from_u64(pts.reshape(-1), ctx.device), level, float(o.q[level])))
        cts.append(ctx.ct_import(he.from_u64(c[0].data, ctx.device), level, scale))
    b = he.Batch(ctx, plans, pms)
    outs = b.run(cts)
    for out, want in zip(outs, wants):
        assert np.array_equal(he.as_u64(ctx.ct_export(out)), want)


def test_batch_rejects_partitioned_plans(he):
    import torch

    ctx = he.Context(5, [60, 40, 40], [60], 3, seed=1)
    plan = he.Plan(64, 4, ctx.slots)  # m > N': two output ciphertexts
    ctx.keygen(list(range(1, plan.m_prime)))
    pm = ctx.encode_matrix(plan, torch.zeros((64, 4), dtype=torch.float64, device="cuda"), 2)
    with pytest.raises(he.HEError) as e:
        he.Batch(ctx, [plan], [pm])
    assert e.value.status == he.HE_EINVAL


@pytest.mark.parametrize("form", [0, 1])
def test_batch_stage_forms_bit_identical(he, form):
    """The batch's ModUp / ModDown / rescale as one CTA per limb-poly (form 0) or as clusters
    (form 1) give the single calls' ciphertexts bit for bit, at N = 8192 with an m' = 1 job and
    uneven shapes; the first run's tuning reports both forms' times."""
    ctx = he.Context(13, [60, 40, 40], [60], 3, seed=8)
    shapes = [(16, 64), (256, 1024), (100, 300), (4096, 2), (7, 4000)]
    jobs = _jobs(he, ctx, shapes, 3, 2.0**40)
    b = he.Batch(ctx, [j[2] for j in jobs], [j[3] for j in jobs])
    b.run([j[4] for j in jobs])  # tunes the loop variant, then the stage form
    t = b.stage_tuning()
    assert t["form"] in (0, 1) and all(ms > 0 for ms in t["form_ms"])
    b.set_stage_form(form)
    for rep in range(2):
        outs = b.run([j[4] for j in jobs])
        for (X, y, plan, pm, ct), o in zip(jobs, outs):
            single = ctx.matmult(plan, pm, [ct])[0]
            assert np.array_equal(he.as_u64(ctx.ct_export(o)), he.as_u64(ctx.ct_export(single)))
