"""The NTT forms for launches of many limb-polys (one CTA, a 2-CTA cluster with one stage through
distributed shared memory, or two phases of column and row sub-transforms) give the same
residues: encoded matrices, plaintext import and export against the oracle's coefficient-form
plaintexts (and random residues), and a MatMult, at N = 4096, 8192, 16384."""
import numpy as np
import pytest

from oracle import ckks, layout

pytestmark = pytest.mark.gpu

PARAMS = {12: (12, [40, 20], [40], 2), 13: (13, [60, 40, 40], [60], 3), 14: (14, [60] + [40] * 6, [60, 60, 60], 3)}


@pytest.fixture(scope="module")
def he():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_00482_gb300 import build as b

    b.build()
    from paper_2405_00482_gb300 import he as h

    return h


@pytest.mark.parametrize("log_n", [12, 13, 14])
def test_forms_agree_with_each_other_and_the_oracle(he, log_n):
    import torch

    lg, qb, pb, d = PARAMS[log_n]
    ctx = he.Context(lg, qb, pb, d, seed=21)
    o = ckks.Oracle(lg, qb, pb, d, seed=21)
    level = o.L - 1
    m, n = ctx.slots // 8, ctx.slots  # m' = N'/8 diagonals: many limb-polys per launch
    rng = np.random.default_rng(log_n)
    X = rng.normal(size=(m, n))
    y = rng.uniform(-1, 1, n)
    plan = he.Plan(m, n, ctx.slots)
    oplan = layout.make_plan(m, n, o.slots)
    ctx.keygen(plan.rotation_steps)
    pts = o.encode_matrix(X[:, :], oplan, level, ext=True) if log_n == 12 else None
    exports, outs = [], []
    cts = ctx.encrypt_vector(plan, torch.from_numpy(y).cuda(), 2.0**40 if log_n > 12 else 2.0**20, level, 3)
    # random canonical residues in the plaintext batch's layout [count][ext][N]
    count, ext = plan.row_blocks * plan.col_blocks * plan.m_prime, level + 1 + len(pb)
    primes = [o.q[i] for i in range(level + 1)] + [o.p[i] for i in range(len(pb))]
    rnd = np.stack([rng.integers(0, q, size=(count, ctx.n), dtype=np.uint64) for q in primes], axis=1)
    for form in range(he.HE_NTT_FORMS):
        ctx.set_ntt_form(form)
        pm = ctx.encode_matrix(plan, torch.from_numpy(X).cuda(), level)
        exports.append(pm.export())
        outs.append(ctx.ct_export(ctx.matmult(plan, pm, cts)[0]))
        if pts is not None:  # import / export of the oracle's plaintexts round-trips in this form
            pmi = ctx.ptmat_import(plan, he.from_u64(pts.reshape(-1), ctx.device), level, float(o.q[level]))
            assert np.array_equal(he.as_u64(pmi.export()).reshape(pts.shape), pts)
        pmr = ctx.ptmat_import(plan, he.from_u64(rnd.reshape(-1), ctx.device), level, 1.0)
        assert np.array_equal(he.as_u64(pmr.export()).reshape(rnd.shape), rnd), f"form {form}"
    for f in range(1, he.HE_NTT_FORMS):
        assert torch.equal(exports[0], exports[f]), f"form {f}"
        assert torch.equal(outs[0], outs[f]), f"form {f}"
    ctx.set_ntt_form(-1)
