"""he_ctx_fork: a context on another stream sharing tables and Galois keys.  Products run on
the parent and the fork at the same time give the ciphertexts one context gives alone; keys
made on either context serve both; the family's tables outlive whichever context goes first."""
import numpy as np
import pytest

from paper_2405_00482_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def he():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2405_00482_gb300 import he as mod

    return mod


def _product(ctx, he, plan, M, v, level, nonce):
    import torch

    P = inputs.PARAMS_N8192
    pm = ctx.encode_matrix(plan, M, level)
    ct = ctx.encrypt(ctx.encode_vector(plan, v, P.scale, level)[0], nonce)
    out = ctx.matmult(plan, pm, [ct])[0]
    return out, torch.stack([ctx.decrypt(out)]), pm


def test_fork_concurrent_products_bit_exact(he):
    import torch

    P = inputs.PARAMS_N8192
    X, r, w = inputs.gradient_and_forward_n8192(seed=3)
    dev = torch.device("cuda")
    dXT, dX = torch.from_numpy(np.ascontiguousarray(X.T)).to(dev), torch.from_numpy(X).to(dev)
    dr, dw = torch.from_numpy(r).to(dev), torch.from_numpy(w).to(dev)
    pg, pf = he.Plan(256, 1024, P.slots), he.Plan(1024, 256, P.slots)
    steps = sorted(set(range(1, pg.m_prime)) | set(range(1, pf.m_prime)))
    # one context, sequential
    solo = he.Context(P.log_n, list(P.q_bits), list(P.p_bits), P.dnum, seed=9)
    solo.keygen(steps)
    want_g, _, _ = _product(solo, he, pg, dXT, dr, P.top, 4)
    want_f, _, _ = _product(solo, he, pf, dX, dw, P.top, 5)
    solo.synchronize()
    # parent + fork, the two products issued on two streams
    ctx = he.Context(P.log_n, list(P.q_bits), list(P.p_bits), P.dnum, seed=9)
    ctx.keygen(steps[: len(steps) // 2])
    fork = ctx.fork()
    fork.keygen(steps)  # the rest, made on the fork, seen by the parent
    fork.synchronize()
    main = torch.cuda.current_stream()
    fork.stream.wait_stream(main)
    got_g, sg, _ = _product(ctx, he, pg, dXT, dr, P.top, 4)
    with torch.cuda.stream(fork.stream):
        got_f, sf, _ = _product(fork, he, pf, dX, dw, P.top, 5)
    main.wait_stream(fork.stream)
    assert np.array_equal(he.as_u64(ctx.ct_export(got_g)), he.as_u64(solo.ct_export(want_g)))
    assert np.array_equal(he.as_u64(ctx.ct_export(got_f)), he.as_u64(solo.ct_export(want_f)))
    res_g = ctx.matmult_decode(pg, sg).cpu().numpy()
    res_f = ctx.matmult_decode(pf, sf).cpu().numpy()
    assert np.abs(res_g - X.T @ r).max() < 1e-4
    assert np.abs(res_f - X @ w).max() < 1e-4
    assert fork.launch_count() > 0


def test_fork_outlives_parent(he):
    import torch

    P = inputs.PARAMS_N8192
    ctx = he.Context(P.log_n, list(P.q_bits), list(P.p_bits), P.dnum, seed=2)
    ctx.keygen([1, 5])
    fork = ctx.fork()
    ct = ctx.encrypt(ctx.encode(torch.linspace(-1, 1, P.slots, dtype=torch.float64, device="cuda"), P.scale, P.top), 1)
    want = he.as_u64(ctx.ct_export(ctx.rotate(ct, 5)))
    del ctx  # tables and keys stay with the fork
    torch.cuda.synchronize()
    with torch.cuda.stream(fork.stream):
        got = fork.rotate(ct, 5)
    fork.synchronize()
    assert np.array_equal(he.as_u64(fork.ct_export(got)), want)
    with pytest.raises(he.HEError) as e:
        fork.rotate(ct, 3)
    assert e.value.status == he.HE_EKEY


def test_ptmat_shared_in_family_foreign_rejected(he):
    """A plaintext matrix encoded on the fork serves the parent; another family's is refused."""
    import torch

    P = inputs.PARAMS_N8192
    ctx = he.Context(P.log_n, list(P.q_bits), list(P.p_bits), P.dnum, seed=2)
    plan = he.Plan(64, 64, P.slots)
    ctx.keygen(list(range(1, plan.m_prime)))
    fork = ctx.fork(torch.cuda.current_stream())
    M = torch.from_numpy(np.random.default_rng(1).normal(size=(64, 64))).cuda()
    y = torch.from_numpy(np.random.default_rng(2).uniform(-1, 1, 64)).cuda()
    pm_fork = fork.encode_matrix(plan, M, P.top)
    pm_ctx = ctx.encode_matrix(plan, M, P.top)
    ct = ctx.encrypt(ctx.encode_vector(plan, y, P.scale, P.top)[0], 1)
    a = he.as_u64(ctx.ct_export(ctx.matmult(plan, pm_fork, [ct])[0]))
    b = he.as_u64(ctx.ct_export(fork.matmult(plan, pm_ctx, [ct])[0]))
    assert np.array_equal(a, b)
    other = he.Context(P.log_n, list(P.q_bits), list(P.p_bits), P.dnum, seed=2)
    other.keygen(list(range(1, plan.m_prime)))
    with pytest.raises(he.HEError) as e:
        other.matmult(plan, pm_ctx, [ct])
    assert e.value.status == he.HE_EINVAL
