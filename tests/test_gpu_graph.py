"""he.Graph: library calls captured into one CUDA graph on a context and its fork.  Encryption
under a device-resident nonce equals encryption under the same integer nonce; each replay
reads the nonce and inputs the buffers hold at that time and gives the eager call's ciphertext."""
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


def test_device_nonce_equals_int_nonce(he):
    import torch

    P = inputs.PARAMS_N8192
    ctx = he.Context(P.log_n, list(P.q_bits), list(P.p_bits), P.dnum, seed=4)
    pt = ctx.encode(torch.linspace(-1, 1, P.slots, dtype=torch.float64, device="cuda"), P.scale, P.top)
    nb = torch.tensor([123456789012, 7], dtype=torch.int64, device="cuda")
    for k, v in ((0, 123456789012), (1, 7)):
        a = he.as_u64(ctx.ct_export(ctx.encrypt(pt, nb[k:k + 1])))
        b = he.as_u64(ctx.ct_export(ctx.encrypt(pt, v)))
        assert np.array_equal(a, b)
    with pytest.raises(ValueError):
        ctx.encrypt(pt, nb)  # two elements


def test_graph_replays_match_eager(he):
    import torch

    P = inputs.PARAMS_N8192
    X, r, w = inputs.gradient_and_forward_n8192(seed=5)
    dev = torch.device("cuda")
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        ctx = he.Context(P.log_n, list(P.q_bits), list(P.p_bits), P.dnum, seed=6)
        fork = ctx.fork()
        pg, pf = he.Plan(256, 1024, P.slots), he.Plan(1024, 256, P.slots)
        ctx.keygen(sorted(set(range(1, pg.m_prime)) | set(range(1, pf.m_prime))))
        dM = [torch.from_numpy(np.ascontiguousarray(X.T)).to(dev), torch.from_numpy(X).to(dev)]
        dv = [torch.from_numpy(r).to(dev), torch.from_numpy(w).to(dev)]
        pms = [ctx.encode_matrix(pg, dM[0], P.top)]
        with torch.cuda.stream(fork.stream):
            pms.append(fork.encode_matrix(pf, dM[1], P.top))
        fork.synchronize()
        pts = [ctx.new_pt(P.top), ctx.new_pt(P.top)]
        cts = [ctx.new_ct(P.top), ctx.new_ct(P.top)]
        outs = [[ctx.new_ct(P.top - 1)], [ctx.new_ct(P.top - 1)]]
        nonce = torch.tensor([100, 101], dtype=torch.int64, device=dev)

        def prod(c, k, plan):
            c.encode_matrix(plan, dM[k], P.top, out=pms[k])
            c.encode_vector(plan, dv[k], P.scale, P.top, outs=[pts[k]])
            c.encrypt(pts[k], nonce[k:k + 1], out=cts[k])
            c.matmult(plan, pms[k], [cts[k]], outs[k])

        def step():
            fork.stream.wait_stream(side)
            prod(ctx, 0, pg)
            with torch.cuda.stream(fork.stream):
                prod(fork, 1, pf)
            side.wait_stream(fork.stream)
            nonce.add_(2)

        g = he.Graph(ctx, step, forks=[fork])  # eager run with nonces 100/101, capture
        assert g.launches > 10
        nonce.copy_(torch.tensor([500, 501]))
        got = []
        for _ in range(2):
            g.replay()
            got.append([he.as_u64(ctx.ct_export(o[0])) for o in outs])
        side.synchronize()
        assert int(nonce[0]) == 504
    # eager reference on a fresh context with the same seed
    ref = he.Context(P.log_n, list(P.q_bits), list(P.p_bits), P.dnum, seed=6)
    ref.keygen(sorted(set(range(1, pg.m_prime)) | set(range(1, pf.m_prime))))
    for rep, base in enumerate((500, 502)):
        for k, plan in ((0, pg), (1, pf)):
            pm = ref.encode_matrix(plan, dM[k], P.top)
            ct = ref.encrypt(ref.encode_vector(plan, dv[k], P.scale, P.top)[0], base + k)
            want = he.as_u64(ref.ct_export(ref.matmult(plan, pm, [ct])[0]))
            assert np.array_equal(got[rep][k], want)
    assert not np.array_equal(got[0][0], got[1][0])  # fresh randomness on each replay


def test_graph_needs_non_default_stream(he):
    import torch

    P = inputs.PARAMS_SMALL
    ctx = he.Context(P.log_n, list(P.q_bits), list(P.p_bits), P.dnum, seed=1, stream=torch.cuda.default_stream())
    with pytest.raises(ValueError):
        he.Graph(ctx, lambda: None)


@pytest.mark.parametrize("log_n,m,n", [(5, 4, 40), (5, 8, 8), (13, 256, 1024), (13, 1024, 256), (13, 64, 9000)])
def test_encrypt_vector_equals_encode_then_encrypt(he, log_n, m, n):
    """he_encrypt_vector (encoded coefficients joined to the error before its NTT at N >= 2^10)
    gives the ciphertexts of encode_vector then encrypt under nonce + c, bit for bit; likewise
    with the nonces in device memory."""
    import torch

    qb, pb, d = [60, 40, 40], [60], 3
    ctx = he.Context(log_n, qb, pb, d, seed=8)
    plan = he.Plan(m, n, ctx.slots)
    y = torch.from_numpy(np.random.default_rng(n).uniform(-1, 1, n)).cuda()
    level, scale = 2, 2.0**40
    pts = ctx.encode_vector(plan, y, scale, level)
    want = [he.as_u64(ctx.ct_export(ctx.encrypt(p, 40 + c))) for c, p in enumerate(pts)]
    got = ctx.encrypt_vector(plan, y, scale, level, 40)
    assert len(got) == plan.col_blocks
    for g, w in zip(got, want):
        assert g.level == level and g.scale == scale
        assert np.array_equal(he.as_u64(ctx.ct_export(g)), w)
    nonces = torch.arange(40, 40 + plan.col_blocks, dtype=torch.int64, device="cuda")
    got = ctx.encrypt_vector(plan, y, scale, level, nonces)
    for g, w in zip(got, want):
        assert np.array_equal(he.as_u64(ctx.ct_export(g)), w)
