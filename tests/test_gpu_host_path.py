"""The host-memory entry points (he_*_host: the party-facing calls of Sec. 3 and Alg. 1) against
their device-memory counterparts, through the C ABI: the same plaintexts, ciphertexts and
decrypted doubles bit for bit, from pageable and from page-locked host memory, and the
serialized ciphertext round trip (he_ct_export_host / he_ct_import_host) on host bytes."""
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

    ctx = he.Context(13, [60, 40, 40], [60], 3, seed=3)
    return he, ctx, torch


@pytest.mark.parametrize("m,n,transposed,pinned", [(256, 1024, True, True), (1024, 256, False, False), (300, 5000, False, True),
                                                  (5000, 300, True, False)])
def test_host_matrix_and_vector_equal_device_path(env, m, n, transposed, pinned):
    he, ctx, torch = env
    rng = np.random.default_rng(m + n)
    X = rng.normal(size=(m, n))
    y = rng.uniform(-1, 1, n)
    plan = he.Plan(m, n, ctx.slots)
    level = 2
    Xh = np.ascontiguousarray(X.T) if transposed else X
    Xt = torch.from_numpy(Xh)
    yt = torch.from_numpy(y)
    if pinned:
        Xt, yt = Xt.pin_memory(), yt.pin_memory()
    pm_h = ctx.encode_matrix_host(plan, Xt, level, transposed=transposed)
    pm_d = ctx.encode_matrix(plan, torch.from_numpy(Xh).cuda(), level, transposed=transposed)
    assert torch.equal(pm_h.export(), pm_d.export())
    # re-encoding in place from host memory gives the same plaintexts
    ctx.encode_matrix_host(plan, Xt, level, out=pm_d, transposed=transposed)
    assert torch.equal(pm_h.export(), pm_d.export())
    cts_h = ctx.encrypt_vector_host(plan, yt, 2.0**40, level, 77)
    cts_d = ctx.encrypt_vector(plan, torch.from_numpy(y).cuda(), 2.0**40, level, 77)
    for a, b in zip(cts_h, cts_d):
        assert torch.equal(a.data, b.data) and a.scale == b.scale and a.level == b.level
    ctx.keygen(list(range(1, plan.m_prime)))
    outs = ctx.matmult(plan, pm_h, cts_h)
    want = ctx.matmult_decrypt(plan, outs).cpu()
    got = torch.empty(plan.m, dtype=torch.float64)
    if pinned:
        got = got.pin_memory()
    ctx.matmult_decrypt_host(plan, outs, out=got)
    ctx.synchronize()
    assert torch.equal(got, want)
    assert float(np.abs(got.numpy() - X @ y).max()) < 1e-4
    # with a mask (Alg. 1): the host mask and the device mask give the same doubles
    mask = rng.uniform(-100, 100, size=(plan.row_blocks, ctx.slots))
    want_m = ctx.matmult_decrypt(plan, outs, mask=torch.from_numpy(mask).cuda()).cpu()
    got_m = ctx.matmult_decrypt_host(plan, outs, mask=mask)
    assert torch.equal(got_m, want_m)


def test_decrypt_host_equals_decrypt(env):
    he, ctx, torch = env
    z = torch.linspace(-1, 1, ctx.slots, dtype=torch.float64).cuda()
    ct = ctx.encrypt(ctx.encode(z, 2.0**40, 2), 5)
    want = ctx.decrypt(ct).cpu()
    assert torch.equal(ctx.decrypt_host(ct), want)
    pinned = torch.empty(ctx.slots, dtype=torch.float64).pin_memory()
    ctx.decrypt_host(ct, out=pinned)
    ctx.synchronize()
    assert torch.equal(pinned, want)


@pytest.mark.parametrize("level", [0, 1, 2])
def test_ciphertext_bytes_round_trip(env, level):
    he, ctx, torch = env
    z = torch.linspace(-1, 1, ctx.slots, dtype=torch.float64).cuda()
    ct = ctx.encrypt(ctx.encode(z, 2.0**40, level), 11 + level)
    data = ctx.ct_export_host(ct)
    nl = level + 1
    assert len(data) == 32 + 8 * nl + 16 * nl * ctx.n
    # the coefficient section is the canonical coefficient form, the primes those of the level
    coef = np.frombuffer(data[32 + 8 * nl:], dtype=np.uint64).reshape(2, nl, ctx.n)
    assert np.array_equal(coef, he.as_u64(ctx.ct_export(ct)))
    assert list(np.frombuffer(data[32:32 + 8 * nl], dtype=np.uint64)) == ctx.primes[:nl]
    back = ctx.ct_import_host(data)
    assert back.level == level and back.scale == ct.scale
    assert torch.equal(back.data, ct.data)


def test_ciphertext_bytes_are_checked(env):
    he, ctx, torch = env
    z = torch.ones(ctx.slots, dtype=torch.float64).cuda()
    ct = ctx.encrypt(ctx.encode(z, 2.0**40, 2), 4)
    data = bytearray(ctx.ct_export_host(ct))
    nl = 3
    for bad in (data[:-8], bytes(b"X") + bytes(data[1:])):
        with pytest.raises(he.HEError) as e:
            ctx.ct_import_host(bytes(bad))
        assert e.value.status == he.HE_EINVAL
    # a coefficient that is not a canonical residue of its prime
    off = 32 + 8 * nl + 8 * 5
    bad = bytearray(data)
    bad[off:off + 8] = int(ctx.primes[0]).to_bytes(8, "little")
    with pytest.raises(he.HEError) as e:
        ctx.ct_import_host(bytes(bad))
    assert e.value.status == he.HE_EINVAL
    # bytes made under another prime chain
    other = he.Context(13, [60, 40, 38], [60], 3, seed=3)
    ct2 = other.encrypt(other.encode(z, 2.0**40, 2), 4)
    with pytest.raises(he.HEError) as e:
        ctx.ct_import_host(other.ct_export_host(ct2))
    assert e.value.status == he.HE_EINVAL
