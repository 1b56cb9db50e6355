"""O3 on many ciphertexts at once (he_rotate_many): bit-identical to one he_rotate per pair and
to the oracle's rotation; argument checks."""
import numpy as np
import pytest

from oracle import ckks

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def he():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2405_00482_gb300 import he as mod

    return mod


@pytest.mark.parametrize("log_n,qb,pb,dnum,count", [(13, [60, 40, 40], [60], 3, 70), (14, [60] + [40] * 6, [60, 60, 60], 3, 9)])
def test_rotate_many_matches_single_rotations(he, log_n, qb, pb, dnum, count):
    import torch

    ctx = he.Context(log_n, qb, pb, dnum, seed=31)
    rng = np.random.default_rng(count)
    level = len(qb) - 1
    cts = [ctx.encrypt(ctx.encode(torch.from_numpy(rng.uniform(-1, 1, ctx.slots)).cuda(), 2.0**40, level), 100 + i) for i in range(count)]
    steps = [int(s) for s in rng.integers(-ctx.slots, ctx.slots, size=count)]
    steps[0] = 0  # identity: a copy
    steps[1] = ctx.slots  # a multiple of N/2: also the identity
    ctx.keygen(sorted(set(s % ctx.slots for s in steps if s % ctx.slots)))
    outs = ctx.rotate_many(cts, steps)
    for c, s, o in zip(cts, steps, outs):
        want = ctx.ct_export(c) if s % ctx.slots == 0 else ctx.ct_export(ctx.rotate(c, s % ctx.slots))
        assert torch.equal(ctx.ct_export(o), want)
    # the results decrypt to the rotated slots (scale 2^40)
    for c, s, o in zip(cts[:5], steps[:5], outs[:5]):
        z = ctx.decrypt(c).cpu().numpy()
        assert np.abs(ctx.decrypt(o).cpu().numpy() - np.roll(z, -s)).max() < 1e-6
    # one level down (fewer digits), still bit-identical to single rotations
    low = [ctx.rescale(c) for c in cts[2:7]]
    for c, s, o in zip(low, steps[2:7], ctx.rotate_many(low, steps[2:7])):
        assert torch.equal(ctx.ct_export(o), ctx.ct_export(ctx.rotate(c, s % ctx.slots)))


def test_rotate_many_bit_exact_against_oracle(he):
    log_n, qb, pb, d = 6, [60, 40, 40], [60], 3
    ctx, o = he.Context(log_n, qb, pb, d, seed=32), ckks.Oracle(log_n, qb, pb, d, seed=32)
    rng = np.random.default_rng(5)
    level, scale = 2, 2.0**40
    cts = [o.encrypt(o.encode(rng.uniform(-1, 1, o.slots), scale, level), level, scale, 10 + i) for i in range(6)]
    steps = [1, 5, 31, 2, 17, 9]
    o.gen_rotation_keys(steps)
    ctx.keygen(steps)
    got = ctx.rotate_many([ctx.ct_import(he.from_u64(c.data, ctx.device), level, scale) for c in cts], steps)
    for g, c, s in zip(got, cts, steps):
        assert np.array_equal(he.as_u64(ctx.ct_export(g)), o.rotate(c, s).data)


def test_rotate_many_argument_checks(he):
    import torch

    ctx = he.Context(6, [60, 40, 40], [60], 3, seed=33)
    cts = [ctx.encrypt(ctx.encode(torch.zeros(4, dtype=torch.float64, device="cuda"), 2.0**40, 2), i) for i in range(3)]
    ctx.keygen([1])
    with pytest.raises(he.HEError) as e:
        ctx.rotate_many(cts, [1, 1, 1], outs=[cts[1], ctx.new_ct(2), ctx.new_ct(2)])  # output overlaps an input
    assert e.value.status == he.HE_EINVAL
    with pytest.raises(he.HEError) as e:
        ctx.rotate_many(cts, [1, 2, 1])  # no key for step 2
    assert e.value.status == he.HE_EKEY
    assert ctx.rotate_many([], []) == []


@pytest.mark.parametrize("log_n,qb,pb,dnum", [(12, [40, 20], [40], 2), (13, [60, 40, 40], [60], 3), (14, [60] + [40] * 6, [60, 60, 60], 3)])
def test_keyswitch_variants_agree(he, log_n, qb, pb, dnum):
    """Every transform variant of the many-rotation key switch (one CTA per limb-poly at two
    thread counts, two phases per transform), pinned in turn: hoisted and many-ciphertext
    rotations bit-identical across variants and to single rotations (the cluster key switch)."""
    import torch

    ctx = he.Context(log_n, qb, pb, dnum, seed=33)
    rng = np.random.default_rng(log_n)
    level, scale = len(qb) - 1, 2.0**20 if log_n == 12 else 2.0**40
    enc = lambda i: ctx.encrypt(ctx.encode(torch.from_numpy(rng.uniform(-1, 1, ctx.slots)).cuda(), scale, level), 200 + i)
    steps = list(range(1, 41))  # at least 32 rotations: the many-rotation key switch
    ctx.keygen(steps)
    ct, cts = enc(0), [enc(1 + i) for i in range(len(steps))]
    results = []
    for v in range(he.HE_KS_VARIANTS):
        ctx.set_keyswitch_variant(v)
        hoisted = torch.stack([ctx.ct_export(o) for o in ctx.rotate_hoisted(ct, steps)])
        many = torch.stack([ctx.ct_export(o) for o in ctx.rotate_many(cts, steps)])
        results.append((hoisted, many))
    ctx.set_keyswitch_variant(-1)
    for v in range(1, he.HE_KS_VARIANTS):
        assert torch.equal(results[v][0], results[0][0]), f"hoisted, variant {v}"
        assert torch.equal(results[v][1], results[0][1]), f"many, variant {v}"
    for s in (1, 7, 40):
        assert torch.equal(results[0][0][s - 1], ctx.ct_export(ctx.rotate(ct, s)))
        assert torch.equal(results[0][1][s - 1], ctx.ct_export(ctx.rotate(cts[s - 1], s)))


@pytest.mark.parametrize("log_n,qb,pb,dnum", [(12, [40, 20], [40], 2), (13, [60, 40, 40], [60], 3), (14, [60] + [40] * 6, [60, 60, 60], 3)])
def test_modup_forms_agree(he, log_n, qb, pb, dnum):
    """The ModUp of many ciphertexts in each NTT form (one CTA per limb-poly, or the two-phase
    inverse and forward transforms of form 2): rotations of 40 different ciphertexts bit-identical
    across forms and to single rotations."""
    import torch

    ctx = he.Context(log_n, qb, pb, dnum, seed=34)
    rng = np.random.default_rng(log_n + 1)
    level, scale = len(qb) - 1, 2.0**20 if log_n == 12 else 2.0**40
    steps = [int(s) for s in rng.integers(1, ctx.slots, size=40)]
    ctx.keygen(sorted(set(steps)))
    cts = [ctx.encrypt(ctx.encode(torch.from_numpy(rng.uniform(-1, 1, ctx.slots)).cuda(), scale, level), 300 + i) for i in range(len(steps))]
    got = []
    for form in range(he.HE_NTT_FORMS):
        ctx.set_ntt_form(form)
        got.append(torch.stack([ctx.ct_export(o) for o in ctx.rotate_many(cts, steps)]))
    ctx.set_ntt_form(-1)
    for f in range(1, he.HE_NTT_FORMS):
        assert torch.equal(got[f], got[0]), f"form {f}"
    for i in (0, 13, 39):
        assert torch.equal(got[0][i], ctx.ct_export(ctx.rotate(cts[i], steps[i])))
