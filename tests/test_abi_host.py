"""C-ABI library on the CPU (no compute calls): it loads, exports every symbol declared in
include/he.h, and its host-side logic (prime chain, sampler table, MatMult planner,
argument checks) agrees with the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import ckks, layout

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def he():
    from paper_2405_00482_gb300 import build as b

    b.build()
    from paper_2405_00482_gb300 import he as h

    return h


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "he.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(he_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(he):
    lib = ctypes.CDLL(he.LIB_PATH)
    names = declared_symbols()
    assert len(names) >= 25
    for name in names:
        assert hasattr(lib, name), name


@pytest.mark.parametrize("log_n,qb,pb,dnum", [(12, [40, 20], [40], 2), (13, [60, 40, 40], [60], 3),
                                               (14, [60] + [40] * 6, [60, 60, 60], 3), (6, [60, 40, 40], [60], 3),
                                               (10, [50, 40, 40, 40], [55, 55], 2)])
def test_prime_chain_agrees_with_oracle(he, log_n, qb, pb, dnum):
    assert he.primes(log_n, qb, pb, dnum) == ckks.gen_primes(log_n, qb + pb)


def test_gaussian_table_agrees_with_oracle(he, oracle_lib):
    t = np.zeros(38, np.uint64)
    oracle_lib.or_cdt_table(t)
    assert [int(v) for v in t] == he.cdt_table()


@pytest.mark.parametrize("m,n", [(1, 1), (3, 5), (16, 64), (64, 16), (256, 1024), (1024, 256), (4096, 4096), (5000, 37),
                                 (37, 5000), (9000, 9000), (4097, 4095), (512, 8192), (16384, 64), (128, 2)])
def test_planner_agrees_with_oracle(he, m, n):
    p = he.Plan(m, n, 4096)
    o = layout.make_plan(m, n, 4096)
    assert (p.m, p.n, p.slots, p.mp, p.np, p.mb, p.nb, p.row_blocks, p.col_blocks, p.m_prime, p.blocks) == (
        o.m, o.n, o.slots, o.mp, o.np_, o.mb, o.nb, o.row_blocks, o.col_blocks, o.m_prime, o.blocks)


def test_invalid_arguments_are_rejected(he):
    with pytest.raises(he.HEError) as e:
        he.Plan(0, 4, 8)
    assert e.value.status == he.HE_EINVAL
    with pytest.raises(he.HEError):
        he.Plan(4, 4, 6)
    with pytest.raises(he.HEError):
        he.primes(13, [70], [60], 1)  # no 70-bit primes
    with pytest.raises(he.HEError):
        he.primes(13, [60, 40], [60], 3)  # more digits than primes
    assert he.lib().he_strerror(he.HE_EKEY) == b"missing Galois key"


def test_loop_variant_table_and_argument_checks(he):
    """The variant table is host data: readable without a device.  Out-of-range variants and
    NULL handles are rejected before anything touches the GPU."""
    shapes = he.loop_variants()
    assert 7 <= len(shapes) <= he.HE_MM_MAX_VARIANTS
    assert all(vec in (1, 2) and grp in (4, 8) and st >= 0 and ga in (0, 1) and (st > 0 or not ga) for vec, grp, st, ga in shapes)
    assert shapes[0] == (2, 4, 0, 0)
    a, b, c, d = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    lib = he.lib()
    for v in (-1, len(shapes)):
        assert lib.he_loop_variant_shape(v, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)) == he.HE_EINVAL
    assert lib.he_ptmat_set_variant(None, 0) == he.HE_EINVAL
    assert lib.he_batch_set_variant(None, 0) == he.HE_EINVAL
    ms = (ctypes.c_float * he.HE_MM_MAX_VARIANTS)()
    assert lib.he_ptmat_tuning(None, ctypes.byref(a), ms) == he.HE_EINVAL
    assert lib.he_ct_bytes(None, 0) == 0 and lib.he_pt_bytes(None, 0) == 0
    # fused key tables: NULL handles and modes out of range
    for mode in (-1, 3):
        assert lib.he_set_key_fusion(None, mode, 0) == he.HE_EINVAL
    assert lib.he_set_key_fusion(None, 1, 0) == he.HE_EINVAL
    assert lib.he_ptmat_key_fusion(None, ctypes.byref(a), ctypes.byref(b), ms) == he.HE_EINVAL
    assert lib.he_ptmat_set_key_fusion(None, 1, -1) == he.HE_EINVAL
    assert lib.he_set_keyswitch_variant(None, 0) == he.HE_EINVAL


@pytest.mark.parametrize("m,n,slots", [(4, 4, 8), (16, 64, 2048), (256, 1024, 4096), (3, 5, 8), (1, 8, 16), (5000, 300, 4096)])
def test_ras_steps_agree_with_oracle(he, m, n, slots):
    assert he.Plan(m, n, slots).ras_steps == layout.ras_steps(layout.make_plan(m, n, slots))


def test_new_entry_points_reject_null_arguments(he):
    """Context forks, device-nonce encryption, vector encryption, transposed matrix encoding and
    the fused decryption check their arguments before any device work (no GPU needed)."""
    lib = he.lib()
    out = ctypes.c_void_p()
    assert lib.he_ctx_fork(None, None, ctypes.byref(out)) == he.HE_EINVAL
    assert lib.he_ctx_fork(None, None, None) == he.HE_EINVAL
    assert lib.he_encrypt_dnonce(None, None, None, None) == he.HE_EINVAL
    assert lib.he_encrypt_vector(None, None, None, 1.0, 0, 0, None, None) == he.HE_EINVAL
    assert lib.he_encode_matrix_transposed(None, None, None, 1, ctypes.byref(out)) == he.HE_EINVAL
    assert lib.he_ptmat_encode_transposed(None, None, None) == he.HE_EINVAL
    assert lib.he_matmult_decrypt(None, None, None, 0, None, None) == he.HE_EINVAL


@pytest.mark.parametrize("m,n", [(4096, 256), (256, 4096), (16, 4), (4, 16), (8, 8), (1, 64)])
def test_transpose_steps_agree_with_oracle(he, m, n):
    """he_cdiag_transpose_steps lists the nonzero steps of the oracle's Eq. 5 reading."""
    want = sorted({r for _, r in layout.transpose_rotations(m, n) if r})
    assert he.Context.cdiag_transpose_steps(m, n) == want


def test_ct_host_level_reads_header(he):
    """The serialized-ciphertext header (magic, version, level) is parsed on the host; bad
    headers are refused."""
    import struct

    lib = he.lib()
    hdr = struct.pack("<IIiidQ", 0x54434548, 1, 13, 2, 2.0**40, 0)
    buf = ctypes.create_string_buffer(hdr, len(hdr))
    lvl = ctypes.c_int32()
    assert lib.he_ct_host_level(buf, len(hdr), ctypes.byref(lvl)) == 0 and lvl.value == 2
    bad = ctypes.create_string_buffer(b"XECT" + hdr[4:], len(hdr))
    assert lib.he_ct_host_level(bad, len(hdr), ctypes.byref(lvl)) == he.HE_EINVAL
    assert lib.he_ct_host_level(buf, 16, ctypes.byref(lvl)) == he.HE_EINVAL


def _bconv_i8(he, v, h, t):
    lib = he.lib()
    a = len(v)
    va, ha, out = (ctypes.c_uint64 * a)(*v), (ctypes.c_uint64 * a)(*h), ctypes.c_uint64()
    assert lib.he_bconv_i8_host(a, va, ha, t, ctypes.byref(out)) == 0
    return out.value


@pytest.mark.parametrize("t", [3, 17, 257])
def test_int8_basis_extension_exhaustive_small_moduli(he, t):
    """The INT8 engine's arithmetic (bytes of v and h, 32-bit sums of byte products, recombination
    in three groups and reduction mod t) equals sum v_i h_i mod t on every pair of residues of a
    small modulus, one and two source primes."""
    r = range(t) if t <= 17 else range(0, t, 7)
    for v0 in r:
        for h0 in r:
            assert _bconv_i8(he, [v0], [h0], t) == (v0 * h0) % t
    if t <= 17:
        for v0 in range(t):
            for v1 in range(t):
                for h0 in range(t):
                    h1 = (v0 + 3 * v1 + h0) % t
                    assert _bconv_i8(he, [v0, v1], [h0, h1], t) == (v0 * h0 + v1 * h1) % t


def test_int8_basis_extension_wide_operands(he):
    """Full-width operands (every byte 255 included) and 60-bit primes, one to four sources."""
    rng = np.random.default_rng(7)
    ts = [ckks.gen_primes(13, [60])[0], ckks.gen_primes(14, [40])[0], (1 << 61) - 1, 3]
    for t in ts:
        for a in (1, 2, 3, 4):
            cases = [[(1 << 64) - 1] * a, [0] * a] + [[int(x) for x in rng.integers(0, 2**63, size=a, dtype=np.uint64)] for _ in range(50)]
            for v in cases:
                for h in cases[:3] + [[int(x) % t for x in v[::-1]]]:
                    assert _bconv_i8(he, v, h, t) == sum(x * y for x, y in zip(v, h)) % t


@pytest.mark.parametrize("m,n,slots,baby", [(256, 1024, 4096, 8), (256, 1024, 4096, 1), (256, 1024, 4096, 64), (16, 16, 16, 4),
                                            (600, 300, 512, 2), (1, 1, 8, 1)])
def test_plan_baby_steps_agree_with_oracle(he, m, n, slots, baby):
    """he_plan_rotation_steps lists the oracle's baby then giant steps; 0 gives 1..m'-1."""
    plan = he.Plan(m, n, slots, baby=baby)
    op = layout.make_plan(m, n, slots)
    bs, gs = layout.bsgs_steps(op, baby)
    assert plan.rotation_steps == bs + gs
    assert he.Plan(m, n, slots).rotation_steps == op.rotation_steps


def test_plan_baby_steps_rejected(he):
    lib = he.lib()
    plan = he.Plan(256, 1024, 4096)
    for bad in (-1, 3, 128, 48):
        assert lib.he_plan_set_baby_steps(plan.handle, bad) == he.HE_EINVAL
    assert lib.he_plan_set_baby_steps(plan.handle, 0) == 0
