"""Python binding of the C ABI in include/he.h (argument marshalling only).

Every computation runs in the CUDA kernels of libhe.so; this module only allocates
device buffers with torch, passes their pointers and the stream, and checks status codes.
Residue buffers are torch.int64 tensors used as raw 64-bit storage (the library treats
them as uint64).  Loading fails loudly if libhe.so has not been built.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhe.so")

HE_OK, HE_EINVAL, HE_ENOMEM, HE_ECUDA, HE_EKEY, HE_ELEVEL, HE_ESCALE, HE_ETIMEOUT, HE_EBUDGET = 0, -1, -2, -3, -4, -5, -6, -7, -8
HE_BCONV_INT64, HE_BCONV_INT8_TC = 0, 1  # basis extension engines of ModUp
HE_NTT_FORMS = 3  # NTT forms of launches of many limb-polys
HE_KS_VARIANTS = 3  # transform variants of the many-rotation key switch
HE_PROF_LOOP, HE_PROF_MATRIX_NTT, HE_PROF_KS_TRANSFORM, HE_PROF_KS_ELEMENTWISE = 0, 1, 2, 3  # profiled kernel classes


class HEError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {_lib().he_strerror(status).decode()} ({status})")
        self.status = status


class HeParams(ctypes.Structure):
    _fields_ = [("log_n", ctypes.c_int32), ("n_q", ctypes.c_int32), ("n_p", ctypes.c_int32), ("dnum", ctypes.c_int32),
                ("q_bits", ctypes.c_int32 * 16), ("p_bits", ctypes.c_int32 * 8)]


class HeCt(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("level", ctypes.c_int32), ("scale", ctypes.c_double)]


HePt = HeCt  # same layout: data, level, scale

_vp, _i32, _i64, _u64, _dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
_SIGS = {
    "he_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "he_params_primes": (ctypes.c_int, [ctypes.POINTER(HeParams), ctypes.POINTER(_u64)]),
    "he_cdt_table": (ctypes.c_int, [ctypes.POINTER(_u64)]),
    "he_ctx_create": (ctypes.c_int, [ctypes.POINTER(HeParams), _u64, _vp, ctypes.POINTER(_vp)]),
    "he_ctx_destroy": (None, [_vp]),
    "he_ctx_fork": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(_vp)]),
    "he_synchronize": (ctypes.c_int, [_vp]),
    "he_ctx_info": (ctypes.c_int, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "he_keygen": (ctypes.c_int, [_vp, ctypes.POINTER(_i32), ctypes.c_int]),
    "he_launch_count": (ctypes.c_int, [_vp, ctypes.POINTER(_i64)]),
    "he_profile_enable": (ctypes.c_int, [_vp, ctypes.c_int]),
    "he_profile_read": (ctypes.c_int, [_vp, ctypes.POINTER(_dbl), ctypes.POINTER(_i64)]),
    "he_profile_read_kind": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(_dbl), ctypes.POINTER(_i64)]),
    "he_encode": (ctypes.c_int, [_vp, _vp, _i64, _dbl, ctypes.c_int, ctypes.POINTER(HePt)]),
    "he_encrypt": (ctypes.c_int, [_vp, ctypes.POINTER(HePt), _u64, ctypes.POINTER(HeCt)]),
    "he_encrypt_dnonce": (ctypes.c_int, [_vp, ctypes.POINTER(HePt), _vp, ctypes.POINTER(HeCt)]),
    "he_encrypt_vector": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_double, ctypes.c_int, _u64, _vp, _vp]),
    "he_matmult_decrypt": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp, _vp]),
    "he_decrypt": (ctypes.c_int, [_vp, ctypes.POINTER(HeCt), _vp]),
    "he_add": (ctypes.c_int, [_vp, ctypes.POINTER(HeCt), ctypes.POINTER(HeCt), ctypes.POINTER(HeCt)]),
    "he_add_plain": (ctypes.c_int, [_vp, ctypes.POINTER(HeCt), ctypes.POINTER(HePt), ctypes.POINTER(HeCt)]),
    "he_matmult_decode_masked": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "he_plan_ras_steps": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int)]),
    "he_ras": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(HeCt), ctypes.POINTER(HeCt)]),
    "he_ras_decode": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "he_mul_plain": (ctypes.c_int, [_vp, ctypes.POINTER(HeCt), ctypes.POINTER(HePt), ctypes.POINTER(HeCt)]),
    "he_rescale": (ctypes.c_int, [_vp, ctypes.POINTER(HeCt), ctypes.POINTER(HeCt)]),
    "he_rotate": (ctypes.c_int, [_vp, ctypes.POINTER(HeCt), _i32, ctypes.POINTER(HeCt)]),
    "he_rotate_many": (ctypes.c_int, [_vp, ctypes.POINTER(HeCt), ctypes.POINTER(ctypes.c_int32), ctypes.c_int, ctypes.POINTER(HeCt)]),
    "he_rotate_hoisted": (ctypes.c_int, [_vp, ctypes.POINTER(HeCt), ctypes.POINTER(_i32), ctypes.c_int, ctypes.POINTER(HeCt)]),
    "he_plan_create": (ctypes.c_int, [_i64, _i64, _i64, ctypes.POINTER(_vp)]),
    "he_plan_query": (ctypes.c_int, [_vp, ctypes.POINTER(_i64)]),
    "he_plan_free": (None, [_vp]),
    "he_plan_set_baby_steps": (ctypes.c_int, [_vp, _i64]),
    "he_plan_rotation_steps": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int)]),
    "he_encode_matrix": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.POINTER(_vp)]),
    "he_ptmat_encode": (ctypes.c_int, [_vp, _vp, _vp]),
    "he_encode_matrix_transposed": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.POINTER(_vp)]),
    "he_ptmat_encode_transposed": (ctypes.c_int, [_vp, _vp, _vp]),
    "he_ct_bytes": (ctypes.c_size_t, [_vp, ctypes.c_int]),
    "he_pt_bytes": (ctypes.c_size_t, [_vp, ctypes.c_int]),
    "he_ptmat_export": (ctypes.c_int, [_vp, _vp, _vp]),
    "he_ptmat_import": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _dbl, ctypes.POINTER(_vp)]),
    "he_ptmat_free": (None, [_vp]),
    "he_encode_vector": (ctypes.c_int, [_vp, _vp, _vp, _dbl, ctypes.c_int, ctypes.POINTER(HePt)]),
    "he_matmult_plain_cipher": (ctypes.c_int, [_vp, _vp, _vp, ctypes.POINTER(HeCt), ctypes.c_int, ctypes.POINTER(HeCt), ctypes.c_int]),
    "he_matmult_plain_cipher_noalloc": (ctypes.c_int, [_vp, _vp, _vp, ctypes.POINTER(HeCt), ctypes.c_int, ctypes.POINTER(HeCt),
                                                        ctypes.c_int]),
    "he_matmult_decode": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "he_batch_create": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp)]),
    "he_batch_run": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(HeCt), ctypes.POINTER(HeCt)]),
    "he_batch_free": (None, [_vp]),
    "he_ptmat_tuning": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)]),
    "he_batch_tuning": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)]),
    "he_loop_variant_count": (ctypes.c_int, []),
    "he_batch_stage_form": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)]),
    "he_batch_set_stage_form": (ctypes.c_int, [_vp, ctypes.c_int]),
    "he_ptmat_set_variant": (ctypes.c_int, [_vp, ctypes.c_int]),
    "he_set_key_fusion": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_size_t]),
    "he_set_keyswitch_variant": (ctypes.c_int, [_vp, ctypes.c_int]),
    "he_ptmat_key_fusion": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)]),
    "he_ptmat_set_key_fusion": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
    "he_batch_set_variant": (ctypes.c_int, [_vp, ctypes.c_int]),
    "he_loop_variant_shape": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                             ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "he_cdiag_encode_weights": (ctypes.c_int, [_vp, _vp, _i64, _i64, ctypes.c_int, ctypes.POINTER(_vp)]),
    "he_cdmat_free": (None, [_vp]),
    "he_cdiag_encode_matrix": (ctypes.c_int, [_vp, _vp, _i64, _i64, _dbl, ctypes.c_int, ctypes.POINTER(HePt)]),
    "he_cdiag_matmult": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(HeCt), ctypes.c_int, ctypes.POINTER(HeCt)]),
    "he_cdiag_decode": (ctypes.c_int, [_vp, _i64, _i64, _i64, _vp, _vp]),
    "he_cdiag_transpose": (ctypes.c_int, [_vp, ctypes.POINTER(HeCt), _i64, _i64, ctypes.POINTER(HeCt)]),
    "he_server_create": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(_vp)]),
    "he_server_submit": (ctypes.c_int, [_vp, _vp, _vp, ctypes.POINTER(HeCt), ctypes.POINTER(HeCt), ctypes.POINTER(_i64)]),
    "he_server_add_ring": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
    "he_server_wait": (ctypes.c_int, [_vp, _i64, _i64, ctypes.POINTER(_dbl)]),
    "he_server_stats": (ctypes.c_int, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(ctypes.c_size_t)]),
    "he_server_free": (None, [_vp]),
    "he_cdiag_transpose_steps": (ctypes.c_int, [_i64, _i64, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int)]),
    "he_encode_matrix_host": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_vp)]),
    "he_ptmat_encode_host": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int]),
    "he_encrypt_vector_host": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_double, ctypes.c_int, _u64, _vp, _vp]),
    "he_decrypt_host": (ctypes.c_int, [_vp, ctypes.POINTER(HeCt), _vp]),
    "he_matmult_decrypt_host": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp, _vp]),
    "he_ct_export_host": (ctypes.c_int, [_vp, ctypes.POINTER(HeCt), _vp, ctypes.POINTER(ctypes.c_size_t)]),
    "he_ct_host_level": (ctypes.c_int, [_vp, ctypes.c_size_t, ctypes.POINTER(_i32)]),
    "he_ct_import_host": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t, ctypes.POINTER(HeCt)]),
    "he_keyswitch_tuning": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)]),
    "he_ntt_form": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)]),
    "he_set_ntt_form": (ctypes.c_int, [_vp, ctypes.c_int]),
    "he_set_basis_extension": (ctypes.c_int, [_vp, ctypes.c_int]),
    "he_get_basis_extension": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int)]),
    "he_bconv_i8_host": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_u64), ctypes.POINTER(_u64), _u64, ctypes.POINTER(_u64)]),
    "he_modup_export": (ctypes.c_int, [_vp, ctypes.POINTER(HeCt), _vp]),
    "he_ct_export": (ctypes.c_int, [_vp, ctypes.POINTER(HeCt), _vp]),
    "he_ct_import": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _dbl, ctypes.POINTER(HeCt)]),
    "he_pt_export": (ctypes.c_int, [_vp, ctypes.POINTER(HePt), _vp]),
    "he_pt_import": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _dbl, ctypes.POINTER(HePt)]),
}

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it first (python -m paper_2405_00482_gb300.build)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def lib():
    return _lib()


def _check(status: int, what: str):
    if status != HE_OK:
        raise HEError(status, what)


def make_params(log_n: int, q_bits, p_bits, dnum: int) -> HeParams:
    p = HeParams()
    p.log_n, p.n_q, p.n_p, p.dnum = log_n, len(q_bits), len(p_bits), dnum
    for i, b in enumerate(q_bits):
        p.q_bits[i] = b
    for i, b in enumerate(p_bits):
        p.p_bits[i] = b
    return p


def primes(log_n: int, q_bits, p_bits, dnum: int) -> list[int]:
    """Host-side prime chain of the library (no GPU needed)."""
    p = make_params(log_n, q_bits, p_bits, dnum)
    out = (_u64 * (len(q_bits) + len(p_bits)))()
    _check(_lib().he_params_primes(ctypes.byref(p), out), "he_params_primes")
    return [int(v) for v in out]


def cdt_table() -> list[int]:
    out = (_u64 * 38)()
    _check(_lib().he_cdt_table(out), "he_cdt_table")
    return [int(v) for v in out]


class Plan:
    """MatMult layout plan (host only): he_plan_create / he_plan_query."""

    FIELDS = ("m", "n", "slots", "mp", "np", "mb", "nb", "row_blocks", "col_blocks", "m_prime", "blocks")

    def __init__(self, m: int, n: int, slots: int, baby: int = 0):
        """baby > 0: the baby-step giant-step schedule with that many baby steps
        (he_plan_set_baby_steps); 0: the diagonal method."""
        h = _vp()
        _check(_lib().he_plan_create(m, n, slots, ctypes.byref(h)), "he_plan_create")
        self.handle = h
        self.baby = baby
        if baby:
            _check(_lib().he_plan_set_baby_steps(h, baby), "he_plan_set_baby_steps")
        info = (_i64 * 11)()
        _check(_lib().he_plan_query(h, info), "he_plan_query")
        for k, v in zip(self.FIELDS, info):
            setattr(self, k, int(v))
        n = ctypes.c_int()
        _check(_lib().he_plan_ras_steps(h, None, ctypes.byref(n)), "he_plan_ras_steps")
        steps = (ctypes.c_int32 * max(n.value, 1))()
        _check(_lib().he_plan_ras_steps(h, steps, ctypes.byref(n)), "he_plan_ras_steps")
        self.ras_steps = [int(v) for v in steps[: n.value]]
        _check(_lib().he_plan_rotation_steps(h, None, ctypes.byref(n)), "he_plan_rotation_steps")
        steps = (ctypes.c_int32 * max(n.value, 1))()
        _check(_lib().he_plan_rotation_steps(h, steps, ctypes.byref(n)), "he_plan_rotation_steps")
        self.rotation_steps = [int(v) for v in steps[: n.value]]

    def __del__(self):
        if getattr(self, "handle", None):
            _lib().he_plan_free(self.handle)
            self.handle = None


@dataclass
class Ciphertext:
    data: torch.Tensor  # int64 [2][level+1][N], NTT form
    level: int
    scale: float

    def c(self) -> HeCt:
        return HeCt(self.data.data_ptr(), self.level, self.scale)


@dataclass
class Plaintext:
    data: torch.Tensor  # int64 [level+1][N], NTT form
    level: int
    scale: float

    def c(self) -> HePt:
        return HePt(self.data.data_ptr(), self.level, self.scale)


HE_MM_MAX_VARIANTS = 8


def loop_variants() -> list:
    """(coefficients per thread, rotation groups, cp.async stages, gathers staged) of every
    loop-kernel variant."""
    out = []
    for v in range(_lib().he_loop_variant_count()):
        a, b, c, d = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(_lib().he_loop_variant_shape(v, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)), "he_loop_variant_shape")
        out.append((a.value, b.value, c.value, d.value))
    return out


def _tuning(fn, handle) -> dict:
    v = ctypes.c_int()
    ms = (ctypes.c_float * HE_MM_MAX_VARIANTS)()
    _check(fn(handle, ctypes.byref(v), ms), "tuning")
    n = _lib().he_loop_variant_count()
    return {"variant": int(v.value), "variant_ms": [round(float(x), 4) for x in ms[:n]]}


class PtMatrix:
    def __init__(self, ctx: "Context", handle, plan: Plan, level: int):
        self.ctx, self.handle, self.plan, self.level = ctx, handle, plan, level

    def tuning(self) -> dict:
        """Loop-kernel variant chosen on the first MatMult and the timed ms of each variant."""
        return _tuning(_lib().he_ptmat_tuning, self.handle)

    def set_variant(self, v: int) -> None:
        """Pin the loop-kernel variant (-1: tune again on the next MatMult)."""
        _check(_lib().he_ptmat_set_variant(self.handle, v), "he_ptmat_set_variant")

    def key_fusion(self) -> dict:
        """Fused key tables (he_ptmat_key_fusion): state 0 not tried, 1 in use, -1 not used; the
        fused form's variant and its timed ms per variant."""
        st, v = ctypes.c_int(), ctypes.c_int()
        ms = (ctypes.c_float * HE_MM_MAX_VARIANTS)()
        _check(_lib().he_ptmat_key_fusion(self.handle, ctypes.byref(st), ctypes.byref(v), ms), "he_ptmat_key_fusion")
        n = _lib().he_loop_variant_count()
        return {"state": int(st.value), "variant": int(v.value), "variant_ms": [round(float(x), 4) for x in ms[:n]]}

    def set_key_fusion(self, on: bool, variant: int = -1) -> None:
        """he_ptmat_set_key_fusion: off (tables freed), eligible again, or pinned to a variant."""
        _check(_lib().he_ptmat_set_key_fusion(self.handle, int(on), variant), "he_ptmat_set_key_fusion")

    def export(self) -> torch.Tensor:
        """Plaintexts [R][C][m'][level+1+K][N] in canonical coefficient form (int64 storage)."""
        p = self.plan
        limbs = self.level + 1 + self.ctx.K
        out = torch.empty((p.row_blocks, p.col_blocks, p.m_prime, limbs, self.ctx.n), dtype=torch.int64, device=self.ctx.device)
        _check(_lib().he_ptmat_export(self.ctx.handle, self.handle, out.data_ptr()), "he_ptmat_export")
        return out

    def __del__(self):
        if getattr(self, "handle", None):
            _lib().he_ptmat_free(self.handle)
            self.handle = None


class Batch:
    """he_batch: many R = C = 1 MatMults run by one persistent kernel under a CUDA graph."""

    def __init__(self, ctx: "Context", plans: list[Plan], pms: list["PtMatrix"]):
        self.ctx, self.plans, self.pms = ctx, plans, pms
        pa = (_vp * len(plans))(*[p.handle.value for p in plans])
        ma = (_vp * len(pms))(*[m.handle.value for m in pms])
        h = _vp()
        _check(_lib().he_batch_create(ctx.handle, len(plans), pa, ma, ctypes.byref(h)), "he_batch_create")
        self.handle = h
        self.level = pms[0].level

    def tuning(self) -> dict:
        return _tuning(_lib().he_batch_tuning, self.handle)

    def set_variant(self, v: int) -> None:
        """Pin the loop-kernel variant (-1: tune again on the next run)."""
        _check(_lib().he_batch_set_variant(self.handle, v), "he_batch_set_variant")

    def stage_tuning(self) -> dict:
        """ModUp / ModDown / rescale stage form (0 one CTA per limb-poly, 1 clusters) and both timings."""
        f = ctypes.c_int()
        ms = (ctypes.c_float * 2)()
        _check(_lib().he_batch_stage_form(self.handle, ctypes.byref(f), ms), "he_batch_stage_form")
        return {"form": int(f.value), "form_ms": [round(float(x), 4) for x in ms]}

    def set_stage_form(self, form: int) -> None:
        _check(_lib().he_batch_set_stage_form(self.handle, form), "he_batch_set_stage_form")

    def run(self, cts: list[Ciphertext], outs: list[Ciphertext] | None = None) -> list[Ciphertext]:
        outs = outs or [self.ctx.new_ct(self.level - 1) for _ in cts]
        ia = (HeCt * len(cts))(*[c.c() for c in cts])
        oa = (HeCt * len(outs))(*[o.c() for o in outs])
        _check(_lib().he_batch_run(self.ctx.handle, self.handle, ia, oa), "he_batch_run")
        for o, a in zip(outs, oa):
            o.level, o.scale = a.level, a.scale
        return outs

    def __del__(self):
        if getattr(self, "handle", None):
            _lib().he_batch_free(self.handle)
            self.handle = None


class WeightMatrix:
    """he_cdmat: encoded weight columns for the VFL-NN forward pass (Alg. 3)."""

    def __init__(self, ctx: "Context", W: torch.Tensor, level: int):
        W = _dev(W, torch.float64)
        self.ctx, self.n, self.K, self.level = ctx, W.shape[0], W.shape[1], level
        h = _vp()
        _check(_lib().he_cdiag_encode_weights(ctx.handle, W.data_ptr(), self.n, self.K, level, ctypes.byref(h)),
               "he_cdiag_encode_weights")
        self.handle = h

    def __del__(self):
        if getattr(self, "handle", None):
            _lib().he_cdmat_free(self.handle)
            self.handle = None


class Server:
    """he_server: continuous-batching request loop (or one request per call with plain=True)."""

    def __init__(self, ctx: "Context", slots: int, level: int, hbm_budget_bytes: int, plain: bool = False):
        self.ctx = ctx
        h = _vp()
        _check(_lib().he_server_create(ctx.handle, slots, level, hbm_budget_bytes, int(plain), ctypes.byref(h)), "he_server_create")
        self.handle = h
        self._keep = {}

    def add_ring(self, ctx: "Context", level: int) -> None:
        """Also serve ctx's family at `level` (he_server_add_ring), before the first submit."""
        _check(_lib().he_server_add_ring(self.handle, ctx.handle, level), "he_server_add_ring")
        self._ctxs = getattr(self, "_ctxs", []) + [ctx]

    def submit(self, plan: Plan, pm: "PtMatrix", ct: Ciphertext, out: Ciphertext) -> int:
        ci, co = ct.c(), out.c()
        rid = _i64()
        _check(_lib().he_server_submit(self.handle, plan.handle, pm.handle, ctypes.byref(ci), ctypes.byref(co), ctypes.byref(rid)),
               "he_server_submit")
        out.level, out.scale = co.level, co.scale
        self._keep[int(rid.value)] = (plan, pm, ct, out)
        return int(rid.value)

    def wait(self, rid: int, timeout_s: float = 60.0) -> float:
        lat = _dbl()
        _check(_lib().he_server_wait(self.handle, rid, int(timeout_s * 1e6), ctypes.byref(lat)), "he_server_wait")
        self._keep.pop(rid, None)
        return float(lat.value)

    def stats(self) -> tuple[int, int, int]:
        c, l, b = _i64(), _i64(), ctypes.c_size_t()
        _check(_lib().he_server_stats(self.handle, ctypes.byref(c), ctypes.byref(l), ctypes.byref(b)), "he_server_stats")
        return int(c.value), int(l.value), int(b.value)

    def close(self):
        if getattr(self, "handle", None):
            _lib().he_server_free(self.handle)
            self.handle = None

    def __del__(self):
        self.close()


def _host(t, dtype) -> torch.Tensor:
    """A contiguous host tensor of `dtype` from a host tensor or numpy array (a view when possible,
    so a pinned tensor stays pinned)."""
    if not isinstance(t, torch.Tensor):
        t = torch.from_numpy(t)
    if t.is_cuda:
        raise ValueError("host tensor expected")
    return t.to(dtype).contiguous()


def _host_out(t: torch.Tensor, numel: int) -> None:
    if t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous() or t.numel() != numel:
        raise ValueError(f"contiguous host float64 tensor of {numel} elements expected")


def _dev(t: torch.Tensor, dtype) -> torch.Tensor:
    if not t.is_cuda:
        raise ValueError("device tensor expected")
    return t.to(dtype).contiguous()


class Graph:
    """The library calls `fn` issues, captured once into a CUDA graph and replayed with one launch.

    `fn` issues its calls on `ctx` (whose stream is the capture stream and must not be the
    legacy default stream) and on any forks, whose streams it joins back to ctx's stream before
    it returns.  It runs once eagerly first (scratch growth and autotuning happen there), then
    under capture.  Inputs and outputs are the device buffers `fn` names: write new inputs into
    them before a replay; encrypt with a device nonce whose buffer changes between replays.
    `launches` is the number of library kernels one replay runs."""

    def __init__(self, ctx: "Context", fn, forks=()):
        if ctx.stream.cuda_stream == 0:
            raise ValueError("capture needs a context on a non-default stream")
        self.ctxs = [ctx, *forks]
        fn()
        for c in self.ctxs:
            c.synchronize()
        l0 = sum(c.launch_count() for c in self.ctxs)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=ctx.stream):
            fn()
        self.launches = sum(c.launch_count() for c in self.ctxs) - l0
        self.stream = ctx.stream

    def replay(self):
        """One replay on the capture context's stream."""
        with torch.cuda.stream(self.stream):
            self.graph.replay()


class Context:
    """he_ctx: parameters, tables, secret key and Galois keys on one CUDA device and stream."""

    def __init__(self, log_n: int, q_bits, p_bits, dnum: int, seed: int = 0, stream: torch.cuda.Stream | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.stream = stream or torch.cuda.current_stream()
        self.params = make_params(log_n, q_bits, p_bits, dnum)
        h = _vp()
        _check(_lib().he_ctx_create(ctypes.byref(self.params), seed, _vp(self.stream.cuda_stream), ctypes.byref(h)), "he_ctx_create")
        self.handle = h
        self.n = 1 << log_n
        self.slots = self.n // 2
        self.L, self.K = len(q_bits), len(p_bits)
        self.primes = primes(log_n, q_bits, p_bits, dnum)
        self.device = torch.device("cuda", torch.cuda.current_device())

    def __del__(self):
        if getattr(self, "handle", None):
            _lib().he_ctx_destroy(self.handle)
            self.handle = None

    def fork(self, stream: torch.cuda.Stream | None = None) -> "Context":
        """A context on `stream` (a new one by default) sharing this one's tables, secret and
        Galois keys, with its own scratch: calls on the two run concurrently.  Tensors the
        fork's calls allocate come from torch's current stream, so call it inside
        `torch.cuda.stream(fork.stream)`."""
        f = object.__new__(Context)
        f.stream = stream or torch.cuda.Stream(device=self.device)
        h = _vp()
        _check(_lib().he_ctx_fork(self.handle, _vp(f.stream.cuda_stream), ctypes.byref(h)), "he_ctx_fork")
        f.handle = h
        for k in ("params", "n", "slots", "L", "K", "primes", "device"):
            setattr(f, k, getattr(self, k))
        return f

    # ---- buffers ----
    def new_ct(self, level: int) -> Ciphertext:
        return Ciphertext(torch.empty((2, level + 1, self.n), dtype=torch.int64, device=self.device), level, 0.0)

    def ct_bytes(self, level: int) -> int:
        return int(_lib().he_ct_bytes(self.handle, level))

    def pt_bytes(self, level: int) -> int:
        return int(_lib().he_pt_bytes(self.handle, level))

    def new_pt(self, level: int) -> Plaintext:
        return Plaintext(torch.empty((level + 1, self.n), dtype=torch.int64, device=self.device), level, 0.0)

    def synchronize(self):
        _check(_lib().he_synchronize(self.handle), "he_synchronize")

    def launch_count(self) -> int:
        v = _i64()
        _check(_lib().he_launch_count(self.handle, ctypes.byref(v)), "he_launch_count")
        return int(v.value)

    def profile(self, on: bool):
        _check(_lib().he_profile_enable(self.handle, int(on)), "he_profile_enable")

    def profile_read(self, kind: int = HE_PROF_LOOP) -> tuple[float, int]:
        """(total ms, timed launches) of a profiled kernel class since profile(True)."""
        ms, n = _dbl(), _i64()
        _check(_lib().he_profile_read_kind(self.handle, kind, ctypes.byref(ms), ctypes.byref(n)), "he_profile_read_kind")
        return float(ms.value), int(n.value)

    # ---- keys / encode / encrypt / decrypt ----
    def keygen(self, steps):
        arr = (_i32 * len(steps))(*steps)
        _check(_lib().he_keygen(self.handle, arr, len(steps)), "he_keygen")

    def encode(self, slots: torch.Tensor, scale: float, level: int, out: Plaintext | None = None) -> Plaintext:
        slots = _dev(slots, torch.float64)
        pt = out or self.new_pt(level)
        c = pt.c()
        _check(_lib().he_encode(self.handle, slots.data_ptr(), slots.numel(), scale, level, ctypes.byref(c)), "he_encode")
        pt.level, pt.scale = c.level, c.scale
        return pt

    def encrypt(self, pt: Plaintext, nonce, out: Ciphertext | None = None) -> Ciphertext:
        """`nonce` an int, or a one-element int64 device tensor read when the kernels run (for
        a captured Graph: write a fresh nonce there before each replay)."""
        ct = out or self.new_ct(pt.level)
        p, c = pt.c(), ct.c()
        if isinstance(nonce, torch.Tensor):
            if nonce.numel() != 1 or nonce.dtype != torch.int64 or not nonce.is_cuda:
                raise ValueError("device nonce: one int64 element on the GPU")
            _check(_lib().he_encrypt_dnonce(self.handle, ctypes.byref(p), _vp(nonce.data_ptr()), ctypes.byref(c)), "he_encrypt_dnonce")
        else:
            _check(_lib().he_encrypt(self.handle, ctypes.byref(p), nonce, ctypes.byref(c)), "he_encrypt")
        ct.level, ct.scale = c.level, c.scale
        return ct

    def decrypt(self, ct: Ciphertext, out: torch.Tensor | None = None) -> torch.Tensor:
        out = out if out is not None else torch.empty(self.slots, dtype=torch.float64, device=self.device)
        c = ct.c()
        _check(_lib().he_decrypt(self.handle, ctypes.byref(c), out.data_ptr()), "he_decrypt")
        return out

    # ---- O1..O4, rescale ----
    def add(self, a: Ciphertext, b: Ciphertext) -> Ciphertext:
        out = self.new_ct(a.level)
        ca, cb, co = a.c(), b.c(), out.c()
        _check(_lib().he_add(self.handle, ctypes.byref(ca), ctypes.byref(cb), ctypes.byref(co)), "he_add")
        out.scale = co.scale
        return out

    def add_plain(self, ct: Ciphertext, pt: Plaintext, out: Ciphertext | None = None) -> Ciphertext:
        """O1 with a plaintext at the ciphertext's scale: (c0 + pt, c1)."""
        out = out if out is not None else self.new_ct(ct.level)
        c, p, o = ct.c(), pt.c(), out.c()
        _check(_lib().he_add_plain(self.handle, ctypes.byref(c), ctypes.byref(p), ctypes.byref(o)), "he_add_plain")
        out.level, out.scale = o.level, o.scale
        return out

    def ras(self, plan: Plan, ct: Ciphertext, out: Ciphertext | None = None) -> Ciphertext:
        """Ciphertext rotate-and-sum over plan.ras_steps (the non-lazy form of Sec. 4.3)."""
        out = out if out is not None else self.new_ct(ct.level)
        c, o = ct.c(), out.c()
        _check(_lib().he_ras(self.handle, plan.handle, ctypes.byref(c), ctypes.byref(o)), "he_ras")
        out.level, out.scale = o.level, o.scale
        return out

    def ras_decode(self, plan: Plan, slots: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        slots = _dev(slots, torch.float64)
        out = out if out is not None else torch.empty(plan.m, dtype=torch.float64, device=self.device)
        _check(_lib().he_ras_decode(self.handle, plan.handle, slots.data_ptr(), out.data_ptr()), "he_ras_decode")
        return out

    def mul_plain(self, ct: Ciphertext, pt: Plaintext) -> Ciphertext:
        out = self.new_ct(ct.level)
        c, p, o = ct.c(), pt.c(), out.c()
        _check(_lib().he_mul_plain(self.handle, ctypes.byref(c), ctypes.byref(p), ctypes.byref(o)), "he_mul_plain")
        out.scale = o.scale
        return out

    def rotate_many(self, cts: list[Ciphertext], steps: list[int], outs: list[Ciphertext] | None = None) -> list[Ciphertext]:
        """outs[i] = RotL(cts[i], steps[i]) for many ciphertexts, one launch per stage."""
        outs = outs or [self.new_ct(c.level) for c in cts]
        ia = (HeCt * len(cts))(*[c.c() for c in cts])
        oa = (HeCt * len(outs))(*[o.c() for o in outs])
        st = (ctypes.c_int32 * len(steps))(*steps)
        _check(_lib().he_rotate_many(self.handle, ia, st, len(cts), oa), "he_rotate_many")
        for o, a in zip(outs, oa):
            o.level, o.scale = a.level, a.scale
        return outs

    def rescale(self, ct: Ciphertext) -> Ciphertext:
        out = self.new_ct(max(ct.level - 1, 0))
        c, o = ct.c(), out.c()
        _check(_lib().he_rescale(self.handle, ctypes.byref(c), ctypes.byref(o)), "he_rescale")
        out.level, out.scale = o.level, o.scale
        return out

    def rotate(self, ct: Ciphertext, step: int, out: Ciphertext | None = None) -> Ciphertext:
        out = out if out is not None else self.new_ct(ct.level)
        c, o = ct.c(), out.c()
        _check(_lib().he_rotate(self.handle, ctypes.byref(c), step, ctypes.byref(o)), "he_rotate")
        out.level, out.scale = o.level, o.scale
        return out

    def rotate_hoisted(self, ct: Ciphertext, steps, outs: list[Ciphertext] | None = None) -> list[Ciphertext]:
        outs = outs or [self.new_ct(ct.level) for _ in steps]
        arr = (HeCt * len(steps))(*[o.c() for o in outs])
        st = (_i32 * len(steps))(*steps)
        c = ct.c()
        _check(_lib().he_rotate_hoisted(self.handle, ctypes.byref(c), st, len(steps), arr), "he_rotate_hoisted")
        for o, a in zip(outs, arr):
            o.level, o.scale = a.level, a.scale
        return outs

    # ---- MatMult ----
    def encode_matrix(self, plan: Plan, X: torch.Tensor, level: int, out: PtMatrix | None = None,
                      transposed: bool = False) -> PtMatrix:
        """Diagonal plaintexts of X (plan.m x plan.n); transposed=True: X given as its n x m
        transpose (no transposed copy made)."""
        X = _dev(X, torch.float64)
        want = (plan.n, plan.m) if transposed else (plan.m, plan.n)
        if X.numel() != plan.m * plan.n or (X.dim() == 2 and tuple(X.shape) != want):
            raise ValueError(f"matrix of shape {want} expected, got {tuple(X.shape)}")
        if out is not None:
            fn = "he_ptmat_encode_transposed" if transposed else "he_ptmat_encode"
            _check(getattr(_lib(), fn)(self.handle, out.handle, X.data_ptr()), fn)
            return out
        h = _vp()
        fn = "he_encode_matrix_transposed" if transposed else "he_encode_matrix"
        _check(getattr(_lib(), fn)(self.handle, plan.handle, X.data_ptr(), level, ctypes.byref(h)), fn)
        return PtMatrix(self, h, plan, level)

    def ptmat_import(self, plan: Plan, coeffs: torch.Tensor, level: int, scale: float) -> PtMatrix:
        coeffs = _dev(coeffs, torch.int64)
        h = _vp()
        _check(_lib().he_ptmat_import(self.handle, plan.handle, coeffs.data_ptr(), level, scale, ctypes.byref(h)), "he_ptmat_import")
        return PtMatrix(self, h, plan, level)

    def encode_vector(self, plan: Plan, y: torch.Tensor, scale: float, level: int, outs: list[Plaintext] | None = None) -> list[Plaintext]:
        y = _dev(y, torch.float64)
        pts = outs or [self.new_pt(level) for _ in range(plan.col_blocks)]
        arr = (HePt * len(pts))(*[p.c() for p in pts])
        _check(_lib().he_encode_vector(self.handle, plan.handle, y.data_ptr(), scale, level, arr), "he_encode_vector")
        for p, a in zip(pts, arr):
            p.level, p.scale = a.level, a.scale
        return pts

    def encrypt_vector(self, plan: Plan, y: torch.Tensor, scale: float, level: int, nonce,
                       outs: list[Ciphertext] | None = None) -> list[Ciphertext]:
        """encode_vector then encrypt of each column block c in one call (he_encrypt_vector): nonce
        an int (block c under nonce + c) or an int64 device tensor of col_blocks nonces read when
        the kernels run."""
        y = _dev(y, torch.float64)
        cts = outs or [self.new_ct(level) for _ in range(plan.col_blocks)]
        arr = (HeCt * len(cts))(*[c.c() for c in cts])
        if isinstance(nonce, torch.Tensor):
            if nonce.numel() != plan.col_blocks or nonce.dtype != torch.int64 or not nonce.is_cuda:
                raise ValueError("device nonces: col_blocks int64 elements on the GPU")
            n_host, n_dev = 0, _vp(nonce.data_ptr())
        else:
            n_host, n_dev = nonce, None
        _check(_lib().he_encrypt_vector(self.handle, plan.handle, y.data_ptr(), scale, level, n_host, n_dev, arr), "he_encrypt_vector")
        for c, a in zip(cts, arr):
            c.level, c.scale = a.level, a.scale
        return cts

    def matmult(self, plan: Plan, pm: PtMatrix, cts: list[Ciphertext], outs: list[Ciphertext] | None = None) -> list[Ciphertext]:
        outs = outs or [self.new_ct(pm.level - 1) for _ in range(plan.row_blocks)]
        ins = (HeCt * len(cts))(*[c.c() for c in cts])
        oa = (HeCt * len(outs))(*[o.c() for o in outs])
        _check(_lib().he_matmult_plain_cipher(self.handle, plan.handle, pm.handle, ins, len(cts), oa, len(outs)), "he_matmult_plain_cipher")
        for o, a in zip(outs, oa):
            o.level, o.scale = a.level, a.scale
        return outs

    def matmult_noalloc(self, plan: Plan, pm: PtMatrix, cts: list[Ciphertext], outs: list[Ciphertext]) -> list[Ciphertext]:
        """he_matmult_plain_cipher_noalloc: the library allocates nothing; `outs` must be given."""
        ins = (HeCt * len(cts))(*[c.c() for c in cts])
        oa = (HeCt * len(outs))(*[o.c() for o in outs])
        _check(_lib().he_matmult_plain_cipher_noalloc(self.handle, plan.handle, pm.handle, ins, len(cts), oa, len(outs)),
               "he_matmult_plain_cipher_noalloc")
        for o, a in zip(outs, oa):
            o.level, o.scale = a.level, a.scale
        return outs

    def matmult_decode(self, plan: Plan, slots: torch.Tensor, out: torch.Tensor | None = None,
                       mask: torch.Tensor | None = None) -> torch.Tensor:
        """Lazy RaS of the decrypted slots [R][N/2]; with mask, of (slots - mask) (Alg. 1)."""
        slots = _dev(slots, torch.float64)
        out = out if out is not None else torch.empty(plan.m, dtype=torch.float64, device=self.device)
        if mask is None:
            _check(_lib().he_matmult_decode(self.handle, plan.handle, slots.data_ptr(), out.data_ptr()), "he_matmult_decode")
        else:
            mask = _dev(mask, torch.float64)
            _check(_lib().he_matmult_decode_masked(self.handle, plan.handle, slots.data_ptr(), mask.data_ptr(), out.data_ptr()),
                   "he_matmult_decode_masked")
        return out

    def matmult_decrypt(self, plan: Plan, cts: list[Ciphertext], out: torch.Tensor | None = None,
                        mask: torch.Tensor | None = None) -> torch.Tensor:
        """decrypt of each output ciphertext then matmult_decode in one call (he_matmult_decrypt)."""
        out = out if out is not None else torch.empty(plan.m, dtype=torch.float64, device=self.device)
        arr = (HeCt * len(cts))(*[c.c() for c in cts])
        mp = None
        if mask is not None:
            mask = _dev(mask, torch.float64)
            mp = _vp(mask.data_ptr())
        _check(_lib().he_matmult_decrypt(self.handle, plan.handle, arr, len(cts), mp, _vp(out.data_ptr())), "he_matmult_decrypt")
        return out

    # ---- VFL-NN forward pass with the encrypted matrix diagonally encoded (Alg. 3) ----
    def cdiag_encode_matrix(self, A: torch.Tensor, scale: float, level: int) -> list[Plaintext]:
        A = _dev(A, torch.float64)
        m, n = A.shape
        pts = [self.new_pt(level) for _ in range(min(m, n))]
        arr = (HePt * len(pts))(*[p.c() for p in pts])
        _check(_lib().he_cdiag_encode_matrix(self.handle, A.data_ptr(), m, n, scale, level, arr), "he_cdiag_encode_matrix")
        for p, a in zip(pts, arr):
            p.level, p.scale = a.level, a.scale
        return pts

    def cdiag_matmult(self, W: WeightMatrix, cts: list[Ciphertext], outs: list[Ciphertext] | None = None) -> list[Ciphertext]:
        outs = outs or [self.new_ct(W.level - 1) for _ in range(W.K)]
        ia = (HeCt * len(cts))(*[c.c() for c in cts])
        oa = (HeCt * len(outs))(*[o.c() for o in outs])
        _check(_lib().he_cdiag_matmult(self.handle, W.handle, ia, len(cts), oa), "he_cdiag_matmult")
        for o, a in zip(outs, oa):
            o.level, o.scale = a.level, a.scale
        return outs

    @staticmethod
    def cdiag_transpose_steps(m: int, n: int) -> list[int]:
        """Rotation steps he_cdiag_transpose needs keys for (he_cdiag_transpose_steps)."""
        cnt = ctypes.c_int()
        _check(_lib().he_cdiag_transpose_steps(m, n, None, ctypes.byref(cnt)), "he_cdiag_transpose_steps")
        arr = (ctypes.c_int32 * max(cnt.value, 1))()
        _check(_lib().he_cdiag_transpose_steps(m, n, arr, ctypes.byref(cnt)), "he_cdiag_transpose_steps")
        return [int(v) for v in arr[: cnt.value]]

    def cdiag_transpose(self, cts: list[Ciphertext], m: int, n: int) -> list[Ciphertext]:
        outs = [self.new_ct(cts[0].level) for _ in range(min(m, n))]
        ia = (HeCt * len(cts))(*[c.c() for c in cts])
        oa = (HeCt * len(outs))(*[o.c() for o in outs])
        _check(_lib().he_cdiag_transpose(self.handle, ia, m, n, oa), "he_cdiag_transpose")
        for o, a in zip(outs, oa):
            o.level, o.scale = a.level, a.scale
        return outs

    def cdiag_decode(self, m: int, n: int, slots: torch.Tensor) -> torch.Tensor:
        slots = _dev(slots, torch.float64)
        K = slots.shape[0]
        Z = torch.empty((m, K), dtype=torch.float64, device=self.device)
        _check(_lib().he_cdiag_decode(self.handle, m, n, K, slots.data_ptr(), Z.data_ptr()), "he_cdiag_decode")
        return Z

    # ---- host-memory forms (the party-facing calls; inputs and results in host memory) ----
    def encode_matrix_host(self, plan: Plan, X, level: int, out: PtMatrix | None = None, transposed: bool = False) -> PtMatrix:
        """he_encode_matrix_host / he_ptmat_encode_host: X a host tensor or array (m x n, or its
        n x m transpose with transposed=True)."""
        X = _host(X, torch.float64)
        if X.numel() != plan.m * plan.n:
            raise ValueError(f"matrix of {plan.m * plan.n} elements expected, got {X.numel()}")
        if out is not None:
            _check(_lib().he_ptmat_encode_host(self.handle, out.handle, X.data_ptr(), int(transposed)), "he_ptmat_encode_host")
            return out
        h = _vp()
        _check(_lib().he_encode_matrix_host(self.handle, plan.handle, X.data_ptr(), level, int(transposed), ctypes.byref(h)),
               "he_encode_matrix_host")
        return PtMatrix(self, h, plan, level)

    def encrypt_vector_host(self, plan: Plan, y, scale: float, level: int, nonce,
                            outs: list[Ciphertext] | None = None) -> list[Ciphertext]:
        """he_encrypt_vector_host: y a host tensor or array of n doubles; nonce as in encrypt_vector."""
        y = _host(y, torch.float64)
        if y.numel() != plan.n:
            raise ValueError(f"vector of {plan.n} elements expected, got {y.numel()}")
        cts = outs or [self.new_ct(level) for _ in range(plan.col_blocks)]
        arr = (HeCt * len(cts))(*[c.c() for c in cts])
        if isinstance(nonce, torch.Tensor):
            if nonce.numel() != plan.col_blocks or nonce.dtype != torch.int64 or not nonce.is_cuda:
                raise ValueError("device nonces: col_blocks int64 elements on the GPU")
            n_host, n_dev = 0, _vp(nonce.data_ptr())
        else:
            n_host, n_dev = nonce, None
        _check(_lib().he_encrypt_vector_host(self.handle, plan.handle, y.data_ptr(), scale, level, n_host, n_dev, arr),
               "he_encrypt_vector_host")
        for c, a in zip(cts, arr):
            c.level, c.scale = a.level, a.scale
        return cts

    def decrypt_host(self, ct: Ciphertext, out: torch.Tensor | None = None) -> torch.Tensor:
        """he_decrypt_host: N/2 slot values into a host tensor (valid on return unless `out` is
        pinned, in which case after synchronize())."""
        out = out if out is not None else torch.empty(self.slots, dtype=torch.float64)
        _host_out(out, self.slots)
        c = ct.c()
        _check(_lib().he_decrypt_host(self.handle, ctypes.byref(c), out.data_ptr()), "he_decrypt_host")
        return out

    def matmult_decrypt_host(self, plan: Plan, cts: list[Ciphertext], out: torch.Tensor | None = None, mask=None) -> torch.Tensor:
        """he_matmult_decrypt_host: the m results into a host tensor (valid on return unless `out`
        is pinned, in which case after synchronize()); mask a host [row_blocks][N/2] array or None."""
        out = out if out is not None else torch.empty(plan.m, dtype=torch.float64)
        _host_out(out, plan.m)
        arr = (HeCt * len(cts))(*[c.c() for c in cts])
        mp = None
        if mask is not None:
            mask = _host(mask, torch.float64)
            mp = _vp(mask.data_ptr())
        _check(_lib().he_matmult_decrypt_host(self.handle, plan.handle, arr, len(cts), mp, _vp(out.data_ptr())),
               "he_matmult_decrypt_host")
        return out

    def ct_export_host(self, ct: Ciphertext) -> bytes:
        """he_ct_export_host: the ciphertext serialized into bytes (header, primes, coefficients)."""
        c = ct.c()
        n = ctypes.c_size_t()
        _check(_lib().he_ct_export_host(self.handle, ctypes.byref(c), None, ctypes.byref(n)), "he_ct_export_host")
        buf = ctypes.create_string_buffer(n.value)
        _check(_lib().he_ct_export_host(self.handle, ctypes.byref(c), buf, ctypes.byref(n)), "he_ct_export_host")
        return buf.raw[: n.value]

    def ct_import_host(self, data: bytes) -> Ciphertext:
        """he_ct_import_host: a ciphertext from bytes made by ct_export_host under the same parameters."""
        buf = ctypes.create_string_buffer(bytes(data), len(data))
        lvl = _i32()
        _check(_lib().he_ct_host_level(buf, len(data), ctypes.byref(lvl)), "he_ct_host_level")
        ct = self.new_ct(int(lvl.value))
        c = ct.c()
        _check(_lib().he_ct_import_host(self.handle, buf, len(data), ctypes.byref(c)), "he_ct_import_host")
        ct.level, ct.scale = c.level, c.scale
        return ct

    def keyswitch_tuning(self) -> dict:
        """Transform variant of the many-rotation key switch (he_keyswitch_tuning): -1 before tuning."""
        v = ctypes.c_int()
        ms = (ctypes.c_float * HE_KS_VARIANTS)()
        _check(_lib().he_keyswitch_tuning(self.handle, ctypes.byref(v), ms), "he_keyswitch_tuning")
        return {"variant": int(v.value), "variant_ms": [round(float(x), 4) for x in ms],
                "variants": ["one CTA per limb-poly, usual threads", "one CTA per limb-poly, 512 threads, <= 64 registers",
                             "two phases of small CTAs per transform"]}

    def set_keyswitch_variant(self, v: int) -> None:
        """Pin the many-rotation key switch's transform variant (-1: time again)."""
        _check(_lib().he_set_keyswitch_variant(self.handle, v), "he_set_keyswitch_variant")

    def ntt_form(self) -> dict:
        """NTT form of launches of many limb-polys (he_ntt_form): 0 one CTA, 1 a 2-CTA cluster per
        limb-poly, 2 two phases (columns, then rows)."""
        f = ctypes.c_int()
        ms = (ctypes.c_float * HE_NTT_FORMS)()
        _check(_lib().he_ntt_form(self.handle, ctypes.byref(f), ms), "he_ntt_form")
        return {"form": int(f.value), "form_ms": [round(float(x), 4) for x in ms],
                "forms": ["one CTA per limb-poly", "2-CTA cluster per limb-poly", "two phases: 64-point columns, then rows"]}

    def set_ntt_form(self, form: int) -> None:
        _check(_lib().he_set_ntt_form(self.handle, form), "he_set_ntt_form")

    def set_key_fusion(self, mode: int, max_bytes: int = 0) -> None:
        """Fused key tables for the context family's encoded matrices (he_set_key_fusion):
        0 never, 1 when an encoding is multiplied again (default), 2 at the first MatMult."""
        _check(_lib().he_set_key_fusion(self.handle, mode, max_bytes), "he_set_key_fusion")

    # ---- basis extension engine of ModUp ----
    def set_basis_extension(self, engine: int) -> None:
        """HE_BCONV_INT64 (exact 64-bit products) or HE_BCONV_INT8_TC (byte-split products on the
        tensor cores, recombined exactly): same results, for this context's later calls."""
        _check(_lib().he_set_basis_extension(self.handle, engine), "he_set_basis_extension")

    def basis_extension(self) -> int:
        v = ctypes.c_int()
        _check(_lib().he_get_basis_extension(self.handle, ctypes.byref(v)), "he_get_basis_extension")
        return int(v.value)

    def modup_export(self, ct: Ciphertext, out: torch.Tensor) -> torch.Tensor:
        """ModUp digits of ct's c1, [ndig][level+1+K][N] canonical coefficient form (he_modup_export)."""
        c = ct.c()
        _check(_lib().he_modup_export(self.handle, ctypes.byref(c), out.data_ptr()), "he_modup_export")
        return out

    # ---- canonical coefficient form ----
    def ct_export(self, ct: Ciphertext) -> torch.Tensor:
        out = torch.empty_like(ct.data)
        c = ct.c()
        _check(_lib().he_ct_export(self.handle, ctypes.byref(c), out.data_ptr()), "he_ct_export")
        return out

    def ct_import(self, coeffs: torch.Tensor, level: int, scale: float) -> Ciphertext:
        coeffs = _dev(coeffs, torch.int64)
        ct = self.new_ct(level)
        c = ct.c()
        _check(_lib().he_ct_import(self.handle, coeffs.data_ptr(), level, scale, ctypes.byref(c)), "he_ct_import")
        ct.scale = scale
        return ct

    def pt_export(self, pt: Plaintext) -> torch.Tensor:
        out = torch.empty_like(pt.data)
        p = pt.c()
        _check(_lib().he_pt_export(self.handle, ctypes.byref(p), out.data_ptr()), "he_pt_export")
        return out

    def pt_import(self, coeffs: torch.Tensor, level: int, scale: float) -> Plaintext:
        coeffs = _dev(coeffs, torch.int64)
        pt = self.new_pt(level)
        p = pt.c()
        _check(_lib().he_pt_import(self.handle, coeffs.data_ptr(), level, scale, ctypes.byref(p)), "he_pt_import")
        pt.scale = scale
        return pt


def as_u64(t: torch.Tensor):
    """Device int64 residue tensor -> host numpy uint64 array."""
    return t.detach().cpu().numpy().view("uint64")


def from_u64(a, device) -> torch.Tensor:
    import numpy as np

    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).to(device)
