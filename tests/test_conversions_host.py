"""Host mirrors of the FFT kernels' integer conversions and of the sampler's 128-bit reduction,
checked against the conversions they replace (no GPU).  The device code avoids GB300's FP64
pipe; these tests pin the methods, written here with the same steps on 64-bit integers and
IEEE single precision:

- double -> (hi, lo) float pair: hi = the significand rounded to 24 bits (ties to even, a carry
  raising the exponent), lo = the remainder in units of the last place, converted and scaled; the
  same pair as two FP64 conversions for 2^-60 <= |x| < 2^101;
- uint64 -> double rounded to nearest, from the leading bit's position;
- float -> double by re-biasing the exponent (normal floats);
- the nearest integer to hi + lo as rint(hi) plus the rounded remainder, exact except within
  2^-24 of a half-integer;
- (hi 2^64 + lo) mod q by Barrett reduction of hi, Montgomery reduction and a Montgomery product
  by 2^128 mod q."""
from fractions import Fraction
import math
import struct

import numpy as np
import pytest

RNG = np.random.default_rng(20251203)
M64 = (1 << 64) - 1


def dbits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def bits_d(u):
    return struct.unpack("<d", struct.pack("<Q", u))[0]


def fbits(f):
    return struct.unpack("<I", struct.pack("<f", f))[0]


def bits_f(u):
    return float(struct.unpack("<f", struct.pack("<I", u))[0])


def f32(x):
    return float(np.float32(x))


def df_from_ref(x):
    h = f32(x)
    return h, f32(x - h)


def df_from_int(x):
    b = dbits(x)
    E = (b >> 52) & 0x7FF
    if not (1023 - 60 <= E <= 1023 + 100):
        return df_from_ref(x)
    M = (b & ((1 << 52) - 1)) | (1 << 52)
    Mh, r = M >> 29, M & ((1 << 29) - 1)
    Mh += 1 if (r > (1 << 28) or (r == (1 << 28) and (Mh & 1))) else 0
    rem = M - (Mh << 29)
    sgn = b >> 63
    hi = bits_f((sgn << 31) | ((E - 896 + (Mh >> 24)) << 23) | (Mh & 0x7FFFFF))
    scale = bits_f((E - 1075 + 127) << 23)
    lo = f32(np.float32(np.float32(-rem if sgn else rem) * np.float32(scale)))
    return hi, lo


def u64_to_double_rn(u):
    if u == 0:
        return 0.0
    e = u.bit_length() - 1
    if e <= 52:
        mant = u << (52 - e)
    else:
        sh = e - 52
        mant, rem, half = u >> sh, u & ((1 << sh) - 1), 1 << (sh - 1)
        mant += 1 if (rem > half or (rem == half and (mant & 1))) else 0
        if mant >> 53:
            mant >>= 1
            e += 1
    return bits_d(((e + 1023) << 52) | (mant & ((1 << 52) - 1)))


def f2d_exact(f):
    b = fbits(f)
    e = (b >> 23) & 0xFF
    if e in (0, 0xFF):
        return float(np.float64(np.float32(f)))
    return bits_d(((b >> 31) << 63) | ((e + 896) << 52) | ((b & 0x7FFFFF) << 29))


def rint_f(x):
    x = np.float32(x)
    if abs(x) < np.float32(8388608.0):
        m = np.float32(math.copysign(8388608.0, x))
        return np.float32(np.float32(x + m) - m)
    return x


def f2ll_integral(f):
    b = fbits(float(f))
    e = ((b >> 23) & 0xFF) - 150
    m = (b & 0x7FFFFF) | 0x800000
    v = m << e if e >= 0 else (m >> -e if e > -24 else 0)
    return -v if b >> 31 else v


def df_round_ll(hi, lo):
    rh = rint_f(hi)
    d = np.float32(np.float32(np.float32(hi) - rh) + np.float32(lo))
    return f2ll_integral(rh) + f2ll_integral(rint_f(d))


def random_doubles(n):
    mags = RNG.integers(-70, 110, n)
    x = RNG.uniform(-1, 1, n) * np.ldexp(1.0, mags)
    x[::7] = np.floor(x[::7]) + 0.5  # halves
    return [float(v) for v in x]


def test_df_from_matches_fp64_conversions():
    for x in random_doubles(20000) + [0.0, -0.0, 1.0, -1.0, 2.0**100, 2.0**-60, 3.0 * 2.0**-61]:
        h, l = df_from_int(x)
        hr, lr = df_from_ref(x)
        assert fbits(h) == fbits(hr) and (l == lr or (l == 0 and lr == 0)), x
    # significands whose 29 dropped bits are exactly half a unit (ties to even both ways)
    for m in range(1 << 20, (1 << 20) + 64):
        x = math.ldexp((m << 29 | (1 << 28)) + 0.0, -40)
        assert df_from_int(x)[0] == df_from_ref(x)[0]


def test_u64_to_double_rounds_to_nearest_even():
    us = [int(v) for v in RNG.integers(0, 2**63, 20000, dtype=np.int64)]
    us += [(1 << 53) + 1, (1 << 53) + 3, (1 << 64) - 1, (1 << 60) + (1 << 7), 1, 0, (1 << 62) - 1]
    for u in us:
        assert dbits(u64_to_double_rn(u)) == dbits(float(u)), u


def test_f2d_exact():
    for b in list(RNG.integers(0, 2**32, 20000, dtype=np.uint64)) + [0x00800000, 0x7F7FFFFF, 0x80000000, 0x00000001]:
        f = bits_f(int(b))
        if f != f:
            continue
        assert dbits(f2d_exact(f)) == dbits(float(np.float64(np.float32(f))))


def test_df_round_matches_exact_rounding_outside_the_tie_window():
    for x in random_doubles(20000):
        if abs(x) >= 2.0**62:
            continue
        hi, lo = df_from_ref(x)
        ex = Fraction(hi) + Fraction(lo)
        fl = math.floor(ex)
        frac = ex - fl
        got = df_round_ll(hi, lo)
        if abs(frac - Fraction(1, 2)) <= Fraction(1, 2**23) * max(1, abs(Fraction(lo))):
            assert got in (fl, fl + 1)
        else:
            assert got == (fl + 1 if frac > Fraction(1, 2) else fl), x


@pytest.mark.parametrize("bits", [20, 40, 60])
def test_mod128_is_the_residue(bits):
    qs = []
    while len(qs) < 6:
        q = int(RNG.integers(2**(bits - 1), 2**bits)) | 1
        qs.append(q)
    for q in qs:
        mu = (1 << 64) // q
        qinv = (-pow(q, -1, 1 << 64)) & M64
        r2 = (1 << 128) % q

        def barrett(x):
            r = (x - ((x * mu) >> 64) * q) & M64
            return r - q if r >= q else r

        def redc(hi, lo):
            m = (lo * qinv) & M64
            r = hi + ((m * q) >> 64) + (1 if lo else 0)
            return r - q if r >= q else r

        def mont_mul(a, b):
            t = a * b
            return redc(t >> 64, t & M64)

        cases = [(int(RNG.integers(0, 2**63)) * 2 + int(RNG.integers(0, 2)), int(RNG.integers(0, 2**63)) * 2 + int(RNG.integers(0, 2)))
                 for _ in range(400)]
        cases += [(0, 0), (M64, M64), (M64, 0), (0, M64), (q - 1, 0), (q, 1)]
        for hi, lo in cases:
            assert mont_mul(redc(barrett(hi), lo), r2) == ((hi << 64) | lo) % q
