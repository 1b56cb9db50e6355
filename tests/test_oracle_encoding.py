"""Pins of the oracle's CKKS encoding (Sec. 2.2): FFT form against the defining sums,
closed forms, round trips and the slot rotation induced by X -> X^5."""
import numpy as np
import pytest

from oracle import encoding as E


@pytest.mark.parametrize("n", [8, 64, 1024])
def test_fft_encode_equals_definition(n):
    rng = np.random.default_rng(n)
    z = rng.uniform(-1, 1, n // 2)
    a = E.encode_real(z, 2.0**30, n)
    b = E.encode_direct_real(z, 2.0**30, n)
    assert np.abs(a - b).max() < 1e-6 * 2**30 / n * 10
    m = E.encode(z, 2.0**30, n)
    assert np.allclose(E.decode(m, 2.0**30, n), E.decode_direct(m, 2.0**30, n), atol=1e-9)


def test_round_trip():
    n = 8192
    z = np.random.default_rng(0).uniform(-1, 1, n // 2)
    m = E.encode(z, 2.0**40, n)
    out = E.decode(m, 2.0**40, n)
    # rounding error 1/2 per coefficient, decode gain sqrt(N)
    assert np.abs(out.real - z).max() < 4 * np.sqrt(n) / 2**40
    assert np.abs(out.imag).max() < 4 * np.sqrt(n) / 2**40


def test_closed_forms():
    n = 64
    # a constant vector is the constant polynomial
    m = E.encode(np.full(n // 2, 3.0), 1.0, n)
    assert m[0] == 3 and not m[1:].any()
    # the monomial X^k has slot j equal to zeta^(k 5^j)
    e = E.slot_exponents(n)
    for k in (1, 3, n - 1):
        mono = np.zeros(n)
        mono[k] = 1.0
        want = np.exp(1j * np.pi * k * e / n)
        assert np.allclose(E.decode(mono, 1.0, n), want, atol=1e-12)
    # real-linear
    rng = np.random.default_rng(1)
    x, y = rng.normal(size=n // 2), rng.normal(size=n // 2)
    assert np.allclose(E.encode_real(2 * x - y, 1.0, n), 2 * E.encode_real(x, 1.0, n) - E.encode_real(y, 1.0, n))


def _automorph_real(m, g):
    n = len(m)
    out = np.zeros(n)
    for k in range(n):
        t = (k * g) % (2 * n)
        if t < n:
            out[t] = m[k]
        else:
            out[t - n] = -m[k]
    return out


@pytest.mark.parametrize("r", [1, 2, 7, 31])
def test_x_to_x5_rotates_slots_left(r):
    """phi_{5^r}(m) decodes to RotL(z, r): the rotation direction of Sec. 3.1.1."""
    n = 64
    z = np.random.default_rng(r).uniform(-1, 1, n // 2)
    m = E.encode_real(z, 1.0, n)
    out = E.decode(_automorph_real(m, pow(5, r, 2 * n)), 1.0, n)
    assert np.allclose(out.real, np.roll(z, -r), atol=1e-12)
    # and the conjugate Galois element 2N-1 leaves real slots unchanged
    assert np.allclose(E.decode(_automorph_real(m, 2 * n - 1), 1.0, n).real, z, atol=1e-12)
