"""CKKS encoding and decoding on the CPU (oracle side).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the library.

Sec. 2.2: a cleartext vector of N' = N/2 slots is mapped to an integer polynomial
of Z_q[X]/(X^N+1) by the CKKS canonical-embedding encoding.  Slot j sits at the
root zeta^(5^j mod 2N), zeta = exp(i pi / N); the conjugate root carries the
conjugate value, so a real vector gives a real polynomial.

Definition (all j < N', k < N):
    encode:  m_k = rint( scale * (2/N) * Re( sum_j z_j zeta^(-k 5^j) ) )   (round half to even)
    decode:  z_j = (1/scale) * sum_k m_k zeta^(k 5^j)

`encode_direct` / `decode_direct` are those sums written out (O(N^2)); `encode` /
`decode` evaluate the same sums with a length-N FFT over all 2N-th odd roots.
"""
from __future__ import annotations

import numpy as np


def slot_exponents(n: int) -> np.ndarray:
    """e_j = 5^j mod 2N for j < N/2 (the root exponent of slot j)."""
    e = np.empty(n // 2, dtype=np.int64)
    v = 1
    for j in range(n // 2):
        e[j] = v
        v = (v * 5) % (2 * n)
    return e


def _pad(z, n):
    z = np.asarray(z, dtype=np.complex128)
    out = np.zeros(n // 2, dtype=np.complex128)
    out[: len(z)] = z
    return out


def encode_real(z, scale: float, n: int) -> np.ndarray:
    """scale * sigma^{-1}(z) before rounding (float64 vector of length N), by FFT.

    With F(e) the value at root zeta^e (z_j at e_j, conj(z_j) at 2N - e_j) and e = 2t + 1:
        m_k = (1/N) sum_t F(2t+1) zeta^(-k(2t+1)) = (1/N) zeta^(-k) * DFT(F(2t+1))[k].
    """
    z = _pad(z, n)
    e = slot_exponents(n)
    F = np.zeros(n, dtype=np.complex128)
    F[(e - 1) // 2] = z
    F[(2 * n - e - 1) // 2] = np.conj(z)
    k = np.arange(n)
    twist = np.exp(-1j * np.pi * k / n)
    m = (twist * np.fft.fft(F)).real / n
    return scale * m


def encode(z, scale: float, n: int) -> np.ndarray:
    """Integer coefficients (int64), round half to even."""
    return np.rint(encode_real(z, scale, n)).astype(np.int64)


def encode_direct_real(z, scale: float, n: int) -> np.ndarray:
    """The defining sum, O(N^2): scale * (2/N) Re(sum_j z_j zeta^(-k e_j))."""
    z = _pad(z, n)
    # exponent k*e_j reduced mod 2N keeps the angle argument small and exact
    ke = np.mod(np.outer(np.arange(n, dtype=np.int64), slot_exponents(n)), 2 * n).astype(np.float64)
    w = np.exp(-1j * np.pi * ke / n)
    return scale * (2.0 / n) * (w @ z).real


def decode(m, scale: float, n: int) -> np.ndarray:
    """Slots of an integer (or real) coefficient vector, by inverse FFT:
    z_j = (1/scale) sum_k m_k zeta^k exp(2 pi i k t_j / N),  e_j = 2 t_j + 1."""
    m = np.asarray(m, dtype=np.float64)
    k = np.arange(n)
    v = np.fft.ifft(m * np.exp(1j * np.pi * k / n)) * n
    t = (slot_exponents(n) - 1) // 2
    return v[t] / scale


def decode_direct(m, scale: float, n: int) -> np.ndarray:
    """The defining sum, O(N^2)."""
    m = np.asarray(m, dtype=np.float64)
    ke = np.mod(np.outer(slot_exponents(n), np.arange(n, dtype=np.int64)), 2 * n).astype(np.float64)
    return (np.exp(1j * np.pi * ke / n) @ m) / scale
