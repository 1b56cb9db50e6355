"""Pins of the oracle's integer arithmetic: primes, negacyclic products, automorphisms, Philox.

Each check compares the oracle with something other than itself: sympy's primality
test, a schoolbook product, numpy's polynomial convolution, the coefficient-packing
example of Sec. 3.2, numpy's Philox-4x64-10, and algebraic identities.
"""
import json
import os

import numpy as np
import pytest
import sympy

from oracle import ckks

GOLD = os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")


def test_is_prime_matches_sympy(oracle_lib):
    rng = np.random.default_rng(3)
    cands = [int(v) | 1 for v in rng.integers(1 << 40, 1 << 62, size=300, dtype=np.int64)]
    # Carmichael numbers and strong pseudoprimes to small bases
    cands += [561, 1105, 1729, 2465, 2821, 6601, 3215031751, 2152302898747, 3474749660383, 341550071728321]
    for c in cands:
        assert bool(oracle_lib.or_is_prime(c)) == sympy.isprime(c), c


@pytest.mark.parametrize("log_n,bits", [(12, [40, 20, 40]), (13, [60, 40, 40, 60]), (14, [60] + [40] * 6 + [60] * 3), (4, [60, 40])])
def test_prime_chain(log_n, bits):
    primes = ckks.gen_primes(log_n, bits)
    two_n = 2 << log_n
    assert len(set(primes)) == len(primes)
    for i, (q, b) in enumerate(zip(primes, bits)):
        assert sympy.isprime(q)
        assert q % two_n == 1
        assert q.bit_length() == b
        # nothing larger below 2^b qualifies, except primes taken earlier in the chain
        c = q + two_n
        while c < (1 << b):
            assert (not sympy.isprime(c)) or c in primes[:i], (q, c)
            c += two_n


def _rand_poly(rng, n, q):
    return np.array([int(v) % q for v in rng.integers(0, 1 << 62, size=n, dtype=np.int64)], dtype=np.uint64)


@pytest.mark.parametrize("n", [4, 16, 64, 256])
def test_poly_mul_equals_schoolbook(oracle_lib, n):
    rng = np.random.default_rng(n)
    log_n = n.bit_length() - 1
    for q in ckks.gen_primes(log_n, [60, 40, 30]):
        a, b = _rand_poly(rng, n, q), _rand_poly(rng, n, q)
        s, f = np.zeros(n, np.uint64), np.zeros(n, np.uint64)
        oracle_lib.or_negacyclic_schoolbook(n, q, a, b, s)
        oracle_lib.or_poly_mul(n, q, a, b, f)
        assert np.array_equal(s, f)


def test_schoolbook_matches_numpy_convolution(oracle_lib):
    """Small integers: the negacyclic product is the plain product folded with X^N = -1."""
    rng = np.random.default_rng(7)
    n, q = 32, ckks.gen_primes(5, [40])[0]
    a = rng.integers(-50, 50, size=n)
    b = rng.integers(-50, 50, size=n)
    full = np.convolve(a, b)  # degree 2N-2
    want = full[:n].copy()
    want[: n - 1] -= full[n:]
    out = np.zeros(n, np.uint64)
    oracle_lib.or_negacyclic_schoolbook(n, q, (a % q).astype(np.uint64), (b % q).astype(np.uint64), out)
    assert np.array_equal(out, (want % q).astype(np.uint64))


def test_coefficient_packing_example(oracle_lib):
    """Sec. 3.2: in Z_q[X]/(X^16+1), coefficient 2i+1 of X~ y~ is row i's dot product."""
    ex = json.load(open(GOLD))["cheetah_product"]
    rng = np.random.default_rng(11)
    vals = {f"{r}{c}": int(rng.integers(1, 1000)) for r in "ABCD" for c in "01"}
    vals.update({"M0": int(rng.integers(1, 1000)), "M1": int(rng.integers(1, 1000))})
    n = ex["ring_degree"]
    q = ckks.gen_primes(4, [50])[0]
    x = np.zeros(n, np.uint64)
    y = np.zeros(n, np.uint64)
    for i, s in enumerate(ex["x_coeffs"]):
        x[i] = vals[s]
    for i, s in enumerate(ex["y_coeffs"]):
        y[i] = vals[s]
    out = np.zeros(n, np.uint64)
    oracle_lib.or_negacyclic_schoolbook(n, q, x, y, out)
    for pos, row in ex["dot_positions"].items():
        assert int(out[int(pos)]) == vals[row + "0"] * vals["M0"] + vals[row + "1"] * vals["M1"]


def test_ntt_round_trip_and_evaluation(oracle_lib):
    """Forward transform = evaluation at the odd powers of a primitive 2N-th root."""
    n = 16
    q = ckks.gen_primes(4, [30])[0]
    rng = np.random.default_rng(5)
    a = _rand_poly(rng, n, q)
    f = a.copy()
    oracle_lib.or_ntt_forward(n, q, f)
    # find the primitive 2N-th root psi with f[0] = a(psi), then check f[k] = a(psi^(2k+1))
    psi = None
    for k0 in range(1, 200):
        cand = pow(k0, (q - 1) // (2 * n), q)
        if pow(cand, n, q) == q - 1 and sum(int(a[j]) * pow(cand, j, q) for j in range(n)) % q == int(f[0]):
            psi = cand
            break
    assert psi is not None
    for k in range(n):
        r = pow(psi, 2 * k + 1, q)
        assert sum(int(a[j]) * pow(r, j, q) for j in range(n)) % q == int(f[k])
    oracle_lib.or_ntt_inverse(n, q, f)
    assert np.array_equal(f, a)


def test_automorphism_is_ring_homomorphism_and_composes(oracle_lib):
    n = 64
    q = ckks.gen_primes(6, [40])[0]
    rng = np.random.default_rng(9)
    a, b = _rand_poly(rng, n, q), _rand_poly(rng, n, q)
    ab = np.zeros(n, np.uint64)
    oracle_lib.or_poly_mul(n, q, a, b, ab)
    for g1, g2 in [(5, 25), (3, 2 * n - 1), (125, 7)]:
        pa, pb, pab, lhs = (np.zeros(n, np.uint64) for _ in range(4))
        oracle_lib.or_automorph(n, q, g1, a, pa)
        oracle_lib.or_automorph(n, q, g1, b, pb)
        oracle_lib.or_automorph(n, q, g1, ab, pab)
        oracle_lib.or_poly_mul(n, q, pa, pb, lhs)
        assert np.array_equal(lhs, pab)
        t, u, v = (np.zeros(n, np.uint64) for _ in range(3))
        oracle_lib.or_automorph(n, q, g2, a, t)
        oracle_lib.or_automorph(n, q, g1, t, u)
        oracle_lib.or_automorph(n, q, (g1 * g2) % (2 * n), a, v)
        assert np.array_equal(u, v)
    # X -> X^g sends the monomial X^k to X^(kg) with X^N = -1
    for k in [0, 1, 5, n - 1]:
        mono = np.zeros(n, np.uint64)
        mono[k] = 1
        out = np.zeros(n, np.uint64)
        oracle_lib.or_automorph(n, q, 5, mono, out)
        e = (5 * k) % (2 * n)
        want = np.zeros(n, np.uint64)
        want[e % n] = 1 if e < n else q - 1
        assert np.array_equal(out, want)


def test_philox_matches_numpy(oracle_lib):
    """numpy's Philox is Philox-4x64-10 and increments the counter before each block."""
    for key in ([0, 0], [5, 7], [2**64 - 1, 12345]):
        for ctr in ([0, 0, 0, 0], [17, 3, 9, 0], [2**64 - 2, 1, 2, 3]):
            g = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(ctr, dtype=np.uint64))
            want = g.random_raw(4)
            nxt = list(ctr)
            nxt[0] = (nxt[0] + 1) % 2**64
            if nxt[0] == 0:
                nxt[1] += 1
            out = np.zeros(4, np.uint64)
            oracle_lib.or_philox4x64(np.array(nxt, dtype=np.uint64), np.array(key, dtype=np.uint64), out)
            assert np.array_equal(out, want.astype(np.uint64))


def test_samplers_distributions(oracle_lib):
    n = 1 << 16
    s = np.zeros(n, np.int64)
    oracle_lib.or_sample_ternary(n, 42, s)
    counts = np.array([(s == v).sum() for v in (-1, 0, 1)])
    assert counts.sum() == n
    chi2 = (((counts - n / 3) ** 2) / (n / 3)).sum()
    assert chi2 < 13.8  # 2 dof, p = 0.001

    e = np.zeros(n, np.int64)
    oracle_lib.or_sample_gauss(n, 42, 3, 0, e)
    assert np.abs(e).max() <= 19
    ys = np.arange(-19, 20)
    rho = np.exp(-(ys.astype(float) ** 2) / (2 * 3.2**2))
    p = rho / rho.sum()
    obs = np.array([(e == y).sum() for y in ys])
    keep = p * n > 5
    chi2 = (((obs[keep] - n * p[keep]) ** 2) / (n * p[keep])).sum()
    assert chi2 < 45.0  # ~20 dof, p = 0.001
    assert abs(e.std() - 3.2) < 0.05

    q = ckks.gen_primes(13, [60])[0]
    u = np.zeros(n, np.uint64)
    oracle_lib.or_sample_uniform(n, 42, 4, 9, 2, q, u)
    assert int(u.max()) < q
    assert abs(u.astype(float).mean() / q - 0.5) < 0.01
    # streams differ by tag, nonce and limb
    u2 = np.zeros(n, np.uint64)
    oracle_lib.or_sample_uniform(n, 42, 4, 10, 2, q, u2)
    assert not np.array_equal(u, u2)


def test_cdt_table_shape(oracle_lib):
    t = np.zeros(38, np.uint64)
    oracle_lib.or_cdt_table(t)
    assert np.all(np.diff(t.astype(object)) > 0)
    assert int(t[-1]) < 2**40
    # the 40-bit thresholds reproduce the probabilities to 2^-40
    ys = np.arange(-19, 20)
    rho = np.exp(-(ys.astype(float) ** 2) / 20.48)
    cdf = np.cumsum(rho / rho.sum())[:38]
    assert np.abs(t.astype(float) / 2**40 - cdf).max() < 1e-11
