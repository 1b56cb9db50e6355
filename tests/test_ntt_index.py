"""Host-side check of the NTT passes' shared-memory addressing: element base + (k << lg) of a
pass sits at SIDX(base) - SIDX(off) + SIDX(k << lg), SIDX(x) = x + (x >> 5), for every pass shape
the one-CTA and cluster transforms use (log N = 4..14), so the kernels address a set's elements
as one base plus constant offsets."""
import numpy as np
import pytest


def sidx(x):
    return x + (x >> 5)


def one_cta_passes(logn):
    out, s0, first = [], 0, logn % 4
    while s0 < logn:  # forward: the remainder pass first
        nb = first if (s0 == 0 and first) else 4
        out.append(("f", s0, nb))
        s0 += nb
    s0 = 0
    while s0 < logn:  # inverse: the remainder pass last
        nb = min(4, logn - s0)
        out.append(("i", s0, nb))
        s0 += nb
    return out


def cluster_passes(logn):  # radix-2 passes on a slice of N/8: forward stages 3.., inverse ..logn-4
    return [("f", s0, 1) for s0 in range(3, logn)] + [("i", s0, 1) for s0 in range(0, logn - 3)]


def check(logn, kind, s0, nb, off, sets):
    lg_t0 = logn - 1 - s0 if kind == "f" else s0
    lg = lg_t0 - (nb - 1) if kind == "f" else s0
    gshift = lg_t0 + 1 if kind == "f" else s0 + nb
    g, low = sets >> lg, sets & ((1 << lg) - 1)
    base = (g << gshift) + low
    for k in range(1 << nb):
        x = base + (k << lg)
        assert np.array_equal(sidx(x - off), sidx(base) - sidx(off) + sidx(k << lg))


@pytest.mark.parametrize("logn", range(4, 15))
def test_pass_addressing(logn):
    N = 1 << logn
    for kind, s0, nb in one_cta_passes(logn):
        check(logn, kind, s0, nb, 0, np.arange(N >> nb, dtype=np.int64))
    if logn >= 10:
        NS = N >> 3
        for kind, s0, nb in cluster_passes(logn):
            for rank in range(8):
                check(logn, kind, s0, nb, rank * NS, np.arange(rank * (NS >> nb), (rank + 1) * (NS >> nb), dtype=np.int64))
