"""Host-side check of the lane schedules of the cluster transforms (no GPU): which elements each
lane holds at each stage when butterflies are spread over lanes that swap elements by warp
shuffle, written with the index formulas of the kernels and run on element labels.

- the cross-CTA stages of the cluster NTT (four lanes per offset; forward pairs c with c + 4, + 2,
  + 1, inverse with + 1, + 2, + 4) and of the cluster FFT (2^(CLG-1) lanes, pairs c with c + 2^st),
  and the fused inverse-then-forward step of the ModUp (the forward stages start on the inverse's
  last pairs);
- the two-stage passes of the NTT (forward and inverse) and of the FFT (two lanes per set of four);
- the row phase's radix-16 pass on lane pairs (eight elements per lane, one swap before the last
  stage);
- the pass schedules (every stage exactly once, the forward transform's last pass flagged) and the
  thread counts (whole warps in every iteration of a shuffle loop).

Each stage's pairs must be exactly the butterflies of the stage-by-stage transform, each element
written once at the end: the values are then those of the radix-2 form, which the GPU tests
compare bit for bit."""
import pytest


def ins_bit(v, b):
    return (v & ((1 << b) - 1)) | ((v >> b) << (b + 1))


def del_bit(v, b):
    return (v & ((1 << b) - 1)) | ((v >> (b + 1)) << b)


def stage_pairs(n, b):
    """The butterflies of a radix-2 stage over n elements pairing c with c + 2^b."""
    return {(c, c | (1 << b)) for c in range(n) if not (c >> b) & 1}


def run_cross(bits, lanes):
    """Lane p starts with the pair (ins(p, b0), + 2^b0); before each later stage it takes its pair
    from the lanes that held the two elements (element c at lane del(c, b_prev), slot bit b_prev
    of c).  Returns the pairs of every stage and the final holdings."""
    hold = {p: (ins_bit(p, bits[0]), ins_bit(p, bits[0]) | (1 << bits[0])) for p in range(lanes)}
    seen = [set(hold.values())]
    for st in range(1, len(bits)):
        b, bp = bits[st], bits[st - 1]
        new = {}
        for p in range(lanes):
            nlo = ins_bit(p, b)
            nhi = nlo | (1 << b)
            a = hold[del_bit(nlo, bp)]
            c = hold[del_bit(nhi, bp)]
            x0 = a[(nlo >> bp) & 1]
            x1 = c[(nhi >> bp) & 1]
            assert (x0, x1) == (nlo, nhi)
            new[p] = (x0, x1)
        hold = new
        seen.append(set(hold.values()))
    return seen, hold


@pytest.mark.parametrize("fwd", [True, False])
def test_ntt_cross_step(fwd):
    bits = (2, 1, 0) if fwd else (0, 1, 2)
    seen, hold = run_cross(bits, 4)
    for st, b in enumerate(bits):
        assert seen[st] == stage_pairs(8, b)
    # the final stores: lane p writes its lo and lo + 2^b_last, every element once
    written = sorted(x for p in range(4) for x in hold[p])
    assert written == list(range(8))
    for p in range(4):
        lo = ins_bit(p, bits[-1])
        assert hold[p] == (lo, lo | (1 << bits[-1]))


def test_modup_inverse_then_forward():
    _, hold = run_cross((0, 1, 2), 4)
    # the forward stages take each lane's holdings as their first pair: (ins(p, 2), + 4)
    for p in range(4):
        assert hold[p] == (ins_bit(p, 2), ins_bit(p, 2) | 4)
    seen, hold2 = run_cross((2, 1, 0), 4)
    assert seen[0] == stage_pairs(8, 2)
    assert sorted(x for p in range(4) for x in hold2[p]) == list(range(8))


@pytest.mark.parametrize("clg", [1, 2, 3])
def test_fft_cross_step(clg):
    bits = tuple(range(clg))
    seen, hold = run_cross(bits, max(1, (1 << clg) // 2))
    for st, b in enumerate(bits):
        assert seen[st] == stage_pairs(1 << clg, b)
    assert sorted(x for p in hold for x in hold[p]) == list(range(1 << clg))


def test_ntt_forward_pair_pass():
    # elements k of a set (stride 2^lg_tl); stage s0 pairs k, k + 2, stage s0 + 1 pairs k, k + 1
    x = {p: [p, p + 2] for p in (0, 1)}
    assert {tuple(v) for v in x.values()} == {(0, 2), (1, 3)}
    send = {p: x[p][0] if p else x[p][1] for p in (0, 1)}
    for p in (0, 1):
        got = send[p ^ 1]
        if p:
            x[p][0] = got
        else:
            x[p][1] = got
    assert x[0] == [0, 1] and x[1] == [2, 3]
    # stored at 2p, 2p + 1
    assert sorted(k for p in (0, 1) for k in (2 * p, 2 * p + 1)) == [0, 1, 2, 3]


def test_ntt_inverse_pair_pass():
    # stage s0 pairs k, k + 1 (lane p: 2p, 2p + 1), stage s0 + 1 pairs k, k + 2 (lane p: p, p + 2)
    x = {p: [2 * p, 2 * p + 1] for p in (0, 1)}
    send = {p: x[p][0] if p else x[p][1] for p in (0, 1)}
    for p in (0, 1):
        got = send[p ^ 1]
        if p:
            x[p][0] = got
        else:
            x[p][1] = got
    assert x[0] == [0, 2] and x[1] == [1, 3]
    assert sorted(k for p in (0, 1) for k in (p, p + 2)) == [0, 1, 2, 3]


def test_fft_pair_pass():
    # stage s0 pairs (0, 1), (2, 3) (lane p: 2p, 2p + 1); then (0, 2), (1, 3) (lane p: p, p + 2)
    x = {p: [2 * p, 2 * p + 1] for p in (0, 1)}
    sent = {p: x[p][0] if p else x[p][1] for p in (0, 1)}
    y = {}
    for p in (0, 1):
        got = sent[p ^ 1]
        y[p] = [got, x[p][1]] if p else [x[p][0], got]
    assert y[0] == [0, 2] and y[1] == [1, 3]


def test_row_pass_radix16_on_lane_pairs():
    # lane p holds k = 2i + p, i < 8
    r = {p: [2 * i + p for i in range(8)] for p in (0, 1)}
    for j in range(3):  # stages with k-distance 8, 4, 2 stay within a lane (i-distance 4, 2, 1)
        hi = 4 >> j
        pairs = set()
        for p in (0, 1):
            for i in range(8):
                if (i & (2 * hi - 1)) < hi:
                    pairs.add((r[p][i], r[p][i + hi]))
        assert pairs == stage_pairs(16, 3 - j)
    got = {p: [r[p ^ 1][u] if (p ^ 1) else r[p ^ 1][4 + u] for u in range(4)] for p in (0, 1)}
    pairs, stored = set(), []
    for p in (0, 1):
        for u in range(4):
            i = 4 * p + u
            a = got[p][u] if p else r[p][u]
            b = r[p][4 + u] if p else got[p][u]
            assert (a, b) == (2 * i, 2 * i + 1)
            pairs.add((a, b))
            stored += [2 * i, 2 * i + 1]
    assert pairs == stage_pairs(16, 0)
    assert sorted(stored) == list(range(16))


@pytest.mark.parametrize("logn", range(10, 17))
def test_cluster_ntt_schedules(logn):
    fwd, s0 = [], 3
    while s0 + 1 < logn:
        fwd.append((s0, 2, s0 + 2 == logn))
        s0 += 2
    if (logn - 3) & 1:
        fwd.append((logn - 1, 1, True))
    stages = [s for s0, nb, _ in fwd for s in range(s0, s0 + nb)]
    assert stages == list(range(3, logn))
    assert [last for *_, last in fwd] == [False] * (len(fwd) - 1) + [True]
    inv, s0 = [], 0
    while s0 + 1 < logn - 3:
        inv.append((s0, 2))
        s0 += 2
    if (logn - 3) & 1:
        inv.append((logn - 4, 1))
    assert [s for s0, nb in inv for s in range(s0, s0 + nb)] == list(range(0, logn - 3))
    # shuffle loops: NS / 2 lane-slots (pairs and cross step), blockDim = min(512, NS / 2)
    NS = 1 << (logn - 3)
    threads = min(512, NS // 2)
    assert (NS // 2) % 32 == 0 and (NS // 2) % threads == 0 and threads % 32 == 0


@pytest.mark.parametrize("logn", range(10, 17))
@pytest.mark.parametrize("clg", [1, 2, 3])
def test_cluster_fft_schedules(logn, clg):
    lg_ms = logn - 1 - clg
    MS = 1 << lg_ms
    passes, s0 = [], 0
    while s0 + 1 < lg_ms:
        passes.append((s0, 2))
        s0 += 2
    if lg_ms & 1:
        passes.append((lg_ms - 1, 1))
    assert [s for s0, nb in passes for s in range(s0, s0 + nb)] == list(range(lg_ms))
    threads = min(512, max(32, MS // 2))
    assert (MS // 2) % 32 == 0 and (MS // 2) % threads == 0


@pytest.mark.parametrize("m,n,log_n", [(256, 1024, 13), (1024, 256, 13), (16, 64, 12), (64, 16, 12), (9000, 2, 13), (300, 5000, 13),
                                       (700, 300, 13), (4096, 256, 14), (100, 20, 11), (20, 100, 10)])
def test_decode_rotate_and_sum_terms(m, n, log_n):
    """The decode's rotate-and-sum epilogue (DecodeRas): row rem of a block goes to CTA rem mod CL,
    its terms s < nb/m' read slot ((rem >> lm) << lnb) + (rem mod m') + (s << lm).  Over a block's
    rows every slot is read at most once, so each CTA's rows x terms fit the MS doubles of its
    twiddle copy (the fast path's condition) for the cluster sizes the decoder picks."""
    from oracle import layout

    slots = 1 << (log_n - 1)
    p = layout.make_plan(m, n, slots)
    mb, nb, mp = p.mb, p.nb, p.m_prime
    lm, lnb = mp.bit_length() - 1, nb.bit_length() - 1
    terms = nb >> lm
    seen = set()
    for rem in range(mb):
        for s in range(terms):
            j = ((rem >> lm) << lnb) + (rem & (mp - 1)) + (s << lm)
            assert 0 <= j < slots and j not in seen
            seen.add(j)
    for clg in (1, 2, 3):
        MS = slots >> clg
        for rank in range(1 << clg):
            rows = ((mb - 1 - rank) >> clg) + 1 if rank < mb else 0
            assert rows * terms <= MS
