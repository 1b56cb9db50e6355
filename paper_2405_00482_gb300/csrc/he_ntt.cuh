// he_ntt.cuh -- negacyclic NTT of one limb-poly held in shared memory (device functions).
//
// Forward: Cooley-Tukey, natural order in, bit-reversed order out, twiddles psi^brv(m+i)
// (psi a primitive 2N-th root mod q): out[k] = a(psi^(2 brv(k) + 1)).
// Inverse: Gentleman-Sande with psi^-brv(m+i), bit-reversed in, natural out; the caller's
// store multiplies by N^-1 (the inverse leaves values in [0, 2q)).
//
// Schedule: the log N stages are grouped into passes of up to 4 stages.  In a pass each
// thread loads the 2^nb elements that interact over those stages into registers, runs the
// radix-2 butterflies there and writes them back, so a N = 8192 transform makes 4 trips
// through shared memory instead of 13.  Butterflies are Harvey's lazy form: forward values
// stay in [0, 4q), inverse values in [0, 2q); products use Shoup's precomputed quotients
// (twiddle tables hold (w, floor(w 2^64 / q)) pairs).  Any block size works: each thread loops
// over the radix-16 sets it owns.
#pragma once
#include <cooperative_groups.h>

#include "he_internal.cuh"

namespace cg = cooperative_groups;

#define HE_NTT_RADIX_LOG 4

// Shared-memory position of element k: one pad word per 32 removes the bank conflicts of the
// strided passes (a CTA needs ntt_smem_words(N) = N + N/32 words).
#define SIDX(k) ((k) + ((k) >> 5))

// s[SIDX(k)] = f(src[k]) for k < len, thread t taking k = t + u blockDim.x: eight global loads in
// flight per thread before the first is used, instead of one load and its wait per element
template <class T, class F>
__device__ __forceinline__ void stage_in(uint64_t *s, const T *__restrict__ src, int len, F f) {
    constexpr int U = 8;
    const int stride = blockDim.x;
    for (int k0 = threadIdx.x; k0 < len; k0 += U * stride) {
        T v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int k = k0 + u * stride;
            v[u] = k < len ? src[k] : T(0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int k = k0 + u * stride;
            if (k < len) s[SIDX(k)] = f(v[u]);
        }
    }
}

// s[SIDX(k)] = f(s[SIDX(k)], src[k]) for k < len, with the same eight loads in flight per thread
template <class T, class F>
__device__ __forceinline__ void stage_acc(uint64_t *s, const T *__restrict__ src, int len, F f) {
    constexpr int U = 8;
    const int stride = blockDim.x;
    for (int k0 = threadIdx.x; k0 < len; k0 += U * stride) {
        T v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int k = k0 + u * stride;
            v[u] = k < len ? src[k] : T(0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int k = k0 + u * stride;
            if (k < len) s[SIDX(k)] = f(s[SIDX(k)], v[u]);
        }
    }
}

// Twiddle access: entry idx of the bit-reversed table (idx = m + j for a stage with m groups).
// TwGlobal reads the table in global memory; the cluster forms read a per-slice copy in shared
// memory (see tw_prefetch).
struct TwGlobal {
    const ulonglong2 *tw;
    __device__ __forceinline__ ulonglong2 operator()(int, int idx) const { return tw[idx]; }
    // entry i of the 2^j (forward) or 2^(NB-j-1) (inverse) consecutive ones that stage j of a
    // pass gives set group g, entry idx of the bit-reversed table
    __device__ __forceinline__ ulonglong2 at(int, int, int, int m, int idx) const { return tw[idx]; }
};

// The radix-16 pass whose sets are its groups (g = set: the forward transform's last pass, the
// inverse's first) reads, at stage j, entries that lie 2^j (or 2^(3-j)) apart for neighbouring
// threads, so a warp's load touches up to 32 lines.  These accessors read a copy of those
// entries ordered [stage j][entry i][set g] (G = N/16 sets), one coalesced line run per load.
struct TwLastFwd {
    const ulonglong2 *t4;
    int G;
    __device__ __forceinline__ ulonglong2 at(int j, int g, int i, int, int) const { return t4[((1 << j) - 1 + i) * G + g]; }
};
struct TwFirstInv {
    const ulonglong2 *t4;
    int G;
    __device__ __forceinline__ ulonglong2 at(int j, int g, int i, int, int) const { return t4[(16 - (16 >> j) + i) * G + g]; }
};

// NB forward stages s0..s0+NB-1 on the 2^NB elements of one set held in registers, r[k] the
// element base + (k << lg_tl) of a set whose stage-s0 group is g (g = base >> (log N - s0)):
// at stage s0 + j element k meets twiddle entry m + (g << j) + (k >> (NB - j)), m = 2^(s0+j),
// the 2^j consecutive entries loaded once per stage.  Harvey's lazy butterfly: inputs below 4q,
// outputs below 4q.  Without CORR the top input is not brought below 2q first: each stage then
// adds less than 2q to the bound, so canonical inputs stay below (1 + 2 log N) q, which fits in
// 64 bits for q < 2^59 and log N <= 14 (the caller reduces at the end).
template <int NB, class TWA, bool CORR = true>
__device__ __forceinline__ void ntt_fwd_radix(uint64_t (&r)[1 << NB], TWA tw, uint64_t q, int s0, int g) {
    constexpr int E = 1 << NB;
    const uint64_t two_q = 2 * q;
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        const int h = E >> (j + 1);
        const int m = 1 << (s0 + j);
        ulonglong2 wj[E / 2];
#pragma unroll
        for (int i = 0; i < (1 << j); ++i) wj[i] = tw.at(j, g, i, m, m + (g << j) + i);
#pragma unroll
        for (int k = 0; k < E; ++k) {
            if ((k & (2 * h - 1)) < h) {
                const ulonglong2 w = wj[k >> (NB - j)];
                uint64_t X = r[k];
                if constexpr (CORR) X = X >= two_q ? X - two_q : X;
                const uint64_t T = mul_shoup_lazy(r[k + h], w.x, w.y, q);
                r[k] = X + T;
                r[k + h] = X - T + two_q;
            }
        }
    }
}
// primes for which the forward transform may skip the lazy correction (see ntt_fwd_radix)
#define HE_NTT_NOCORR_Q (1ull << 59)

// A pass over sets [set0, set1) of stages s0..s0+NB-1; element x lives at s[SIDX(x - off)].
// The whole transform in one CTA uses set0 = 0, set1 = N >> NB, off = 0; a cluster member
// holding the slice [off, off + N/8) uses the sets whose elements fall in its slice.
template <int NB, class TWA, bool CORR = true>
__device__ __forceinline__ void ntt_fwd_pass(uint64_t *s, TWA tw, uint64_t q, int logn, int s0, bool last, int set0 = 0, int set1 = -1,
                                             int off = 0) {
    constexpr int E = 1 << NB;
    const int N = 1 << logn;
    if (set1 < 0) set1 = N >> NB;
    const int lg_t0 = logn - 1 - s0;          // t0 = N / 2^(s0+1)
    const int lg_tl = lg_t0 - (NB - 1);       // stride between a set's elements
    const uint64_t two_q = 2 * q;
    for (int set = set0 + threadIdx.x; set < set1; set += blockDim.x) {
        const int g = set >> lg_tl, low = set & ((1 << lg_tl) - 1);
        const int base = (g << (lg_t0 + 1)) + low;
        // element base + (k << lg_tl) sits at sb + SIDX(k << lg_tl): the low five bits of base
        // plus those of k << lg_tl stay below 32 for every pass shape (and off is a multiple of
        // 32), so the padding splits over the sum
        const int sb = SIDX(base) - SIDX(off);
        uint64_t r[E];
#pragma unroll
        for (int k = 0; k < E; ++k) r[k] = s[sb + SIDX(k << lg_tl)];
        // element x = base + (k << lg_tl) meets twiddle m + (x >> (lg_t0 - j + 1)) at stage
        // s0 + j, which is m + (g << j) + (k >> (NB - j))
        ntt_fwd_radix<NB, TWA, CORR>(r, tw, q, s0, g);
        if (CORR && last) {
#pragma unroll
            for (int k = 0; k < E; ++k) {
                uint64_t v = r[k];
                v = v >= two_q ? v - two_q : v;
                r[k] = v >= q ? v - q : v;
            }
        }
#pragma unroll
        for (int k = 0; k < E; ++k) s[sb + SIDX(k << lg_tl)] = r[k];
    }
    __syncthreads();
}

// NB inverse stages s0..s0+NB-1 on the 2^NB elements of one set held in registers, r[k] the
// element base + (k << s0) of a set whose group at the pass's last stage is g
// (g = base >> (s0 + NB)): at stage s0 + j element k meets twiddle entry
// m + (g << (NB - j - 1)) + (k >> (j + 1)), m = N >> (s0 + j + 1).  Gentleman-Sande lazy
// butterflies: inputs and outputs below 2q.
template <int NB, class TWA>
__device__ __forceinline__ void ntt_inv_radix(uint64_t (&r)[1 << NB], TWA itw, uint64_t q, int N, int s0, int g) {
    constexpr int E = 1 << NB;
    const uint64_t two_q = 2 * q;
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        const int h = 1 << j;
        const int m = N >> (s0 + j + 1);
        ulonglong2 wj[E / 2];
#pragma unroll
        for (int i = 0; i < (E >> (j + 1)); ++i) wj[i] = itw.at(j, g, i, m, m + (g << (NB - j - 1)) + i);
#pragma unroll
        for (int k = 0; k < E; ++k) {
            if ((k & (2 * h - 1)) < h) {
                const ulonglong2 w = wj[k >> (j + 1)];
                const uint64_t U = r[k], V = r[k + h];
                uint64_t X = U + V;
                r[k] = X >= two_q ? X - two_q : X;
                r[k + h] = mul_shoup_lazy(U - V + two_q, w.x, w.y, q);
            }
        }
    }
}

template <int NB, class TWA>
__device__ __forceinline__ void ntt_inv_pass(uint64_t *s, TWA itw, uint64_t q, int logn, int s0, int set0 = 0, int set1 = -1,
                                             int off = 0) {
    constexpr int E = 1 << NB;
    const int N = 1 << logn;
    if (set1 < 0) set1 = N >> NB;
    const int lg_t0 = s0;  // t of the pass's first stage
    for (int set = set0 + threadIdx.x; set < set1; set += blockDim.x) {
        const int g = set >> lg_t0, low = set & ((1 << lg_t0) - 1);
        const int base = (g << (lg_t0 + NB)) + low;
        const int sb = SIDX(base) - SIDX(off);  // as in the forward pass
        uint64_t r[E];
#pragma unroll
        for (int k = 0; k < E; ++k) r[k] = s[sb + SIDX(k << lg_t0)];
        // element x = base + (k << lg_t0) meets twiddle m + (x >> (lg_t0 + j + 1)), which is
        // m + (g << (NB - j - 1)) + (k >> (j + 1)): 2^(NB-j-1) consecutive entries
        ntt_inv_radix<NB>(r, itw, q, N, s0, g);
#pragma unroll
        for (int k = 0; k < E; ++k) s[sb + SIDX(k << lg_t0)] = r[k];
    }
    __syncthreads();
}

// Two radix-2 stages per pass with two lanes per set of four elements, which swap one element by
// warp shuffle between the stages: the butterflies, twiddles and lazy bounds of ntt_fwd_pass<2> /
// ntt_inv_pass<2>, with each thread holding one butterfly's pair per stage (the thread count of a
// radix-2 pass) and one trip through shared memory and one barrier per two stages.
// 2 (set1 - set0) must be a multiple of blockDim.x and of 32, so whole warps run each iteration.
__device__ __forceinline__ uint64_t shfl64_xor1(uint64_t v) {
    return ((uint64_t)__shfl_xor_sync(0xffffffffu, (unsigned)(v >> 32), 1) << 32) | __shfl_xor_sync(0xffffffffu, (unsigned)v, 1);
}
// forward stages s0, s0 + 1: elements base + k 2^lg_tl; stage s0 pairs k, k + 2 (lane p: k = p),
// stage s0 + 1 pairs k, k + 1 (lane p: k = 2p)
template <class TWA>
__device__ __forceinline__ void ntt_fwd_pass_pair(uint64_t *s, TWA tw, uint64_t q, int logn, int s0, bool last, int set0, int set1, int off) {
    const int lg_t0 = logn - 1 - s0, lg_tl = lg_t0 - 1;
    const uint64_t two_q = 2 * q;
    const int p = threadIdx.x & 1;
    for (int t = 2 * set0 + (int)threadIdx.x; t < 2 * set1; t += blockDim.x) {
        const int set = t >> 1, g = set >> lg_tl, low = set & ((1 << lg_tl) - 1);
        const int sb = SIDX((g << (lg_t0 + 1)) + low) - SIDX(off);
        uint64_t x0 = s[sb + SIDX(p << lg_tl)], x1 = s[sb + SIDX((p + 2) << lg_tl)];
        const int m0 = 1 << s0, m1 = 2 << s0;
        ulonglong2 w = tw.at(0, g, 0, m0, m0 + g);
        uint64_t X = x0 >= two_q ? x0 - two_q : x0;
        uint64_t T = mul_shoup_lazy(x1, w.x, w.y, q);
        x0 = X + T;
        x1 = X - T + two_q;
        const uint64_t got = shfl64_xor1(p ? x0 : x1);
        if (p) x0 = got;
        else x1 = got;
        w = tw.at(1, g, p, m1, m1 + (g << 1) + p);
        X = x0 >= two_q ? x0 - two_q : x0;
        T = mul_shoup_lazy(x1, w.x, w.y, q);
        x0 = X + T;
        x1 = X - T + two_q;
        if (last) {
            x0 = x0 >= two_q ? x0 - two_q : x0;
            x0 = x0 >= q ? x0 - q : x0;
            x1 = x1 >= two_q ? x1 - two_q : x1;
            x1 = x1 >= q ? x1 - q : x1;
        }
        s[sb + SIDX((2 * p) << lg_tl)] = x0;
        s[sb + SIDX((2 * p + 1) << lg_tl)] = x1;
    }
    __syncthreads();
}
// inverse stages s0, s0 + 1: elements base + k 2^s0; stage s0 pairs k, k + 1 (lane p: k = 2p),
// stage s0 + 1 pairs k, k + 2 (lane p: k = p)
template <class TWA>
__device__ __forceinline__ void ntt_inv_pass_pair(uint64_t *s, TWA itw, uint64_t q, int logn, int s0, int set0, int set1, int off) {
    const int N = 1 << logn;
    const uint64_t two_q = 2 * q;
    const int p = threadIdx.x & 1;
    for (int t = 2 * set0 + (int)threadIdx.x; t < 2 * set1; t += blockDim.x) {
        const int set = t >> 1, g = set >> s0, low = set & ((1 << s0) - 1);
        const int sb = SIDX((g << (s0 + 2)) + low) - SIDX(off);
        uint64_t x0 = s[sb + SIDX((2 * p) << s0)], x1 = s[sb + SIDX((2 * p + 1) << s0)];
        const int m0 = N >> (s0 + 1), m1 = N >> (s0 + 2);
        ulonglong2 w = itw.at(0, g, p, m0, m0 + (g << 1) + p);
        uint64_t X = x0 + x1, D = x0 - x1 + two_q;
        x0 = X >= two_q ? X - two_q : X;
        x1 = mul_shoup_lazy(D, w.x, w.y, q);
        const uint64_t got = shfl64_xor1(p ? x0 : x1);
        if (p) x0 = got;
        else x1 = got;
        w = itw.at(1, g, 0, m1, m1 + g);
        X = x0 + x1;
        D = x0 - x1 + two_q;
        x0 = X >= two_q ? X - two_q : X;
        x1 = mul_shoup_lazy(D, w.x, w.y, q);
        s[sb + SIDX(p << s0)] = x0;
        s[sb + SIDX((p + 2) << s0)] = x1;
    }
    __syncthreads();
}

// Four forward stages s0..s0+3 (a radix-16 set) on two lanes of eight elements: lane p holds the
// elements k = 2i + p (i < 8) of the set base + k 2^lg_tl, so stages s0..s0+2 (pairs k, k + 8,
// + 4, + 2) stay within a lane; before stage s0 + 3 (pairs 2i, 2i + 1) the lanes swap four
// elements by shuffle and lane p takes i = 4p .. 4p + 3.  The butterflies, twiddles and lazy
// bounds of ntt_fwd_pass<4, TWA, CORR> with the registers of a radix-8 pass per thread.
// 2 (set1 - set0) must be a multiple of blockDim.x and of 32.
template <class TWA, bool CORR = true>
__device__ __forceinline__ void ntt_fwd_pass16_lanes(uint64_t *s, TWA tw, uint64_t q, int logn, int s0, bool last, int set0, int set1, int off) {
    const int lg_t0 = logn - 1 - s0, lg_tl = lg_t0 - 3;
    const uint64_t two_q = 2 * q;
    const int p = threadIdx.x & 1;
    auto bfly = [&](uint64_t &a, uint64_t &b, ulonglong2 w) {
        uint64_t X = a;
        if constexpr (CORR) X = X >= two_q ? X - two_q : X;
        const uint64_t T = mul_shoup_lazy(b, w.x, w.y, q);
        a = X + T;
        b = X - T + two_q;
    };
    for (int t = 2 * set0 + (int)threadIdx.x; t < 2 * set1; t += blockDim.x) {
        const int set = t >> 1, g = set >> lg_tl, low = set & ((1 << lg_tl) - 1);
        const int sb = SIDX((g << (lg_t0 + 1)) + low) - SIDX(off);
        uint64_t r[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) r[i] = s[sb + SIDX((2 * i + p) << lg_tl)];
#pragma unroll
        for (int j = 0; j < 3; ++j) {  // element k = 2i + p meets entry m + (g << j) + (k >> (4 - j))
            const int hi = 4 >> j, m = 1 << (s0 + j);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                if ((i & (2 * hi - 1)) < hi) {
                    const int e = (2 * i + p) >> (4 - j);
                    bfly(r[i], r[i + hi], tw.at(j, g, e, m, m + (g << j) + e));
                }
            }
        }
        uint64_t got[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint64_t v = p ? r[u] : r[4 + u];
            got[u] = ((uint64_t)__shfl_xor_sync(0xffffffffu, (unsigned)(v >> 32), 1) << 32) | __shfl_xor_sync(0xffffffffu, (unsigned)v, 1);
        }
        const int m3 = 8 << s0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = 4 * p + u;  // the pair (2i, 2i + 1), twiddle entry m3 + (g << 3) + i
            uint64_t a = p ? got[u] : r[u], b = p ? r[4 + u] : got[u];
            bfly(a, b, tw.at(3, g, i, m3, m3 + (g << 3) + i));
            if (CORR && last) {
                a = a >= two_q ? a - two_q : a;
                a = a >= q ? a - q : a;
                b = b >= two_q ? b - two_q : b;
                b = b >= q ? b - q : b;
            }
            s[sb + SIDX((2 * i) << lg_tl)] = a;
            s[sb + SIDX((2 * i + 1) << lg_tl)] = b;
        }
    }
    __syncthreads();
}

// ---- two-phase transforms of many limb-polys (NTT form 2) ----
// With N = 64 C (C = 2^(log N - 6)), stages 0..5 of the forward transform only combine the 64
// elements x = l C + c of one column c (their stage-s group x >> (log N - s) = l >> (6 - s) does
// not depend on c), and stages 6..log N - 1 only the C elements of one row x = b C + m; the
// inverse transform runs the same stages in the other order (rows first).  A column phase takes
// NTT2_TC columns of one limb-poly per CTA (two radix-8 passes in registers, one exchange through
// shared memory); a row phase NTT2_TR rows per CTA (a radix-2^NB1 and a radix-2^(log N - 6 - NB1)
// pass).  The butterflies and their stage order are those of the one-CTA form, so the values are
// the same.  Forward: for primes below HE_NTT_NOCORR_Q the butterflies skip the lazy correction
// (ntt_fwd_radix) and the row phase reduces with one Barrett step at the end; the other primes
// end with the usual two conditional subtractions.  Inverse: values stay below 2q; the column
// phase hands each output to a store functor (the caller's scaling).
#define NTT2_TC 16
#define NTT2_TR 16
#define NTT2_THREADS 128
__host__ __device__ constexpr int ntt2_cols_smem_words() { return 64 * (NTT2_TC + 1); }
// shared-memory row stride of a row phase: one pad word per 8 elements, rows r and r + 1 on
// opposite halves of the banks
__host__ __device__ constexpr int ntt2_row_pitch(int lb) {
    return ((1 << lb) + (1 << lb) / 8) % 16 == 0 ? (1 << lb) + (1 << lb) / 8 + 8 : (1 << lb) + (1 << lb) / 8;
}
__host__ __device__ constexpr int ntt2_rows_smem_words(int lb) { return NTT2_TR * ntt2_row_pitch(lb); }
// the forward row phase's staged slice: NTT2_TR rows with one pad word per 32
__host__ __device__ constexpr int ntt2_frows_smem_words(int lb) { return NTT2_TR * (1 << lb) + NTT2_TR * (1 << lb) / 32; }
__device__ __forceinline__ int ntt2_at(int m) { return m + (m >> 3); }

// canonical residue of v 2^64 mod q for a signed v (Shoup product by 2^64 mod q of |v|)
__device__ __forceinline__ uint64_t signed_to_mont(int64_t v, uint64_t r1, uint64_t r1s, uint64_t q) {
    const uint64_t a = v >= 0 ? (uint64_t)v : 0ull - (uint64_t)v;
    const uint64_t r = mul_shoup(a, r1, r1s, q);
    return (v < 0 && r != 0) ? q - r : r;
}

// forward stages 0-5 of columns c0 .. c0 + NTT2_TC - 1 of one limb-poly: load(x) gives the
// canonical input of element x; writes the stage-5 values to dst[x]
template <int LOGN, class LOAD>
__device__ __forceinline__ void ntt2_fwd_cols(uint64_t *sm, LOAD load, uint64_t *dst, int c0, TwGlobal tw, uint64_t q) {
    constexpr int C = (1 << LOGN) >> 6, PAD = NTT2_TC + 1;
    static_assert(NTT2_THREADS == 8 * NTT2_TC, "one thread per (column, set of 8)");
    const int c = threadIdx.x % NTT2_TC, r = threadIdx.x / NTT2_TC;
    const bool corr = q >= HE_NTT_NOCORR_Q;
    uint64_t v[8];
    // stages 0-2 on the column's elements l = r + 8 i (one group at stage 0)
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = load((int64_t)(r + 8 * i) * C + c0 + c);
    if (corr) ntt_fwd_radix<3, TwGlobal, true>(v, tw, q, 0, 0);
    else ntt_fwd_radix<3, TwGlobal, false>(v, tw, q, 0, 0);
#pragma unroll
    for (int i = 0; i < 8; ++i) sm[(r + 8 * i) * PAD + c] = v[i];
    __syncthreads();
    // stages 3-5 on l = 8 r + i: group r at stage 3
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = sm[(8 * r + i) * PAD + c];
    if (corr) ntt_fwd_radix<3, TwGlobal, true>(v, tw, q, 3, r);
    else ntt_fwd_radix<3, TwGlobal, false>(v, tw, q, 3, r);
#pragma unroll
    for (int i = 0; i < 8; ++i) dst[(int64_t)(8 * r + i) * C + c0 + c] = v[i];
}

// forward stages 6 .. log N - 1 of rows b0 .. b0 + NTT2_TR - 1 of one limb-poly, in place;
// canonical outputs.  The rows are staged into shared memory (sm: ntt2_rows_smem_words) as the
// slice [b0 R, (b0 + NTT2_TR) R) of the transform and run through the one-CTA form's passes of up
// to three stages (ntt_fwd_pass over the sets whose elements fall in the slice, as a cluster
// member does), so a thread holds 8 values at a time.
template <int LOGN>
__device__ __forceinline__ void ntt2_fwd_rows(uint64_t *sm, uint64_t *poly, int b0, TwGlobal tw, uint64_t q, uint64_t mu) {
    constexpr int LB = LOGN - 6, R = 1 << LB, LEN = NTT2_TR * R;
    const int off = b0 * R;  // a multiple of 32, so SIDX splits over the offset
    stage_in(sm, poly + off, LEN, [](uint64_t v) { return v; });
    __syncthreads();
    const bool corr = q >= HE_NTT_NOCORR_Q;
    if constexpr (LB == 7) {  // stages 6-8 as a radix-8 pass, 9-12 as a radix-16 one on lane pairs
        if (corr) {
            ntt_fwd_pass<3, TwGlobal, true>(sm, tw, q, LOGN, 6, false, off >> 3, (off + LEN) >> 3, off);
            ntt_fwd_pass16_lanes<TwGlobal, true>(sm, tw, q, LOGN, 9, true, off >> 4, (off + LEN) >> 4, off);
        } else {
            ntt_fwd_pass<3, TwGlobal, false>(sm, tw, q, LOGN, 6, false, off >> 3, (off + LEN) >> 3, off);
            ntt_fwd_pass16_lanes<TwGlobal, false>(sm, tw, q, LOGN, 9, false, off >> 4, (off + LEN) >> 4, off);
        }
    } else
#pragma unroll
    for (int s0 = 6; s0 < LOGN; s0 += 3) {
        const bool last = s0 + 3 >= LOGN;
        if (LOGN - s0 >= 3) {
            if (corr) ntt_fwd_pass<3, TwGlobal, true>(sm, tw, q, LOGN, s0, last, off >> 3, (off + LEN) >> 3, off);
            else ntt_fwd_pass<3, TwGlobal, false>(sm, tw, q, LOGN, s0, false, off >> 3, (off + LEN) >> 3, off);
        } else if (LOGN - s0 == 2) {
            if (corr) ntt_fwd_pass<2, TwGlobal, true>(sm, tw, q, LOGN, s0, last, off >> 2, (off + LEN) >> 2, off);
            else ntt_fwd_pass<2, TwGlobal, false>(sm, tw, q, LOGN, s0, false, off >> 2, (off + LEN) >> 2, off);
        } else {
            if (corr) ntt_fwd_pass<1, TwGlobal, true>(sm, tw, q, LOGN, s0, last, off >> 1, (off + LEN) >> 1, off);
            else ntt_fwd_pass<1, TwGlobal, false>(sm, tw, q, LOGN, s0, false, off >> 1, (off + LEN) >> 1, off);
        }
    }
    // without the lazy correction the values are below (1 + 2 log N) q: one Barrett step
    for (int k = threadIdx.x; k < LEN; k += NTT2_THREADS) {
        const uint64_t v = sm[SIDX(k)];
        poly[off + k] = corr ? v : reduce_barrett(v, q, mu);
    }
}

// inverse stages 0 .. log N - 7 of rows b0 .. b0 + NTT2_TR - 1 of one limb-poly (inputs below 2q),
// from src to dst (which may be src): a radix-2^NBA pass on consecutive elements, then one of
// stride 2^NBA
template <int LOGN, int NBA>
__device__ __forceinline__ void ntt2_inv_rows(uint64_t *sm, const uint64_t *src, uint64_t *dst, int b0, TwGlobal itw, uint64_t q) {
    constexpr int N = 1 << LOGN, LB = LOGN - 6, R = 1 << LB, NBB = LB - NBA, RP = ntt2_row_pitch(LB);
    constexpr int SA = R >> NBA, SB = R >> NBB;  // sets per row of the two passes
    const uint64_t *in0 = src + (int64_t)b0 * R;
    uint64_t *row0 = dst + (int64_t)b0 * R;
    // stages 0 .. NBA - 1 on m = 2^NBA e + i: group at stage NBA - 1 is b 2^(LB - NBA) + e
    for (int set = threadIdx.x; set < NTT2_TR * SA; set += NTT2_THREADS) {
        const int rb = set / SA, e = set % SA;
        uint64_t v[1 << NBA];
        const ulonglong2 *s2 = reinterpret_cast<const ulonglong2 *>(in0 + (int64_t)rb * R + (e << NBA));
#pragma unroll
        for (int i = 0; i < (1 << NBA) / 2; ++i) {
            const ulonglong2 t = s2[i];
            v[2 * i] = t.x;
            v[2 * i + 1] = t.y;
        }
        ntt_inv_radix<NBA>(v, itw, q, N, 0, ((b0 + rb) << (LB - NBA)) + e);
#pragma unroll
        for (int i = 0; i < (1 << NBA); ++i) sm[rb * RP + ntt2_at((e << NBA) + i)] = v[i];
    }
    __syncthreads();
    // stages NBA .. LB - 1 on m = j + 2^NBA i: group b at stage LB - 1
    for (int set = threadIdx.x; set < NTT2_TR * SB; set += NTT2_THREADS) {
        const int rb = set / SB, j = set % SB;
        uint64_t v[1 << NBB];
#pragma unroll
        for (int i = 0; i < (1 << NBB); ++i) v[i] = sm[rb * RP + ntt2_at(j + SB * i)];
        ntt_inv_radix<NBB>(v, itw, q, N, NBA, b0 + rb);
#pragma unroll
        for (int i = 0; i < (1 << NBB); ++i) row0[(int64_t)rb * R + j + SB * i] = v[i];
    }
}

// inverse stages log N - 6 .. log N - 1 of columns c0 .. c0 + NTT2_TC - 1 of one limb-poly:
// reads poly[x] (below 2q), hands each result (below 2q) to store(x, v)
template <int LOGN, class STORE>
__device__ __forceinline__ void ntt2_inv_cols(uint64_t *sm, const uint64_t *poly, int c0, TwGlobal itw, uint64_t q, STORE store) {
    constexpr int N = 1 << LOGN, LB = LOGN - 6, C = 1 << LB, PAD = NTT2_TC + 1;
    const int c = threadIdx.x % NTT2_TC, r = threadIdx.x / NTT2_TC;
    uint64_t v[8];
    // stages LB .. LB + 2 on l = 8 r + i: group r at stage LB + 2
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = poly[(int64_t)(8 * r + i) * C + c0 + c];
    ntt_inv_radix<3>(v, itw, q, N, LB, r);
#pragma unroll
    for (int i = 0; i < 8; ++i) sm[(8 * r + i) * PAD + c] = v[i];
    __syncthreads();
    // stages LB + 3 .. LB + 5 on l = r + 8 i: one group
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = sm[(r + 8 * i) * PAD + c];
    ntt_inv_radix<3>(v, itw, q, N, LB + 3, 0);
#pragma unroll
    for (int i = 0; i < 8; ++i) store((int64_t)(r + 8 * i) * C + c0 + c, v[i]);
}

// Per prime the twiddle block holds, in 16-byte pairs (w, Shoup quotient): the forward table
// [N], the inverse table [N], then the stage-ordered copies [15 N/16] of the forward transform's
// last pass and [15 N/16] of the inverse transform's first pass (none below N = 16).
__host__ __device__ __forceinline__ size_t tw_t4_pairs(int logn) { return logn >= 4 ? (size_t)15 << (logn - 4) : 0; }
__host__ __device__ __forceinline__ size_t tw_prime_words(int logn) { return ((size_t)4 << logn) + 4 * tw_t4_pairs(logn); }
// from the forward (inverse) table of a prime to its copy for the last (first) pass
__device__ __forceinline__ const ulonglong2 *tw_last_fwd(const ulonglong2 *tw, int logn) { return tw + (2 << logn); }
__device__ __forceinline__ const ulonglong2 *tw_first_inv(const ulonglong2 *itw, int logn) { return itw + (1 << logn) + tw_t4_pairs(logn); }

// in-place forward transform of canonical residues in s[SIDX(0..N)); output canonical
// The stage count left over by the radix-16 passes (log N mod 4) runs first: the early stages use
// few distinct twiddles (stage t has 2^t), so a short pass there costs little, while the last
// stages touch N/2 distinct twiddles and belong in full passes that load them together.
__device__ __forceinline__ void ntt_fwd_smem(uint64_t *s, const ulonglong2 *__restrict__ tw, uint64_t q, int logn) {
    int s0 = 0;
    while (s0 < logn) {
        const int first = logn % HE_NTT_RADIX_LOG;
        const int nb = (s0 == 0 && first) ? first : HE_NTT_RADIX_LOG;
        const bool last = s0 + nb == logn;
        switch (nb) {
            case 4:
                if (last) ntt_fwd_pass<4>(s, TwLastFwd{tw_last_fwd(tw, logn), 1 << (logn - 4)}, q, logn, s0, last);
                else ntt_fwd_pass<4>(s, TwGlobal{tw}, q, logn, s0, last);
                break;
            case 3: ntt_fwd_pass<3>(s, TwGlobal{tw}, q, logn, s0, last); break;
            case 2: ntt_fwd_pass<2>(s, TwGlobal{tw}, q, logn, s0, last); break;
            default: ntt_fwd_pass<1>(s, TwGlobal{tw}, q, logn, s0, last); break;
        }
        s0 += nb;
    }
}

// ntt_fwd_smem for a ring size known at compile time (LOGN >= 4): the pass schedule, strides,
// twiddle offsets and shared-memory offsets fold to constants
template <int LOGN>
__device__ __forceinline__ void ntt_fwd_smem_c(uint64_t *s, const ulonglong2 *__restrict__ tw, uint64_t q) {
    static_assert(LOGN >= 4 && LOGN <= 16, "compile-time ring size");
    constexpr int R = HE_NTT_RADIX_LOG, FIRST = LOGN % R, NPASS = (LOGN + R - 1) / R;
#pragma unroll
    for (int pi = 0; pi < NPASS; ++pi) {
        const int nb = (pi == 0 && FIRST) ? FIRST : R;
        const int s0 = pi == 0 ? 0 : (FIRST ? FIRST : R) + (pi - 1) * R;
        const bool last = pi == NPASS - 1;
        switch (nb) {
            case 4:
                if (last) ntt_fwd_pass<4>(s, TwLastFwd{tw_last_fwd(tw, LOGN), 1 << (LOGN - 4)}, q, LOGN, s0, last);
                else ntt_fwd_pass<4>(s, TwGlobal{tw}, q, LOGN, s0, last);
                break;
            case 3: ntt_fwd_pass<3>(s, TwGlobal{tw}, q, LOGN, s0, last); break;
            case 2: ntt_fwd_pass<2>(s, TwGlobal{tw}, q, LOGN, s0, last); break;
            default: ntt_fwd_pass<1>(s, TwGlobal{tw}, q, LOGN, s0, last); break;
        }
    }
}

// ntt_inv_smem for a ring size known at compile time (LOGN >= 4)
template <int LOGN>
__device__ __forceinline__ void ntt_inv_smem_c(uint64_t *s, const ulonglong2 *__restrict__ itw, uint64_t q) {
    static_assert(LOGN >= 4 && LOGN <= 16, "compile-time ring size");
    constexpr int R = HE_NTT_RADIX_LOG, NPASS = (LOGN + R - 1) / R;
#pragma unroll
    for (int pi = 0; pi < NPASS; ++pi) {
        const int s0 = pi * R, nb = LOGN - s0 < R ? LOGN - s0 : R;
        switch (nb) {
            case 4:
                if (s0 == 0) ntt_inv_pass<4>(s, TwFirstInv{tw_first_inv(itw, LOGN), 1 << (LOGN - 4)}, q, LOGN, s0);
                else ntt_inv_pass<4>(s, TwGlobal{itw}, q, LOGN, s0);
                break;
            case 3: ntt_inv_pass<3>(s, TwGlobal{itw}, q, LOGN, s0); break;
            case 2: ntt_inv_pass<2>(s, TwGlobal{itw}, q, LOGN, s0); break;
            default: ntt_inv_pass<1>(s, TwGlobal{itw}, q, LOGN, s0); break;
        }
    }
}

// in-place inverse transform without the N^-1 factor; input canonical, output in [0, 2q)
__device__ __forceinline__ void ntt_inv_smem(uint64_t *s, const ulonglong2 *__restrict__ itw, uint64_t q, int logn) {
    int s0 = 0;
    while (s0 < logn) {
        const int nb = logn - s0 < HE_NTT_RADIX_LOG ? logn - s0 : HE_NTT_RADIX_LOG;
        switch (nb) {
            case 4:
                if (s0 == 0) ntt_inv_pass<4>(s, TwFirstInv{tw_first_inv(itw, logn), 1 << (logn - 4)}, q, logn, s0);
                else ntt_inv_pass<4>(s, TwGlobal{itw}, q, logn, s0);
                break;
            case 3: ntt_inv_pass<3>(s, TwGlobal{itw}, q, logn, s0); break;
            case 2: ntt_inv_pass<2>(s, TwGlobal{itw}, q, logn, s0); break;
            default: ntt_inv_pass<1>(s, TwGlobal{itw}, q, logn, s0); break;
        }
        s0 += nb;
    }
}

// ---------------------------------------------------------------------------------------
// Cluster form: HE_NTT_CL CTAs (one thread-block cluster) share one limb-poly, CTA `rank`
// holding the slice [rank N/CL, (rank+1) N/CL) in its shared memory (padded layout, local
// index x - rank N/CL).  The stages whose butterflies span slices (the first 3 forward, the
// last 3 inverse) are one radix-8 step through distributed shared memory: element j + c N/CL
// lives in CTA c at local index j, and each CTA takes 1/CL of the offsets j.  The other stages
// run on each slice one stage at a time (radix-2 passes).  Used for launches of few limb-polys,
// where one CTA per limb-poly would leave most SMs idle.
#define HE_NTT_CL HE_NTT_CL_SIZE
// local passes of the cluster form are radix 2, one butterfly per thread per stage (N/16 threads
// per CTA, at most 512): a cluster transform is latency-bound, and on GB300 the most warps with
// the shortest chains finished it soonest (radix 8 > radix 4 > radix 2 in time)
#define HE_NTT_CL_RADIX_LOG 1

// The local stages of a cluster member touch NS - 1 twiddles of its slice (NS = N/8): forward
// stage t (3 <= t < log N, m = 2^t) the m/8 entries m + rank m/8 + j; inverse stage t
// (0 <= t < log N - 3, m = N / 2^(t+1)) likewise.  tw_slice_issue puts them in shared memory,
// ordered by stage, behind the slice's data: forward stage m from (m/8 - 1), inverse stage m
// from (N/2 - m)/4.  The copy is one round of asynchronous 16-byte copies, waited for before the
// transform, so the passes do not wait on global memory.
__device__ __forceinline__ int cl_tw_offset_words(int logn) {  // the slice's padded data, in words
    const int NS = 1 << (logn - 3);
    return NS + (NS >> 5);
}
template <bool FWD>
__device__ __forceinline__ void tw_slice_issue(ulonglong2 *stw, const ulonglong2 *__restrict__ tw, int logn, int rank) {
    const int NS = 1 << (logn - 3);
    for (int i = threadIdx.x; i < NS - 1; i += blockDim.x) {
        int b = 0, c = FWD ? 1 : NS >> 1, m = FWD ? 8 : 1 << (logn - 1);
        while (i >= b + c) {
            b += c;
            c = FWD ? c << 1 : c >> 1;
            m = FWD ? m << 1 : m >> 1;
        }
        const unsigned sa = (unsigned)__cvta_generic_to_shared(stw + i);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(tw + m + rank * (m >> 3) + (i - b)) : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void tw_slice_wait() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// the dynamic shared memory, for a kernel that starts a copy into it before calling a body that
// declares its own (every extern __shared__ array starts at the same address)
__device__ __forceinline__ uint64_t *s_dyn() {
    extern __shared__ uint64_t s_dyn_words[];
    return s_dyn_words;
}

// Kernels call this as soon as they know their prime, before loading their data, so the twiddle
// copy overlaps the loads; the cluster transform waits for it.  Nothing in the one-CTA form.
template <bool CL, bool FWD>
__device__ __forceinline__ void tw_prefetch(uint64_t *s, const ulonglong2 *__restrict__ tw, int logn) {
    if constexpr (CL)
        tw_slice_issue<FWD>(reinterpret_cast<ulonglong2 *>(s + cl_tw_offset_words(logn)), tw, logn, (int)cg::this_cluster().block_rank());
}
struct TwSliceFwd {
    const ulonglong2 *stw;
    int rank;
    __device__ __forceinline__ ulonglong2 operator()(int m, int idx) const { return stw[idx - m + (1 - rank) * (m >> 3) - 1]; }
    __device__ __forceinline__ ulonglong2 at(int, int, int, int m, int idx) const { return (*this)(m, idx); }
};
struct TwSliceInv {
    const ulonglong2 *stw;
    int rank, half_n;
    __device__ __forceinline__ ulonglong2 operator()(int m, int idx) const { return stw[((half_n - m) >> 2) + idx - m - rank * (m >> 3)]; }
    __device__ __forceinline__ ulonglong2 at(int, int, int, int m, int idx) const { return (*this)(m, idx); }
};

// The cross-CTA stages of the cluster form: the 8 elements j + c NS of an offset j, one per CTA,
// go through three radix-2 stages (forward: c paired with c + 4, then c + 2, then c + 1;
// inverse: c + 1, c + 2, c + 4).  Four adjacent lanes share an offset, lane p holding the pair of
// one butterfly per stage (the stage's bit inserted into p), and between stages they swap
// elements by warp shuffles, so every thread of the CTA takes part.  A stage's twiddle does not
// depend on j: forward tw[2^st + (c >> (3 - st))], inverse tw[(4 >> st) + (c >> (st + 1))] for
// the pair's lower element c; cross_tw_load reads them before the cluster barrier.
__device__ __forceinline__ int ins_bit(int v, int b) { return (v & ((1 << b) - 1)) | ((v >> b) << (b + 1)); }
__device__ __forceinline__ int del_bit(int v, int b) { return (v & ((1 << b) - 1)) | ((v >> (b + 1)) << b); }
template <bool FWD>
__device__ __forceinline__ int cross_bit(int st) { return FWD ? 2 - st : st; }
template <bool FWD>
__device__ __forceinline__ void cross_tw_load(ulonglong2 w[3], const ulonglong2 *__restrict__ tw) {
    const int p = threadIdx.x & 3;
#pragma unroll
    for (int st = 0; st < 3; ++st) {
        const int c = ins_bit(p, cross_bit<FWD>(st));
        w[st] = FWD ? tw[(1 << st) + (c >> (3 - st))] : tw[(4 >> st) + (c >> (st + 1))];
    }
}
__device__ __forceinline__ uint64_t shfl64(uint64_t v, int src) {
    return ((uint64_t)__shfl_sync(0xffffffffu, (unsigned)(v >> 32), src) << 32) | __shfl_sync(0xffffffffu, (unsigned)v, src);
}
// the three stages on lane p's pair (x0, x1) = elements (lo, lo + 2^b) of stage 0's bit b
template <bool FWD>
__device__ __forceinline__ void cross_stages(uint64_t &x0, uint64_t &x1, int &lo, int p, int lane_base, const ulonglong2 w[3], uint64_t q) {
    const uint64_t two_q = 2 * q;
#pragma unroll
    for (int st = 0; st < 3; ++st) {
        if (st > 0) {
            // this lane's pair from the lanes that held them at stage st - 1 (element c at lane
            // c with that stage's bit removed, in the slot given by the bit)
            const int b = cross_bit<FWD>(st), bp = cross_bit<FWD>(st - 1);
            const int nlo = ins_bit(p, b), nhi = nlo | (1 << b);
            const int sl = lane_base + del_bit(nlo, bp), sh = lane_base + del_bit(nhi, bp);
            const uint64_t a0 = shfl64(x0, sl), a1 = shfl64(x1, sl), b0 = shfl64(x0, sh), b1 = shfl64(x1, sh);
            x0 = (nlo >> bp) & 1 ? a1 : a0;
            x1 = (nhi >> bp) & 1 ? b1 : b0;
            lo = nlo;
        }
        if (FWD) {  // Cooley-Tukey, lazy: inputs in [0, 4q)
            const uint64_t X = x0 >= two_q ? x0 - two_q : x0;
            const uint64_t T = mul_shoup_lazy(x1, w[st].x, w[st].y, q);
            x0 = X + T;
            x1 = X - T + two_q;
        } else {  // Gentleman-Sande, inputs in [0, 2q)
            const uint64_t X = x0 + x1, D = x0 - x1 + two_q;
            x0 = X >= two_q ? X - two_q : X;
            x1 = mul_shoup_lazy(D, w[st].x, w[st].y, q);
        }
    }
}
template <bool FWD>
__device__ __forceinline__ void ntt_cross_step(uint64_t *s, const ulonglong2 w[3], uint64_t q, int logn) {
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int NS = 1 << (logn - 3), per = NS >> 3;
    const int p = threadIdx.x & 3, lane_base = (threadIdx.x & 31) & ~3;
    // 4 lanes per offset: NS / 2 of them, a multiple of 32 (NS >= 128), and blockDim.x a multiple
    // of 32, so whole warps run each iteration and the shuffles see every lane
    for (int t = threadIdx.x; t < per * 4; t += blockDim.x) {
        const int j = SIDX(rank * per + (t >> 2));
        int lo = ins_bit(p, cross_bit<FWD>(0));
        uint64_t x0 = cl.map_shared_rank(s, lo)[j], x1 = cl.map_shared_rank(s, lo | (1 << cross_bit<FWD>(0)))[j];
        cross_stages<FWD>(x0, x1, lo, p, lane_base, w, q);
        cl.map_shared_rank(s, lo)[j] = x0;
        cl.map_shared_rank(s, lo | (1 << cross_bit<FWD>(2)))[j] = x1;
    }
}
// An inverse transform's three cross-CTA stages (prime qi, twiddles wi), an elementwise map f to
// another prime t's residues, then a forward transform's three cross-CTA stages (prime t,
// twiddles wf), in one pass through distributed shared memory: the inverse's last stage and the
// forward's first both pair c and c + 4, so each lane already holds its forward pair.  The same
// values as ntt_cross_step<false>, f on every element, then ntt_cross_step<true>.
template <class F>
__device__ __forceinline__ void ntt_cross_inv_fwd(uint64_t *s, const ulonglong2 wi[3], uint64_t qi, F f, const ulonglong2 wf[3], uint64_t t, int logn) {
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int NS = 1 << (logn - 3), per = NS >> 3;
    const int p = threadIdx.x & 3, lane_base = (threadIdx.x & 31) & ~3;
    for (int u = threadIdx.x; u < per * 4; u += blockDim.x) {
        const int j = SIDX(rank * per + (u >> 2));
        int lo = ins_bit(p, cross_bit<false>(0));
        uint64_t x0 = cl.map_shared_rank(s, lo)[j], x1 = cl.map_shared_rank(s, lo | (1 << cross_bit<false>(0)))[j];
        cross_stages<false>(x0, x1, lo, p, lane_base, wi, qi);  // lo = ins_bit(p, 2) = ins_bit(p, cross_bit<true>(0))
        x0 = f(x0);
        x1 = f(x1);
        cross_stages<true>(x0, x1, lo, p, lane_base, wf, t);
        cl.map_shared_rank(s, lo)[j] = x0;
        cl.map_shared_rank(s, lo | (1 << cross_bit<true>(2)))[j] = x1;
    }
}

// the local stages (3 .. log N - 1) of ntt_fwd_cluster, after its cross-CTA stages and a cluster
// barrier that follows the slice's twiddle copy
template <int LOGN>
__device__ __forceinline__ void ntt_fwd_cluster_local(uint64_t *s, uint64_t q, int logn) {
    const int rank = (int)cg::this_cluster().block_rank();
    const int NS = 1 << (logn - 3), off = rank * NS;
    const TwSliceFwd tws{reinterpret_cast<const ulonglong2 *>(s + cl_tw_offset_words(logn)), rank};
#pragma unroll(LOGN > 0 ? 16 : 1)
    for (int s0 = 3; s0 + 1 < (LOGN > 0 ? LOGN : 16); s0 += 2) {  // stages in pairs, the last alone if odd
        if (s0 + 1 >= logn) break;
        ntt_fwd_pass_pair(s, tws, q, logn, s0, s0 + 2 == logn, rank * (NS / 4), (rank + 1) * (NS / 4), off);
    }
    if (((logn - 3) & 1) != 0) ntt_fwd_pass<1>(s, tws, q, logn, logn - 1, true, rank * (NS / 2), (rank + 1) * (NS / 2), off);
}

// forward transform of a slice held by each CTA of the cluster; output canonical, bit-reversed
// positions [rank N/8, (rank+1) N/8) in this CTA.  s must have cl_tw_offset_words(logn) words of
// data followed by room for N/8 twiddle pairs, whose copy tw_prefetch<true, true> started.
// LOGN > 0: the ring size at compile time (logn == LOGN), so the pass loop unrolls and every
// index folds to a constant; 0: runtime
template <int LOGN = 0>
__device__ __forceinline__ void ntt_fwd_cluster(uint64_t *s, const ulonglong2 *__restrict__ tw, uint64_t q, int logn) {
    cg::cluster_group cl = cg::this_cluster();
    ulonglong2 wx[3];
    cross_tw_load<true>(wx, tw);
    tw_slice_wait();
    cl.sync();
    ntt_cross_step<true>(s, wx, q, logn);
    cl.sync();
    ntt_fwd_cluster_local<LOGN>(s, q, logn);
}

// the local stages (0 .. log N - 4) of ntt_inv_cluster: waits for the slice's twiddle copy and
// ends with a block barrier, before the cluster barrier of the cross-CTA stages
template <int LOGN>
__device__ __forceinline__ void ntt_inv_cluster_local(uint64_t *s, uint64_t q, int logn) {
    const int rank = (int)cg::this_cluster().block_rank();
    const int NS = 1 << (logn - 3), off = rank * NS;
    tw_slice_wait();
    __syncthreads();
    const TwSliceInv tws{reinterpret_cast<const ulonglong2 *>(s + cl_tw_offset_words(logn)), rank, 1 << (logn - 1)};
#pragma unroll(LOGN > 0 ? 16 : 1)
    for (int s0 = 0; s0 + 1 < (LOGN > 0 ? LOGN - 3 : 16); s0 += 2) {  // stages in pairs, the last alone if odd
        if (s0 + 1 >= logn - 3) break;
        ntt_inv_pass_pair(s, tws, q, logn, s0, rank * (NS / 4), (rank + 1) * (NS / 4), off);
    }
    if (((logn - 3) & 1) != 0) ntt_inv_pass<1>(s, tws, q, logn, logn - 4, rank * (NS / 2), (rank + 1) * (NS / 2), off);
}

// inverse transform (without N^-1) of the slices; output in [0, 2q), natural order (twiddle copy
// started by tw_prefetch<true, false>)
template <int LOGN = 0>
__device__ __forceinline__ void ntt_inv_cluster(uint64_t *s, const ulonglong2 *__restrict__ itw, uint64_t q, int logn) {
    cg::cluster_group cl = cg::this_cluster();
    ulonglong2 wx[3];
    cross_tw_load<false>(wx, itw);
    ntt_inv_cluster_local<LOGN>(s, q, logn);
    cl.sync();
    ntt_cross_step<false>(s, wx, q, logn);
    cl.sync();
}

// the cluster form is used for rings of at least 2^10 (slices of at least 128 elements)
#define HE_NTT_CL_MIN_LOGN 10
__device__ __forceinline__ int cl_slice_threads(int logn) { return min(512, 1 << (logn - 3 - HE_NTT_CL_RADIX_LOG)); }

// Kernels over a batch of limb-polys: in the plain form one CTA transforms a whole limb-poly
// (grid = polys); in the cluster form (CL) a cluster of HE_NTT_CL CTAs shares one limb-poly,
// each CTA handling the slice [rank N/8, (rank+1) N/8) (grid = polys * HE_NTT_CL).
template <bool CL>
__device__ __forceinline__ void slice_of(int logn, int &poly, int &off, int &len) {
    const int N = 1 << logn;
    if (CL) {
        poly = blockIdx.x / HE_NTT_CL;
        len = N / HE_NTT_CL;
        off = (int)cg::this_cluster().block_rank() * len;
    } else {
        poly = blockIdx.x;
        len = N;
        off = 0;
    }
}

template <bool CL, int LOGN = 0>
__device__ __forceinline__ void fwd_any(uint64_t *s, const ulonglong2 *tw, uint64_t q, int logn) {
    if constexpr (CL) ntt_fwd_cluster<LOGN>(s, tw, q, logn);
    else if constexpr (LOGN > 0) ntt_fwd_smem_c<LOGN>(s, tw, q);
    else ntt_fwd_smem(s, tw, q, logn);
}
template <bool CL, int LOGN = 0>
__device__ __forceinline__ void inv_any(uint64_t *s, const ulonglong2 *tw, uint64_t q, int logn) {
    if constexpr (CL) ntt_inv_cluster<LOGN>(s, tw, q, logn);
    else if constexpr (LOGN > 0) ntt_inv_smem_c<LOGN>(s, tw, q);
    else ntt_inv_smem(s, tw, q, logn);
}

// ---------------------------------------------------------------------------------------
// Pair form: a 2-CTA cluster per limb-poly, CTA r holding the half [r N/2, (r+1) N/2) in its shared
// memory (padded layout, local index x - r N/2).  A throughput form for launches of many
// limb-polys: twice the CTAs, each with half the work, so 256 limb-polys on 152 SMs become 512
// halves spread 3-4 per SM instead of 1-2 transforms per SM.  Only the forward transform's first
// stage (the inverse's last) pairs elements of the two halves, x and x + N/2: one step through
// distributed shared memory, each CTA taking half of those butterflies.  Every other stage runs in
// the radix-16 passes of the one-CTA form, on the CTA's half of the sets (its groups lie wholly in
// one half), with the same twiddle tables.  The butterflies are those of the one-CTA form, so the
// output is the same canonical transform.
template <int LOGN>
__device__ __forceinline__ void pair_cross_step(uint64_t *s, ulonglong2 w, uint64_t q, bool fwd) {
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    constexpr int NS = 1 << (LOGN - 1);
    uint64_t *a = cl.map_shared_rank(s, 0), *b = cl.map_shared_rank(s, 1);
    const uint64_t two_q = 2 * q;
    for (int j = rank * (NS / 2) + threadIdx.x; j < (rank + 1) * (NS / 2); j += blockDim.x) {
        const uint64_t U = a[SIDX(j)], V = b[SIDX(j)];
        if (fwd) {  // Cooley-Tukey stage 0, inputs canonical
            const uint64_t T = mul_shoup_lazy(V, w.x, w.y, q);
            a[SIDX(j)] = U + T;
            b[SIDX(j)] = U - T + two_q;
        } else {  // Gentleman-Sande last stage, inputs in [0, 2q)
            const uint64_t X = U + V;
            a[SIDX(j)] = X >= two_q ? X - two_q : X;
            b[SIDX(j)] = mul_shoup_lazy(U - V + two_q, w.x, w.y, q);
        }
    }
}

// forward transform of the two halves (canonical in, canonical bit-reversed out); every thread of
// both CTAs calls it after its half is in shared memory
template <int LOGN>
__device__ __forceinline__ void ntt_fwd_pair(uint64_t *s, const ulonglong2 *__restrict__ tw, uint64_t q) {
    static_assert(LOGN >= 6, "pair form: halves of at least 32 elements");
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    constexpr int R = HE_NTT_RADIX_LOG, LOC = LOGN - 1, FIRST = LOC % R, NPASS = (LOC + R - 1) / R;
    constexpr int NS = 1 << LOC;
    cl.sync();
    pair_cross_step<LOGN>(s, tw[1], q, true);
    cl.sync();
#pragma unroll
    for (int pi = 0; pi < NPASS; ++pi) {
        const int nb = (pi == 0 && FIRST) ? FIRST : R;
        const int s0 = 1 + (pi == 0 ? 0 : (FIRST ? FIRST : R) + (pi - 1) * R);
        const bool last = pi == NPASS - 1;
        const int E = 1 << nb;
        const int set0 = rank * (NS / E), set1 = (rank + 1) * (NS / E), off = rank * NS;
        switch (nb) {
            case 4:
                if (last) ntt_fwd_pass<4>(s, TwLastFwd{tw_last_fwd(tw, LOGN), 1 << (LOGN - 4)}, q, LOGN, s0, last, set0, set1, off);
                else ntt_fwd_pass<4>(s, TwGlobal{tw}, q, LOGN, s0, last, set0, set1, off);
                break;
            case 3: ntt_fwd_pass<3>(s, TwGlobal{tw}, q, LOGN, s0, last, set0, set1, off); break;
            case 2: ntt_fwd_pass<2>(s, TwGlobal{tw}, q, LOGN, s0, last, set0, set1, off); break;
            default: ntt_fwd_pass<1>(s, TwGlobal{tw}, q, LOGN, s0, last, set0, set1, off); break;
        }
    }
}

// inverse transform (without N^-1) of the two halves: input canonical, output in [0, 2q); every
// thread of both CTAs calls it after writing its part of the half to shared memory
template <int LOGN>
__device__ __forceinline__ void ntt_inv_pair(uint64_t *s, const ulonglong2 *__restrict__ itw, uint64_t q) {
    static_assert(LOGN >= 6, "pair form: halves of at least 32 elements");
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    constexpr int R = HE_NTT_RADIX_LOG, LOC = LOGN - 1, NPASS = (LOC + R - 1) / R;
    constexpr int NS = 1 << LOC;
    __syncthreads();  // the half staged by this CTA's threads (the local passes come first)
#pragma unroll
    for (int pi = 0; pi < NPASS; ++pi) {
        const int s0 = pi * R, nb = LOC - s0 < R ? LOC - s0 : R;
        const int E = 1 << nb;
        const int set0 = rank * (NS / E), set1 = (rank + 1) * (NS / E), off = rank * NS;
        switch (nb) {
            case 4:
                if (s0 == 0) ntt_inv_pass<4>(s, TwFirstInv{tw_first_inv(itw, LOGN), 1 << (LOGN - 4)}, q, LOGN, s0, set0, set1, off);
                else ntt_inv_pass<4>(s, TwGlobal{itw}, q, LOGN, s0, set0, set1, off);
                break;
            case 3: ntt_inv_pass<3>(s, TwGlobal{itw}, q, LOGN, s0, set0, set1, off); break;
            case 2: ntt_inv_pass<2>(s, TwGlobal{itw}, q, LOGN, s0, set0, set1, off); break;
            default: ntt_inv_pass<1>(s, TwGlobal{itw}, q, LOGN, s0, set0, set1, off); break;
        }
    }
    cl.sync();
    pair_cross_step<LOGN>(s, itw[1], q, false);
    cl.sync();
}

// dynamic shared memory and threads of a pair-form CTA: a half (padded), one radix-16 set per thread
__host__ __device__ __forceinline__ size_t pair_smem_bytes(int logn) { return ((size_t)1 << (logn - 1)) * 8 + ((size_t)1 << (logn - 1)) / 32 * 8; }
__host__ __device__ constexpr int pair_threads_c(int logn) { return (1 << (logn - 1 - HE_NTT_RADIX_LOG)) > 512 ? 512 : (1 << (logn - 1 - HE_NTT_RADIX_LOG)); }
__host__ __device__ __forceinline__ int pair_threads(int logn) { return pair_threads_c(logn); }

// twiddle table of prime index p: which = 0 forward (psi^brv(k), Shoup), 1 inverse (psi^-brv(k), Shoup)
__device__ __forceinline__ const ulonglong2 *twiddles(const uint64_t *d_tw, int p, int which, int logn) {
    return reinterpret_cast<const ulonglong2 *>(d_tw + (size_t)p * tw_prime_words(logn) + ((size_t)which << (logn + 1)));
}
