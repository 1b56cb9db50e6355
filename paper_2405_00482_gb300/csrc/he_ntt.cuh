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
#include "he_internal.cuh"

#define HE_NTT_RADIX_LOG 4

// Shared-memory position of element k: one pad word per 32 removes the bank conflicts of the
// strided passes (a CTA needs ntt_smem_words(N) = N + N/32 words).
#define SIDX(k) ((k) + ((k) >> 5))

template <int NB>
__device__ __forceinline__ void ntt_fwd_pass(uint64_t *s, const ulonglong2 *__restrict__ tw, uint64_t q, int logn, int s0, bool last) {
    constexpr int E = 1 << NB;
    const int N = 1 << logn;
    const int lg_t0 = logn - 1 - s0;          // t0 = N / 2^(s0+1)
    const int lg_tl = lg_t0 - (NB - 1);       // stride between a set's elements
    const uint64_t two_q = 2 * q;
    for (int set = threadIdx.x; set < (N >> NB); set += blockDim.x) {
        const int g = set >> lg_tl, low = set & ((1 << lg_tl) - 1);
        const int base = (g << (lg_t0 + 1)) + low;
        uint64_t r[E];
#pragma unroll
        for (int k = 0; k < E; ++k) r[k] = s[SIDX(base + (k << lg_tl))];
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            const int h = E >> (j + 1);
            const int m = 1 << (s0 + j);
            const int lg_2t = lg_t0 - j + 1;
#pragma unroll
            for (int k = 0; k < E; ++k) {
                if ((k & (2 * h - 1)) < h) {
                    const int x = base + (k << lg_tl);
                    const ulonglong2 w = tw[m + (x >> lg_2t)];
                    uint64_t X = r[k];
                    X = X >= two_q ? X - two_q : X;
                    const uint64_t T = mul_shoup_lazy(r[k + h], w.x, w.y, q);
                    r[k] = X + T;
                    r[k + h] = X - T + two_q;
                }
            }
        }
        if (last) {
#pragma unroll
            for (int k = 0; k < E; ++k) {
                uint64_t v = r[k];
                v = v >= two_q ? v - two_q : v;
                r[k] = v >= q ? v - q : v;
            }
        }
#pragma unroll
        for (int k = 0; k < E; ++k) s[SIDX(base + (k << lg_tl))] = r[k];
    }
    __syncthreads();
}

template <int NB>
__device__ __forceinline__ void ntt_inv_pass(uint64_t *s, const ulonglong2 *__restrict__ itw, uint64_t q, int logn, int s0) {
    constexpr int E = 1 << NB;
    const int N = 1 << logn;
    const int lg_t0 = s0;  // t of the pass's first stage
    const uint64_t two_q = 2 * q;
    for (int set = threadIdx.x; set < (N >> NB); set += blockDim.x) {
        const int g = set >> lg_t0, low = set & ((1 << lg_t0) - 1);
        const int base = (g << (lg_t0 + NB)) + low;
        uint64_t r[E];
#pragma unroll
        for (int k = 0; k < E; ++k) r[k] = s[SIDX(base + (k << lg_t0))];
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            const int h = 1 << j;
            const int m = N >> (s0 + j + 1);
            const int lg_2t = lg_t0 + j + 1;
#pragma unroll
            for (int k = 0; k < E; ++k) {
                if ((k & (2 * h - 1)) < h) {
                    const int x = base + (k << lg_t0);
                    const ulonglong2 w = itw[m + (x >> lg_2t)];
                    const uint64_t U = r[k], V = r[k + h];
                    uint64_t X = U + V;
                    r[k] = X >= two_q ? X - two_q : X;
                    r[k + h] = mul_shoup_lazy(U - V + two_q, w.x, w.y, q);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < E; ++k) s[SIDX(base + (k << lg_t0))] = r[k];
    }
    __syncthreads();
}

// in-place forward transform of canonical residues in s[SIDX(0..N)); output canonical
__device__ __forceinline__ void ntt_fwd_smem(uint64_t *s, const ulonglong2 *__restrict__ tw, uint64_t q, int logn) {
    int s0 = 0;
    while (s0 < logn) {
        const int nb = logn - s0 < HE_NTT_RADIX_LOG ? logn - s0 : HE_NTT_RADIX_LOG;
        const bool last = s0 + nb == logn;
        switch (nb) {
            case 4: ntt_fwd_pass<4>(s, tw, q, logn, s0, last); break;
            case 3: ntt_fwd_pass<3>(s, tw, q, logn, s0, last); break;
            case 2: ntt_fwd_pass<2>(s, tw, q, logn, s0, last); break;
            default: ntt_fwd_pass<1>(s, tw, q, logn, s0, last); break;
        }
        s0 += nb;
    }
}

// in-place inverse transform without the N^-1 factor; input canonical, output in [0, 2q)
__device__ __forceinline__ void ntt_inv_smem(uint64_t *s, const ulonglong2 *__restrict__ itw, uint64_t q, int logn) {
    int s0 = 0;
    while (s0 < logn) {
        const int nb = logn - s0 < HE_NTT_RADIX_LOG ? logn - s0 : HE_NTT_RADIX_LOG;
        switch (nb) {
            case 4: ntt_inv_pass<4>(s, itw, q, logn, s0); break;
            case 3: ntt_inv_pass<3>(s, itw, q, logn, s0); break;
            case 2: ntt_inv_pass<2>(s, itw, q, logn, s0); break;
            default: ntt_inv_pass<1>(s, itw, q, logn, s0); break;
        }
        s0 += nb;
    }
}

// twiddle table of prime index p: which = 0 forward (psi^brv(k), Shoup), 1 inverse (psi^-brv(k), Shoup)
__device__ __forceinline__ const ulonglong2 *twiddles(const uint64_t *d_tw, int p, int which, int logn) {
    return reinterpret_cast<const ulonglong2 *>(d_tw + (((size_t)p * 2 + which) << (logn + 1)));
}
