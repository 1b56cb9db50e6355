// he_ntt.cuh -- negacyclic NTT of one limb-poly held in shared memory (device functions).
//
// Forward: Cooley-Tukey, natural order in, bit-reversed order out, twiddles psi^brv(m+i)
// (psi a primitive 2N-th root mod q): out[k] = a(psi^(2 brv(k) + 1)).
// Inverse: Gentleman-Sande with psi^-brv(m+i), bit-reversed in, natural out, times N^-1
// (applied by the caller's store).  Twiddle products use Shoup's precomputed quotients.
#pragma once
#include "he_internal.cuh"

__device__ __forceinline__ void ntt_fwd_smem(uint64_t *s, const uint64_t *__restrict__ tw, const uint64_t *__restrict__ tws,
                                             uint64_t q, int logn) {
    const int half = 1 << (logn - 1);
    for (int lg_m = 0; lg_m < logn; ++lg_m) {
        const int lg_t = logn - 1 - lg_m;
        const int m = 1 << lg_m, tmask = (1 << lg_t) - 1;
        for (int j = threadIdx.x; j < half; j += blockDim.x) {
            const int i = j >> lg_t;
            const int i1 = (i << (lg_t + 1)) + (j & tmask);
            const int i2 = i1 + (1 << lg_t);
            const uint64_t w = __ldg(tw + m + i), wp = __ldg(tws + m + i);
            const uint64_t U = s[i1];
            const uint64_t V = mul_shoup(s[i2], w, wp, q);
            s[i1] = add_mod(U, V, q);
            s[i2] = sub_mod(U, V, q);
        }
        __syncthreads();
    }
}

__device__ __forceinline__ void ntt_inv_smem(uint64_t *s, const uint64_t *__restrict__ itw, const uint64_t *__restrict__ itws,
                                             uint64_t q, int logn) {
    const int half = 1 << (logn - 1);
    for (int lg_t = 0; lg_t < logn; ++lg_t) {
        const int lg_m = logn - 1 - lg_t;
        const int m = 1 << lg_m, tmask = (1 << lg_t) - 1;
        for (int j = threadIdx.x; j < half; j += blockDim.x) {
            const int i = j >> lg_t;
            const int i1 = (i << (lg_t + 1)) + (j & tmask);
            const int i2 = i1 + (1 << lg_t);
            const uint64_t w = __ldg(itw + m + i), wp = __ldg(itws + m + i);
            const uint64_t U = s[i1], V = s[i2];
            s[i1] = add_mod(U, V, q);
            s[i2] = mul_shoup(sub_mod(U, V, q), w, wp, q);
        }
        __syncthreads();
    }
}

// twiddle table of prime index p: which = 0 psi_rev, 1 its Shoup quotients, 2 psi^-1 rev, 3 quotients
__device__ __forceinline__ const uint64_t *twiddles(const uint64_t *d_tw, int p, int which, int logn) {
    return d_tw + (((size_t)p * 4 + which) << logn);
}
