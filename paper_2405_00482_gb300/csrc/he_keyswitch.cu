// he_keyswitch.cu -- key switching of many rotations after their decomposition (O3/O4, Sec. 2.2).
//
// Rotation j of a launch has Galois element g_j, key_j, input ciphertext ct_j and ModUp digits
// D_j = D + j d_stride (d_stride 0: one decomposition shared by every rotation, O4's hoisting).
// With u_c = sum_d phi_g(D_d) key_{d,c} over Q_level U P (c = 0, 1):
//   ks_p_kernel, per (j, c, P limb i): u_c on p_i, inverse NTT, times N^-1 [(P/p_i)^-1] -> pc_j[c][i]
//   ks_q_kernel, per (j, c, Q limb l): conv_l = sum_i pc_j[c][i] (P/p_i mod q_l), NTT, then
//     out_j[c][l] = (u_c on q_l - conv_l) P^-1, plus phi_g(c0)[l] for c = 0,
// with u_c on q_l formed in the same kernel, so the Q part of u_c is never stored.  This is
// ModDown (x_Q - Conv_{P->Q}(x_P)) P^-1 of hybrid key switching; every step is exact modular
// arithmetic, so the outputs are the canonical residues that a separate inner product,
// automorphism and ModDown give, bit for bit.
//
// The inner products gather D at the automorphism's source index (L2: the digits are shared or
// small) and stream the keys from HBM.  Each thread forms KS_U coefficients at once with every
// load of those coefficients (all digits when their count is known at compile time) issued
// before the first product, so a thread's loads overlap instead of queueing one after another.
#include "he_internal.cuh"
#include "he_ntt.cuh"

namespace {

struct KsGeom {
    const uint64_t *D;   // digits [ndig][ext][N] of rotation j at D + j d_stride
    int64_t d_stride;
    uint64_t *pc;        // [count][2][K][N]: converted P limbs in coefficient form
    int32_t ndig, ext, nl, L, LK, K;
};

constexpr int KS_U = 4;  // coefficients per thread per round: k, k + B, .., k + (KS_U - 1) B

// r[v] = sum_d D_d[ue][src[v]] key[d][c][kl][kk[v]] mod q for the coefficients v with kk[v] < len
// (key in Montgomery form: one REDC per 8 digits).  ND > 0: the digit count at compile time.
template <int ND>
__device__ __forceinline__ void ks_dot_u(uint64_t (&r)[KS_U], const uint64_t *__restrict__ D, int ndig_rt, int ext, int ue,
                                         const uint64_t *__restrict__ key, int c, int kl, int LK, int64_t N, const uint32_t (&src)[KS_U],
                                         const int (&kk)[KS_U], int len, int off, uint64_t q, uint64_t qinv) {
#pragma unroll
    for (int v = 0; v < KS_U; ++v) r[v] = 0;
    // a coefficient past len reads coefficient 0 (in bounds; its result is not stored), so every
    // load is unconditional and all of them are issued before the first product
    int ki[KS_U];
#pragma unroll
    for (int v = 0; v < KS_U; ++v) ki[v] = kk[v] < len ? kk[v] : 0;
    if constexpr (ND > 0) {
        static_assert(ND <= 8, "one REDC per 8 products");
        uint64_t dv[ND][KS_U], kv[ND][KS_U];
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            const uint64_t *Dd = D + ((int64_t)d * ext + ue) * N, *Kd = key + ((int64_t)(d * 2 + c) * LK + kl) * N + off;
#pragma unroll
            for (int v = 0; v < KS_U; ++v) {
                dv[d][v] = __ldg(Dd + src[v]);
                kv[d][v] = __ldg(Kd + ki[v]);
            }
        }
#pragma unroll
        for (int v = 0; v < KS_U; ++v) {
            u128 t = 0;
#pragma unroll
            for (int d = 0; d < ND; ++d) t += (u128)dv[d][v] * kv[d][v];
            r[v] = redc128(t, q, qinv);
        }
    } else {
        for (int d0 = 0; d0 < ndig_rt; d0 += 8) {
            u128 t[KS_U];
#pragma unroll
            for (int v = 0; v < KS_U; ++v) t[v] = 0;
            for (int d = d0; d < ndig_rt && d < d0 + 8; ++d) {
                const uint64_t *Dd = D + ((int64_t)d * ext + ue) * N, *Kd = key + ((int64_t)(d * 2 + c) * LK + kl) * N + off;
                uint64_t dv[KS_U], kv[KS_U];
#pragma unroll
                for (int v = 0; v < KS_U; ++v) {
                    dv[v] = __ldg(Dd + src[v]);
                    kv[v] = __ldg(Kd + ki[v]);
                }
#pragma unroll
                for (int v = 0; v < KS_U; ++v) t[v] += (u128)dv[v] * kv[v];
            }
#pragma unroll
            for (int v = 0; v < KS_U; ++v) r[v] = add_mod(r[v], redc128(t[v], q, qinv), q);
        }
    }
}

template <bool CL, int LOGN, int ND>
__global__ void ks_p_kernel(const RotTable jobs, KsGeom kg, ModDownConst md, const uint64_t *__restrict__ d_tw, const ModConst *__restrict__ mc,
                            int logn_rt) {
    HE_GRID_DEP();
    const int logn = LOGN ? LOGN : logn_rt;
    extern __shared__ uint64_t s[];
    const int64_t N = (int64_t)1 << logn;
    int item, off, len;
    slice_of<CL>(logn, item, off, len);
    const int j = item / (2 * kg.K), c = (item / kg.K) % 2, i = item % kg.K;
    const int pr = md.p_prime[i];
    const uint64_t q = mc[pr].q, qinv = mc[pr].qinv;
    const ulonglong2 *itw = twiddles(d_tw, pr, 1, logn);
    tw_prefetch<CL, false>(s, itw, logn);
    const RotJob jb = jobs.j[j];
    const uint64_t *D = kg.D + j * kg.d_stride;
    const int B = blockDim.x;
    for (int k0 = threadIdx.x; k0 < len; k0 += KS_U * B) {
        uint32_t src[KS_U];
        int kk[KS_U];
#pragma unroll
        for (int v = 0; v < KS_U; ++v) {
            kk[v] = k0 + v * B;
            src[v] = automorph_src((uint32_t)(off + kk[v]), jb.g, logn);
        }
        uint64_t r[KS_U];
        ks_dot_u<ND>(r, D, kg.ndig, kg.ext, kg.nl + i, jb.key, c, kg.L + i, kg.LK, N, src, kk, len, off, q, qinv);
#pragma unroll
        for (int v = 0; v < KS_U; ++v)
            if (kk[v] < len) s[SIDX(kk[v])] = r[v];
    }
    __syncthreads();
    inv_any<CL, LOGN>(s, itw, q, logn);
    uint64_t *dst = kg.pc + (((int64_t)j * 2 + c) * kg.K + i) * N + off;
    const uint64_t ni = mc[pr].ninv, nis = mc[pr].ninv_shoup;
    for (int k = threadIdx.x; k < len; k += B) dst[k] = mul_shoup(mul_shoup(s[SIDX(k)], ni, nis, q), md.inv[i], md.inv_shoup[i], q);
}

template <bool CL, int LOGN, int ND>
__global__ void ks_q_kernel(const RotTable jobs, KsGeom kg, ModDownConst md, const uint64_t *__restrict__ d_tw, const ModConst *__restrict__ mc,
                            int logn_rt) {
    HE_GRID_DEP();
    const int logn = LOGN ? LOGN : logn_rt;
    extern __shared__ uint64_t s[];
    const int64_t N = (int64_t)1 << logn;
    int item, off, len;
    slice_of<CL>(logn, item, off, len);
    const int j = item / (2 * kg.nl), c = (item / kg.nl) % 2, l = item % kg.nl;
    const int pl = md.q_prime[l];
    const uint64_t q = mc[pl].q, qinv = mc[pl].qinv;
    const ulonglong2 *tw = twiddles(d_tw, pl, 0, logn);
    tw_prefetch<CL, true>(s, tw, logn);
    const uint64_t *pc = kg.pc + ((int64_t)j * 2 + c) * kg.K * N + off;
    const int B = blockDim.x;
    for (int k0 = threadIdx.x; k0 < len; k0 += KS_U * B) {
        uint64_t acc[KS_U];
#pragma unroll
        for (int v = 0; v < KS_U; ++v) acc[v] = 0;
        for (int i = 0; i < kg.K; ++i) {
            uint64_t x[KS_U];
#pragma unroll
            for (int v = 0; v < KS_U; ++v) x[v] = k0 + v * B < len ? pc[(int64_t)i * N + k0 + v * B] : 0;
#pragma unroll
            for (int v = 0; v < KS_U; ++v) acc[v] = add_mod(acc[v], mul_shoup(x[v], md.hat[i][l], md.hat_shoup[i][l], q), q);
        }
#pragma unroll
        for (int v = 0; v < KS_U; ++v)
            if (k0 + v * B < len) s[SIDX(k0 + v * B)] = acc[v];
    }
    __syncthreads();
    fwd_any<CL, LOGN>(s, tw, q, logn);
    const RotJob jb = jobs.j[j];
    const uint64_t *D = kg.D + j * kg.d_stride;
    uint64_t *o = jb.out + ((int64_t)c * kg.nl + l) * N + off;
    const uint64_t *c0 = jb.ct + (int64_t)l * N;
    const uint64_t pinv = md.pinv[l], pinvs = md.pinv_shoup[l];
    for (int k0 = threadIdx.x; k0 < len; k0 += KS_U * B) {
        uint32_t src[KS_U];
        int kk[KS_U];
        uint64_t a0[KS_U];
#pragma unroll
        for (int v = 0; v < KS_U; ++v) {
            kk[v] = k0 + v * B;
            src[v] = automorph_src((uint32_t)(off + kk[v]), jb.g, logn);
            a0[v] = (c == 0 && kk[v] < len) ? c0[src[v]] : 0;
        }
        uint64_t x[KS_U];
        ks_dot_u<ND>(x, D, kg.ndig, kg.ext, l, jb.key, c, l, kg.LK, N, src, kk, len, off, q, qinv);
#pragma unroll
        for (int v = 0; v < KS_U; ++v) {
            if (kk[v] >= len) continue;
            uint64_t y = mul_shoup(sub_mod(x[v], s[SIDX(kk[v])], q), pinv, pinvs, q);
            if (c == 0) y = add_mod(y, a0[v], q);
            o[kk[v]] = y;
        }
    }
}

// ---- the same key switch for many rotations, in four launches ----
// With many rotations the inner products' automorphism gathers and key streams run in
// elementwise kernels (no shared memory, many warps per SM to hide their latency), and the
// transforms in kernels that do nothing else:
//   ks_up_kernel    u_c on the P limbs, NTT form -> pc_j[c][i]                       (elementwise)
//   ks_pintt_kernel pc_j[c][i] -> inverse NTT, times N^-1 [(P/p_i)^-1]                (transform)
//   ks_conv_kernel  conv_l = sum_i pc_j[c][i] (P/p_i mod q_l), NTT -> cv_j[c][l]      (transform)
//   ks_out_kernel   out_j[c][l] = (u_c on q_l - cv_j[c][l]) P^-1 (+ phi_g(c0)[l])    (elementwise)
// The values are those of ks_p_kernel / ks_q_kernel, bit for bit.

// grid (N / 256, count * 2 * K): thread per coefficient of one (j, c, P limb i)
template <int ND>
__global__ void __launch_bounds__(256) ks_up_kernel(const RotTable jobs, KsGeom kg, const ModConst *__restrict__ mc, int logn) {
    HE_GRID_DEP();
    const int64_t N = (int64_t)1 << logn;
    const int item = blockIdx.y;
    const int j = item / (2 * kg.K), c = (item / kg.K) % 2, i = item % kg.K;
    const int pr = kg.L + i;
    const uint64_t q = mc[pr].q, qinv = mc[pr].qinv;
    const RotJob jb = jobs.j[j];
    const uint64_t *D = kg.D + j * kg.d_stride;
    uint32_t src[KS_U];
    int kk[KS_U];
    const int k0 = blockIdx.x * (256 * KS_U) + threadIdx.x;
#pragma unroll
    for (int v = 0; v < KS_U; ++v) {
        kk[v] = k0 + v * 256;
        src[v] = automorph_src((uint32_t)kk[v], jb.g, logn);
    }
    uint64_t r[KS_U];
    ks_dot_u<ND>(r, D, kg.ndig, kg.ext, kg.nl + i, jb.key, c, kg.L + i, kg.LK, N, src, kk, (int)N, 0, q, qinv);
    uint64_t *dst = kg.pc + (int64_t)item * N;
#pragma unroll
    for (int v = 0; v < KS_U; ++v)
        if (kk[v] < N) dst[kk[v]] = r[v];
}

// in place on pc: item (j, c, i).  TPB 512: the one-CTA form with 512 threads and at most 64
// registers (two CTAs per SM); 256: the usual thread count; 0: the cluster form
template <bool CL, int LOGN, int TPB>
__global__ void __launch_bounds__(512, TPB == 512 ? 2 : 1) ks_pintt_kernel(KsGeom kg, ModDownConst md, const uint64_t *__restrict__ d_tw, const ModConst *__restrict__ mc, int logn_rt) {
    HE_GRID_DEP();
    const int logn = LOGN ? LOGN : logn_rt;
    extern __shared__ uint64_t s[];
    const int64_t N = (int64_t)1 << logn;
    int item, off, len;
    slice_of<CL>(logn, item, off, len);
    const int i = item % kg.K;
    const int pr = md.p_prime[i];
    const uint64_t q = mc[pr].q;
    const ulonglong2 *itw = twiddles(d_tw, pr, 1, logn);
    tw_prefetch<CL, false>(s, itw, logn);
    uint64_t *x = kg.pc + (int64_t)item * N + off;
    stage_in(s, x, len, [](uint64_t v) { return v; });
    __syncthreads();
    inv_any<CL, LOGN>(s, itw, q, logn);
    const uint64_t ni = mc[pr].ninv, nis = mc[pr].ninv_shoup;
    for (int k = threadIdx.x; k < len; k += blockDim.x) x[k] = mul_shoup(mul_shoup(s[SIDX(k)], ni, nis, q), md.inv[i], md.inv_shoup[i], q);
}

// item (j, c, l): cv_j[c][l] = NTT(sum_i pc_j[c][i] (P/p_i mod q_l))
template <bool CL, int LOGN, int TPB>
__global__ void __launch_bounds__(512, TPB == 512 ? 2 : 1) ks_conv_kernel(KsGeom kg, uint64_t *cv, ModDownConst md, const uint64_t *__restrict__ d_tw, const ModConst *__restrict__ mc,
                               int logn_rt) {
    HE_GRID_DEP();
    const int logn = LOGN ? LOGN : logn_rt;
    extern __shared__ uint64_t s[];
    const int64_t N = (int64_t)1 << logn;
    int item, off, len;
    slice_of<CL>(logn, item, off, len);
    const int jc = item / kg.nl, l = item % kg.nl;
    const int pl = md.q_prime[l];
    const uint64_t q = mc[pl].q;
    const ulonglong2 *tw = twiddles(d_tw, pl, 0, logn);
    tw_prefetch<CL, true>(s, tw, logn);
    const uint64_t *pc = kg.pc + (int64_t)jc * kg.K * N + off;
    const uint64_t h0 = md.hat[0][l], h0s = md.hat_shoup[0][l];
    stage_in(s, pc, len, [=](uint64_t v) { return mul_shoup(v, h0, h0s, q); });
    __syncthreads();
    for (int i = 1; i < kg.K; ++i) {
        for (int k = threadIdx.x; k < len; k += blockDim.x)
            s[SIDX(k)] = add_mod(s[SIDX(k)], mul_shoup(pc[(int64_t)i * N + k], md.hat[i][l], md.hat_shoup[i][l], q), q);
        __syncthreads();
    }
    fwd_any<CL, LOGN>(s, tw, q, logn);
    uint64_t *o = cv + (int64_t)item * N + off;
    for (int k = threadIdx.x; k < len; k += blockDim.x) o[k] = s[SIDX(k)];
}

// ---- transform variant 2: the two transforms in two phases each (he_ntt.cuh, NTT form 2) ----
// P limbs: the inverse row phase, then the inverse column phase scaled by N^-1 [(P/p_i)^-1] (the
// values of ks_pintt_kernel); Q limbs: the forward column phase on the conversion
// sum_i pc_j[c][i] (P/p_i mod q_l), then the forward row phase (the values of ks_conv_kernel).
template <int LOGN, int NBA>
__global__ void __launch_bounds__(NTT2_THREADS) ks2_pinv_rows_kernel(KsGeom kg, ModDownConst md, const uint64_t *__restrict__ d_tw,
                                                                   const ModConst *__restrict__ mc) {
    HE_GRID_DEP();
    constexpr int N = 1 << LOGN, TILES = 64 / NTT2_TR;
    __shared__ uint64_t sm[ntt2_rows_smem_words(LOGN - 6)];
    const int item = blockIdx.x / TILES, b0 = (blockIdx.x % TILES) * NTT2_TR;
    const int pr = md.p_prime[item % kg.K];
    uint64_t *x = kg.pc + (int64_t)item * N;
    ntt2_inv_rows<LOGN, NBA>(sm, x, x, b0, TwGlobal{twiddles(d_tw, pr, 1, LOGN)}, mc[pr].q);
}

template <int LOGN>
__global__ void __launch_bounds__(NTT2_THREADS, 8) ks2_pinv_cols_kernel(KsGeom kg, ModDownConst md, const uint64_t *__restrict__ d_tw,
                                                                      const ModConst *__restrict__ mc) {
    HE_GRID_DEP();
    constexpr int N = 1 << LOGN, TILES = (N >> 6) / NTT2_TC;
    __shared__ uint64_t sm[ntt2_cols_smem_words()];
    const int item = blockIdx.x / TILES, c0 = (blockIdx.x % TILES) * NTT2_TC;
    const int i = item % kg.K, pr = md.p_prime[i];
    const uint64_t q = mc[pr].q, ni = mc[pr].ninv, nis = mc[pr].ninv_shoup, f = md.inv[i], fs = md.inv_shoup[i];
    uint64_t *x = kg.pc + (int64_t)item * N;
    ntt2_inv_cols<LOGN>(sm, x, c0, TwGlobal{twiddles(d_tw, pr, 1, LOGN)}, q,
                        [=](int64_t k, uint64_t v) { x[k] = mul_shoup(mul_shoup(v, ni, nis, q), f, fs, q); });
}

template <int LOGN>
__global__ void __launch_bounds__(NTT2_THREADS, 8) ks2_conv_cols_kernel(KsGeom kg, uint64_t *cv, ModDownConst md, const uint64_t *__restrict__ d_tw,
                                                                      const ModConst *__restrict__ mc) {
    HE_GRID_DEP();
    constexpr int N = 1 << LOGN, TILES = (N >> 6) / NTT2_TC;
    __shared__ uint64_t sm[ntt2_cols_smem_words()];
    const int item = blockIdx.x / TILES, c0 = (blockIdx.x % TILES) * NTT2_TC;
    const int jc = item / kg.nl, l = item % kg.nl, pl = md.q_prime[l];
    const uint64_t q = mc[pl].q, h0 = md.hat[0][l], h0s = md.hat_shoup[0][l];
    const uint64_t *pc = kg.pc + (int64_t)jc * kg.K * N;
    ntt2_fwd_cols<LOGN>(
        sm,
        [&](int64_t x) {
            uint64_t v = mul_shoup(pc[x], h0, h0s, q);
            for (int i = 1; i < kg.K; ++i) v = add_mod(v, mul_shoup(pc[(int64_t)i * N + x], md.hat[i][l], md.hat_shoup[i][l], q), q);
            return v;
        },
        cv + (int64_t)item * N, c0, TwGlobal{twiddles(d_tw, pl, 0, LOGN)}, q);
}

template <int LOGN>
__global__ void __launch_bounds__(NTT2_THREADS, 8) ks2_conv_rows_kernel(uint64_t *cv, int nl, ModDownConst md, const uint64_t *__restrict__ d_tw,
                                                                      const ModConst *__restrict__ mc) {
    HE_GRID_DEP();
    constexpr int N = 1 << LOGN, TILES = 64 / NTT2_TR;
    __shared__ uint64_t sm[ntt2_frows_smem_words(LOGN - 6)];
    const int item = blockIdx.x / TILES, b0 = (blockIdx.x % TILES) * NTT2_TR;
    const int pl = md.q_prime[item % nl];
    ntt2_fwd_rows<LOGN>(sm, cv + (int64_t)item * N, b0, TwGlobal{twiddles(d_tw, pl, 0, LOGN)}, mc[pl].q, mc[pl].mu);
}

// the four launches of transform variant 2 (log N = 12, 13, 14)
void ks2_transforms(int logn, const KsGeom &kg, uint64_t *cv, const ModDownConst &md, const uint64_t *tw, const ModConst *mc, int np, int nq,
                    cudaStream_t st) {
    const int tiles_c = (1 << (logn - 6)) / NTT2_TC, tiles_r = 64 / NTT2_TR;
    auto go = [&](auto L, auto NB) {
        constexpr int LG = decltype(L)::value, NB1 = decltype(NB)::value;
        launch_k(ks2_pinv_rows_kernel<LG, LG - 6 - NB1>, (unsigned)(np * tiles_r), NTT2_THREADS, 0, st, kg, md, tw, mc);
        launch_k(ks2_pinv_cols_kernel<LG>, (unsigned)(np * tiles_c), NTT2_THREADS, 0, st, kg, md, tw, mc);
        launch_k(ks2_conv_cols_kernel<LG>, (unsigned)(nq * tiles_c), NTT2_THREADS, 0, st, kg, cv, md, tw, mc);
        launch_k(ks2_conv_rows_kernel<LG>, (unsigned)(nq * tiles_r), NTT2_THREADS, 0, st, cv, kg.nl, md, tw, mc);
    };
    if (logn == 12) go(std::integral_constant<int, 12>{}, std::integral_constant<int, 3>{});
    else if (logn == 13) go(std::integral_constant<int, 13>{}, std::integral_constant<int, 4>{});
    else go(std::integral_constant<int, 14>{}, std::integral_constant<int, 4>{});
}

// grid (N / (256 KS_U), count * 2 * nl): thread per KS_U coefficients of one (j, c, Q limb l)
template <int ND>
__global__ void __launch_bounds__(256) ks_out_kernel(const RotTable jobs, KsGeom kg, const uint64_t *__restrict__ cv, ModDownConst md,
                                                     const ModConst *__restrict__ mc, int logn) {
    HE_GRID_DEP();
    const int64_t N = (int64_t)1 << logn;
    const int item = blockIdx.y;
    const int j = item / (2 * kg.nl), c = (item / kg.nl) % 2, l = item % kg.nl;
    const int pl = md.q_prime[l];
    const uint64_t q = mc[pl].q, qinv = mc[pl].qinv;
    const RotJob jb = jobs.j[j];
    const uint64_t *D = kg.D + j * kg.d_stride;
    const uint64_t *c0 = jb.ct + (int64_t)l * N, *cvl = cv + (int64_t)item * N;
    uint32_t src[KS_U];
    int kk[KS_U];
    uint64_t a0[KS_U], w[KS_U];
    const int k0 = blockIdx.x * (256 * KS_U) + threadIdx.x;
#pragma unroll
    for (int v = 0; v < KS_U; ++v) {
        kk[v] = k0 + v * 256;
        src[v] = automorph_src((uint32_t)kk[v], jb.g, logn);  // in range for any kk (its low log N bits)
        w[v] = __ldg(cvl + (kk[v] < N ? kk[v] : 0));
        a0[v] = c == 0 ? __ldg(c0 + src[v]) : 0;
    }
    uint64_t x[KS_U];
    ks_dot_u<ND>(x, D, kg.ndig, kg.ext, l, jb.key, c, l, kg.LK, N, src, kk, (int)N, 0, q, qinv);
    uint64_t *o = jb.out + ((int64_t)c * kg.nl + l) * N;
#pragma unroll
    for (int v = 0; v < KS_U; ++v) {
        if (kk[v] >= N) continue;
        uint64_t y = mul_shoup(sub_mod(x[v], w[v], q), md.pinv[l], md.pinv_shoup[l], q);
        if (c == 0) y = add_mod(y, a0[v], q);
        o[kk[v]] = y;
    }
}

// instance for (cluster form, ring size, digit count): 3 digits (the parameter sets' top
// levels) at compile time, every other count at run time
template <bool CL, class F>
auto ks_pick(int logn, int ndig, F f) {
    return by_logn(logn, [&](auto L) { return ndig == 3 ? f.template operator()<CL, L.value, 3>() : f.template operator()<CL, L.value, 0>(); });
}

}  // namespace

size_t keyswitch_many_pc_words(const he_ctx *ctx, int count) {
    const int c = count < HE_ROT_CHUNK ? count : HE_ROT_CHUNK;
    return (size_t)c * 2 * (ctx->K + ctx->L) * ctx->n;  // pc [c][2][K][N], then cv [c][2][nl][N] (nl <= L)
}

void launch_keyswitch_many(he_ctx *ctx, const RotJob *jobs, int count, int level, const uint64_t *D, int64_t d_stride, uint64_t *pc) {
    const ModUpConst &mu = ctx->modup[level];
    const ModDownConst &md = ctx->moddown[level];
    const int logn = ctx->log_n;
    cudaStream_t st = ctx->stream;
    const uint64_t *tw = ctx->d_tw;
    const ModConst *mc = ctx->d_mc;
    const int cmax = count < HE_ROT_CHUNK ? count : HE_ROT_CHUNK;
    uint64_t *cv = pc + (size_t)cmax * 2 * ctx->K * ctx->n;  // [cmax][2][level+1][N] after pc [cmax][2][K][N]
    // one chunk's launches with transform variant v (0: ntt_threads per CTA, 1: 512 threads,
    // 2: two phases of small CTAs per transform)
    auto issue = [&](int c0, int v) {
        const int n = count - c0 < HE_ROT_CHUNK ? count - c0 : HE_ROT_CHUNK;
        RotTable tab{};
        for (int j = 0; j < n; ++j) tab.j[j] = jobs[c0 + j];
        KsGeom kg{};
        kg.D = D + c0 * d_stride;
        kg.d_stride = d_stride;
        kg.pc = pc;  // pc and cv are reused by each chunk: the chunks run in stream order
        kg.ndig = mu.ndig;
        kg.ext = mu.ext;
        kg.nl = level + 1;
        kg.L = ctx->L;
        kg.LK = ctx->L + ctx->K;
        kg.K = ctx->K;
        const int np = n * 2 * ctx->K, nq = n * 2 * (level + 1);
        if (use_cluster(logn, nq)) {
            // few rotations: two cluster launches, the inner products inside the transforms
            ctx->launches += 2;
            const auto kp = ks_pick<true>(logn, mu.ndig, []<bool CL, int LOGN, int ND>() { return ks_p_kernel<CL, LOGN, ND>; });
            const auto kq = ks_pick<true>(logn, mu.ndig, []<bool CL, int LOGN, int ND>() { return ks_q_kernel<CL, LOGN, ND>; });
            launch_cluster(kp, np * HE_NTT_CL_SIZE, cl_threads(logn), cl_smem_bytes(logn), st, tab, kg, md, tw, mc, logn);
            launch_cluster(kq, nq * HE_NTT_CL_SIZE, cl_threads(logn), cl_smem_bytes(logn), st, tab, kg, md, tw, mc, logn);
            return;
        }
        const unsigned eblocks = (unsigned)((ctx->n + 256 * KS_U - 1) / (256 * KS_U));
        ctx->launches += 4;
        // CUDA-event timing of the transforms and of the elementwise kernels, when profiling
        cudaEvent_t *pe = prof_pair(ctx, HE_PROF_KS_ELEMENTWISE), *pt = nullptr;
        if (pe) cudaEventRecord(pe[0], st);
        if (mu.ndig == 3)
            launch_k(ks_up_kernel<3>, dim3(eblocks, (unsigned)np), 256, 0, st, tab, kg, mc, logn);
        else
            launch_k(ks_up_kernel<0>, dim3(eblocks, (unsigned)np), 256, 0, st, tab, kg, mc, logn);
        if (pe) {
            cudaEventRecord(pe[1], st);
            pt = prof_pair(ctx, HE_PROF_KS_TRANSFORM);
            if (pt) cudaEventRecord(pt[0], st);
        }
        // the transforms: cluster form for few limb-polys, else one CTA each, or two phases each
        const bool wide = v == 1 && logn >= 12;
        if (v == 2 && logn >= 12 && logn <= 14) {
            ctx->launches += 2;
            ks2_transforms(logn, kg, cv, md, tw, mc, np, nq, st);
        } else if (use_cluster(logn, np))
            launch_cluster(by_logn(logn, [](auto L) { return ks_pintt_kernel<true, L.value, 0>; }), np * HE_NTT_CL_SIZE, cl_threads(logn),
                           cl_smem_bytes(logn), st, kg, md, tw, mc, logn);
        else if (wide)
            launch_k(by_logn(logn, [](auto L) { return ks_pintt_kernel<false, L.value, 512>; }), np, 512, ntt_smem_bytes(logn), st, kg, md, tw, mc, logn);
        else
            launch_k(by_logn(logn, [](auto L) { return ks_pintt_kernel<false, L.value, 256>; }), np, ntt_threads(logn), ntt_smem_bytes(logn), st, kg, md, tw,
                     mc, logn);
        if (v == 2 && logn >= 12 && logn <= 14)
            ;  // both transforms launched above
        else if (wide)
            launch_k(by_logn(logn, [](auto L) { return ks_conv_kernel<false, L.value, 512>; }), nq, 512, ntt_smem_bytes(logn), st, kg, cv, md, tw, mc, logn);
        else
            launch_k(by_logn(logn, [](auto L) { return ks_conv_kernel<false, L.value, 256>; }), nq, ntt_threads(logn), ntt_smem_bytes(logn), st, kg, cv, md,
                     tw, mc, logn);
        cudaEvent_t *pe2 = nullptr;
        if (pt) {
            cudaEventRecord(pt[1], st);
            pe2 = prof_pair(ctx, HE_PROF_KS_ELEMENTWISE);
            if (pe2) cudaEventRecord(pe2[0], st);
        }
        if (mu.ndig == 3)
            launch_k(ks_out_kernel<3>, dim3(eblocks, (unsigned)nq), 256, 0, st, tab, kg, (const uint64_t *)cv, md, mc, logn);
        else
            launch_k(ks_out_kernel<0>, dim3(eblocks, (unsigned)nq), 256, 0, st, tab, kg, (const uint64_t *)cv, md, mc, logn);
        if (pe2) cudaEventRecord(pe2[1], st);
    };
    // the first launch of at least 32 rotations on a context chooses the transform variant by timing
    // both on its first chunk (the launches overwrite their outputs with the same values, so
    // repeating them changes nothing); not under stream capture, where the usual thread count is taken
    if (ctx->ks_variant < 0 && cmax >= 32 && !use_cluster(logn, cmax * 2 * (level + 1))) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(st, &cs);
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (cs == cudaStreamCaptureStatusNone && cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
            int best = 0;
            for (int v = 0; v < (logn >= 12 && logn <= 14 ? HE_KS_VARIANTS : 2); ++v) {
                float ms = 1e30f;
                for (int rep = 0; rep < 3; ++rep) {
                    cudaEventRecord(e0, st);
                    issue(0, v);
                    cudaEventRecord(e1, st);
                    if (cudaEventSynchronize(e1) != cudaSuccess) break;
                    float t = 0.0f;
                    cudaEventElapsedTime(&t, e0, e1);
                    if (rep > 0 && t < ms) ms = t;
                }
                ctx->ks_tune_ms[v] = ms;
                if (ms < ctx->ks_tune_ms[best]) best = v;
            }
            ctx->ks_variant = best;
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
    for (int c0 = 0; c0 < count; c0 += HE_ROT_CHUNK) issue(c0, ctx->ks_variant < 0 ? 0 : ctx->ks_variant);
}

void keyswitch_set_smem_limits(int max_bytes) {
    auto set = [max_bytes](auto k) { cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes); };
    for (int logn : {0, 12, 13, 14})
        for (int nd : {0, 3}) {
            set(ks_pick<true>(logn, nd, []<bool CL, int LOGN, int ND>() { return ks_p_kernel<CL, LOGN, ND>; }));
            set(ks_pick<false>(logn, nd, []<bool CL, int LOGN, int ND>() { return ks_p_kernel<CL, LOGN, ND>; }));
            set(ks_pick<true>(logn, nd, []<bool CL, int LOGN, int ND>() { return ks_q_kernel<CL, LOGN, ND>; }));
            set(ks_pick<false>(logn, nd, []<bool CL, int LOGN, int ND>() { return ks_q_kernel<CL, LOGN, ND>; }));
        }
    each_logn([&](auto L) {
        set(ks_pintt_kernel<true, L.value, 0>);
        set(ks_pintt_kernel<false, L.value, 256>);
        set(ks_pintt_kernel<false, L.value, 512>);
        set(ks_conv_kernel<true, L.value, 0>);
        set(ks_conv_kernel<false, L.value, 256>);
        set(ks_conv_kernel<false, L.value, 512>);
    });
}

extern "C" int he_set_keyswitch_variant(he_ctx *ctx, int variant) {
    if (!ctx || variant < -1 || variant >= HE_KS_VARIANTS) return HE_EINVAL;
    if (variant == 2 && (ctx->log_n < 12 || ctx->log_n > 14)) return HE_EINVAL;
    ctx->ks_variant = variant;
    return HE_OK;
}

extern "C" int he_keyswitch_tuning(const he_ctx *ctx, int *variant, float *ms) {
    if (!ctx || !variant) return HE_EINVAL;
    *variant = ctx->ks_variant;
    if (ms)
        for (int v = 0; v < HE_KS_VARIANTS; ++v) ms[v] = ctx->ks_tune_ms[v];
    return HE_OK;
}
