// he_ops.cu -- ciphertext arithmetic, hybrid key switching and the PackVFL MatMult loop.
//
// Key switching (O3/O4, Sec. 2.2) uses hybrid decomposition with dnum digits:
//   D = ModUp(c1): each digit's residues extended to Q_level U P by exact fast base conversion;
//   u_c = sum_d phi_g(D_d) * evk_{g,d,c}           (NTT domain; phi_g is an index gather);
//   ModDown(x) = (x_Q - Conv_{P->Q}(x_P)) * P^-1.
// The MatMult loop (Eq. 2/3, Tab. 2) keeps sum_i pt_i * u^(i) in Q U P and divides by P once.
#include "he_internal.cuh"
#include "he_ntt.cuh"


namespace {

__global__ void add_kernel(const uint64_t *__restrict__ a, const uint64_t *__restrict__ b, uint64_t *out, LimbMap map,
                           const ModConst *__restrict__ mc, int logn) {
    HE_GRID_DEP();
    const int N = 1 << logn;
    const int l = blockIdx.y, g = blockIdx.z;
    const uint64_t q = mc[map.prime[l]].q;
    const int64_t base = ((int64_t)g * map.n + l) * N;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) out[base + k] = add_mod(a[base + k], b[base + k], q);
}

// ct [2][nl][N] times pt [>= nl][N] (canonical): two Montgomery steps give the canonical product
__global__ void mul_plain_kernel(const uint64_t *__restrict__ ct, const uint64_t *__restrict__ pt, uint64_t *out, int nl,
                                 const ModConst *__restrict__ mc, int logn) {
    HE_GRID_DEP();
    const int N = 1 << logn;
    const int l = blockIdx.y, c = blockIdx.z;
    const ModConst m = mc[l];
    const int64_t base = ((int64_t)c * nl + l) * N;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
        uint64_t t = mont_mul(ct[base + k], pt[(int64_t)l * N + k], m.q, m.qinv);  // a b 2^-64
        out[base + k] = mont_mul(t, m.r2, m.q, m.qinv);                          // a b
    }
}

__global__ void automorph_kernel(const uint64_t *__restrict__ in, uint64_t *__restrict__ out, uint32_t g, int logn) {
    HE_GRID_DEP();
    const int N = 1 << logn;
    const int64_t base = (int64_t)blockIdx.y * N;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) out[base + k] = in[base + automorph_src(k, g, logn)];
}

// ModUp body for (d, u): digit-own limbs are copied from the NTT-form input; the others are
// converted from the coefficient-form digit limbs and transformed.  CL: this CTA handles the
// slice [off, off + len) of a cluster-shared limb-poly.
template <bool CL>
__device__ __forceinline__ void modup_body(const uint64_t *__restrict__ c1_ntt, const uint64_t *__restrict__ c1_coef, uint64_t *D,
                                           const ModUpConst &mu, int d, int u, uint64_t *s, const uint64_t *__restrict__ d_tw,
                                           const ModConst *__restrict__ mc, int logn, int off, int len) {
    const int N = 1 << logn;
    const int lo = d * mu.alpha;
    const int hi = lo + mu.alpha < mu.nq ? lo + mu.alpha : mu.nq;
    const int p = mu.ext_prime[u];
    const uint64_t t = mc[p].q;
    uint64_t *dst = D + ((int64_t)d * mu.ext + u) * N + off;
    if (u >= lo && u < hi) {  // uniform over the whole cluster
        for (int k = threadIdx.x; k < len; k += blockDim.x) dst[k] = c1_ntt[(int64_t)u * N + off + k];
        return;
    }
    tw_prefetch<CL, true>(s, twiddles(d_tw, p, 0, logn), logn);
    const int na = hi - lo;
    // sum over the digit's primes of [x_i (Qd/q_i)^-1]_{q_i} (Qd/q_i mod t), one source limb at a
    // time with its loads staged (eight in flight per thread)
    for (int i = 0; i < na; ++i) {
        const uint64_t qi = mc[lo + i].q, iv = mu.inv[d][i], ivs = mu.inv_shoup[d][i], h = mu.hat[d][i][u], hs = mu.hat_shoup[d][i][u];
        const uint64_t *src = c1_coef + (int64_t)(lo + i) * N + off;
        auto term = [=](uint64_t x) { return mul_shoup(mul_shoup(x, iv, ivs, qi), h, hs, t); };
        if (i == 0)
            stage_in(s, src, len, term);
        else
            stage_acc(s, src, len, [=](uint64_t a, uint64_t x) { return add_mod(a, term(x), t); });
    }
    __syncthreads();
    fwd_any<CL>(s, twiddles(d_tw, p, 0, logn), t, logn);
    for (int k = threadIdx.x; k < len; k += blockDim.x) dst[k] = s[SIDX(k)];
}

template <bool CL>
__global__ void modup_kernel(const uint64_t *__restrict__ c1_ntt, const uint64_t *__restrict__ c1_coef, uint64_t *D, ModUpConst mu,
                             const uint64_t *__restrict__ d_tw, const ModConst *__restrict__ mc, int logn) {
    HE_GRID_DEP();
    extern __shared__ uint64_t s[];
    int item, off, len;
    slice_of<CL>(logn, item, off, len);
    modup_body<CL>(c1_ntt, c1_coef, D, mu, item / mu.ext, item % mu.ext, s, d_tw, mc, logn, off, len);
}

// u_c[u][k] = sum_d D[d][u][src(k)] * keyM[d][c][kl(u)][k], REDC in groups of at most 8 terms
__global__ void ks_inner_kernel(const uint64_t *__restrict__ D, int ndig, int ext, LimbMap emap, int nq, int L, int LK, uint32_t g, const uint64_t *__restrict__ key, uint64_t *out,
                                const ModConst *__restrict__ mc, int logn) {
    HE_GRID_DEP();
    const int N = 1 << logn;
    const int u = blockIdx.y;
    const int p = emap.prime[u];
    const int kl = u < nq ? u : L + (u - nq);
    const uint64_t q = mc[p].q, qinv = mc[p].qinv;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
        const uint32_t src = automorph_src(k, g, logn);
        uint64_t r0 = 0, r1 = 0;
        for (int d0 = 0; d0 < ndig; d0 += 8) {
            u128 t0 = 0, t1 = 0;
            for (int d = d0; d < ndig && d < d0 + 8; ++d) {
                const uint64_t dv = D[((int64_t)d * ext + u) * N + src];
                t0 += (u128)dv * key[((int64_t)(d * 2 + 0) * LK + kl) * N + k];
                t1 += (u128)dv * key[((int64_t)(d * 2 + 1) * LK + kl) * N + k];
            }
            r0 = add_mod(r0, redc128(t0, q, qinv), q);
            r1 = add_mod(r1, redc128(t1, q, qinv), q);
        }
        out[((int64_t)0 * ext + u) * N + k] = r0;
        out[((int64_t)1 * ext + u) * N + k] = r1;
    }
}

// ModDown body for (c, j): conv = Conv_{P->q_j}(x_P, coefficient form) -> NTT ->
// out = add_c + (x_j - conv) P^-1.  CL: slice [off, off + len) of a cluster-shared limb-poly.
template <bool CL>
__device__ __forceinline__ void moddown_body(const uint64_t *__restrict__ x, int ext, const uint64_t *__restrict__ xp_coef,
                                             const ModDownConst &md, const uint64_t *__restrict__ ad, uint64_t *out, int c, int j,
                                             uint64_t *s, const uint64_t *__restrict__ d_tw, const ModConst *__restrict__ mc, int logn,
                                             int off, int len) {
    const int N = 1 << logn;
    const int pj = md.q_prime[j];
    const uint64_t q = mc[pj].q;
    tw_prefetch<CL, true>(s, twiddles(d_tw, pj, 0, logn), logn);
    const uint64_t *xp = xp_coef + (int64_t)c * md.K * N + off;
    for (int i = 0; i < md.K; ++i) {  // conversion of the P limbs, loads staged as in modup_body
        const uint64_t pi = mc[md.p_prime[i]].q, iv = md.inv[i], ivs = md.inv_shoup[i], h = md.hat[i][j], hs = md.hat_shoup[i][j];
        auto term = [=](uint64_t x) { return mul_shoup(mul_shoup(x, iv, ivs, pi), h, hs, q); };
        if (i == 0)
            stage_in(s, xp, len, term);
        else
            stage_acc(s, xp + (int64_t)i * N, len, [=](uint64_t a, uint64_t x) { return add_mod(a, term(x), q); });
    }
    __syncthreads();
    fwd_any<CL>(s, twiddles(d_tw, pj, 0, logn), q, logn);
    const uint64_t *xj = x + ((int64_t)c * ext + j) * N + off;
    uint64_t *o = out + ((int64_t)c * md.nq + j) * N + off;
    const uint64_t *a = ad ? ad + (int64_t)j * N + off : nullptr;
    for (int k = threadIdx.x; k < len; k += blockDim.x) {
        uint64_t v = mul_shoup(sub_mod(xj[k], s[SIDX(k)], q), md.pinv[j], md.pinv_shoup[j], q);
        if (a) v = add_mod(v, a[k], q);
        o[k] = v;
    }
}

template <bool CL>
__global__ void moddown_kernel(const uint64_t *__restrict__ x, int ext, const uint64_t *__restrict__ xp_coef, ModDownConst md,
                               const uint64_t *__restrict__ add0, const uint64_t *__restrict__ add1, uint64_t *out,
                               const uint64_t *__restrict__ d_tw, const ModConst *__restrict__ mc, int logn) {
    HE_GRID_DEP();
    extern __shared__ uint64_t s[];
    int item, off, len;
    slice_of<CL>(logn, item, off, len);
    const int c = item / md.nq, j = item % md.nq;
    moddown_body<CL>(x, ext, xp_coef, md, c == 0 ? add0 : add1, out, c, j, s, d_tw, mc, logn, off, len);
}

struct RescaleConst {
    uint64_t ql, half;
    uint64_t inv[HE_MAX_Q], inv_shoup[HE_MAX_Q];  // q_l^-1 mod q_j
};

// Rescale body for (c, j), j < level: v = centred(last limb) mod q_j -> NTT ->
// out = (c_j - v) q_l^-1.  CL: slice [off, off + len) of a cluster-shared limb-poly.
template <bool CL>
__device__ __forceinline__ void rescale_body(const uint64_t *__restrict__ ct, int level, const uint64_t *__restrict__ last_coef,
                                             const RescaleConst &rc, uint64_t *out, int c, int j, uint64_t *s,
                                             const uint64_t *__restrict__ d_tw, const ModConst *__restrict__ mc, int logn, int off, int len) {
    const int N = 1 << logn;
    const uint64_t q = mc[j].q;
    tw_prefetch<CL, true>(s, twiddles(d_tw, j, 0, logn), logn);
    const uint64_t *lc = last_coef + (int64_t)c * N + off;
    const uint64_t ql = rc.ql, half = rc.half, mu = mc[j].mu;
    stage_in(s, lc, len, [=](uint64_t x) {
        uint64_t r = x + half;
        if (r >= ql) r -= ql;
        return reduce_signed((int64_t)r - (int64_t)half, q, mu);
    });
    __syncthreads();
    fwd_any<CL>(s, twiddles(d_tw, j, 0, logn), q, logn);
    const uint64_t *cj = ct + ((int64_t)c * (level + 1) + j) * N + off;
    uint64_t *o = out + ((int64_t)c * level + j) * N + off;
    for (int k = threadIdx.x; k < len; k += blockDim.x) o[k] = mul_shoup(sub_mod(cj[k], s[SIDX(k)], q), rc.inv[j], rc.inv_shoup[j], q);
}

template <bool CL>
__global__ void rescale_kernel(const uint64_t *__restrict__ ct, int level, const uint64_t *__restrict__ last_coef, RescaleConst rc,
                               uint64_t *out, const uint64_t *__restrict__ d_tw, const ModConst *__restrict__ mc, int logn) {
    HE_GRID_DEP();
    extern __shared__ uint64_t s[];
    int item, off, len;
    slice_of<CL>(logn, item, off, len);
    rescale_body<CL>(ct, level, last_coef, rc, out, item / level, item % level, s, d_tw, mc, logn, off, len);
}

// ---- cluster forms with the inverse NTT inside: one launch per stage instead of two ----
// Each cluster item transforms the limb-polys it needs back to coefficient form itself (a
// cluster inverse NTT of the input slice, then the N^-1 scaling of the separate inverse-NTT
// kernel), so ModUp, ModDown and rescale no longer wait on a preceding inverse-NTT launch and its
// round trip through global memory.  The per-element operations and their order are those of
// modup_body / moddown_body / rescale_body fed by that kernel, so results are bit-identical.
// Shared memory: the slice, its twiddles, and an accumulator slice.

// cluster inverse NTT of the slice [off, off + len) of limb-poly src (NTT form, prime index pr);
// canonical coefficients are then s[SIDX(k)] * N^-1 (applied by the caller with mul_shoup)
template <int LOGN = 0>
__device__ __forceinline__ void cl_intt_slice(uint64_t *s, const uint64_t *__restrict__ src, int pr, const uint64_t *__restrict__ d_tw,
                                              const ModConst *__restrict__ mc, int logn, int len, bool tw_issued = false) {
    const ulonglong2 *itw = twiddles(d_tw, pr, 1, logn);
    if (!tw_issued) tw_prefetch<true, false>(s, itw, logn);
    for (int k = threadIdx.x; k < len; k += blockDim.x) s[SIDX(k)] = src[k];
    __syncthreads();
    ntt_inv_cluster<LOGN>(s, itw, mc[pr].q, logn);
}
__device__ __forceinline__ uint64_t *cl_acc_slice(uint64_t *s, int logn) { return s + cl_tw_offset_words(logn) + 2 * (1 << (logn - 3)); }

// LOGN > 0: the ring size at compile time (logn_rt == LOGN)
// ModUp item (d, u) of one ciphertext (c1 in NTT form) as a cluster, the inverse NTT inside
template <int LOGN = 0>
__device__ __forceinline__ void modup_cl_fused_body(const uint64_t *__restrict__ c1_ntt, uint64_t *D, const ModUpConst &mu, int item,
                                                    const uint64_t *__restrict__ d_tw, const ModConst *__restrict__ mc, int logn, int off,
                                                    int len, bool tw_issued = false) {
    extern __shared__ uint64_t s[];
    const int N = 1 << logn;
    const int d = item / mu.ext, u = item % mu.ext;
    const int lo = d * mu.alpha;
    const int hi = lo + mu.alpha < mu.nq ? lo + mu.alpha : mu.nq;
    const int p = mu.ext_prime[u];
    const uint64_t t = mc[p].q;
    uint64_t *dst = D + ((int64_t)d * mu.ext + u) * N + off;
    if (u >= lo && u < hi) {  // uniform over the whole cluster
        for (int k = threadIdx.x; k < len; k += blockDim.x) dst[k] = c1_ntt[(int64_t)u * N + off + k];
        return;
    }
    if (hi - lo == 1) {
        // one limb per digit: its inverse transform's cross-CTA stages, the conversion to t and
        // the forward transform's cross-CTA stages in one pass (ntt_cross_inv_fwd); the same
        // operations as the general path below
        const int i = lo;
        const uint64_t qi = mc[i].q;
        const ulonglong2 *itw = twiddles(d_tw, i, 1, logn), *tw = twiddles(d_tw, p, 0, logn);
        if (!tw_issued) tw_prefetch<true, false>(s, itw, logn);
        for (int k = threadIdx.x; k < len; k += blockDim.x) s[SIDX(k)] = c1_ntt[(int64_t)i * N + off + k];
        __syncthreads();
        ulonglong2 wi[3], wf[3];
        cross_tw_load<false>(wi, itw);
        cross_tw_load<true>(wf, tw);
        ntt_inv_cluster_local<LOGN>(s, qi, logn);
        tw_prefetch<true, true>(s, tw, logn);  // the inverse copy is no longer read
        cg::this_cluster().sync();
        const ModConst mi = mc[i];
        const uint64_t inv = mu.inv[d][0], inv_s = mu.inv_shoup[d][0], hat = mu.hat[d][0][u], hat_s = mu.hat_shoup[d][0][u];
        ntt_cross_inv_fwd(
            s, wi, qi,
            [&](uint64_t x) { return mul_shoup(mul_shoup(mul_shoup(x, mi.ninv, mi.ninv_shoup, qi), inv, inv_s, qi), hat, hat_s, t); }, wf, t,
            logn);
        tw_slice_wait();
        cg::this_cluster().sync();
        ntt_fwd_cluster_local<LOGN>(s, t, logn);
        for (int k = threadIdx.x; k < len; k += blockDim.x) dst[k] = s[SIDX(k)];
        return;
    }
    uint64_t *acc = cl_acc_slice(s, logn);
    for (int k = threadIdx.x; k < len; k += blockDim.x) acc[k] = 0;
    for (int i = lo; i < hi; ++i) {
        cl_intt_slice<LOGN>(s, c1_ntt + (int64_t)i * N + off, i, d_tw, mc, logn, len, tw_issued && i == lo);
        const uint64_t qi = mc[i].q;
        for (int k = threadIdx.x; k < len; k += blockDim.x) {
            uint64_t v = mul_shoup(s[SIDX(k)], mc[i].ninv, mc[i].ninv_shoup, qi);
            v = mul_shoup(v, mu.inv[d][i - lo], mu.inv_shoup[d][i - lo], qi);
            acc[k] = add_mod(acc[k], mul_shoup(v, mu.hat[d][i - lo][u], mu.hat_shoup[d][i - lo][u], t), t);
        }
        __syncthreads();
    }
    const ulonglong2 *tw = twiddles(d_tw, p, 0, logn);
    tw_prefetch<true, true>(s, tw, logn);
    for (int k = threadIdx.x; k < len; k += blockDim.x) s[SIDX(k)] = acc[k];
    __syncthreads();
    ntt_fwd_cluster<LOGN>(s, tw, t, logn);
    for (int k = threadIdx.x; k < len; k += blockDim.x) dst[k] = s[SIDX(k)];
}

template <int LOGN = 0>
__global__ void modup_cl_fused_kernel(const uint64_t *__restrict__ c1_ntt, uint64_t *D, ModUpConst mu, const uint64_t *__restrict__ d_tw,
                                      const ModConst *__restrict__ mc, int logn_rt) {
    HE_GRID_LAUNCH();
    const int logn = LOGN ? LOGN : logn_rt;
    int item, off, len;
    slice_of<true>(logn, item, off, len);
    // the first inverse transform's twiddle copy (a context table) before the wait
    const int d = item / mu.ext, u = item % mu.ext, lo = d * mu.alpha;
    const bool own = u >= lo && u < (lo + mu.alpha < mu.nq ? lo + mu.alpha : mu.nq);
    if (!own) tw_prefetch<true, false>(s_dyn(), twiddles(d_tw, lo, 1, logn), logn);
    HE_GRID_WAIT();
    modup_cl_fused_body<LOGN>(c1_ntt, D, mu, item, d_tw, mc, logn, off, len, !own);
}

// ModDown of component c, output limb j: conversion of the K special-prime limbs (each brought
// to coefficient form here), NTT, out = add_c + (x_j - conv) P^-1
// LOGN > 0: the ring size at compile time (logn_rt == LOGN)
template <int LOGN = 0>
__global__ void moddown_cl_fused_kernel(const uint64_t *__restrict__ x, int ext, ModDownConst md, const uint64_t *__restrict__ add0,
                                        const uint64_t *__restrict__ add1, uint64_t *out, const uint64_t *__restrict__ d_tw,
                                        const ModConst *__restrict__ mc, int logn_rt) {
    HE_GRID_DEP();
    const int logn = LOGN ? LOGN : logn_rt;
    extern __shared__ uint64_t s[];
    const int N = 1 << logn;
    int item, off, len;
    slice_of<true>(logn, item, off, len);
    const int c = item / md.nq, j = item % md.nq;
    const int pj = md.q_prime[j];
    const uint64_t q = mc[pj].q;
    uint64_t *acc = cl_acc_slice(s, logn);
    for (int k = threadIdx.x; k < len; k += blockDim.x) acc[k] = 0;
    for (int i = 0; i < md.K; ++i) {
        const int pr = md.p_prime[i];
        cl_intt_slice<LOGN>(s, x + ((int64_t)c * ext + md.nq + i) * N + off, pr, d_tw, mc, logn, len);
        const uint64_t pi = mc[pr].q;
        for (int k = threadIdx.x; k < len; k += blockDim.x) {
            uint64_t v = mul_shoup(s[SIDX(k)], mc[pr].ninv, mc[pr].ninv_shoup, pi);
            v = mul_shoup(v, md.inv[i], md.inv_shoup[i], pi);
            acc[k] = add_mod(acc[k], mul_shoup(v, md.hat[i][j], md.hat_shoup[i][j], q), q);
        }
        __syncthreads();
    }
    const ulonglong2 *tw = twiddles(d_tw, pj, 0, logn);
    tw_prefetch<true, true>(s, tw, logn);
    for (int k = threadIdx.x; k < len; k += blockDim.x) s[SIDX(k)] = acc[k];
    __syncthreads();
    ntt_fwd_cluster<LOGN>(s, tw, q, logn);
    const uint64_t *xj = x + ((int64_t)c * ext + j) * N + off;
    uint64_t *o = out + ((int64_t)c * md.nq + j) * N + off;
    const uint64_t *ad = c == 0 ? add0 : add1;
    const uint64_t *a = ad ? ad + (int64_t)j * N + off : nullptr;
    for (int k = threadIdx.x; k < len; k += blockDim.x) {
        uint64_t v = mul_shoup(sub_mod(xj[k], s[SIDX(k)], q), md.pinv[j], md.pinv_shoup[j], q);
        if (a) v = add_mod(v, a[k], q);
        o[k] = v;
    }
}

// rescale of component c, output limb j < level: the last limb in coefficient form (here),
// centred, reduced mod q_j, NTT, out = (c_j - v) q_l^-1
// LOGN > 0: the ring size at compile time (logn_rt == LOGN)
template <int LOGN = 0>
__global__ void rescale_cl_fused_kernel(const uint64_t *__restrict__ ct, int level, RescaleConst rc, uint64_t *out,
                                        const uint64_t *__restrict__ d_tw, const ModConst *__restrict__ mc, int logn_rt) {
    HE_GRID_DEP();
    const int logn = LOGN ? LOGN : logn_rt;
    extern __shared__ uint64_t s[];
    const int N = 1 << logn;
    int item, off, len;
    slice_of<true>(logn, item, off, len);
    const int c = item / level, j = item % level;
    const uint64_t q = mc[j].q, ql = mc[level].q;
    uint64_t *lc = cl_acc_slice(s, logn);
    cl_intt_slice<LOGN>(s, ct + ((int64_t)c * (level + 1) + level) * N + off, level, d_tw, mc, logn, len);
    for (int k = threadIdx.x; k < len; k += blockDim.x) lc[k] = mul_shoup(s[SIDX(k)], mc[level].ninv, mc[level].ninv_shoup, ql);
    __syncthreads();
    const ulonglong2 *tw = twiddles(d_tw, j, 0, logn);
    tw_prefetch<true, true>(s, tw, logn);
    for (int k = threadIdx.x; k < len; k += blockDim.x) {
        uint64_t r = lc[k] + rc.half;
        if (r >= rc.ql) r -= rc.ql;
        const int64_t centred = (int64_t)r - (int64_t)rc.half;
        s[SIDX(k)] = reduce_signed(centred, q, mc[j].mu);
    }
    __syncthreads();
    ntt_fwd_cluster<LOGN>(s, tw, q, logn);
    const uint64_t *cj = ct + ((int64_t)c * (level + 1) + j) * N + off;
    uint64_t *o = out + ((int64_t)c * level + j) * N + off;
    for (int k = threadIdx.x; k < len; k += blockDim.x) o[k] = mul_shoup(sub_mod(cj[k], s[SIDX(k)], q), rc.inv[j], rc.inv_shoup[j], q);
}

// ModDown then rescale (the MatMult epilogue).  Component c, output limb j < L (L = md.nq - 1,
// the limb the rescale drops); a_i the P limbs in coefficient form and conv_t their conversion to
// q_t.  ModDown gives sum_t = add_c[t] + (x_t - NTT(conv_t)) P^-1 and the rescale
// out_j = (sum_j - NTT([INTT(sum_L)]_j)) q_L^-1, [.]_j the centred lift reduced mod q_j.  The NTT
// being linear mod q_j, out_j = (add_c[j] + x_j P^-1 - NTT(w_j)) q_L^-1 with
// w_j = conv_j P^-1 + [INTT(sum_L)]_j, and INTT(sum_L) = INTT(add_c[L] + x_L P^-1) - conv_L P^-1.
// Each step is exact arithmetic mod a prime, so the output is the canonical residue the two
// separate stages give, bit for bit.  Two launches, each one cluster transform deep:
// moddown_rescale_intt_kernel brings every input limb the combination needs to coefficient form
// at once (per component the K limbs of P, already scaled by [(P/p_i)^-1]_{p_i}, and
// add_c[L] + x_L P^-1), into tmp [2][K+1][N]; moddown_rescale_ntt_kernel forms w_j per coefficient
// and transforms it.  (One launch doing the K + 2 transforms in a row took longer.)
template <int LOGN = 0>
__device__ __forceinline__ void moddown_rescale_intt_body(const uint64_t *__restrict__ x, int ext, const ModDownConst &md,
                                                          const uint64_t *__restrict__ add0, const uint64_t *__restrict__ add1, uint64_t *tmp,
                                                          int item, const uint64_t *__restrict__ d_tw, const ModConst *__restrict__ mc, int logn,
                                                          int off, int len, bool tw_issued = false) {
    extern __shared__ uint64_t s[];
    const int N = 1 << logn;
    const int c = item / (md.K + 1), r = item % (md.K + 1);
    const int L = md.nq - 1;
    uint64_t *o = tmp + ((int64_t)c * (md.K + 1) + r) * N + off;
    if (r < md.K) {  // P limb r: INTT, N^-1, [(P/p_r)^-1]
        const int pr = md.p_prime[r];
        const uint64_t pi = mc[pr].q;
        cl_intt_slice<LOGN>(s, x + ((int64_t)c * ext + md.nq + r) * N + off, pr, d_tw, mc, logn, len, tw_issued);
        for (int k = threadIdx.x; k < len; k += blockDim.x) {
            const uint64_t v = mul_shoup(s[SIDX(k)], mc[pr].ninv, mc[pr].ninv_shoup, pi);
            o[k] = mul_shoup(v, md.inv[r], md.inv_shoup[r], pi);
        }
        return;
    }
    // add_c[L] + x_L P^-1, INTT, N^-1
    const int pl = md.q_prime[L];
    const uint64_t ql = mc[pl].q;
    const ulonglong2 *itw = twiddles(d_tw, pl, 1, logn);
    if (!tw_issued) tw_prefetch<true, false>(s, itw, logn);
    const uint64_t *xl = x + ((int64_t)c * ext + L) * N + off;
    const uint64_t *ad = c == 0 ? add0 : add1;
    const uint64_t *al = ad ? ad + (int64_t)L * N + off : nullptr;
    for (int k = threadIdx.x; k < len; k += blockDim.x) {
        uint64_t v = mul_shoup(xl[k], md.pinv[L], md.pinv_shoup[L], ql);
        if (al) v = add_mod(v, al[k], ql);
        s[SIDX(k)] = v;
    }
    __syncthreads();
    ntt_inv_cluster<LOGN>(s, itw, ql, logn);
    for (int k = threadIdx.x; k < len; k += blockDim.x) o[k] = mul_shoup(s[SIDX(k)], mc[pl].ninv, mc[pl].ninv_shoup, ql);
}

template <int LOGN = 0>
__global__ void moddown_rescale_intt_kernel(const uint64_t *__restrict__ x, int ext, ModDownConst md, const uint64_t *__restrict__ add0,
                                            const uint64_t *__restrict__ add1, uint64_t *tmp, const uint64_t *__restrict__ d_tw,
                                            const ModConst *__restrict__ mc, int logn_rt) {
    HE_GRID_LAUNCH();
    const int logn = LOGN ? LOGN : logn_rt;
    int item, off, len;
    slice_of<true>(logn, item, off, len);
    const int r = item % (md.K + 1);  // the inverse transform's twiddle copy (a context table) before the wait
    tw_prefetch<true, false>(s_dyn(), twiddles(d_tw, r < md.K ? md.p_prime[r] : md.q_prime[md.nq - 1], 1, logn), logn);
    HE_GRID_WAIT();
    moddown_rescale_intt_body<LOGN>(x, ext, md, add0, add1, tmp, item, d_tw, mc, logn, off, len, true);
}

template <int LOGN = 0>
__device__ __forceinline__ void moddown_rescale_ntt_body(const uint64_t *__restrict__ x, int ext, const ModDownConst &md, const RescaleConst &rc,
                                                         const uint64_t *__restrict__ add0, const uint64_t *__restrict__ add1,
                                                         const uint64_t *__restrict__ tmp, uint64_t *out, int item, const uint64_t *__restrict__ d_tw,
                                                         const ModConst *__restrict__ mc, int logn, int off, int len, bool tw_issued = false) {
    extern __shared__ uint64_t s[];
    const int N = 1 << logn;
    const int L = md.nq - 1;
    const int c = item / L, j = item % L;
    const int pj = md.q_prime[j], pl = md.q_prime[L];
    const uint64_t q = mc[pj].q, ql = mc[pl].q;
    const ulonglong2 *tw = twiddles(d_tw, pj, 0, logn);
    if (!tw_issued) tw_prefetch<true, true>(s, tw, logn);
    const uint64_t *tc = tmp + (int64_t)c * (md.K + 1) * N + off;
    for (int k = threadIdx.x; k < len; k += blockDim.x) {
        // conv_j and conv_L of the scaled P limbs, in limb order
        uint64_t acc_j = 0, acc_l = 0;
        for (int i = 0; i < md.K; ++i) {
            const uint64_t v = tc[(int64_t)i * N + k];
            acc_j = add_mod(acc_j, mul_shoup(v, md.hat[i][j], md.hat_shoup[i][j], q), q);
            acc_l = add_mod(acc_l, mul_shoup(v, md.hat[i][L], md.hat_shoup[i][L], ql), ql);
        }
        // sum_L in coefficient form, centred, reduced mod q_j; w_j = conv_j P^-1 + [sum_L]_j
        const uint64_t sl = sub_mod(tc[(int64_t)md.K * N + k], mul_shoup(acc_l, md.pinv[L], md.pinv_shoup[L], ql), ql);
        uint64_t rr = sl + rc.half;
        if (rr >= rc.ql) rr -= rc.ql;
        const int64_t centred = (int64_t)rr - (int64_t)rc.half;
        s[SIDX(k)] = add_mod(mul_shoup(acc_j, md.pinv[j], md.pinv_shoup[j], q), reduce_signed(centred, q, mc[pj].mu), q);
    }
    __syncthreads();
    // the combination's other inputs of the first two iterations, loaded before the transform
    const uint64_t *xj = x + ((int64_t)c * ext + j) * N + off;
    const uint64_t *ad = c == 0 ? add0 : add1;
    const uint64_t *aj = ad ? ad + (int64_t)j * N + off : nullptr;
    uint64_t xv[2], av[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int k = threadIdx.x + r * blockDim.x;
        if (k < len) {
            xv[r] = xj[k];
            av[r] = aj ? aj[k] : 0;
        }
    }
    ntt_fwd_cluster<LOGN>(s, tw, q, logn);
    uint64_t *o = out + ((int64_t)c * L + j) * N + off;
    int r = 0;
    for (int k = threadIdx.x; k < len; k += blockDim.x, ++r) {
        uint64_t v = mul_shoup(r == 0 ? xv[0] : (r == 1 ? xv[1] : xj[k]), md.pinv[j], md.pinv_shoup[j], q);
        if (aj) v = add_mod(v, r == 0 ? av[0] : (r == 1 ? av[1] : aj[k]), q);
        o[k] = mul_shoup(sub_mod(v, s[SIDX(k)], q), rc.inv[j], rc.inv_shoup[j], q);
    }
}

template <int LOGN = 0>
__global__ void moddown_rescale_ntt_kernel(const uint64_t *__restrict__ x, int ext, ModDownConst md, RescaleConst rc,
                                           const uint64_t *__restrict__ add0, const uint64_t *__restrict__ add1, const uint64_t *__restrict__ tmp,
                                           uint64_t *out, const uint64_t *__restrict__ d_tw, const ModConst *__restrict__ mc, int logn_rt) {
    HE_GRID_LAUNCH();
    const int logn = LOGN ? LOGN : logn_rt;
    int item, off, len;
    slice_of<true>(logn, item, off, len);
    // the forward transform's twiddle copy (a context table) before the wait
    tw_prefetch<true, true>(s_dyn(), twiddles(d_tw, md.q_prime[item % (md.nq - 1)], 0, logn), logn);
    HE_GRID_WAIT();
    moddown_rescale_ntt_body<LOGN>(x, ext, md, rc, add0, add1, tmp, out, item, d_tw, mc, logn, off, len, true);
}

// ---- many rotations: O3 of different ciphertexts, each by its own step, one launch per stage ----
// (the same definition as launch_rotate: ModUp of c1, key-switch inner product after the
// automorphism, ModDown, plus the automorphism of c0; bit-identical to one he_rotate per job)
struct RotGeom {
    int32_t nl, ext, K, L, LK;
    uint64_t *coef, *D, *pcoef;  // per-job scratch: c1 in coefficient form, ModUp digits, converted P limbs
    int64_t coef_w, d_w, p_w;    // their strides
};

__global__ void rot_intt_c1_kernel(const RotTable jobs, RotGeom rg, const uint64_t *__restrict__ d_tw, const ModConst *__restrict__ mc,
                                   int logn) {
    HE_GRID_DEP();
    extern __shared__ uint64_t s[];
    const int N = 1 << logn;
    const int j = blockIdx.x / rg.nl, l = blockIdx.x % rg.nl;
    const uint64_t q = mc[l].q;
    const uint64_t *src = jobs.j[j].ct + ((int64_t)rg.nl + l) * N;
    stage_in(s, src, N, [](uint64_t v) { return v; });
    __syncthreads();
    ntt_inv_smem(s, twiddles(d_tw, l, 1, logn), q, logn);
    uint64_t *dst = rg.coef + j * rg.coef_w + (int64_t)l * N;
    for (int k = threadIdx.x; k < N; k += blockDim.x) dst[k] = mul_shoup(s[SIDX(k)], mc[l].ninv, mc[l].ninv_shoup, q);
}

__global__ void rot_modup_kernel(const RotTable jobs, RotGeom rg, ModUpConst mu, const uint64_t *__restrict__ d_tw,
                                 const ModConst *__restrict__ mc, int logn) {
    HE_GRID_DEP();
    extern __shared__ uint64_t s[];
    const int per = mu.ndig * mu.ext;
    const int j = blockIdx.x / per, rest = blockIdx.x % per;
    modup_body<false>(jobs.j[j].ct + (int64_t)rg.nl * (1 << logn), rg.coef + j * rg.coef_w, rg.D + j * rg.d_w, mu, rest / mu.ext, rest % mu.ext, s,
                      d_tw, mc, logn, 0, 1 << logn);
}

// ---- the same ModUp in two phases per transform (NTT form 2, he_ntt.cuh): the inverse NTT of
// every c1 limb as rows (from the job's ciphertext into coef) then columns scaled by N^-1, and
// every (j, d, u) target as columns on the conversion then rows; the digit's own limbs are
// copied from the NTT-form input by the column launch and skipped by the row launch.  The values
// of rot_intt_c1_kernel and rot_modup_kernel. ----
template <int LOGN, int NBA>
__global__ void __launch_bounds__(NTT2_THREADS) rot2_intt_rows_kernel(const RotTable jobs, RotGeom rg, const uint64_t *__restrict__ d_tw,
                                                                    const ModConst *__restrict__ mc) {
    HE_GRID_DEP();
    constexpr int N = 1 << LOGN, TILES = 64 / NTT2_TR;
    __shared__ uint64_t sm[ntt2_rows_smem_words(LOGN - 6)];
    const int item = blockIdx.x / TILES, b0 = (blockIdx.x % TILES) * NTT2_TR;
    const int j = item / rg.nl, l = item % rg.nl;
    ntt2_inv_rows<LOGN, NBA>(sm, jobs.j[j].ct + ((int64_t)rg.nl + l) * N, rg.coef + j * rg.coef_w + (int64_t)l * N, b0,
                             TwGlobal{twiddles(d_tw, l, 1, LOGN)}, mc[l].q);
}

template <int LOGN>
__global__ void __launch_bounds__(NTT2_THREADS, 8) rot2_intt_cols_kernel(RotGeom rg, const uint64_t *__restrict__ d_tw, const ModConst *__restrict__ mc) {
    HE_GRID_DEP();
    constexpr int N = 1 << LOGN, TILES = (N >> 6) / NTT2_TC;
    __shared__ uint64_t sm[ntt2_cols_smem_words()];
    const int item = blockIdx.x / TILES, c0 = (blockIdx.x % TILES) * NTT2_TC;
    const int j = item / rg.nl, l = item % rg.nl;
    const uint64_t q = mc[l].q, ni = mc[l].ninv, nis = mc[l].ninv_shoup;
    uint64_t *x = rg.coef + j * rg.coef_w + (int64_t)l * N;
    ntt2_inv_cols<LOGN>(sm, x, c0, TwGlobal{twiddles(d_tw, l, 1, LOGN)}, q, [=](int64_t k, uint64_t v) { x[k] = mul_shoup(v, ni, nis, q); });
}

template <int LOGN>
__global__ void __launch_bounds__(NTT2_THREADS, 8) rot2_modup_cols_kernel(const RotTable jobs, RotGeom rg, ModUpConst mu,
                                                                        const uint64_t *__restrict__ d_tw, const ModConst *__restrict__ mc) {
    HE_GRID_DEP();
    constexpr int N = 1 << LOGN, C = N >> 6, TILES = C / NTT2_TC;
    __shared__ uint64_t sm[ntt2_cols_smem_words()];
    const int item = blockIdx.x / TILES, c0 = (blockIdx.x % TILES) * NTT2_TC;
    const int per = mu.ndig * mu.ext, j = item / per, d = (item % per) / mu.ext, u = item % mu.ext;
    const int lo = d * mu.alpha, hi = lo + mu.alpha < mu.nq ? lo + mu.alpha : mu.nq;
    const int p = mu.ext_prime[u];
    const uint64_t t = mc[p].q;
    uint64_t *dst = rg.D + j * rg.d_w + ((int64_t)d * mu.ext + u) * N;
    if (u >= lo && u < hi) {  // the digit's own limb: its NTT form is the input's (uniform over the CTA)
        const uint64_t *src = jobs.j[j].ct + ((int64_t)rg.nl + u) * N;
        for (int e = threadIdx.x; e < 64 * NTT2_TC; e += NTT2_THREADS) {
            const int64_t x = (int64_t)(e / NTT2_TC) * C + c0 + e % NTT2_TC;
            dst[x] = src[x];
        }
        return;
    }
    const uint64_t *coef = rg.coef + j * rg.coef_w;
    // sum over the digit's primes of [x_i (Qd/q_i)^-1]_{q_i} (Qd/q_i mod t), as in modup_body
    ntt2_fwd_cols<LOGN>(
        sm,
        [&](int64_t x) {
            uint64_t a = 0;
            for (int i = 0; i < hi - lo; ++i) {
                const uint64_t qi = mc[lo + i].q;
                const uint64_t term = mul_shoup(mul_shoup(coef[(int64_t)(lo + i) * N + x], mu.inv[d][i], mu.inv_shoup[d][i], qi), mu.hat[d][i][u],
                                                mu.hat_shoup[d][i][u], t);
                a = i == 0 ? term : add_mod(a, term, t);
            }
            return a;
        },
        dst, c0, TwGlobal{twiddles(d_tw, p, 0, LOGN)}, t);
}

template <int LOGN>
__global__ void __launch_bounds__(NTT2_THREADS, 8) rot2_modup_rows_kernel(RotGeom rg, ModUpConst mu, const uint64_t *__restrict__ d_tw,
                                                                        const ModConst *__restrict__ mc) {
    HE_GRID_DEP();
    constexpr int N = 1 << LOGN, TILES = 64 / NTT2_TR;
    __shared__ uint64_t sm[ntt2_frows_smem_words(LOGN - 6)];
    const int item = blockIdx.x / TILES, b0 = (blockIdx.x % TILES) * NTT2_TR;
    const int per = mu.ndig * mu.ext, j = item / per, d = (item % per) / mu.ext, u = item % mu.ext;
    const int lo = d * mu.alpha, hi = lo + mu.alpha < mu.nq ? lo + mu.alpha : mu.nq;
    if (u >= lo && u < hi) return;  // copied, already in NTT form
    const int p = mu.ext_prime[u];
    ntt2_fwd_rows<LOGN>(sm, rg.D + j * rg.d_w + ((int64_t)d * mu.ext + u) * N, b0, TwGlobal{twiddles(d_tw, p, 0, LOGN)}, mc[p].q, mc[p].mu);
}

// ModUp of the jobs' c1 (NTT form) as clusters, item (j, d, u), the inverse NTT inside: for
// launches of few rotations (at most HE_ROT_CL_MAX_ITEMS items, 8 CTAs each), where one CTA per
// limb-poly would leave most SMs idle
#define HE_ROT_CL_MAX_ITEMS 128
template <int LOGN = 0>
__global__ void rot_modup_cl_kernel(const RotTable jobs, RotGeom rg, ModUpConst mu, const uint64_t *__restrict__ d_tw,
                                    const ModConst *__restrict__ mc, int logn_rt) {
    HE_GRID_DEP();
    const int logn = LOGN ? LOGN : logn_rt;
    int item, off, len;
    slice_of<true>(logn, item, off, len);
    const int per = mu.ndig * mu.ext;
    const int j = item / per;
    modup_cl_fused_body<LOGN>(jobs.j[j].ct + (int64_t)rg.nl * (1 << logn), rg.D + j * rg.d_w, mu, item % per, d_tw, mc, logn, off, len);
}

// ---- batch forms: the same bodies over a job table (one job = one MatMult, R = C = 1) ----
// iNTT of limbs [first, first + count) of component `comp` of the job's buffer `which`
// (0: input ciphertext, 1: accumulator acc, 2: pre-rescale sum) into scratch.
__global__ void batch_intt_c1_kernel(const MMJob *__restrict__ jobs, BatchGeom bg, const uint64_t *__restrict__ d_tw,
                                     const ModConst *__restrict__ mc, int logn) {
    HE_GRID_DEP();
    extern __shared__ uint64_t s[];
    const int N = 1 << logn;
    const int j = blockIdx.x / bg.nq, l = blockIdx.x % bg.nq;
    if (jobs[j].m_prime <= 1) return;
    const uint64_t q = mc[l].q;
    const uint64_t *src = jobs[j].ct + ((int64_t)bg.nq + l) * N;
    stage_in(s, src, N, [](uint64_t v) { return v; });
    __syncthreads();
    ntt_inv_smem(s, twiddles(d_tw, l, 1, logn), q, logn);
    uint64_t *dst = bg.coef + (int64_t)j * bg.coef_words + (int64_t)l * N;
    for (int k = threadIdx.x; k < N; k += blockDim.x) dst[k] = mul_shoup(s[SIDX(k)], mc[l].ninv, mc[l].ninv_shoup, q);
}

__global__ void batch_modup_kernel(const MMJob *__restrict__ jobs, BatchGeom bg, ModUpConst mu, const uint64_t *__restrict__ d_tw,
                                   const ModConst *__restrict__ mc, int logn) {
    HE_GRID_DEP();
    extern __shared__ uint64_t s[];
    const int per = mu.ndig * mu.ext;
    const int j = blockIdx.x / per, rest = blockIdx.x % per;
    if (jobs[j].m_prime <= 1) return;
    modup_body<false>(jobs[j].ct + (int64_t)bg.nq * (1 << logn), bg.coef + (int64_t)j * bg.coef_words, bg.D + (int64_t)j * bg.d_words, mu,
                      rest / mu.ext, rest % mu.ext, s, d_tw, mc, logn, 0, 1 << logn);
}

// iNTT of the P limbs of both accumulator components: block (j, c, i) -> tmp_j [c][K][N]
__global__ void batch_intt_p_kernel(const MMJob *__restrict__ jobs, BatchGeom bg, const uint64_t *__restrict__ d_tw,
                                    const ModConst *__restrict__ mc, int logn) {
    HE_GRID_DEP();
    extern __shared__ uint64_t s[];
    const int N = 1 << logn;
    const int per = 2 * bg.K;
    const int j = blockIdx.x / per, c = (blockIdx.x % per) / bg.K, i = blockIdx.x % bg.K;
    if (jobs[j].m_prime == 0) return;  // empty slot
    const int p = bg.L + i;
    const uint64_t q = mc[p].q;
    const uint64_t *src = bg.acc + (int64_t)j * bg.acc_words + ((int64_t)c * bg.ext + bg.nq + i) * N;
    stage_in(s, src, N, [](uint64_t v) { return v; });
    __syncthreads();
    ntt_inv_smem(s, twiddles(d_tw, p, 1, logn), q, logn);
    uint64_t *dst = bg.tmp + (int64_t)j * bg.tmp_words + ((int64_t)c * bg.K + i) * N;
    for (int k = threadIdx.x; k < N; k += blockDim.x) dst[k] = mul_shoup(s[SIDX(k)], mc[p].ninv, mc[p].ninv_shoup, q);
}

__global__ void batch_moddown_kernel(const MMJob *__restrict__ jobs, BatchGeom bg, ModDownConst md, const uint64_t *__restrict__ d_tw,
                                     const ModConst *__restrict__ mc, int logn) {
    HE_GRID_DEP();
    extern __shared__ uint64_t s[];
    const int per = 2 * md.nq;
    const int j = blockIdx.x / per, c = (blockIdx.x % per) / md.nq, l = blockIdx.x % md.nq;
    if (jobs[j].m_prime == 0) return;  // empty slot
    const uint64_t *cacc = bg.cacc + (int64_t)j * bg.cacc_words;
    moddown_body<false>(bg.acc + (int64_t)j * bg.acc_words, bg.ext, bg.tmp + (int64_t)j * bg.tmp_words, md,
                        cacc + (int64_t)c * md.nq * (1 << logn), bg.sum + (int64_t)j * bg.sum_words, c, l, s, d_tw, mc, logn, 0, 1 << logn);
}

// iNTT of the last limb of both sum components -> tmp_j + 2K N
__global__ void batch_intt_last_kernel(const MMJob *__restrict__ jobs, BatchGeom bg, const uint64_t *__restrict__ d_tw,
                                       const ModConst *__restrict__ mc, int logn) {
    HE_GRID_DEP();
    extern __shared__ uint64_t s[];
    const int N = 1 << logn;
    const int j = blockIdx.x / 2, c = blockIdx.x % 2;
    if (jobs[j].m_prime == 0) return;  // empty slot
    const int p = bg.level;
    const uint64_t q = mc[p].q;
    const uint64_t *src = bg.sum + (int64_t)j * bg.sum_words + ((int64_t)c * bg.nq + bg.level) * N;
    stage_in(s, src, N, [](uint64_t v) { return v; });
    __syncthreads();
    ntt_inv_smem(s, twiddles(d_tw, p, 1, logn), q, logn);
    uint64_t *dst = bg.tmp + (int64_t)j * bg.tmp_words + ((int64_t)2 * bg.K + c) * N;
    for (int k = threadIdx.x; k < N; k += blockDim.x) dst[k] = mul_shoup(s[SIDX(k)], mc[p].ninv, mc[p].ninv_shoup, q);
}

__global__ void batch_rescale_kernel(const MMJob *__restrict__ jobs, BatchGeom bg, RescaleConst rc, const uint64_t *__restrict__ d_tw,
                                     const ModConst *__restrict__ mc, int logn) {
    HE_GRID_DEP();
    extern __shared__ uint64_t s[];
    const int per = 2 * bg.level;
    const int j = blockIdx.x / per, c = (blockIdx.x % per) / bg.level, l = blockIdx.x % bg.level;
    if (jobs[j].m_prime == 0) return;  // empty slot
    rescale_body<false>(bg.sum + (int64_t)j * bg.sum_words, bg.level, bg.tmp + (int64_t)j * bg.tmp_words + (int64_t)2 * bg.K * (1 << logn),
                        rc, jobs[j].out, c, l, s, d_tw, mc, logn, 0, 1 << logn);
}

// ---- batch stages as clusters (stage form 1): for batches with few jobs (a serving lane's),
// where one CTA per limb-poly leaves most SMs idle and each stage waits a whole one-CTA
// transform.  ModUp of every job in one launch (inverse NTT inside), then ModDown and rescale in
// two launches, each item one 8-CTA cluster; empty slots (m' = 0, or m' = 1 for ModUp) return at
// once, uniformly over their cluster.  The same bodies as the single MatMult's cluster kernels,
// so the results are bit-identical to the one-CTA stages.
template <int LOGN = 0>
__global__ void batch_modup_cl_kernel(const MMJob *__restrict__ jobs, BatchGeom bg, ModUpConst mu, const uint64_t *__restrict__ d_tw,
                                      const ModConst *__restrict__ mc, int logn_rt) {
    HE_GRID_DEP();
    const int logn = LOGN ? LOGN : logn_rt;
    int item, off, len;
    slice_of<true>(logn, item, off, len);
    const int per = mu.ndig * mu.ext, j = item / per;
    if (jobs[j].m_prime <= 1) return;
    modup_cl_fused_body<LOGN>(jobs[j].ct + (int64_t)bg.nq * (1 << logn), bg.D + (int64_t)j * bg.d_words, mu, item % per, d_tw, mc, logn, off, len);
}

template <int LOGN = 0>
__global__ void batch_mdr_intt_cl_kernel(const MMJob *__restrict__ jobs, BatchGeom bg, ModDownConst md, const uint64_t *__restrict__ d_tw,
                                         const ModConst *__restrict__ mc, int logn_rt) {
    HE_GRID_DEP();
    const int logn = LOGN ? LOGN : logn_rt;
    int item, off, len;
    slice_of<true>(logn, item, off, len);
    const int per = 2 * (md.K + 1), j = item / per;
    if (jobs[j].m_prime == 0) return;
    const uint64_t *cacc = bg.cacc + (int64_t)j * bg.cacc_words;
    moddown_rescale_intt_body<LOGN>(bg.acc + (int64_t)j * bg.acc_words, bg.ext, md, cacc, cacc + (int64_t)bg.nq * (1 << logn),
                                    bg.tmp + (int64_t)j * bg.tmp_words, item % per, d_tw, mc, logn, off, len);
}

template <int LOGN = 0>
__global__ void batch_mdr_ntt_cl_kernel(const MMJob *__restrict__ jobs, BatchGeom bg, ModDownConst md, RescaleConst rc, const uint64_t *__restrict__ d_tw,
                                        const ModConst *__restrict__ mc, int logn_rt) {
    HE_GRID_DEP();
    const int logn = LOGN ? LOGN : logn_rt;
    int item, off, len;
    slice_of<true>(logn, item, off, len);
    const int per = 2 * bg.level, j = item / per;
    if (jobs[j].m_prime == 0) return;
    const uint64_t *cacc = bg.cacc + (int64_t)j * bg.cacc_words;
    moddown_rescale_ntt_body<LOGN>(bg.acc + (int64_t)j * bg.acc_words, bg.ext, md, rc, cacc, cacc + (int64_t)bg.nq * (1 << logn),
                                   bg.tmp + (int64_t)j * bg.tmp_words, jobs[j].out, item % per, d_tw, mc, logn, off, len);
}

// The double-hoisted MatMult loop.  For every coefficient k of extended limb u:
//   acc_c[u][k]  = sum_{i>=1} ptM_i[u][k] * redc(sum_d D[d][u][src_i(k)] keyM_i[d][c][kl(u)][k])
//   cacc_0[u][k] = ptM_0 * c0[u][k] + sum_{i>=1} ptM_i[u][k] * c0[u][src_i(k)]   (u in Q_level)
//   cacc_1[u][k] = ptM_0 * c1[u][k]
// Variants (chosen per encoded matrix or batch by timing them, see mm_variant): a block of
// MM_THREADS threads covers LANES = MM_THREADS / G lanes of VEC consecutive coefficients of one
// limb and splits the rotations i = 1..m'-1 into G interleaved groups; the group sums meet in
// shared memory.  With VEC = 2 a lane's pair (k, k+1), k even, gathers the aligned pair
// (src, src ^ 1) of each digit, so every load is 16 bytes; VEC = 1 halves the registers and
// doubles the warps.  Each lane loads the next rotation step's operands while it computes the
// current one.  Products are accumulated in 128 bits and reduced once per lazy_terms(q) terms
// (8 for q < 2^61: 8 q^2 < q 2^64; 2^24 for the 40-bit primes).
#define MM_THREADS 256

__device__ __forceinline__ uint64_t fold(u128 t, uint64_t q, uint64_t qinv) { return redc128(t, q, qinv); }
// t 2^-64 mod q for any t < 2^128: the high word is reduced mod q first (Barrett), so the
// Montgomery step's input is below q 2^64
__device__ __forceinline__ uint64_t fold_wide(u128 t, uint64_t q, uint64_t qinv, uint64_t mu) {
    return redc(reduce_barrett((uint64_t)(t >> 64), q, mu), (uint64_t)t, q, qinv);
}

template <int VEC>
__device__ __forceinline__ void ldv(const uint64_t *p, uint64_t (&o)[VEC]) {
    if constexpr (VEC == 2) {
        const ulonglong2 t = __ldg(reinterpret_cast<const ulonglong2 *>(p));
        o[0] = t.x;
        o[1] = t.y;
    } else {
        o[0] = __ldg(p);
    }
}
// gather of VEC values at the automorphism image of k..k+VEC-1 (src of k given)
template <int VEC>
__device__ __forceinline__ void gatherv(const uint64_t *base, uint32_t src, uint64_t (&o)[VEC]) {
    if constexpr (VEC == 2) {
        const ulonglong2 t = *reinterpret_cast<const ulonglong2 *>(base + (src & ~1u));
        o[0] = (src & 1) ? t.y : t.x;
        o[1] = (src & 1) ? t.x : t.y;
    } else {
        o[0] = base[src];
    }
}
template <int VEC>
__device__ __forceinline__ void stv(uint64_t *p, const uint64_t (&v)[VEC]) {
    if constexpr (VEC == 2) {
        *reinterpret_cast<ulonglong2 *>(p) = make_ulonglong2(v[0], v[1]);
    } else {
        p[0] = v[0];
    }
}

// Asynchronous global -> shared copies of a thread's own operands.  Only the issuing thread
// reads the destination (after cp_async_wait), so no block barrier is involved; the "memory"
// clobbers keep the compiler from moving shared-memory reads across the issue or the wait.
template <int BYTES>
__device__ __forceinline__ void cp_async(uint64_t *smem, const uint64_t *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory");
}

// One block: `lanes` (<= MM_THREADS / G) lanes of VEC consecutive coefficients each, thread t
// serving lane t % lanes in rotation group t / lanes; the calling thread's lane starts at
// coefficient k of extended limb u (k >= N: no lane).  Every thread of the block calls it (it
// synchronises once).  red: 3*VEC*MM_THREADS words.  With S > 0 stages (fixed digit count only) each thread streams its key and plaintext
// operands through S private stages of pipe, so S rotation steps of HBM loads are in flight
// without occupying registers.  With GA the digit and c0 gathers (L2 hits) go through the same
// stages; without, they keep the one-step register prefetch.  keys / galois may point to shared
// memory (the kernels stage the tables there), so no global round trip precedes a step's loads.
//
// With FK (fused keys, staged forms with a fixed digit count only) the key operands of step i are
// the encoded matrix's fused tables F_i[d][c][u][k] = keyM_i[d][c][kl(u)][k] ptM_i[u][k] 2^-64
// (fuse_keys_kernel) in place of the Galois key, so that
//   acc_c[u][k] = redc(sum_i sum_d D[d][u][src_i(k)] F_i[d][c][u][k]),
// the same residue as the two-level form: no per-step reduction and no second product.  The
// 128-bit sums then take up to 2^(128 - 2 bits(q)) products (64 for q < 2^61); their high word is
// reduced mod q before the Montgomery step, whose input must stay below q 2^64.
template <int NDIG, int VEC, int G, int S, bool GA, bool FK = false>
__device__ __forceinline__ void mm_tile(const uint64_t *__restrict__ ct, const uint64_t *__restrict__ D, const uint64_t *__restrict__ pts,
                                        const uint64_t *const *keys, const uint32_t *galois, int m_prime,
                                        int ndig_rt, int ext, int nq, int L, int LK, int u, int k, int lanes, uint64_t *acc,
                                        uint64_t *cacc, int accumulate, const ModConst *__restrict__ mc, int logn, uint64_t *red,
                                        uint64_t *pipe, const uint64_t *__restrict__ fused = nullptr) {
    static_assert(!FK || (NDIG > 0 && S > 0), "fused key tables: staged forms with a fixed digit count");
    const int N = 1 << logn;
    const int ndig = NDIG > 0 ? NDIG : ndig_rt;
    const int kl = u < nq ? u : L + (u - nq), p = kl;
    const uint64_t q = mc[p].q, qinv = mc[p].qinv;
    const bool inq = u < nq;
    const int lane = threadIdx.x % lanes, grp = threadIdx.x / lanes;
    auto R = [&](int g, int which, int j) -> uint64_t & { return red[((g * 3 + which) * VEC + j) * lanes + lane]; };

    uint64_t r0[VEC], r1[VEC], rc[VEC];
#pragma unroll
    for (int j = 0; j < VEC; ++j) r0[j] = r1[j] = rc[j] = 0;
    if (k < N) {
        u128 t0[VEC], t1[VEC], tc[VEC];
#pragma unroll
        for (int j = 0; j < VEC; ++j) t0[j] = t1[j] = tc[j] = 0;
        int pending = 0;
        constexpr int ND = NDIG > 0 ? NDIG : 8;
        // steps per reduction of the 128-bit sums: each step adds one product of two residues
        // (lazy_terms); with FK, ND products of two residues, and the sums are reduced with
        // fold_wide, which only needs them below 2^128: 2^(128 - 2 bits(q)) / ND steps
        const int period = lazy_terms(q);
        const int qb = 64 - __clzll((long long)q);
        const int fk_period = FK ? ((128 - 2 * qb < 24 ? 1 << (128 - 2 * qb) : 1 << 24) / ND) : 0;
        constexpr int SP = NDIG > 0 ? S : 0;
        if constexpr (SP > 0) {
            // slot (stage, field f, thread) at pipe[((stage F + f) MM_THREADS + tid) VEC]: fields
            // 2d, 2d+1 key digit d; 2 ND the plaintext; with GA, 2 ND + 1 + d digit d's gather
            // and 3 ND + 1 the c0 gather (aligned pairs when VEC = 2)
            constexpr int F = 2 * ND + 1 + (GA ? ND + 1 : 0);
            auto slot = [&](int st, int f) { return pipe + ((st * F + f) * MM_THREADS + (int)threadIdx.x) * VEC; };
            // GA with VEC = 2: bit st is the parity of the gather source staged in stage st (set when
            // the gathers are issued, read when they are consumed), so the source index is computed
            // once per step
            uint32_t odd_bits = 0;
            auto issue = [&](int t) {
                const int i = 1 + grp + t * G;
                if (i < m_prime) {
                    const int st = t % SP;
                    if constexpr (FK) {
                        const uint64_t *f = fused + ((int64_t)(i - 1) * 2 * ND * ext + u) * N + k;
#pragma unroll
                        for (int d = 0; d < 2 * ND; ++d) cp_async<8 * VEC>(slot(st, d), f + (int64_t)d * ext * N);
                        if (inq) cp_async<8 * VEC>(slot(st, 2 * ND), pts + ((int64_t)i * ext + u) * N + k);
                    } else {
                        const uint64_t *key = keys[i - 1];
#pragma unroll
                        for (int d = 0; d < ND; ++d) {
                            cp_async<8 * VEC>(slot(st, 2 * d), key + ((int64_t)(d * 2 + 0) * LK + kl) * N + k);
                            cp_async<8 * VEC>(slot(st, 2 * d + 1), key + ((int64_t)(d * 2 + 1) * LK + kl) * N + k);
                        }
                        cp_async<8 * VEC>(slot(st, 2 * ND), pts + ((int64_t)i * ext + u) * N + k);
                    }
                    if constexpr (GA) {
                        const uint32_t src = automorph_src(k, galois[i - 1], logn);
                        const uint32_t sa = VEC == 2 ? (src & ~1u) : src;
                        if constexpr (VEC == 2) odd_bits = (odd_bits & ~(1u << st)) | ((src & 1u) << st);
#pragma unroll
                        for (int d = 0; d < ND; ++d) cp_async<8 * VEC>(slot(st, 2 * ND + 1 + d), D + ((int64_t)d * ext + u) * N + sa);
                        if (inq) cp_async<8 * VEC>(slot(st, 3 * ND + 1), ct + (int64_t)u * N + sa);
                    }
                }
                cp_async_commit();
            };
            uint64_t dv[ND][VEC], cv[VEC];
            // gathered operands of step t: from the stage (GA) or straight from global memory
            auto gather = [&](int t) {
                const int i = 1 + grp + t * G;
                if (i >= m_prime) return;
                if constexpr (GA) {
                    const int st = t % SP;
                    // the staged aligned pair holds (src, src ^ 1) in ascending order: coefficient j
                    // reads word j ^ odd, as two 8-byte shared-memory loads at offsets odd, 1 - odd
                    const int odd = VEC == 2 ? (int)((odd_bits >> st) & 1u) : 0;
#pragma unroll
                    for (int d = 0; d < ND; ++d) {
                        const uint64_t *g = slot(st, 2 * ND + 1 + d);
#pragma unroll
                        for (int j = 0; j < VEC; ++j) dv[d][j] = g[j ^ odd];
                    }
                    if (inq) {
                        const uint64_t *g = slot(st, 3 * ND + 1);
#pragma unroll
                        for (int j = 0; j < VEC; ++j) cv[j] = g[j ^ odd];
                    }
                } else {
                    const uint32_t src = automorph_src(k, galois[i - 1], logn);
#pragma unroll
                    for (int d = 0; d < ND; ++d) gatherv<VEC>(D + ((int64_t)d * ext + u) * N, src, dv[d]);
                    if (inq) gatherv<VEC>(ct + (int64_t)u * N, src, cv);
                }
            };
#pragma unroll
            for (int t = 0; t < SP; ++t) issue(t);
            if constexpr (!GA) gather(0);
            for (int t = 0; 1 + grp + t * G < m_prime; ++t) {
                cp_async_wait<SP - 1>();
                const int st = t % SP;
                if constexpr (GA) gather(t);
                if constexpr (FK) {
                    // t0, t1: sum over steps and digits of D F; tc: sum of c0 ptM
#pragma unroll
                    for (int d = 0; d < ND; ++d) {
                        const uint64_t *a = slot(st, 2 * d), *b = slot(st, 2 * d + 1);
#pragma unroll
                        for (int j = 0; j < VEC; ++j) {
                            t0[j] += (u128)dv[d][j] * a[j];
                            t1[j] += (u128)dv[d][j] * b[j];
                        }
                    }
                    uint64_t pmc[VEC], c0v[VEC];
                    if (inq) {
                        const uint64_t *pp = slot(st, 2 * ND);
#pragma unroll
                        for (int j = 0; j < VEC; ++j) {
                            pmc[j] = pp[j];
                            c0v[j] = cv[j];
                        }
                    }
                    issue(t + SP);
                    if constexpr (!GA) gather(t + 1);
                    if (inq) {
#pragma unroll
                        for (int j = 0; j < VEC; ++j) tc[j] += (u128)c0v[j] * pmc[j];
                    }
                    if (++pending == fk_period) {
                        const uint64_t mu = mc[p].mu;
#pragma unroll
                        for (int j = 0; j < VEC; ++j) {
                            r0[j] = add_mod(r0[j], fold_wide(t0[j], q, qinv, mu), q);
                            r1[j] = add_mod(r1[j], fold_wide(t1[j], q, qinv, mu), q);
                            rc[j] = add_mod(rc[j], fold_wide(tc[j], q, qinv, mu), q);
                            t0[j] = t1[j] = tc[j] = 0;
                        }
                        pending = 0;
                    }
                    continue;
                }
                u128 s0[VEC], s1[VEC];
#pragma unroll
                for (int j = 0; j < VEC; ++j) s0[j] = s1[j] = 0;
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    const uint64_t *a = slot(st, 2 * d), *b = slot(st, 2 * d + 1);
#pragma unroll
                    for (int j = 0; j < VEC; ++j) {
                        s0[j] += (u128)dv[d][j] * a[j];
                        s1[j] += (u128)dv[d][j] * b[j];
                    }
                }
                uint64_t pmc[VEC], c0v[VEC];
                const uint64_t *pp = slot(st, 2 * ND);
#pragma unroll
                for (int j = 0; j < VEC; ++j) {
                    pmc[j] = pp[j];
                    c0v[j] = cv[j];
                }
                issue(t + SP);
                if constexpr (!GA) gather(t + 1);
#pragma unroll
                for (int j = 0; j < VEC; ++j) {
                    t0[j] += (u128)fold(s0[j], q, qinv) * pmc[j];
                    t1[j] += (u128)fold(s1[j], q, qinv) * pmc[j];
                    if (inq) tc[j] += (u128)c0v[j] * pmc[j];
                }
                if (++pending == period) {
#pragma unroll
                    for (int j = 0; j < VEC; ++j) {
                        r0[j] = add_mod(r0[j], fold(t0[j], q, qinv), q);
                        r1[j] = add_mod(r1[j], fold(t1[j], q, qinv), q);
                        rc[j] = add_mod(rc[j], fold(tc[j], q, qinv), q);
                        t0[j] = t1[j] = tc[j] = 0;
                    }
                    pending = 0;
                }
            }
            cp_async_wait<0>();
            if constexpr (FK) {
                const uint64_t mu = mc[p].mu;
#pragma unroll
                for (int j = 0; j < VEC; ++j) {
                    r0[j] = add_mod(r0[j], fold_wide(t0[j], q, qinv, mu), q);
                    r1[j] = add_mod(r1[j], fold_wide(t1[j], q, qinv, mu), q);
                    rc[j] = add_mod(rc[j], fold_wide(tc[j], q, qinv, mu), q);
                    t0[j] = t1[j] = tc[j] = 0;
                }
            }
        } else {
            uint64_t dv[ND][VEC], kv0[ND][VEC], kv1[ND][VEC], pm[VEC], cv[VEC];
            auto fetch = [&](int i) {
                const uint32_t src = automorph_src(k, galois[i - 1], logn);
                const uint64_t *key = keys[i - 1];
    #pragma unroll
                for (int d = 0; d < ND; ++d) {
                    if (NDIG == 0 && d >= ndig) break;
                    gatherv<VEC>(D + ((int64_t)d * ext + u) * N, src, dv[d]);
                    ldv<VEC>(key + ((int64_t)(d * 2 + 0) * LK + kl) * N + k, kv0[d]);
                    ldv<VEC>(key + ((int64_t)(d * 2 + 1) * LK + kl) * N + k, kv1[d]);
                }
                ldv<VEC>(pts + ((int64_t)i * ext + u) * N + k, pm);
                if (inq) gatherv<VEC>(ct + (int64_t)u * N, src, cv);
            };
            int i = 1 + grp;
            if (i < m_prime) fetch(i);
            while (i < m_prime) {
                u128 s0[VEC], s1[VEC];
    #pragma unroll
                for (int j = 0; j < VEC; ++j) s0[j] = s1[j] = 0;
    #pragma unroll
                for (int d = 0; d < ND; ++d) {
                    if (NDIG == 0 && d >= ndig) break;
    #pragma unroll
                    for (int j = 0; j < VEC; ++j) {
                        s0[j] += (u128)dv[d][j] * kv0[d][j];
                        s1[j] += (u128)dv[d][j] * kv1[d][j];
                    }
                }
                uint64_t pmc[VEC], c0v[VEC];
    #pragma unroll
                for (int j = 0; j < VEC; ++j) {
                    pmc[j] = pm[j];
                    c0v[j] = cv[j];
                }
                const int next = i + G;
                if (next < m_prime) fetch(next);
    #pragma unroll
                for (int j = 0; j < VEC; ++j) {
                    t0[j] += (u128)fold(s0[j], q, qinv) * pmc[j];
                    t1[j] += (u128)fold(s1[j], q, qinv) * pmc[j];
                    if (inq) tc[j] += (u128)c0v[j] * pmc[j];
                }
                if (++pending == period) {
    #pragma unroll
                    for (int j = 0; j < VEC; ++j) {
                        r0[j] = add_mod(r0[j], fold(t0[j], q, qinv), q);
                        r1[j] = add_mod(r1[j], fold(t1[j], q, qinv), q);
                        rc[j] = add_mod(rc[j], fold(tc[j], q, qinv), q);
                        t0[j] = t1[j] = tc[j] = 0;
                    }
                    pending = 0;
                }
                i = next;
            }
        }
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
            r0[j] = add_mod(r0[j], fold(t0[j], q, qinv), q);
            r1[j] = add_mod(r1[j], fold(t1[j], q, qinv), q);
            rc[j] = add_mod(rc[j], fold(tc[j], q, qinv), q);
        }
    }
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
        R(grp, 0, j) = r0[j];
        R(grp, 1, j) = r1[j];
        R(grp, 2, j) = rc[j];
    }
    __syncthreads();
    if (grp == 0 && k < N) {
        uint64_t a0[VEC], a1[VEC], cc0[VEC], cc1[VEC];
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
            a0[j] = R(0, 0, j);
            a1[j] = R(0, 1, j);
            cc0[j] = R(0, 2, j);
            cc1[j] = 0;
            for (int g = 1; g < G; ++g) {
                a0[j] = add_mod(a0[j], R(g, 0, j), q);
                a1[j] = add_mod(a1[j], R(g, 1, j), q);
                cc0[j] = add_mod(cc0[j], R(g, 2, j), q);
            }
        }
        if (inq) {  // i = 0: no rotation
            uint64_t p0[VEC], c0[VEC], c1[VEC];
            ldv<VEC>(pts + (int64_t)u * N + k, p0);
            ldv<VEC>(ct + (int64_t)u * N + k, c0);
            ldv<VEC>(ct + ((int64_t)nq + u) * N + k, c1);
#pragma unroll
            for (int j = 0; j < VEC; ++j) {
                cc0[j] = add_mod(cc0[j], mont_mul(c0[j], p0[j], q, qinv), q);
                cc1[j] = mont_mul(c1[j], p0[j], q, qinv);
            }
        }
        uint64_t *A0 = acc + (int64_t)u * N + k, *A1 = acc + ((int64_t)ext + u) * N + k;
        if (accumulate) {
#pragma unroll
            for (int j = 0; j < VEC; ++j) {
                a0[j] = add_mod(A0[j], a0[j], q);
                a1[j] = add_mod(A1[j], a1[j], q);
            }
        }
        stv<VEC>(A0, a0);
        stv<VEC>(A1, a1);
        if (inq) {
            uint64_t *C0 = cacc + (int64_t)u * N + k, *C1 = cacc + ((int64_t)nq + u) * N + k;
            if (accumulate) {
#pragma unroll
                for (int j = 0; j < VEC; ++j) {
                    cc0[j] = add_mod(C0[j], cc0[j], q);
                    cc1[j] = add_mod(C1[j], cc1[j], q);
                }
            }
            stv<VEC>(C0, cc0);
            stv<VEC>(C1, cc1);
        }
    }
}

// dynamic shared memory of the pipelined form
constexpr size_t mm_pipe_bytes(int ndig, int vec, int stages, bool ga) {
    return ndig > 0 && stages > 0 ? (size_t)stages * (2 * ndig + 1 + (ga ? ndig + 1 : 0)) * MM_THREADS * vec * sizeof(uint64_t) : 0;
}

// Key-pointer and Galois-element tables of up to MM_TABLE rotations are copied to shared memory
// (one round trip per CTA) so that a step's loads do not wait on a table load; longer tables
// are read from global memory.
#define MM_TABLE 512
struct MMTables {
    const uint64_t *keys[MM_TABLE];
    uint32_t gal[MM_TABLE];
};
__device__ __forceinline__ void stage_tables(MMTables &tb, const uint64_t *const *keys, const uint32_t *galois, int m_prime,
                                             const uint64_t *const *&k_use, const uint32_t *&g_use) {
    if (m_prime - 1 <= MM_TABLE) {  // uniform over the block
        for (int i = threadIdx.x; i < m_prime - 1; i += blockDim.x) {
            tb.keys[i] = keys[i];
            tb.gal[i] = galois[i];
        }
        __syncthreads();
        k_use = tb.keys;
        g_use = tb.gal;
    } else {
        k_use = keys;
        g_use = galois;
    }
}

// single MatMult: the ext * N / VEC lanes of the extended limbs, in limb-major order, are cut
// into runs of blockDim.x / G lanes, one per block, whose size the launcher picks so that the
// blocks spread evenly over the multiprocessors (a run may cross a limb boundary); with FK,
// fused = the plaintext block's fused key tables [m'-1][NDIG][2][ext][N]
template <int NDIG, int VEC, int G, int S, bool GA, bool FK = false>
__global__ void __launch_bounds__(MM_THREADS, VEC == 2 ? 2 : 3) matmult_loop_kernel(
    const uint64_t *__restrict__ ct, const uint64_t *__restrict__ D, const uint64_t *__restrict__ pts,
    const uint64_t *const *__restrict__ keys, const uint32_t *__restrict__ galois, int m_prime, int ndig_rt, int ext, int nq, int L,
    int LK, uint64_t *acc, uint64_t *cacc, int accumulate, const ModConst *__restrict__ mc, int logn, const uint64_t *__restrict__ fused) {
    HE_GRID_DEP();
    __shared__ uint64_t red[G * 3 * VEC * (MM_THREADS / G)];
    __shared__ MMTables tb;
    extern __shared__ uint4 mm_pipe[];
    const uint64_t *const *k_use;
    const uint32_t *g_use;
    stage_tables(tb, keys, galois, m_prime, k_use, g_use);
    const int lanes = (int)blockDim.x / G, per_limb = (1 << logn) / VEC;
    const int flat = (int)blockIdx.x * lanes + (int)threadIdx.x % lanes;
    int u = flat / per_limb, k = (flat % per_limb) * VEC;
    if (u >= ext) {  // past the last limb: no lane
        u = 0;
        k = 1 << logn;
    }
    mm_tile<NDIG, VEC, G, S, GA, FK>(ct, D, pts, k_use, g_use, m_prime, ndig_rt, ext, nq, L, LK, u, k, lanes, acc, cacc, accumulate, mc, logn,
                                     red, reinterpret_cast<uint64_t *>(mm_pipe), fused);
}

// Fused key tables of an encoded matrix (see mm_tile): one thread per (plaintext block, step
// i >= 1, extended limb u, coefficient pair),
//   F[b][i-1][d][c][u][k] = keyM_i[d][c][kl(u)][k] ptM_{b,i}[u][k] 2^-64 mod q_u,
// i.e. the Montgomery form of key_i pt_{b,i}.
__global__ void __launch_bounds__(256) fuse_keys_kernel(const uint64_t *__restrict__ pts, const uint64_t *const *__restrict__ keys,
                                                       uint64_t *__restrict__ fused, int64_t total, int m_prime, int ndig, int ext, int nq,
                                                       int L, int LK, const ModConst *__restrict__ mc, int logn) {
    HE_GRID_DEP();
    const int64_t N = (int64_t)1 << logn, half = N / 2;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = 2 * (idx % half);
        int64_t rest = idx / half;
        const int u = (int)(rest % ext);
        rest /= ext;
        const int i = (int)(rest % (m_prime - 1)) + 1;
        const int64_t b = rest / (m_prime - 1);
        const int kl = u < nq ? u : L + (u - nq);
        const uint64_t q = mc[kl].q, qinv = mc[kl].qinv;
        const ulonglong2 pt = __ldg(reinterpret_cast<const ulonglong2 *>(pts + ((b * m_prime + i) * ext + u) * N + k));
        const uint64_t *key = keys[i - 1] + (int64_t)kl * N + k;
        uint64_t *f = fused + ((b * (m_prime - 1) + (i - 1)) * 2 * ndig * ext + u) * N + k;
        for (int dc = 0; dc < 2 * ndig; ++dc) {
            const ulonglong2 kv = __ldg(reinterpret_cast<const ulonglong2 *>(key + (int64_t)dc * LK * N));
            *reinterpret_cast<ulonglong2 *>(f + (int64_t)dc * ext * N) = make_ulonglong2(mont_mul(kv.x, pt.x, q, qinv), mont_mul(kv.y, pt.y, q, qinv));
        }
    }
}

// batch: persistent CTAs pull (tile, limb, job) items from an ordered queue
template <int NDIG, int VEC, int G, int S, bool GA>
__global__ void __launch_bounds__(MM_THREADS, VEC == 2 ? 2 : 3) matmult_batch_loop_kernel(
    const MMJob *__restrict__ jobs, const int32_t *__restrict__ order, int n_items, unsigned int *counter, BatchGeom bg,
    const ModConst *__restrict__ mc, int logn) {
    HE_GRID_DEP();
    __shared__ uint64_t red[G * 3 * VEC * (MM_THREADS / G)];
    __shared__ MMTables tb;
    __shared__ int item_s;
    extern __shared__ uint4 mm_pipe[];
    const int N = 1 << logn;
    constexpr int TILE = (MM_THREADS / G) * VEC;
    const int tiles = (N + TILE - 1) / TILE;
    for (;;) {
        if (threadIdx.x == 0) item_s = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int item = item_s;
        __syncthreads();
        if (item >= n_items) return;
        const int code = order[item];
        const int j = code / (tiles * bg.ext), rest = code % (tiles * bg.ext);
        const int u = rest / tiles, tile = rest % tiles;
        const MMJob &jb = jobs[j];
        if (jb.m_prime == 0) continue;  // empty slot
        const uint64_t *const *k_use;
        const uint32_t *g_use;
        stage_tables(tb, jb.keys, jb.galois, jb.m_prime, k_use, g_use);
        constexpr int LANES = MM_THREADS / G;
        mm_tile<NDIG, VEC, G, S, GA>(jb.ct, bg.D + (int64_t)j * bg.d_words, jb.pts, k_use, g_use, jb.m_prime, bg.ndig, bg.ext, bg.nq, bg.L,
                                     bg.LK, u, tile * TILE + VEC * ((int)threadIdx.x % LANES), LANES, bg.acc + (int64_t)j * bg.acc_words,
                                     bg.cacc + (int64_t)j * bg.cacc_words, 0, mc, logn, red, reinterpret_cast<uint64_t *>(mm_pipe));
        __syncthreads();
    }
}

}  // namespace

// ---- variant dispatch ----
// variant v: (coefficients per thread VEC, rotation groups G, cp.async stages S, gathers through
// the stages GA); S = 0 is the register-prefetch form
struct MMShape {
    int vec, grp, stages;
    bool ga;
};
constexpr MMShape kMMShapes[] = {{2, 4, 0, false}, {1, 4, 0, false}, {1, 8, 0, false}, {2, 8, 0, false},
                                 {2, 4, 3, false}, {2, 4, 2, true},  {1, 4, 2, true},  {1, 8, 2, true}};
constexpr int kMMVariants = (int)(sizeof(kMMShapes) / sizeof(kMMShapes[0]));
static_assert(kMMVariants <= HE_MM_MAX_VARIANTS, "variant table");

int mm_variant_count() { return kMMVariants; }
int mm_variant_tile(int v) { return (MM_THREADS / kMMShapes[v].grp) * kMMShapes[v].vec; }
void mm_variant_shape(int v, int *vec, int *grp, int *stages, int *ga) {
    *vec = kMMShapes[v].vec;
    *grp = kMMShapes[v].grp;
    *stages = kMMShapes[v].stages;
    *ga = kMMShapes[v].ga ? 1 : 0;
}

namespace {

// calls f.template operator()<NDIG, VEC, G, S, GA>() for variant v and digit count ndig
// (NDIG = 0: any digit count, register form)
template <int VEC, int G, int S, bool GA, typename F>
void mm_dispatch_nd(int ndig, F &&f) {
    switch (ndig) {
        case 1: f.template operator()<1, VEC, G, S, GA>(); break;
        case 2: f.template operator()<2, VEC, G, S, GA>(); break;
        case 3: f.template operator()<3, VEC, G, S, GA>(); break;
        default: f.template operator()<0, VEC, G, 0, false>(); break;
    }
}
// the fused-key forms: staged variants (4-7) with 1-3 digits
template <int VEC, int G, int S, bool GA, typename F>
void mm_dispatch_fk_nd(int ndig, F &&f) {
    switch (ndig) {
        case 1: f.template operator()<1, VEC, G, S, GA>(); break;
        case 2: f.template operator()<2, VEC, G, S, GA>(); break;
        default: f.template operator()<3, VEC, G, S, GA>(); break;
    }
}
template <typename F>
void mm_dispatch_fk(int v, int ndig, F &&f) {
    switch (v) {
        case 5: mm_dispatch_fk_nd<2, 4, 2, true>(ndig, f); break;
        case 6: mm_dispatch_fk_nd<1, 4, 2, true>(ndig, f); break;
        case 7: mm_dispatch_fk_nd<1, 8, 2, true>(ndig, f); break;
        default: mm_dispatch_fk_nd<2, 4, 3, false>(ndig, f); break;
    }
}
template <typename F>
void mm_dispatch(int v, int ndig, F &&f) {
    switch (v) {
        case 1: mm_dispatch_nd<1, 4, 0, false>(ndig, f); break;
        case 2: mm_dispatch_nd<1, 8, 0, false>(ndig, f); break;
        case 3: mm_dispatch_nd<2, 8, 0, false>(ndig, f); break;
        case 4: mm_dispatch_nd<2, 4, 3, false>(ndig, f); break;
        case 5: mm_dispatch_nd<2, 4, 2, true>(ndig, f); break;
        case 6: mm_dispatch_nd<1, 4, 2, true>(ndig, f); break;
        case 7: mm_dispatch_nd<1, 8, 2, true>(ndig, f); break;
        default: mm_dispatch_nd<2, 4, 0, false>(ndig, f); break;
    }
}

}  // namespace

// Lanes per block of the single-MatMult loop kernel: the multiple of 32 / G (whole warps) up to
// MM_THREADS / G that minimises lanes x ceil(blocks / SMs), the lanes the busiest
// multiprocessor serves (ties: the larger run).  For ext = 4, N = 8192, VEC = 2 on 152 SMs this
// is 56 (293 blocks, at most 2 per SM) instead of 64 (256 blocks: 104 SMs with 2, 48 with 1).
int mm_block_lanes(int v, int64_t total_lanes, int sms) {
    const int g = kMMShapes[v].grp, lmax = MM_THREADS / g, step = 32 / g;
    int best = lmax;
    int64_t best_cost = -1;
    for (int l = lmax; l >= step; l -= step) {
        const int64_t blocks = (total_lanes + l - 1) / l;
        const int64_t cost = (int64_t)l * ((blocks + sms - 1) / sms);
        if (best_cost < 0 || cost < best_cost) {
            best = l;
            best_cost = cost;
        }
    }
    return best;
}

void mm_launch_variant(he_ctx *ctx, int v, const uint64_t *ct, const uint64_t *D, const uint64_t *pts, const uint64_t *const *keys,
                       const uint32_t *galois, int m_prime, int ndig, int ext, int nq, uint64_t *acc, uint64_t *cacc, int accumulate,
                       const uint64_t *fused) {
    const int64_t total = (int64_t)ext * (ctx->n / kMMShapes[v].vec);
    const int lanes = mm_block_lanes(v, total, ctx->sms);
    const unsigned grid = (unsigned)((total + lanes - 1) / lanes), threads = (unsigned)(lanes * kMMShapes[v].grp);
    ctx->launches++;
    if (fused && mm_variant_fusable(v, ndig)) {
        mm_dispatch_fk(v, ndig, [&]<int NDIG, int VEC, int G, int S, bool GA>() {
            launch_k(matmult_loop_kernel<NDIG, VEC, G, S, GA, true>, grid, threads, mm_pipe_bytes(NDIG, VEC, S, GA), ctx->stream, ct, D, pts, keys,
                     galois, m_prime, ndig, ext, nq, ctx->L, ctx->L + ctx->K, acc, cacc, accumulate, ctx->d_mc, ctx->log_n, fused);
        });
        return;
    }
    mm_dispatch(v, ndig, [&]<int NDIG, int VEC, int G, int S, bool GA>() {
        launch_k(matmult_loop_kernel<NDIG, VEC, G, S, GA>, grid, threads, mm_pipe_bytes(NDIG, VEC, S, GA), ctx->stream, ct, D, pts, keys, galois,
                 m_prime, ndig, ext, nq, ctx->L, ctx->L + ctx->K, acc, cacc, accumulate, ctx->d_mc, ctx->log_n, (const uint64_t *)nullptr);
    });
}

bool mm_variant_fusable(int v, int ndig) { return ndig >= 1 && ndig <= 3 && kMMShapes[v].stages > 0; }

void launch_fuse_keys(he_ctx *ctx, he_ptmat *pm) {
    const he_plan &p = pm->plan;
    const int ndig = ctx->modup[pm->level].ndig, nq = pm->level + 1;
    const int64_t total = (int64_t)p.row_blocks * p.col_blocks * (p.m_prime - 1) * pm->ext * (ctx->n / 2);
    if (total <= 0) return;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    ctx->launches++;
    launch_k(fuse_keys_kernel, (unsigned)blocks, 256, 0, ctx->stream, (const uint64_t *)pm->data, (const uint64_t *const *)pm->d_keys, pm->fused,
             total, (int)p.m_prime, ndig, pm->ext, nq, ctx->L, ctx->L + ctx->K, (const ModConst *)ctx->d_mc, ctx->log_n);
}

void mm_launch_batch_variant(int v, dim3 grid, cudaStream_t st, const MMJob *jobs, const int32_t *order, int n_items, unsigned int *counter,
                             const BatchGeom &bg, const ModConst *mc, int logn) {
    mm_dispatch(v, bg.ndig, [&]<int NDIG, int VEC, int G, int S, bool GA>() {
        launch_k(matmult_batch_loop_kernel<NDIG, VEC, G, S, GA>, grid, MM_THREADS, mm_pipe_bytes(NDIG, VEC, S, GA), st, jobs, order, n_items, counter,
                                                                                                                 bg, mc, logn);
    });
}

// resident CTAs per SM of the batch kernel of variant v (the persistent grid is this times the SMs)
int mm_batch_ctas_per_sm(int v, int ndig) {
    int n = 0;
    mm_dispatch(v, ndig, [&]<int NDIG, int VEC, int G, int S, bool GA>() {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, matmult_batch_loop_kernel<NDIG, VEC, G, S, GA>, MM_THREADS,
                                                      mm_pipe_bytes(NDIG, VEC, S, GA));
    });
    return n > 0 ? n : 1;
}

namespace {

// ---- cleartext layout (Eq. 2 after Eq. 3) and lazy rotate-and-sum (Sec. 4.3) ----
// Every size of a plan but m and n is a power of two (slots, padded and block sizes, m', block
// counts), so the index arithmetic below is shifts and masks: log2 of such a size.
__device__ __forceinline__ int lg2p(int64_t v) { return __ffsll(v) - 1; }

// trans: X holds the n x m transpose of the matrix (entry (row, col) at X[col m + row])
__global__ void layout_matrix_kernel(he_plan p, const double *__restrict__ X, double *out, int64_t total, int trans) {
    HE_GRID_DEP();
    const int ls = lg2p(p.slots), lm = lg2p(p.m_prime), lc = lg2p(p.col_blocks), lnb = lg2p(p.nb), lmb = lg2p(p.mb);
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t s = idx & (p.slots - 1);
        int64_t rest = idx >> ls;
        const int64_t i = rest & (p.m_prime - 1);
        if (p.baby) s = (s - (i - (i & (p.baby - 1)))) & (p.slots - 1);  // BSGS: RotR(e_i, g B), i = g B + b
        rest >>= lm;
        const int64_t c = rest & (p.col_blocks - 1), r = rest >> lc;
        const int64_t b = s >> lnb, jj = s & (p.nb - 1);
        const int64_t row = (r << lmb) + (b << lm) + (jj & (p.m_prime - 1));
        const int64_t col = (c << lnb) + ((i + jj) & (p.nb - 1));
        out[idx] = (row < p.m && col < p.n) ? X[trans ? col * p.m + row : row * p.n + col] : 0.0;
    }
}

__global__ void layout_vector_kernel(he_plan p, const double *__restrict__ y, double *out) {
    HE_GRID_DEP();
    const int ls = lg2p(p.slots), lnb = lg2p(p.nb);
    const int64_t total = p.col_blocks * p.slots;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = idx >> ls, s = idx & (p.slots - 1);
        const int64_t col = (c << lnb) + (s & (p.nb - 1));
        out[idx] = col < p.n ? y[col] : 0.0;
    }
}

// y[r mb + b m' + t] = sum_{s < nb/m'} (slots - mask)[r][b nb + t + s m'] (mask may be null)
__global__ void lazy_ras_kernel(he_plan p, const double *__restrict__ slots, const double *__restrict__ mask, double *y) {
    HE_GRID_DEP();
    const int lmb = lg2p(p.mb), lm = lg2p(p.m_prime), lnb = lg2p(p.nb), ls = lg2p(p.slots);
    const int64_t terms = p.nb >> lm;
    for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < p.m; row += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = row >> lmb, rem = row & (p.mb - 1);
        const int64_t b = rem >> lm, t = rem & (p.m_prime - 1);
        const int64_t off = (r << ls) + (b << lnb) + t;
        double acc = 0.0;  // summed in order s = 0, 1, ...; the unrolling only issues the loads early
#pragma unroll 8
        for (int64_t s = 0; s < terms; ++s) acc += mask ? slots[off + (s << lm)] - mask[off + (s << lm)] : slots[off + (s << lm)];
        y[row] = acc;
    }
}

// after the ciphertext rotate-and-sum: y[r mb + b m' + t] = slots[r][b nb + t]
__global__ void ras_gather_kernel(he_plan p, const double *__restrict__ slots, double *y) {
    HE_GRID_DEP();
    const int lmb = lg2p(p.mb), lm = lg2p(p.m_prime), lnb = lg2p(p.nb), ls = lg2p(p.slots);
    for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < p.m; row += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = row >> lmb, rem = row & (p.mb - 1);
        const int64_t b = rem >> lm, t = rem & (p.m_prime - 1);
        y[row] = slots[(r << ls) + (b << lnb) + t];
    }
}

inline dim3 elem_grid(int n, int y, int z = 1) { return dim3((n + 255) / 256, y, z); }

}  // namespace

// next start/end event pair of profiled kernel class `kind`, or nullptr when profiling is off
cudaEvent_t *prof_pair(he_ctx *ctx, int kind) {
    if (!ctx->prof_on) return nullptr;
    std::vector<cudaEvent_t> &evs = ctx->prof_events[kind];
    if (ctx->prof_used[kind] + 2 > evs.size()) {
        cudaEvent_t a, b;
        if (cudaEventCreate(&a) != cudaSuccess) return nullptr;
        if (cudaEventCreate(&b) != cudaSuccess) {
            cudaEventDestroy(a);
            return nullptr;
        }
        evs.push_back(a);
        evs.push_back(b);
    }
    cudaEvent_t *ev = evs.data() + ctx->prof_used[kind];
    ctx->prof_used[kind] += 2;
    return ev;
}

namespace {

}  // namespace

void launch_add(he_ctx *ctx, const uint64_t *a, const uint64_t *b, uint64_t *out, int groups, const LimbMap &map) {
    ctx->launches++;
    launch_k(add_kernel, elem_grid(ctx->n, map.n, groups), 256, 0, ctx->stream, a, b, out, map, ctx->d_mc, ctx->log_n);
}

void launch_mul_plain(he_ctx *ctx, const uint64_t *ct, const uint64_t *pt, uint64_t *out, int level) {
    ctx->launches++;
    launch_k(mul_plain_kernel, elem_grid(ctx->n, level + 1, 2), 256, 0, ctx->stream, ct, pt, out, level + 1, ctx->d_mc, ctx->log_n);
}

void launch_automorph(he_ctx *ctx, const uint64_t *in, uint64_t *out, int groups, const LimbMap &map, uint32_t g) {
    ctx->launches++;
    launch_k(automorph_kernel, elem_grid(ctx->n, groups * map.n), 256, 0, ctx->stream, in, out, g, ctx->log_n);
}

static size_t cl_fused_smem_bytes(int logn) { return cl_smem_bytes(logn) + ((size_t)8 << (logn - 3)); }

void launch_modup(he_ctx *ctx, const uint64_t *c1_ntt, int level, uint64_t *D, uint64_t *tmp_coeff) {
    const ModUpConst &mu = ctx->modup[level];
    const int items = mu.ndig * mu.ext;
    if (ctx->bconv == HE_BCONV_INT8_TC) {  // c1 to coefficient form, then the tensor-core conversion and the NTTs
        LimbMap qm{};
        qm.n = level + 1;
        for (int l = 0; l <= level; ++l) qm.prime[l] = l;
        launch_ntt_inv_strided(ctx, c1_ntt, 0, tmp_coeff, 0, 1, qm);
        launch_modup_i8(ctx, nullptr, 1, level, c1_ntt, tmp_coeff, 0, D, 0);
        return;
    }
    ctx->launches++;
    if (use_cluster(ctx->log_n, items)) {  // the inverse NTT of c1 happens inside
        launch_cluster(by_logn(ctx->log_n, [](auto L) { return modup_cl_fused_kernel<L.value>; }), items * HE_NTT_CL_SIZE, cl_threads(ctx->log_n), cl_fused_smem_bytes(ctx->log_n), ctx->stream, c1_ntt,
                       D, mu, (const uint64_t *)ctx->d_tw, (const ModConst *)ctx->d_mc, ctx->log_n);
        return;
    }
    LimbMap qmap{};
    qmap.n = level + 1;
    for (int l = 0; l <= level; ++l) qmap.prime[l] = l;
    launch_ntt_inv_strided(ctx, c1_ntt, 0, tmp_coeff, 0, 1, qmap);
    launch_k(modup_kernel<false>, items, ntt_threads(ctx->log_n), ntt_smem_bytes(ctx->log_n), ctx->stream, c1_ntt, tmp_coeff, D, mu, ctx->d_tw,
             ctx->d_mc, ctx->log_n);
}

void launch_ks_inner(he_ctx *ctx, const uint64_t *D, int level, uint32_t g, const uint64_t *key, uint64_t *u) {
    const ModUpConst &mu = ctx->modup[level];
    LimbMap emap{};
    emap.n = mu.ext;
    for (int v = 0; v < mu.ext; ++v) emap.prime[v] = mu.ext_prime[v];
    ctx->launches++;
    launch_k(ks_inner_kernel, elem_grid(ctx->n, mu.ext), 256, 0, ctx->stream, D, mu.ndig, mu.ext, emap, level + 1, ctx->L,
                                                                        ctx->L + ctx->K, g, key, u, ctx->d_mc, ctx->log_n);
}

void launch_moddown(he_ctx *ctx, const uint64_t *x, int level, int ncomp, const uint64_t *add0, const uint64_t *add1, uint64_t *out,
                    uint64_t *tmp) {
    const ModDownConst &md = ctx->moddown[level];
    const int ext = level + 1 + ctx->K;
    const int items = ncomp * md.nq;
    ctx->launches++;
    if (use_cluster(ctx->log_n, items)) {  // the inverse NTT of the P limbs happens inside
        launch_cluster(by_logn(ctx->log_n, [](auto L) { return moddown_cl_fused_kernel<L.value>; }), items * HE_NTT_CL_SIZE, cl_threads(ctx->log_n), cl_fused_smem_bytes(ctx->log_n), ctx->stream, x,
                       ext, md, add0, add1, out, (const uint64_t *)ctx->d_tw, (const ModConst *)ctx->d_mc, ctx->log_n);
        return;
    }
    LimbMap pmap{};
    pmap.n = ctx->K;
    for (int i = 0; i < ctx->K; ++i) pmap.prime[i] = ctx->L + i;
    // P limbs of every component into coefficient form: tmp [ncomp][K][N]
    launch_ntt_inv_strided(ctx, x + (int64_t)(level + 1) * ctx->n, (int64_t)ext * ctx->n, tmp, (int64_t)ctx->K * ctx->n, ncomp, pmap);
    launch_k(moddown_kernel<false>, items, ntt_threads(ctx->log_n), ntt_smem_bytes(ctx->log_n), ctx->stream, x, ext, tmp, md, add0, add1, out,
             ctx->d_tw, ctx->d_mc, ctx->log_n);
}

static RescaleConst make_rescale_const(const he_ctx *ctx, int level) {
    RescaleConst rc{};
    rc.ql = ctx->primes[level];
    rc.half = rc.ql / 2;
    for (int j = 0; j < level; ++j) {
        const uint64_t q = ctx->primes[j];
        // q_l^-1 mod q_j by Fermat, host side
        uint64_t base = rc.ql % q, e = q - 2, r = 1;
        while (e) {
            if (e & 1) r = (uint64_t)((u128)r * base % q);
            base = (uint64_t)((u128)base * base % q);
            e >>= 1;
        }
        rc.inv[j] = r;
        rc.inv_shoup[j] = (uint64_t)(((u128)r << 64) / q);
    }
    return rc;
}

void launch_rescale(he_ctx *ctx, const uint64_t *ct, int level, uint64_t *out, uint64_t *tmp) {
    const RescaleConst rc = make_rescale_const(ctx, level);
    ctx->launches++;
    if (use_cluster(ctx->log_n, 2 * level)) {  // the inverse NTT of the last limb happens inside
        launch_cluster(by_logn(ctx->log_n, [](auto L) { return rescale_cl_fused_kernel<L.value>; }), 2 * level * HE_NTT_CL_SIZE, cl_threads(ctx->log_n), cl_fused_smem_bytes(ctx->log_n), ctx->stream,
                       ct, level, rc, out, (const uint64_t *)ctx->d_tw, (const ModConst *)ctx->d_mc, ctx->log_n);
        return;
    }
    LimbMap lmap{};
    lmap.n = 1;
    lmap.prime[0] = level;
    const int64_t N = ctx->n;
    launch_ntt_inv_strided(ctx, ct + (int64_t)level * N, (int64_t)(level + 1) * N, tmp, N, 2, lmap);
    launch_k(rescale_kernel<false>, 2 * level, ntt_threads(ctx->log_n), ntt_smem_bytes(ctx->log_n), ctx->stream, ct, level, tmp, rc, out, ctx->d_tw,
             ctx->d_mc, ctx->log_n);
}

bool moddown_rescale_fused(const he_ctx *ctx, int level) { return level >= 1 && use_cluster(ctx->log_n, 2 * level); }

void launch_moddown_rescale(he_ctx *ctx, const uint64_t *x, int level, const uint64_t *add0, const uint64_t *add1, uint64_t *out,
                            uint64_t *tmp) {
    const ModDownConst &md = ctx->moddown[level];
    const RescaleConst rc = make_rescale_const(ctx, level);
    const int ext = level + 1 + ctx->K;
    ctx->launches += 2;
    launch_cluster(by_logn(ctx->log_n, [](auto L) { return moddown_rescale_intt_kernel<L.value>; }), 2 * (ctx->K + 1) * HE_NTT_CL_SIZE,
                   cl_threads(ctx->log_n), cl_smem_bytes(ctx->log_n), ctx->stream, x, ext, md, add0, add1, tmp, (const uint64_t *)ctx->d_tw,
                   (const ModConst *)ctx->d_mc, ctx->log_n);
    launch_cluster(by_logn(ctx->log_n, [](auto L) { return moddown_rescale_ntt_kernel<L.value>; }), 2 * level * HE_NTT_CL_SIZE, cl_threads(ctx->log_n),
                   cl_smem_bytes(ctx->log_n), ctx->stream, x, ext, md, rc, add0, add1, (const uint64_t *)tmp, out, (const uint64_t *)ctx->d_tw,
                   (const ModConst *)ctx->d_mc, ctx->log_n);
}

void launch_matmult_loop(he_ctx *ctx, const he_ptmat *pm, int r, int c, const uint64_t *ct, const uint64_t *D, uint64_t *acc,
                         uint64_t *cacc, int accumulate) {
    const int level = pm->level;
    const ModUpConst &mu = ctx->modup[level];
    const he_plan &p = pm->plan;
    const uint64_t *pts = pm->data + (((int64_t)r * p.col_blocks + c) * p.m_prime) * pm->ext * ctx->n;
    const bool fk = pm->fuse_state == 1 && pm->fused && pm->fused_gen == pm->enc_gen && pm->fvariant >= 0;
    const uint64_t *fused = fk ? pm->fused + ((int64_t)r * p.col_blocks + c) * (p.m_prime - 1) * 2 * mu.ndig * pm->ext * ctx->n : nullptr;
    cudaEvent_t *ev = prof_pair(ctx, HE_PROF_LOOP);
    if (ev) cudaEventRecord(ev[0], ctx->stream);
    mm_launch_variant(ctx, fk ? pm->fvariant : (pm->variant < 0 ? 0 : pm->variant), ct, D, pts, pm->d_keys, pm->d_galois, (int)p.m_prime,
                      mu.ndig, mu.ext, level + 1, acc, cacc, accumulate, fused);
    if (ev) cudaEventRecord(ev[1], ctx->stream);
}

// best of three timed launches (after one untimed) of variant v on block (0, 0); 1e30 on error
static float time_loop_variant(he_ctx *ctx, he_ptmat *pm, int v, const uint64_t *ct, const uint64_t *D, uint64_t *acc, uint64_t *cacc,
                               const uint64_t *fused, cudaEvent_t a, cudaEvent_t b) {
    const ModUpConst &mu = ctx->modup[pm->level];
    float ms = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(a, ctx->stream);
        mm_launch_variant(ctx, v, ct, D, pm->data, pm->d_keys, pm->d_galois, (int)pm->plan.m_prime, mu.ndig, mu.ext, pm->level + 1, acc, cacc, 0,
                          fused);
        cudaEventRecord(b, ctx->stream);
        if (cudaEventSynchronize(b) != cudaSuccess) break;
        float t = 0.0f;
        cudaEventElapsedTime(&t, a, b);
        if (rep > 0 && t < ms) ms = t;
    }
    return ms;
}

// Time the fused-key forms of the staged variants on this matrix (its tables built) and keep the
// fastest in pm->fvariant; the caller compares it with the two-level form.  Synchronises.
int tune_matmult_fused(he_ctx *ctx, he_ptmat *pm, const uint64_t *ct, const uint64_t *D, uint64_t *acc, uint64_t *cacc) {
    const int ndig = ctx->modup[pm->level].ndig;
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return HE_ECUDA;
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return HE_ECUDA;
    }
    int best = -1;
    for (int v = 0; v < mm_variant_count(); ++v) {
        pm->fuse_ms[v] = 0.0f;
        if (!mm_variant_fusable(v, ndig)) continue;
        pm->fuse_ms[v] = time_loop_variant(ctx, pm, v, ct, D, acc, cacc, pm->fused, a, b);
        if (best < 0 || pm->fuse_ms[v] < pm->fuse_ms[best]) best = v;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    pm->fvariant = best;
    return cudaGetLastError() == cudaSuccess ? HE_OK : HE_ECUDA;
}

// Time every loop-kernel variant once on this matrix's first product (the results are identical:
// modular sums do not depend on the order) and keep the fastest.  Synchronises the stream.
int tune_matmult_loop(he_ctx *ctx, he_ptmat *pm, const uint64_t *ct, const uint64_t *D, uint64_t *acc, uint64_t *cacc) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return HE_ECUDA;
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return HE_ECUDA;
    }
    int best = 0;
    float best_ms = 1e30f;
    for (int v = 0; v < mm_variant_count(); ++v) {
        // one untimed launch (it also loads the variant's code), then the best of three
        const float ms = time_loop_variant(ctx, pm, v, ct, D, acc, cacc, nullptr, a, b);
        pm->tune_ms[v] = ms;
        if (ms < best_ms) {
            best_ms = ms;
            best = v;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    pm->variant = best;
    return cudaGetLastError() == cudaSuccess ? HE_OK : HE_ECUDA;
}

// Same launch as launch_matmult_loop, with the Galois-key pointer table and Galois elements
// supplied by the caller instead of the encoded matrix's own tables.
void launch_matmult_loop_with_tables(he_ctx *ctx, const he_ptmat *pm, int r, int c, const uint64_t *ct, const uint64_t *D,
                                     const uint64_t *const *keys, const uint32_t *galois, uint64_t *acc, uint64_t *cacc, int accumulate) {
    const int level = pm->level;
    const ModUpConst &mu = ctx->modup[level];
    const he_plan &p = pm->plan;
    const uint64_t *pts = pm->data + (((int64_t)r * p.col_blocks + c) * p.m_prime) * pm->ext * ctx->n;
    mm_launch_variant(ctx, pm->variant < 0 ? 0 : pm->variant, ct, D, pts, keys, galois, (int)p.m_prime, mu.ndig, mu.ext, level + 1, acc, cacc,
                      accumulate, nullptr);
}

void launch_layout_matrix(he_ctx *ctx, const he_plan &p, const double *X, double *slots, int trans) {
    int64_t total = p.row_blocks * p.col_blocks * p.m_prime * p.slots;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 65535 * 8) blocks = 65535 * 8;
    ctx->launches++;
    launch_k(layout_matrix_kernel, blocks, 256, 0, ctx->stream, p, X, slots, total, trans);
}

void launch_layout_vector(he_ctx *ctx, const he_plan &p, const double *y, double *slots) {
    int blocks = (int)((p.col_blocks * p.slots + 255) / 256);
    ctx->launches++;
    launch_k(layout_vector_kernel, blocks, 256, 0, ctx->stream, p, y, slots);
}

void launch_lazy_ras(he_ctx *ctx, const he_plan &p, const double *slots, const double *mask, double *y) {
    int blocks = (int)((p.m + 255) / 256);
    ctx->launches++;
    launch_k(lazy_ras_kernel, blocks, 256, 0, ctx->stream, p, slots, mask, y);
}

void launch_ras_gather(he_ctx *ctx, const he_plan &p, const double *slots, double *y) {
    int blocks = (int)((p.m + 255) / 256);
    ctx->launches++;
    launch_k(ras_gather_kernel, blocks, 256, 0, ctx->stream, p, slots, y);
}

// Whole batched MatMult on `stream`: ModUp of every input, one persistent loop launch over the
// (tile, limb, job) queue, ModDown and rescale of every output.  Seven launches and two copies
// in total, whatever the job count; the caller may capture them in a CUDA graph.
int launch_matmult_batch(he_ctx *ctx, he_batch *b, cudaStream_t stream) {
    const BatchGeom &bg = b->bg;
    const int count = b->count, thr = ntt_threads(ctx->log_n), level = bg.level;
    const size_t smem = ntt_smem_bytes(ctx->log_n);
    const ModUpConst &mu = ctx->modup[level];
    const ModDownConst &md = ctx->moddown[level];
    const RescaleConst rc = make_rescale_const(ctx, level);
    if (cudaMemcpyAsync(b->d_jobs, b->h_jobs, sizeof(MMJob) * count, cudaMemcpyHostToDevice, stream) != cudaSuccess) return HE_ECUDA;
    if (cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned int), stream) != cudaSuccess) return HE_ECUDA;
    const int v = b->variant < 0 ? 0 : b->variant;
    const dim3 pgrid((unsigned)b->ctas_v[v]);
    const int logn = ctx->log_n;
    if (b->stage_form == 1 && logn >= HE_NTT_CL_MIN_LOGN && level >= 1) {
        // stages as clusters: ModUp, loop, ModDown + rescale (four launches)
        const int cl = cl_threads(logn);
        launch_cluster(by_logn(logn, [](auto L) { return batch_modup_cl_kernel<L.value>; }), count * mu.ndig * mu.ext * HE_NTT_CL_SIZE, cl,
                       cl_fused_smem_bytes(logn), stream, (const MMJob *)b->d_jobs, bg, mu, (const uint64_t *)ctx->d_tw, (const ModConst *)ctx->d_mc, logn);
        mm_launch_batch_variant(v, pgrid, stream, b->d_jobs, b->d_order_v[v], b->n_items_v[v], b->d_counter, bg, ctx->d_mc, logn);
        launch_cluster(by_logn(logn, [](auto L) { return batch_mdr_intt_cl_kernel<L.value>; }), count * 2 * (ctx->K + 1) * HE_NTT_CL_SIZE, cl,
                       cl_smem_bytes(logn), stream, (const MMJob *)b->d_jobs, bg, md, (const uint64_t *)ctx->d_tw, (const ModConst *)ctx->d_mc, logn);
        launch_cluster(by_logn(logn, [](auto L) { return batch_mdr_ntt_cl_kernel<L.value>; }), count * 2 * level * HE_NTT_CL_SIZE, cl,
                       cl_smem_bytes(logn), stream, (const MMJob *)b->d_jobs, bg, md, rc, (const uint64_t *)ctx->d_tw, (const ModConst *)ctx->d_mc, logn);
        ctx->launches += 4;
        return cudaGetLastError() == cudaSuccess ? HE_OK : HE_ECUDA;
    }
    launch_k(batch_intt_c1_kernel, count * bg.nq, thr, smem, stream, b->d_jobs, bg, ctx->d_tw, ctx->d_mc, ctx->log_n);
    launch_k(batch_modup_kernel, count * mu.ndig * mu.ext, thr, smem, stream, b->d_jobs, bg, mu, ctx->d_tw, ctx->d_mc, ctx->log_n);
    mm_launch_batch_variant(v, pgrid, stream, b->d_jobs, b->d_order_v[v], b->n_items_v[v], b->d_counter, bg, ctx->d_mc, ctx->log_n);
    launch_k(batch_intt_p_kernel, count * 2 * bg.K, thr, smem, stream, b->d_jobs, bg, ctx->d_tw, ctx->d_mc, ctx->log_n);
    launch_k(batch_moddown_kernel, count * 2 * md.nq, thr, smem, stream, b->d_jobs, bg, md, ctx->d_tw, ctx->d_mc, ctx->log_n);
    launch_k(batch_intt_last_kernel, count * 2, thr, smem, stream, b->d_jobs, bg, ctx->d_tw, ctx->d_mc, ctx->log_n);
    launch_k(batch_rescale_kernel, count * 2 * level, thr, smem, stream, b->d_jobs, bg, rc, ctx->d_tw, ctx->d_mc, ctx->log_n);
    ctx->launches += 7;
    return cudaGetLastError() == cudaSuccess ? HE_OK : HE_ECUDA;
}


static RotGeom rot_geom(const he_ctx *ctx, int level, uint64_t *scratch, int count) {
    const ModUpConst &mu = ctx->modup[level];
    const int64_t N = ctx->n, nl = level + 1;
    RotGeom rg{};
    rg.nl = (int32_t)nl;
    rg.ext = mu.ext;
    rg.K = ctx->K;
    rg.L = ctx->L;
    rg.LK = ctx->L + ctx->K;
    rg.coef_w = nl * N;
    rg.d_w = (int64_t)mu.ndig * mu.ext * N;
    rg.p_w = 2 * (int64_t)ctx->K * N;
    rg.coef = scratch;
    rg.D = rg.coef + count * rg.coef_w;
    rg.pcoef = rg.D + count * rg.d_w;
    return rg;
}

size_t rotate_many_words(const he_ctx *ctx, int level) {
    const ModUpConst &mu = ctx->modup[level];
    const size_t N = ctx->n, nl = level + 1;
    return nl * N + (size_t)mu.ndig * mu.ext * N + 2 * (size_t)ctx->K * N + 2 * nl * N;  // the key switch's pc and cv too
}

// O3 of `count` (<= HE_ROT_CHUNK) different ciphertexts: inverse NTT of every c1, ModUp of every
// digit, then the key switch of all rotations in two launches (launch_keyswitch_many, one
// decomposition each)
void launch_rotate_many(he_ctx *ctx, const RotJob *jobs, int count, int level, uint64_t *scratch) {
    if (count == 0) return;
    const ModUpConst &mu = ctx->modup[level];
    const RotGeom rg = rot_geom(ctx, level, scratch, count);
    const int thr = ntt_threads(ctx->log_n);
    const size_t smem = ntt_smem_bytes(ctx->log_n);
    cudaStream_t st = ctx->stream;
    RotTable tab{};
    for (int j = 0; j < count; ++j) tab.j[j] = jobs[j];
    const int items = count * mu.ndig * mu.ext;
    if (ctx->bconv != HE_BCONV_INT8_TC && ctx->log_n >= HE_NTT_CL_MIN_LOGN && items <= HE_ROT_CL_MAX_ITEMS) {
        // few rotations: one cluster launch does the inverse NTTs and the conversions
        launch_cluster(by_logn(ctx->log_n, [](auto L) { return rot_modup_cl_kernel<L.value>; }), items * HE_NTT_CL_SIZE, cl_threads(ctx->log_n),
                       cl_fused_smem_bytes(ctx->log_n), st, tab, rg, mu, (const uint64_t *)ctx->d_tw, (const ModConst *)ctx->d_mc, ctx->log_n);
        ctx->launches++;
        launch_keyswitch_many(ctx, jobs, count, level, rg.D, rg.d_w, rg.pcoef);
        return;
    }
    if (ctx->bconv != HE_BCONV_INT8_TC && use_two_phase(ctx, items)) {
        const int tiles_c = (ctx->n >> 6) / NTT2_TC, tiles_r = 64 / NTT2_TR;
        const uint64_t *tw = ctx->d_tw;
        const ModConst *mc = ctx->d_mc;
        auto go = [&](auto L, auto NB) {
            constexpr int LG = decltype(L)::value, NB1 = decltype(NB)::value;
            launch_k(rot2_intt_rows_kernel<LG, LG - 6 - NB1>, (unsigned)(count * rg.nl * tiles_r), NTT2_THREADS, 0, st, tab, rg, tw, mc);
            launch_k(rot2_intt_cols_kernel<LG>, (unsigned)(count * rg.nl * tiles_c), NTT2_THREADS, 0, st, rg, tw, mc);
            launch_k(rot2_modup_cols_kernel<LG>, (unsigned)(items * tiles_c), NTT2_THREADS, 0, st, tab, rg, mu, tw, mc);
            launch_k(rot2_modup_rows_kernel<LG>, (unsigned)(items * tiles_r), NTT2_THREADS, 0, st, rg, mu, tw, mc);
        };
        if (ctx->log_n == 12) go(std::integral_constant<int, 12>{}, std::integral_constant<int, 3>{});
        else if (ctx->log_n == 13) go(std::integral_constant<int, 13>{}, std::integral_constant<int, 4>{});
        else go(std::integral_constant<int, 14>{}, std::integral_constant<int, 4>{});
        ctx->launches += 4;
        launch_keyswitch_many(ctx, jobs, count, level, rg.D, rg.d_w, rg.pcoef);
        return;
    }
    launch_k(rot_intt_c1_kernel, count * rg.nl, thr, smem, st, tab, rg, ctx->d_tw, ctx->d_mc, ctx->log_n);
    ctx->launches++;
    if (ctx->bconv == HE_BCONV_INT8_TC) {
        launch_modup_i8(ctx, &tab, count, level, nullptr, rg.coef, rg.coef_w, rg.D, rg.d_w);
    } else {
        launch_k(rot_modup_kernel, count * mu.ndig * mu.ext, thr, smem, st, tab, rg, mu, ctx->d_tw, ctx->d_mc, ctx->log_n);
        ctx->launches++;
    }
    launch_keyswitch_many(ctx, jobs, count, level, rg.D, rg.d_w, rg.pcoef);
}

void ops_set_smem_limits(int max_bytes) {
    cudaFuncSetAttribute(batch_intt_c1_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
    cudaFuncSetAttribute(batch_modup_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
    cudaFuncSetAttribute(batch_intt_p_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
    cudaFuncSetAttribute(batch_moddown_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
    cudaFuncSetAttribute(batch_intt_last_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
    cudaFuncSetAttribute(batch_rescale_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
    cudaFuncSetAttribute(rot_intt_c1_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
    cudaFuncSetAttribute(rot_modup_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
    cudaFuncSetAttribute(modup_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
    cudaFuncSetAttribute(moddown_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
    cudaFuncSetAttribute(rescale_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
    each_logn([max_bytes](auto L) { cudaFuncSetAttribute(modup_cl_fused_kernel<L.value>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes); });
    each_logn([max_bytes](auto L) { cudaFuncSetAttribute(rot_modup_cl_kernel<L.value>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes); });
    each_logn([max_bytes](auto L) {
        cudaFuncSetAttribute(batch_modup_cl_kernel<L.value>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
        cudaFuncSetAttribute(batch_mdr_intt_cl_kernel<L.value>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
        cudaFuncSetAttribute(batch_mdr_ntt_cl_kernel<L.value>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
    });
    each_logn([max_bytes](auto L) { cudaFuncSetAttribute(moddown_cl_fused_kernel<L.value>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes); });
    each_logn([max_bytes](auto L) { cudaFuncSetAttribute(rescale_cl_fused_kernel<L.value>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes); });
    each_logn([max_bytes](auto L) { cudaFuncSetAttribute(moddown_rescale_intt_kernel<L.value>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes); });
    each_logn([max_bytes](auto L) { cudaFuncSetAttribute(moddown_rescale_ntt_kernel<L.value>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes); });

    for (int v = 0; v < kMMVariants; ++v)
        for (int nd = 0; nd <= 3; ++nd)
            mm_dispatch(v, nd, []<int NDIG, int VEC, int G, int S, bool GA>() {
                const int bytes = (int)mm_pipe_bytes(NDIG, VEC, S, GA);
                if (bytes == 0) return;
                cudaFuncSetAttribute(matmult_loop_kernel<NDIG, VEC, G, S, GA>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
                cudaFuncSetAttribute(matmult_batch_loop_kernel<NDIG, VEC, G, S, GA>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
                cudaFuncSetAttribute(matmult_loop_kernel<NDIG, VEC, G, S, GA>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared);
                cudaFuncSetAttribute(matmult_batch_loop_kernel<NDIG, VEC, G, S, GA>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared);
            });
    for (int v = 0; v < kMMVariants; ++v)
        for (int nd = 1; nd <= 3; ++nd)
            if (mm_variant_fusable(v, nd))
                mm_dispatch_fk(v, nd, []<int NDIG, int VEC, int G, int S, bool GA>() {
                    const int bytes = (int)mm_pipe_bytes(NDIG, VEC, S, GA);
                    cudaFuncSetAttribute(matmult_loop_kernel<NDIG, VEC, G, S, GA, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
                    cudaFuncSetAttribute(matmult_loop_kernel<NDIG, VEC, G, S, GA, true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         (int)cudaSharedmemCarveoutMaxShared);
                });
}
