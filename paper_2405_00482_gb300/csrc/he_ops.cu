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
    const int N = 1 << logn;
    const int l = blockIdx.y, g = blockIdx.z;
    const uint64_t q = mc[map.prime[l]].q;
    const int64_t base = ((int64_t)g * map.n + l) * N;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) out[base + k] = add_mod(a[base + k], b[base + k], q);
}

// ct [2][nl][N] times pt [>= nl][N] (canonical): two Montgomery steps give the canonical product
__global__ void mul_plain_kernel(const uint64_t *__restrict__ ct, const uint64_t *__restrict__ pt, uint64_t *out, int nl,
                                 const ModConst *__restrict__ mc, int logn) {
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
    const int N = 1 << logn;
    const int64_t base = (int64_t)blockIdx.y * N;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) out[base + k] = in[base + automorph_src(k, g, logn)];
}

// ModUp: CTA (d, u).  Digit-own limbs are copied from the NTT-form input; the others are
// converted from the coefficient-form digit limbs and transformed.
__global__ void modup_kernel(const uint64_t *__restrict__ c1_ntt, const uint64_t *__restrict__ c1_coef, uint64_t *D, ModUpConst mu,
                             const uint64_t *__restrict__ d_tw, const ModConst *__restrict__ mc, int logn) {
    extern __shared__ uint64_t s[];
    const int N = 1 << logn;
    const int d = blockIdx.x / mu.ext, u = blockIdx.x % mu.ext;
    const int lo = d * mu.alpha;
    const int hi = lo + mu.alpha < mu.nq ? lo + mu.alpha : mu.nq;
    const int p = mu.ext_prime[u];
    const uint64_t t = mc[p].q;
    uint64_t *dst = D + ((int64_t)d * mu.ext + u) * N;
    if (u >= lo && u < hi) {
        for (int k = threadIdx.x; k < N; k += blockDim.x) dst[k] = c1_ntt[(int64_t)u * N + k];
        return;
    }
    const int na = hi - lo;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        uint64_t acc = 0;
        for (int i = 0; i < na; ++i) {
            const uint64_t qi = mc[lo + i].q;
            uint64_t v = mul_shoup(c1_coef[(int64_t)(lo + i) * N + k], mu.inv[d][i], mu.inv_shoup[d][i], qi);
            acc = add_mod(acc, mul_shoup(v, mu.hat[d][i][u], mu.hat_shoup[d][i][u], t), t);
        }
        s[k] = acc;
    }
    __syncthreads();
    ntt_fwd_smem(s, twiddles(d_tw, p, 0, logn), twiddles(d_tw, p, 1, logn), t, logn);
    for (int k = threadIdx.x; k < N; k += blockDim.x) dst[k] = s[k];
}

// u_c[u][k] = sum_d D[d][u][src(k)] * keyM[d][c][kl(u)][k], REDC in groups of at most 8 terms
__global__ void ks_inner_kernel(const uint64_t *__restrict__ D, int ndig, int ext, LimbMap emap, int nq, int L, int LK, uint32_t g, const uint64_t *__restrict__ key, uint64_t *out,
                                const ModConst *__restrict__ mc, int logn) {
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

// ModDown epilogue: CTA (c, j).  conv = Conv_{P->q_j}(x_P coefficient form) -> NTT ->
// out = addend + (x_j - conv) P^-1.
__global__ void moddown_kernel(const uint64_t *__restrict__ x, int ext, const uint64_t *__restrict__ xp_coef, ModDownConst md,
                               const uint64_t *__restrict__ add0, const uint64_t *__restrict__ add1, uint64_t *out,
                               const uint64_t *__restrict__ d_tw, const ModConst *__restrict__ mc, int logn) {
    extern __shared__ uint64_t s[];
    const int N = 1 << logn;
    const int c = blockIdx.x / md.nq, j = blockIdx.x % md.nq;
    const int pj = md.q_prime[j];
    const uint64_t q = mc[pj].q;
    const uint64_t *xp = xp_coef + (int64_t)c * md.K * N;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        uint64_t acc = 0;
        for (int i = 0; i < md.K; ++i) {
            const uint64_t pi = mc[md.p_prime[i]].q;
            uint64_t v = mul_shoup(xp[(int64_t)i * N + k], md.inv[i], md.inv_shoup[i], pi);
            acc = add_mod(acc, mul_shoup(v, md.hat[i][j], md.hat_shoup[i][j], q), q);
        }
        s[k] = acc;
    }
    __syncthreads();
    ntt_fwd_smem(s, twiddles(d_tw, pj, 0, logn), twiddles(d_tw, pj, 1, logn), q, logn);
    const uint64_t *xj = x + ((int64_t)c * ext + j) * N;
    const uint64_t *ad = c == 0 ? add0 : add1;
    uint64_t *o = out + ((int64_t)c * md.nq + j) * N;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        uint64_t v = mul_shoup(sub_mod(xj[k], s[k], q), md.pinv[j], md.pinv_shoup[j], q);
        if (ad) v = add_mod(v, ad[(int64_t)j * N + k], q);
        o[k] = v;
    }
}

struct RescaleConst {
    uint64_t ql, half;
    uint64_t inv[HE_MAX_Q], inv_shoup[HE_MAX_Q];  // q_l^-1 mod q_j
};

// CTA (c, j), j < level: v = centred(last limb) mod q_j -> NTT -> out = (c_j - v) q_l^-1
__global__ void rescale_kernel(const uint64_t *__restrict__ ct, int level, const uint64_t *__restrict__ last_coef, RescaleConst rc,
                               uint64_t *out, const uint64_t *__restrict__ d_tw, const ModConst *__restrict__ mc, int logn) {
    extern __shared__ uint64_t s[];
    const int N = 1 << logn;
    const int c = blockIdx.x / level, j = blockIdx.x % level;
    const uint64_t q = mc[j].q;
    const uint64_t *lc = last_coef + (int64_t)c * N;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        uint64_t r = lc[k] + rc.half;
        if (r >= rc.ql) r -= rc.ql;
        int64_t centred = (int64_t)r - (int64_t)rc.half;
        s[k] = reduce_signed(centred, q);
    }
    __syncthreads();
    ntt_fwd_smem(s, twiddles(d_tw, j, 0, logn), twiddles(d_tw, j, 1, logn), q, logn);
    const uint64_t *cj = ct + ((int64_t)c * (level + 1) + j) * N;
    uint64_t *o = out + ((int64_t)c * level + j) * N;
    for (int k = threadIdx.x; k < N; k += blockDim.x) o[k] = mul_shoup(sub_mod(cj[k], s[k], q), rc.inv[j], rc.inv_shoup[j], q);
}

// The double-hoisted MatMult loop.  Thread (u, k) of the extended basis:
//   acc_c[u][k]  = sum_{i>=1} ptM_i[u][k] * redc(sum_d D[d][u][src_i(k)] keyM_i[d][c][kl(u)][k])
//   cacc_0[u][k] = ptM_0 * c0[u][k] + sum_{i>=1} ptM_i[u][k] * c0[u][src_i(k)]   (u in Q_level)
//   cacc_1[u][k] = ptM_0 * c1[u][k]
__global__ void matmult_loop_kernel(const uint64_t *__restrict__ ct, const uint64_t *__restrict__ D, const uint64_t *__restrict__ pts,
                                    const uint64_t *const *__restrict__ keys, const uint32_t *__restrict__ galois, int m_prime,
                                    int ndig, int ext, int nq, int L, int LK, LimbMap emap, uint64_t *acc, uint64_t *cacc,
                                    int accumulate, const ModConst *__restrict__ mc, int logn) {
    const int N = 1 << logn;
    const int u = blockIdx.y;
    const int p = emap.prime[u];
    const int kl = u < nq ? u : L + (u - nq);
    const uint64_t q = mc[p].q, qinv = mc[p].qinv;
    const bool inq = u < nq;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
        uint64_t a0 = 0, a1 = 0, cc0 = 0, cc1 = 0;
        const uint64_t pt0 = pts[(int64_t)u * N + k];
        if (inq) {
            cc0 = mont_mul(ct[(int64_t)u * N + k], pt0, q, qinv);
            cc1 = mont_mul(ct[((int64_t)nq + u) * N + k], pt0, q, qinv);
        }
        for (int i = 1; i < m_prime; ++i) {
            const uint32_t src = automorph_src(k, galois[i - 1], logn);
            const uint64_t *key = keys[i - 1];
            u128 t0 = 0, t1 = 0;
            uint64_t u0 = 0, u1 = 0;
            for (int d = 0; d < ndig; ++d) {
                const uint64_t dv = D[((int64_t)d * ext + u) * N + src];
                t0 += (u128)dv * key[((int64_t)(d * 2 + 0) * LK + kl) * N + k];
                t1 += (u128)dv * key[((int64_t)(d * 2 + 1) * LK + kl) * N + k];
                if ((d & 7) == 7) {
                    u0 = add_mod(u0, redc128(t0, q, qinv), q);
                    u1 = add_mod(u1, redc128(t1, q, qinv), q);
                    t0 = t1 = 0;
                }
            }
            u0 = add_mod(u0, redc128(t0, q, qinv), q);
            u1 = add_mod(u1, redc128(t1, q, qinv), q);
            const uint64_t ptm = pts[((int64_t)i * ext + u) * N + k];
            a0 = add_mod(a0, mont_mul(u0, ptm, q, qinv), q);
            a1 = add_mod(a1, mont_mul(u1, ptm, q, qinv), q);
            if (inq) cc0 = add_mod(cc0, mont_mul(ct[(int64_t)u * N + src], ptm, q, qinv), q);
        }
        const int64_t ia0 = (int64_t)u * N + k, ia1 = ((int64_t)ext + u) * N + k;
        if (accumulate) {
            acc[ia0] = add_mod(acc[ia0], a0, q);
            acc[ia1] = add_mod(acc[ia1], a1, q);
        } else {
            acc[ia0] = a0;
            acc[ia1] = a1;
        }
        if (inq) {
            const int64_t ic0 = (int64_t)u * N + k, ic1 = ((int64_t)nq + u) * N + k;
            if (accumulate) {
                cacc[ic0] = add_mod(cacc[ic0], cc0, q);
                cacc[ic1] = add_mod(cacc[ic1], cc1, q);
            } else {
                cacc[ic0] = cc0;
                cacc[ic1] = cc1;
            }
        }
    }
}

// ---- cleartext layout (Eq. 2 after Eq. 3) and lazy rotate-and-sum (Sec. 4.3) ----
__global__ void layout_matrix_kernel(he_plan p, const double *__restrict__ X, double *out, int64_t total) {
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = idx % p.slots;
        int64_t rest = idx / p.slots;
        const int64_t i = rest % p.m_prime;
        rest /= p.m_prime;
        const int64_t c = rest % p.col_blocks, r = rest / p.col_blocks;
        const int64_t b = s / p.nb, jj = s % p.nb;
        const int64_t row = r * p.mb + b * p.m_prime + (jj % p.m_prime);
        const int64_t col = c * p.nb + (i + jj) % p.nb;
        out[idx] = (row < p.m && col < p.n) ? X[row * p.n + col] : 0.0;
    }
}

__global__ void layout_vector_kernel(he_plan p, const double *__restrict__ y, double *out) {
    const int64_t total = p.col_blocks * p.slots;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = idx / p.slots, s = idx % p.slots;
        const int64_t col = c * p.nb + s % p.nb;
        out[idx] = col < p.n ? y[col] : 0.0;
    }
}

__global__ void lazy_ras_kernel(he_plan p, const double *__restrict__ slots, double *y) {
    for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < p.m; row += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = row / p.mb, rem = row % p.mb;
        const int64_t b = rem / p.m_prime, t = rem % p.m_prime;
        const double *sl = slots + r * p.slots + b * p.nb + t;
        double acc = 0.0;
        for (int64_t s = 0; s < p.nb / p.m_prime; ++s) acc += sl[s * p.m_prime];
        y[row] = acc;
    }
}

inline dim3 elem_grid(int n, int y, int z = 1) { return dim3((n + 255) / 256, y, z); }

// next start/end event pair of the profiled kernel, or nullptr when profiling is off
cudaEvent_t *prof_pair(he_ctx *ctx) {
    if (!ctx->prof_on) return nullptr;
    if (ctx->prof_used + 2 > ctx->prof_events.size()) {
        cudaEvent_t a, b;
        if (cudaEventCreate(&a) != cudaSuccess) return nullptr;
        if (cudaEventCreate(&b) != cudaSuccess) {
            cudaEventDestroy(a);
            return nullptr;
        }
        ctx->prof_events.push_back(a);
        ctx->prof_events.push_back(b);
    }
    cudaEvent_t *ev = ctx->prof_events.data() + ctx->prof_used;
    ctx->prof_used += 2;
    return ev;
}

}  // namespace

void launch_add(he_ctx *ctx, const uint64_t *a, const uint64_t *b, uint64_t *out, int groups, const LimbMap &map) {
    ctx->launches++;
    add_kernel<<<elem_grid(ctx->n, map.n, groups), 256, 0, ctx->stream>>>(a, b, out, map, ctx->d_mc, ctx->log_n);
}

void launch_mul_plain(he_ctx *ctx, const uint64_t *ct, const uint64_t *pt, uint64_t *out, int level) {
    ctx->launches++;
    mul_plain_kernel<<<elem_grid(ctx->n, level + 1, 2), 256, 0, ctx->stream>>>(ct, pt, out, level + 1, ctx->d_mc, ctx->log_n);
}

void launch_automorph(he_ctx *ctx, const uint64_t *in, uint64_t *out, int groups, const LimbMap &map, uint32_t g) {
    ctx->launches++;
    automorph_kernel<<<elem_grid(ctx->n, groups * map.n), 256, 0, ctx->stream>>>(in, out, g, ctx->log_n);
}

void launch_modup(he_ctx *ctx, const uint64_t *c1_ntt, int level, uint64_t *D, uint64_t *tmp_coeff) {
    const ModUpConst &mu = ctx->modup[level];
    LimbMap qmap{};
    qmap.n = level + 1;
    for (int l = 0; l <= level; ++l) qmap.prime[l] = l;
    launch_ntt_inv_strided(ctx, c1_ntt, 0, tmp_coeff, 0, 1, qmap);
    ctx->launches++;
    modup_kernel<<<mu.ndig * mu.ext, ntt_threads(ctx->log_n), (size_t)ctx->n * 8, ctx->stream>>>(c1_ntt, tmp_coeff, D, mu, ctx->d_tw,
                                                                                              ctx->d_mc, ctx->log_n);
}

void launch_ks_inner(he_ctx *ctx, const uint64_t *D, int level, uint32_t g, const uint64_t *key, uint64_t *u) {
    const ModUpConst &mu = ctx->modup[level];
    LimbMap emap{};
    emap.n = mu.ext;
    for (int v = 0; v < mu.ext; ++v) emap.prime[v] = mu.ext_prime[v];
    ctx->launches++;
    ks_inner_kernel<<<elem_grid(ctx->n, mu.ext), 256, 0, ctx->stream>>>(D, mu.ndig, mu.ext, emap, level + 1, ctx->L,
                                                                        ctx->L + ctx->K, g, key, u, ctx->d_mc, ctx->log_n);
}

void launch_moddown(he_ctx *ctx, const uint64_t *x, int level, int ncomp, const uint64_t *add0, const uint64_t *add1, uint64_t *out,
                    uint64_t *tmp) {
    const ModDownConst &md = ctx->moddown[level];
    const int ext = level + 1 + ctx->K;
    LimbMap pmap{};
    pmap.n = ctx->K;
    for (int i = 0; i < ctx->K; ++i) pmap.prime[i] = ctx->L + i;
    // P limbs of every component into coefficient form: tmp [ncomp][K][N]
    launch_ntt_inv_strided(ctx, x + (int64_t)(level + 1) * ctx->n, (int64_t)ext * ctx->n, tmp, (int64_t)ctx->K * ctx->n, ncomp, pmap);
    ctx->launches++;
    moddown_kernel<<<ncomp * md.nq, ntt_threads(ctx->log_n), (size_t)ctx->n * 8, ctx->stream>>>(x, ext, tmp, md, add0, add1, out, ctx->d_tw,
                                                                                              ctx->d_mc, ctx->log_n);
}

void launch_rescale(he_ctx *ctx, const uint64_t *ct, int level, uint64_t *out, uint64_t *tmp) {
    LimbMap lmap{};
    lmap.n = 1;
    lmap.prime[0] = level;
    const int64_t N = ctx->n;
    launch_ntt_inv_strided(ctx, ct + (int64_t)level * N, (int64_t)(level + 1) * N, tmp, N, 2, lmap);
    RescaleConst rc{};
    rc.ql = ctx->primes[level];
    rc.half = rc.ql / 2;
    for (int j = 0; j < level; ++j) {
        uint64_t q = ctx->primes[j];
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
    ctx->launches++;
    rescale_kernel<<<2 * level, ntt_threads(ctx->log_n), (size_t)ctx->n * 8, ctx->stream>>>(ct, level, tmp, rc, out, ctx->d_tw, ctx->d_mc,
                                                                                          ctx->log_n);
}

void launch_matmult_loop(he_ctx *ctx, const he_ptmat *pm, int r, int c, const uint64_t *ct, const uint64_t *D, uint64_t *acc,
                         uint64_t *cacc, int accumulate) {
    const int level = pm->level;
    const ModUpConst &mu = ctx->modup[level];
    LimbMap emap{};
    emap.n = mu.ext;
    for (int v = 0; v < mu.ext; ++v) emap.prime[v] = mu.ext_prime[v];
    const he_plan &p = pm->plan;
    const uint64_t *pts = pm->data + (((int64_t)r * p.col_blocks + c) * p.m_prime) * pm->ext * ctx->n;
    cudaEvent_t *ev = prof_pair(ctx);
    if (ev) cudaEventRecord(ev[0], ctx->stream);
    ctx->launches++;
    matmult_loop_kernel<<<elem_grid(ctx->n, mu.ext), 256, 0, ctx->stream>>>(ct, D, pts, pm->d_keys, pm->d_galois, (int)p.m_prime, mu.ndig,
                                                                            mu.ext, level + 1, ctx->L, ctx->L + ctx->K, emap, acc, cacc,
                                                                            accumulate, ctx->d_mc, ctx->log_n);
    if (ev) cudaEventRecord(ev[1], ctx->stream);
}

void launch_layout_matrix(he_ctx *ctx, const he_plan &p, const double *X, double *slots) {
    int64_t total = p.row_blocks * p.col_blocks * p.m_prime * p.slots;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 65535 * 8) blocks = 65535 * 8;
    ctx->launches++;
    layout_matrix_kernel<<<blocks, 256, 0, ctx->stream>>>(p, X, slots, total);
}

void launch_layout_vector(he_ctx *ctx, const he_plan &p, const double *y, double *slots) {
    int blocks = (int)((p.col_blocks * p.slots + 255) / 256);
    ctx->launches++;
    layout_vector_kernel<<<blocks, 256, 0, ctx->stream>>>(p, y, slots);
}

void launch_lazy_ras(he_ctx *ctx, const he_plan &p, const double *slots, double *y) {
    int blocks = (int)((p.m + 255) / 256);
    ctx->launches++;
    lazy_ras_kernel<<<blocks, 256, 0, ctx->stream>>>(p, slots, y);
}

void ops_set_smem_limits(int max_bytes) {
    cudaFuncSetAttribute(modup_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
    cudaFuncSetAttribute(moddown_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
    cudaFuncSetAttribute(rescale_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
}
