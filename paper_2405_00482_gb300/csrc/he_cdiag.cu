// he_cdiag.cu -- VFL-NN forward pass with the encrypted operand diagonally encoded (Alg. 3).
//
// The activation matrix A (m x n) is encrypted as its min(m, n) diagonals e_i (Eq. 2), and
// each weight column w_k is one plaintext p_k (w_k repeated with period n).  Column k of the
// product is  sum_i RotL(w_k, i) (x) [[e_i]]  (Sec. 5.3: no O4 at all), where the plaintext
// rotation RotL(., i) is the automorphism X -> X^(5^i) of p_k; in the NTT domain that is the
// index gather p_k[src_i(t)], so the kernel reads p_k through the gather and never key-switches.
//
// Layout: weight plaintexts transposed to [limb][coefficient][K] (Montgomery form) so that the
// K gathered values of one (coefficient, diagonal) are one contiguous row.
#include <algorithm>
#include <new>
#include <utility>
#include <vector>

#include "he_internal.cuh"
#include "he_ntt.cuh"

#define CD_COLS 8      // columns per lane (16 lanes cover 128 columns of one coefficient)
#define CD_WARPS 8     // warps per block (two coefficients each)
#define CD_MAX_IN 1024 // ciphertexts per launch (kernel-parameter table)
#define CD_MAX_OUT 512 // outputs per rescale launch

struct he_cdmat {
    he_ctx *ctx;
    int64_t n, K;  // rows of W (= columns of A), columns of W
    int level;
    double scale;
    uint64_t *pt;  // [level+1][N][K], NTT + Montgomery form
};

namespace {

struct CtTable {
    const uint64_t *p[CD_MAX_IN];
};
struct OutTable {
    uint64_t *p[CD_MAX_OUT];
};

// pre[k][c][u][t] = sum_i ct_i[c][u][t] * pt_k[u][src_i(t)].  Each half-warp takes one
// coefficient t (two per warp, 2 CD_WARPS per block) and its 16 lanes the CD_COLS columns
// k_base + CD_COLS l + (0..7) each, so a half-warp's gather of weight row (u, src_i(t)) is one
// contiguous run of 128 words, and each diagonal's fixed work (automorphism index, ciphertext
// loads, gather address) is shared by 16 multiply-adds per lane.  Ciphertext words are used once
// and loaded with an evict-first hint, so the weight table (read once per diagonal) stays in L2.
// Products of residues below q are summed lazy_terms(q) at a time in 128 bits (8 for 61-bit primes).
__global__ void __launch_bounds__(CD_WARPS * 32, 2) cdiag_mac_kernel(CtTable cts, int n_ct, int nl, const uint64_t *__restrict__ pt, int K,
                                                                    int k_base, uint64_t *pre, const ModConst *__restrict__ mc, int logn) {
    HE_GRID_DEP();
    const int N = 1 << logn;
    const int u = blockIdx.y;
    const uint64_t q = mc[u].q, qinv = mc[u].qinv;
    const int t = blockIdx.x * (2 * CD_WARPS) + (threadIdx.x >> 4);
    const int k0 = k_base + (threadIdx.x & 15) * CD_COLS;
    if (k0 >= K) return;  // no block-wide synchronisation below
    const int kn = K - k0 < CD_COLS ? K - k0 : CD_COLS;
    const bool vec = kn == CD_COLS && (K & 1) == 0;  // rows start 16-byte aligned when K is even
    const uint32_t two_n_mask = (2u << logn) - 1;
    u128 a0[CD_COLS], a1[CD_COLS];
    uint64_t r0[CD_COLS], r1[CD_COLS];
#pragma unroll
    for (int kk = 0; kk < CD_COLS; ++kk) a0[kk] = a1[kk] = 0, r0[kk] = r1[kk] = 0;
    // operands of diagonal i: c0, c1 at t; weights at row src_i(t)
    uint64_t c0n, c1n, pvn[CD_COLS];
    auto fetch = [&](int i, uint32_t g) {
        const uint32_t src = automorph_src(t, g, logn);
        c0n = __ldcs(cts.p[i] + (int64_t)u * N + t);
        c1n = __ldcs(cts.p[i] + ((int64_t)nl + u) * N + t);
        const uint64_t *row = pt + ((int64_t)u * N + src) * K + k0;
        if (vec) {
#pragma unroll
            for (int kk = 0; kk < CD_COLS; kk += 2) {
                const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2 *>(row + kk));
                pvn[kk] = v.x;
                pvn[kk + 1] = v.y;
            }
        } else {
#pragma unroll
            for (int kk = 0; kk < CD_COLS; ++kk) pvn[kk] = kk < kn ? __ldg(row + kk) : 0;
        }
    };
    uint32_t g = 1;
    int pending = 0;
    const int period = lazy_terms(q);  // diagonals per reduction
    for (int i = 0; i < n_ct; ++i) {
        fetch(i, g);
        g = (uint32_t)(((uint64_t)g * 5u) & two_n_mask);
#pragma unroll
        for (int kk = 0; kk < CD_COLS; ++kk) {
            a0[kk] += (u128)c0n * pvn[kk];
            a1[kk] += (u128)c1n * pvn[kk];
        }
        if (++pending == period) {
#pragma unroll
            for (int kk = 0; kk < CD_COLS; ++kk) {
                r0[kk] = add_mod(r0[kk], redc128(a0[kk], q, qinv), q);
                r1[kk] = add_mod(r1[kk], redc128(a1[kk], q, qinv), q);
                a0[kk] = a1[kk] = 0;
            }
            pending = 0;
        }
    }
    for (int kk = 0; kk < kn; ++kk) {
        r0[kk] = add_mod(r0[kk], redc128(a0[kk], q, qinv), q);
        r1[kk] = add_mod(r1[kk], redc128(a1[kk], q, qinv), q);
        uint64_t *o = pre + (int64_t)(k0 + kk) * 2 * nl * N;
        o[(int64_t)u * N + t] = r0[kk];
        o[((int64_t)nl + u) * N + t] = r1[kk];
    }
}

// encoded columns [K][nl][N] -> transposed [nl][N][K]
__global__ void transpose_cols_kernel(const uint64_t *__restrict__ in, uint64_t *out, int K, int nl, int logn) {
    HE_GRID_DEP();
    const int64_t N = 1 << logn;
    const int64_t total = (int64_t)K * nl * N;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = idx % K, rest = idx / K;  // rest = u * N + t
        out[idx] = in[k * nl * N + rest];
    }
}

struct CdRescale {
    uint64_t ql, half;
    uint64_t inv[HE_MAX_Q], inv_shoup[HE_MAX_Q];
};

// CTA (k, c, j): v = centred(last limb of output k) mod q_j -> NTT -> out_k = (pre_j - v) q_l^-1
__global__ void cdiag_rescale_kernel(const uint64_t *__restrict__ pre, const uint64_t *__restrict__ last, int level, CdRescale rc, OutTable outs,
                                     int k_first, const uint64_t *__restrict__ d_tw, const ModConst *__restrict__ mc, int logn) {
    HE_GRID_DEP();
    extern __shared__ uint64_t s[];
    const int N = 1 << logn, nl = level + 1;
    const int per = 2 * level;
    const int kl = blockIdx.x / per, c = (blockIdx.x % per) / level, j = blockIdx.x % level;
    const int k = k_first + kl;
    const uint64_t q = mc[j].q;
    const uint64_t *lc = last + ((int64_t)k * 2 + c) * N;
    for (int x = threadIdx.x; x < N; x += blockDim.x) {
        uint64_t r = lc[x] + rc.half;
        if (r >= rc.ql) r -= rc.ql;
        s[SIDX(x)] = reduce_signed((int64_t)r - (int64_t)rc.half, q, mc[j].mu);
    }
    __syncthreads();
    ntt_fwd_smem(s, twiddles(d_tw, j, 0, logn), q, logn);
    const uint64_t *cj = pre + (((int64_t)k * 2 + c) * nl + j) * N;
    uint64_t *o = outs.p[kl] + ((int64_t)c * level + j) * N;
    for (int x = threadIdx.x; x < N; x += blockDim.x) o[x] = mul_shoup(sub_mod(cj[x], s[SIDX(x)], q), rc.inv[j], rc.inv_shoup[j], q);
}

// slots of the diagonals e_i[j] = A[j mod m, (i + j) mod n], repeated over the N/2 slots
__global__ void cdiag_layout_kernel(const double *__restrict__ A, int64_t m, int64_t n, int64_t slots, double *out) {
    HE_GRID_DEP();
    const int64_t lo = m < n ? m : n, hi = m < n ? n : m;
    const int64_t total = lo * slots;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / slots, j = (idx % slots) % hi;
        out[idx] = A[(j % m) * n + (i + j) % n];
    }
}

// weight column k repeated with period n: slots[k][s] = W[s mod n][k]
__global__ void cdiag_weights_kernel(const double *__restrict__ W, int64_t n, int64_t K, int64_t slots, double *out) {
    HE_GRID_DEP();
    const int64_t total = K * slots;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = idx / slots, s = idx % slots;
        out[idx] = W[(s % n) * K + k];
    }
}

// Z[r][k] from the decrypted slots of output k: slot r (m >= n) or the sum of the n/m groups (m < n)
__global__ void cdiag_decode_kernel(const double *__restrict__ slots, int64_t m, int64_t n, int64_t K, int64_t n_slots, double *Z) {
    HE_GRID_DEP();
    const int64_t total = m * K;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = idx / K, k = idx % K;
        const double *sl = slots + k * n_slots;
        double v = 0.0;
        const int64_t groups = m >= n ? 1 : n / m;
        for (int64_t g = 0; g < groups; ++g) v += sl[r + g * m];
        Z[idx] = v;
    }
}

int blocks_for(int64_t total) { return (int)std::min<int64_t>((total + 255) / 256, 65535 * 16); }

bool pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

}  // namespace

extern "C" {

int he_cdiag_encode_weights(he_ctx *ctx, const double *W, int64_t n, int64_t K, int level, he_cdmat **out) {
    if (!ctx || !W || !out || !pow2(n) || n > ctx->n / 2 || K < 1 || K > (1 << 20)) return HE_EINVAL;
    if (level < 1 || level >= ctx->L) return HE_ELEVEL;
    *out = nullptr;
    he_cdmat *cm = new (std::nothrow) he_cdmat();
    if (!cm) return HE_ENOMEM;
    const int64_t N = ctx->n, nl = level + 1;
    cm->ctx = ctx;
    cm->n = n;
    cm->K = K;
    cm->level = level;
    cm->scale = (double)ctx->primes[level];
    if (cudaMalloc(&cm->pt, (size_t)nl * N * K * 8) != cudaSuccess) {
        delete cm;
        return HE_ENOMEM;
    }
    uint64_t *s = ctx_scratch(ctx, (size_t)K * (N / 2) + (size_t)K * N + (size_t)K * nl * N);
    if (!s) {
        he_cdmat_free(cm);
        return HE_ENOMEM;
    }
    double *slots = reinterpret_cast<double *>(s);
    int64_t *coef = reinterpret_cast<int64_t *>(s + K * (N / 2));
    uint64_t *cols = s + K * (N / 2) + K * N;
    LimbMap m{};
    m.n = (int)nl;
    for (int l = 0; l < nl; ++l) m.prime[l] = l;
    ctx->launches += 3;
    launch_k(cdiag_weights_kernel, blocks_for(K * (N / 2)), 256, 0, ctx->stream, W, n, K, N / 2, slots);
    launch_encode(ctx, slots, N / 2, N / 2, (int)K, cm->scale, coef);
    launch_ntt_from_int64(ctx, coef, cols, (int)K, m, 1);
    launch_k(transpose_cols_kernel, blocks_for(K * nl * N), 256, 0, ctx->stream, cols, cm->pt, (int)K, (int)nl, ctx->log_n);
    if (cudaGetLastError() != cudaSuccess) {
        he_cdmat_free(cm);
        return HE_ECUDA;
    }
    *out = cm;
    return HE_OK;
}

void he_cdmat_free(he_cdmat *cm) {
    if (!cm) return;
    cudaStreamSynchronize(cm->ctx->stream);
    cudaFree(cm->pt);
    delete cm;
}

int he_cdiag_encode_matrix(he_ctx *ctx, const double *A, int64_t m, int64_t n, double scale, int level, he_pt *outs) {
    if (!ctx || !A || !outs || !pow2(m) || !pow2(n) || std::max(m, n) > ctx->n / 2) return HE_EINVAL;
    if (level < 0 || level >= ctx->L) return HE_ELEVEL;
    const int64_t lo = std::min(m, n), N = ctx->n;
    for (int64_t i = 0; i < lo; ++i)
        if (!outs[i].data) return HE_EINVAL;
    uint64_t *s = ctx_scratch(ctx, (size_t)lo * (N / 2) + (size_t)lo * N);
    if (!s) return HE_ENOMEM;
    double *slots = reinterpret_cast<double *>(s);
    int64_t *coef = reinterpret_cast<int64_t *>(s + lo * (N / 2));
    LimbMap map{};
    map.n = level + 1;
    for (int l = 0; l <= level; ++l) map.prime[l] = l;
    ctx->launches++;
    launch_k(cdiag_layout_kernel, blocks_for(lo * (N / 2)), 256, 0, ctx->stream, A, m, n, N / 2, slots);
    launch_encode(ctx, slots, N / 2, N / 2, (int)lo, scale, coef);
    for (int64_t i = 0; i < lo; ++i) {
        launch_ntt_from_int64(ctx, coef + i * N, outs[i].data, 1, map, 0);
        outs[i].level = level;
        outs[i].scale = scale;
    }
    return cudaGetLastError() == cudaSuccess ? HE_OK : HE_ECUDA;
}

int he_cdiag_matmult(he_ctx *ctx, const he_cdmat *W, const he_ct *cts, int n_ct, he_ct *outs) {
    if (!ctx || !W || !cts || !outs || !same_family(W->ctx, ctx) || n_ct < 1 || n_ct > CD_MAX_IN || n_ct > W->n) return HE_EINVAL;
    const int level = W->level, nl = level + 1;
    for (int i = 0; i < n_ct; ++i) {
        if (!cts[i].data) return HE_EINVAL;
        if (cts[i].level != level) return HE_ELEVEL;
    }
    const int64_t K = W->K, N = ctx->n;
    for (int64_t k = 0; k < K; ++k)
        if (!outs[k].data) return HE_EINVAL;
    uint64_t *pre = ctx_scratch(ctx, (size_t)K * 2 * nl * N + (size_t)K * 2 * N);
    if (!pre) return HE_ENOMEM;
    uint64_t *last = pre + K * 2 * nl * N;
    CtTable tab;
    for (int i = 0; i < n_ct; ++i) tab.p[i] = cts[i].data;
    const int kmax = 16 * CD_COLS;  // columns per launch (16 lanes)
    for (int64_t kb = 0; kb < K; kb += kmax) {
        const dim3 grid((unsigned)(N / (2 * CD_WARPS)), (unsigned)nl);
        ctx->launches++;
        launch_k(cdiag_mac_kernel, grid, CD_WARPS * 32, 0, ctx->stream, tab, n_ct, nl, W->pt, (int)K, (int)kb, pre, ctx->d_mc, ctx->log_n);
    }
    // rescale every output: inverse NTT of the last limb of both components, then per (k, c, j)
    LimbMap lm{};
    lm.n = 1;
    lm.prime[0] = level;
    launch_ntt_inv_strided(ctx, pre + (int64_t)level * N, (int64_t)nl * N, last, N, (int)(2 * K), lm);
    CdRescale rc{};
    rc.ql = ctx->primes[level];
    rc.half = rc.ql / 2;
    for (int j = 0; j < level; ++j) {
        const uint64_t q = ctx->primes[j];
        uint64_t base = rc.ql % q, e = q - 2, r = 1;
        while (e) {
            if (e & 1) r = (uint64_t)((u128)r * base % q);
            base = (uint64_t)((u128)base * base % q);
            e >>= 1;
        }
        rc.inv[j] = r;
        rc.inv_shoup[j] = (uint64_t)(((u128)r << 64) / q);
    }
    for (int64_t kf = 0; kf < K; kf += CD_MAX_OUT) {
        const int kn = (int)std::min<int64_t>(CD_MAX_OUT, K - kf);
        OutTable ot;
        for (int k = 0; k < kn; ++k) ot.p[k] = outs[kf + k].data;
        ctx->launches++;
        launch_k(cdiag_rescale_kernel, kn * 2 * level, ntt_threads(ctx->log_n), ntt_smem_bytes(ctx->log_n), ctx->stream, pre, last, level, rc, ot, (int)kf, ctx->d_tw, ctx->d_mc, ctx->log_n);
    }
    const double scale = cts[0].scale * W->scale / (double)ctx->primes[level];
    for (int64_t k = 0; k < K; ++k) {
        outs[k].level = level - 1;
        outs[k].scale = scale;
    }
    return cudaGetLastError() == cudaSuccess ? HE_OK : HE_ECUDA;
}

}  // extern "C"

// Eq. 5 as read: A^T's diagonal i is RotL(e_k, r) with k = (-i) mod min(m, n) and r = i when
// m >= n, r = (-k) mod n when m < n
static void transpose_source(int64_t m, int64_t n, int64_t i, int64_t *k, int64_t *r) {
    const int64_t lo = std::min(m, n);
    *k = (lo - i) % lo;
    *r = m >= n ? i : (n - *k) % n;
}

extern "C" {

int he_cdiag_transpose_steps(int64_t m, int64_t n, int32_t *steps, int *n_steps) {
    if (!n_steps || !pow2(m) || !pow2(n) || std::max(m, n) > ((int64_t)1 << 30)) return HE_EINVAL;
    const int64_t lo = std::min(m, n);
    std::vector<int32_t> out;
    for (int64_t i = 0; i < lo; ++i) {
        int64_t k, r;
        transpose_source(m, n, i, &k, &r);
        if (r) out.push_back((int32_t)r);
    }
    std::sort(out.begin(), out.end());
    out.erase(std::unique(out.begin(), out.end()), out.end());
    if (steps)
        for (size_t t = 0; t < out.size(); ++t) steps[t] = out[t];
    *n_steps = (int)out.size();
    return HE_OK;
}

int he_cdiag_transpose(he_ctx *ctx, const he_ct *cts, int64_t m, int64_t n, he_ct *outs) {
    if (!ctx || !cts || !outs || !pow2(m) || !pow2(n) || std::max(m, n) > ctx->n / 2) return HE_EINVAL;
    const int64_t lo = std::min(m, n);
    std::vector<std::pair<int64_t, int32_t>> kr((size_t)lo);
    for (int64_t i = 0; i < lo; ++i) {
        int64_t k, r;
        transpose_source(m, n, i, &k, &r);
        kr[(size_t)i] = {k, (int32_t)r};
        if (!cts[k].data || !outs[i].data || outs[i].data == cts[k].data) return HE_EINVAL;
        if (cts[k].level != cts[0].level) return HE_ELEVEL;
    }
    // all rotations in one batch (steps that are multiples of N/2, here r = 0, are copies)
    std::vector<he_ct> ins((size_t)lo);
    std::vector<int32_t> steps((size_t)lo);
    for (int64_t i = 0; i < lo; ++i) {
        ins[(size_t)i] = cts[kr[(size_t)i].first];
        steps[(size_t)i] = kr[(size_t)i].second;
    }
    return he_rotate_many(ctx, ins.data(), steps.data(), (int)lo, outs);
}

int he_cdiag_decode(he_ctx *ctx, int64_t m, int64_t n, int64_t K, const double *slots, double *Z) {
    if (!ctx || !slots || !Z || !pow2(m) || !pow2(n) || K < 1) return HE_EINVAL;
    ctx->launches++;
    launch_k(cdiag_decode_kernel, blocks_for(m * K), 256, 0, ctx->stream, slots, m, n, K, ctx->n / 2, Z);
    return cudaGetLastError() == cudaSuccess ? HE_OK : HE_ECUDA;
}

}  // extern "C"

void cdiag_set_smem_limits(int max_bytes) { cudaFuncSetAttribute(cdiag_rescale_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes); }
