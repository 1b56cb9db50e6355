// he_bconv.cu -- the basis extension of ModUp (hybrid key switching, O3/O4 in Sec. 2.2) on the
// INT8 tensor cores, exact.
//
// For digit d with source primes q_lo..q_hi-1 (alpha_d of them) and a target prime t of
// Q_level U P outside the digit, the fast base conversion is
//     y_t = sum_i v_i h_i  mod t,    v_i = [x_i (Q_d/q_i)^-1]_{q_i},   h_i = (Q_d/q_i) mod t,
// with v_i, h_i < 2^61.  Cutting both into bytes, v_i = sum_a v_{i,a} 2^(8a) and
// h_i = sum_b h_{i,b} 2^(8b), gives sum_i v_i h_i = sum_{s=0..14} C_s 2^(8s) with
//     C_s = sum_i sum_{a+b=s} v_{i,a} h_{i,b},
// a product of a constant byte matrix W[(t, s)][(i, a)] = h_{i, s-a} (0 <= s-a < 8, else 0) and
// the byte matrix V[(i, a)][k] of the coefficients k: an unsigned 8-bit matrix product with
// 32-bit sums, the form the tensor cores take (mma.sync m16n8k32, u8 x u8 -> s32; sm_103a has no
// 8-bit integer kind of tcgen05.mma).  Each C_s is at most 4 * 8 * 255^2 < 2^21, so it is exact,
// and the recombination in three groups of five,
//     Y = lo + mid 2^40 + hi 2^80,  lo = sum_{s<5} C_s 2^(8s),  mid = sum_{s<5} C_{5+s} 2^(8s),
//     hi = sum_{s<5} C_{10+s} 2^(8s)   (each < 2^54),
// reduced as lo mod t + mid (2^40 mod t) + hi (2^80 mod t), is the exact residue y_t: the same
// canonical value as the INT64 engine's sum of products, bit for bit.
//
// Layout: W is K = 32 columns (alpha <= 4 primes x 8 bytes) by 16-row tiles of (target, s) rows;
// the coefficients' V columns are the 32 bytes of their (v_0, .., v_3) words, so a column of B is
// read from shared memory as it lies.  The A fragments of every (level, digit) are built on the
// host at context creation.
#include <string.h>

#include <algorithm>
#include <vector>

#include "he_internal.cuh"
#include "he_ntt.cuh"

namespace {

constexpr int BC_TK = 64;        // coefficients per CTA
constexpr int BC_THREADS = 128;  // 4 warps, two 8-coefficient column tiles each
constexpr int BC_MAX_MT = 23;    // row tiles: up to (HE_MAX_LIMBS - 1) targets x 15 shifts
constexpr int BC_CS = BC_TK + 8; // row stride of the partial sums in shared memory (8 pad words: the
                                 // fragments' 8-byte stores fall on distinct banks)

__host__ __device__ inline uint64_t hd_umulhi(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (uint64_t)(((u128)a * b) >> 64);
#endif
}
__host__ __device__ inline uint64_t hd_shoup(uint64_t x, uint64_t w, uint64_t wp, uint64_t q) {
    const uint64_t r = x * w - hd_umulhi(x, wp) * q;
    return r >= q ? r - q : r;
}
__host__ __device__ inline uint64_t hd_addmod(uint64_t a, uint64_t b, uint64_t q) {
    const uint64_t s = a + b;
    return s >= q ? s - q : s;
}

// y = sum_s C_s 2^(8s) mod q from the 15 partial sums C[s * stride] (each < 2^21)
__host__ __device__ inline uint64_t bconv_recombine(const int32_t *C, int stride, const ModConst &m) {
    uint64_t lo = 0, mid = 0, hi = 0;
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        lo += (uint64_t)(uint32_t)C[s * stride] << (8 * s);
        mid += (uint64_t)(uint32_t)C[(5 + s) * stride] << (8 * s);
        hi += (uint64_t)(uint32_t)C[(10 + s) * stride] << (8 * s);
    }
    uint64_t r = lo - hd_umulhi(lo, m.mu) * m.q;  // Barrett, one correction
    r = r >= m.q ? r - m.q : r;
    r = hd_addmod(r, hd_shoup(mid, m.p40, m.p40_shoup, m.q), m.q);
    return hd_addmod(r, hd_shoup(hi, m.p80, m.p80_shoup, m.q), m.q);
}

// byte (row, col) of the constant matrix W of digit d at a level: row = (target t, shift s),
// col = (source i, byte a)
uint8_t w_byte(const ModUpConst &mu, int d, int row, int col) {
    const int lo = d * mu.alpha, hi = std::min(lo + mu.alpha, mu.nq), al = hi - lo, T = mu.ext - al;
    const int t = row / 15, s = row % 15, i = col / 8, a = col % 8, b = s - a;
    if (t >= T || i >= al || b < 0 || b > 7) return 0;
    const int u = t < lo ? t : t + al;
    return (uint8_t)(mu.hat[d][i][u] >> (8 * b));
}

int row_tiles(const ModUpConst &mu, int d) {
    const int lo = d * mu.alpha, hi = std::min(lo + mu.alpha, mu.nq);
    return ((mu.ext - (hi - lo)) * 15 + 15) / 16;
}

struct BconvArgs {
    RotTable jobs;           // per-job c1 (NTT form) at jobs.j[j].ct + nq N when has_jobs, else c1_ntt
    int32_t has_jobs;
    const uint64_t *c1_ntt;
    const uint64_t *coef;    // c1 in coefficient form, job j at coef + j coef_w
    int64_t coef_w;
    uint64_t *D;             // digits, job j at D + j d_w
    int64_t d_w;
    const uint4 *afrag;      // A fragments of this level: digit d at afrag + aoff[d]
    int32_t aoff[HE_MAX_DNUM];
};

__device__ __forceinline__ void mma_u8(int (&c)[4], const uint4 &a, uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.u8.u8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                 : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
                 : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}

// Grid (ceil(N / BC_TK), ndig, jobs).  Writes the digit's target limbs of D in coefficient form and
// copies its own limbs (NTT form) from c1.
__global__ void __launch_bounds__(BC_THREADS) bconv_i8_kernel(BconvArgs a, ModUpConst mu, const ModConst *__restrict__ mc, int logn) {
    HE_GRID_DEP();
    const int N = 1 << logn;
    const int d = blockIdx.y, j = blockIdx.z, k0 = blockIdx.x * BC_TK;
    const int lo = d * mu.alpha, hi = lo + mu.alpha < mu.nq ? lo + mu.alpha : mu.nq, al = hi - lo, T = mu.ext - al;
    const int MT = (T * 15 + 15) / 16;
    extern __shared__ uint4 smem[];
    uint4 *As = smem;                                                     // [MT][32 lanes]
    uint32_t *Vs = reinterpret_cast<uint32_t *>(As + MT * 32);            // [BC_TK][8]: 32 bytes per coefficient
    int32_t *Cs = reinterpret_cast<int32_t *>(Vs + BC_TK * 8);            // [MT * 16][BC_CS]
    const uint4 *Ag = a.afrag + a.aoff[d];
    for (int x = threadIdx.x; x < MT * 32; x += BC_THREADS) As[x] = Ag[x];
    const uint64_t *coef = a.coef + j * a.coef_w;
    for (int x = threadIdx.x; x < BC_TK * 4; x += BC_THREADS) {
        const int kk = x >> 2, i = x & 3;
        uint64_t v = 0;
        if (i < al && k0 + kk < N) {
            const uint64_t q = mc[lo + i].q;
            v = mul_shoup(coef[(int64_t)(lo + i) * N + k0 + kk], mu.inv[d][i], mu.inv_shoup[d][i], q);
        }
        Vs[kk * 8 + 2 * i] = (uint32_t)v;
        Vs[kk * 8 + 2 * i + 1] = (uint32_t)(v >> 32);
    }
    __syncthreads();
    // warp w: column tiles 2w, 2w+1; lane (g, tg) supplies column g, rows 4tg..4tg+3 and 16+4tg..
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, g = lane >> 2, tg = lane & 3;
    for (int nt = 2 * w; nt < 2 * w + 2; ++nt) {
        const int kk = nt * 8 + g;
        const uint32_t b0 = Vs[kk * 8 + tg], b1 = Vs[kk * 8 + 4 + tg];
        for (int m = 0; m < MT; ++m) {
            int c[4] = {0, 0, 0, 0};
            mma_u8(c, As[m * 32 + lane], b0, b1);
            int32_t *row0 = Cs + (m * 16 + g) * BC_CS + nt * 8 + 2 * tg, *row1 = row0 + 8 * BC_CS;
            row0[0] = c[0];
            row0[1] = c[1];
            row1[0] = c[2];
            row1[1] = c[3];
        }
    }
    __syncthreads();
    const int64_t jd = j * a.d_w;
    for (int x = threadIdx.x; x < T * BC_TK; x += BC_THREADS) {
        const int t = x / BC_TK, kk = x % BC_TK;
        if (k0 + kk >= N) continue;
        const int u = t < lo ? t : t + al;
        a.D[jd + ((int64_t)d * mu.ext + u) * N + k0 + kk] = bconv_recombine(Cs + t * 15 * BC_CS + kk, BC_CS, mc[mu.ext_prime[u]]);
    }
    const uint64_t *c1 = a.has_jobs ? a.jobs.j[j].ct + (int64_t)mu.nq * N : a.c1_ntt;
    for (int x = threadIdx.x; x < al * BC_TK; x += BC_THREADS) {
        const int i = x / BC_TK, kk = x % BC_TK;
        if (k0 + kk >= N) continue;
        a.D[jd + ((int64_t)d * mu.ext + lo + i) * N + k0 + kk] = c1[(int64_t)(lo + i) * N + k0 + kk];
    }
}

// forward NTT, in place, of every digit's target limbs (its own limbs are NTT form already);
// item (j, d, u)
template <bool CL, int LOGN = 0>
__global__ void modup_ntt_kernel(uint64_t *D, int64_t d_w, ModUpConst mu, const uint64_t *__restrict__ d_tw, const ModConst *__restrict__ mc,
                                 int logn_rt) {
    HE_GRID_DEP();
    const int logn = LOGN ? LOGN : logn_rt;
    extern __shared__ uint64_t s[];
    const int N = 1 << logn;
    int item, off, len;
    slice_of<CL>(logn, item, off, len);
    const int per = mu.ndig * mu.ext;
    const int j = item / per, d = (item % per) / mu.ext, u = item % mu.ext;
    const int lo = d * mu.alpha, hi = lo + mu.alpha < mu.nq ? lo + mu.alpha : mu.nq;
    if (u >= lo && u < hi) return;  // uniform over the cluster
    const int p = mu.ext_prime[u];
    const ulonglong2 *tw = twiddles(d_tw, p, 0, logn);
    tw_prefetch<CL, true>(s, tw, logn);
    uint64_t *x = D + j * d_w + ((int64_t)d * mu.ext + u) * N + off;
    stage_in(s, x, len, [](uint64_t v) { return v; });
    __syncthreads();
    fwd_any<CL, LOGN>(s, tw, mc[p].q, logn);
    for (int k = threadIdx.x; k < len; k += blockDim.x) x[k] = s[SIDX(k)];
}

size_t bconv_smem_bytes(int mt) { return (size_t)mt * 32 * 16 + (size_t)BC_TK * 32 + (size_t)mt * 16 * BC_CS * 4; }

}  // namespace

int bconv_i8_tables(he_ctx *ctx) {
    std::vector<uint32_t> tab;
    ctx->bconv_a_off.assign((size_t)ctx->L * ctx->dnum, 0);
    for (int level = 0; level < ctx->L; ++level) {
        const ModUpConst &mu = ctx->modup[level];
        for (int d = 0; d < mu.ndig; ++d) {
            ctx->bconv_a_off[(size_t)level * ctx->dnum + d] = tab.size() / 4;
            const int MT = row_tiles(mu, d);
            if (MT > BC_MAX_MT) return HE_EINVAL;
            for (int m = 0; m < MT; ++m)
                for (int lane = 0; lane < 32; ++lane) {
                    const int g = lane >> 2, tg = lane & 3;
                    for (int reg = 0; reg < 4; ++reg) {  // rows g (regs 0, 2), g + 8 (1, 3); cols 4tg.. (0, 1), 16 + 4tg.. (2, 3)
                        const int row = m * 16 + g + (reg & 1) * 8, col = tg * 4 + (reg >> 1) * 16;
                        uint32_t word = 0;
                        for (int b = 0; b < 4; ++b) word |= (uint32_t)w_byte(mu, d, row, col + b) << (8 * b);
                        tab.push_back(word);
                    }
                }
        }
    }
    if (tab.empty()) return HE_OK;
    if (cudaMalloc(&ctx->d_bconv_a, tab.size() * 4) != cudaSuccess) return HE_ENOMEM;
    ctx->sh->owned[5] = ctx->d_bconv_a;
    return cudaMemcpy(ctx->d_bconv_a, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice) == cudaSuccess ? HE_OK : HE_ECUDA;
}

void launch_modup_i8(he_ctx *ctx, const RotTable *jobs, int count, int level, const uint64_t *c1_ntt, const uint64_t *coef, int64_t coef_w,
                     uint64_t *D, int64_t d_w) {
    if (count == 0) return;
    const ModUpConst &mu = ctx->modup[level];
    BconvArgs a{};
    if (jobs) {
        a.jobs = *jobs;
        a.has_jobs = 1;
    }
    a.c1_ntt = c1_ntt;
    a.coef = coef;
    a.coef_w = coef_w;
    a.D = D;
    a.d_w = d_w;
    a.afrag = reinterpret_cast<const uint4 *>(ctx->d_bconv_a);
    int mt = 0;
    for (int d = 0; d < mu.ndig; ++d) {
        a.aoff[d] = (int32_t)ctx->bconv_a_off[(size_t)level * ctx->dnum + d];
        mt = std::max(mt, row_tiles(mu, d));
    }
    const int logn = ctx->log_n;
    ctx->launches += 2;
    launch_k(bconv_i8_kernel, dim3((unsigned)((ctx->n + BC_TK - 1) / BC_TK), (unsigned)mu.ndig, (unsigned)count), BC_THREADS, bconv_smem_bytes(mt), ctx->stream,
             a, mu, ctx->d_mc, logn);
    const int items = count * mu.ndig * mu.ext;
    if (use_cluster(logn, items))
        launch_cluster(by_logn(logn, [](auto L) { return modup_ntt_kernel<true, L.value>; }), items * HE_NTT_CL_SIZE, cl_threads(logn), cl_smem_bytes(logn),
                       ctx->stream, D, d_w, mu, (const uint64_t *)ctx->d_tw, (const ModConst *)ctx->d_mc, logn);
    else
        launch_k(by_logn(logn, [](auto L) { return modup_ntt_kernel<false, L.value>; }), items, ntt_threads(logn), ntt_smem_bytes(logn), ctx->stream, D,
                 d_w, mu, (const uint64_t *)ctx->d_tw, (const ModConst *)ctx->d_mc, logn);
}

void bconv_set_smem_limits(int max_bytes) {
    cudaFuncSetAttribute(bconv_i8_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
    each_logn([max_bytes](auto L) {
        cudaFuncSetAttribute(modup_ntt_kernel<true, L.value>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
        cudaFuncSetAttribute(modup_ntt_kernel<false, L.value>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
    });
}

extern "C" {

int he_set_basis_extension(he_ctx *ctx, int engine) {
    if (!ctx || (engine != HE_BCONV_INT64 && engine != HE_BCONV_INT8_TC)) return HE_EINVAL;
    if (engine == HE_BCONV_INT8_TC && !ctx->d_bconv_a) return HE_EINVAL;
    ctx->bconv = engine;
    return HE_OK;
}

int he_get_basis_extension(const he_ctx *ctx, int *engine) {
    if (!ctx || !engine) return HE_EINVAL;
    *engine = ctx->bconv;
    return HE_OK;
}

int he_bconv_i8_host(int alpha, const uint64_t *v, const uint64_t *h, uint64_t t, uint64_t *out) {
    if (alpha < 1 || alpha > 4 || !v || !h || !out || t < 3 || t >= (1ull << 62)) return HE_EINVAL;
    // the byte products' sums C_s as the tensor cores form them, then the kernel's recombination
    int32_t C[15] = {};
    for (int i = 0; i < alpha; ++i)
        for (int a = 0; a < 8; ++a)
            for (int b = 0; b < 8; ++b) C[a + b] += (int32_t)((v[i] >> (8 * a)) & 255) * (int32_t)((h[i] >> (8 * b)) & 255);
    ModConst m{};
    m.q = t;
    m.mu = (uint64_t)((((u128)1) << 64) / t);
    const uint64_t r40 = (uint64_t)((((u128)1) << 40) % t);
    m.p40 = r40;
    m.p40_shoup = (uint64_t)(((u128)r40 << 64) / t);
    m.p80 = (uint64_t)((u128)r40 * r40 % t);
    m.p80_shoup = (uint64_t)(((u128)m.p80 << 64) / t);
    *out = bconv_recombine(C, 1, m);
    return HE_OK;
}

}  // extern "C"
