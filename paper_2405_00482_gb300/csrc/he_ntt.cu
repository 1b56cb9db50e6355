// he_ntt.cu -- batched negacyclic NTT / inverse NTT kernels over RNS limbs.
//
// One CTA transforms one limb-poly of N residues staged in shared memory (8N bytes).
// Batch layout: limb l of group g sits at base + g * group_stride + l * N, with prime
// index map.prime[l].  Grid = groups * map.n CTAs.
#include <algorithm>
#include <type_traits>

#include "he_internal.cuh"
#include "he_ntt.cuh"

namespace {

// LOGN > 0: the ring size at compile time (logn_rt == LOGN); 0: at run time
template <bool CL, int LOGN = 0>
__global__ void ntt_fwd_kernel(const uint64_t *__restrict__ in, int64_t in_gs, uint64_t *out, int64_t out_gs, LimbMap map,
                               const uint64_t *__restrict__ d_tw, const ModConst *__restrict__ mc, int logn_rt, int to_mont) {
    HE_GRID_DEP();
    const int logn = LOGN ? LOGN : logn_rt;
    extern __shared__ uint64_t s[];
    const int N = 1 << logn;
    int poly, off, len;
    slice_of<CL>(logn, poly, off, len);
    const int g = poly / map.n, l = poly % map.n;
    const int p = map.prime[l];
    const uint64_t q = mc[p].q;
    tw_prefetch<CL, true>(s, twiddles(d_tw, p, 0, logn), logn);
    const uint64_t *src = in + g * in_gs + (int64_t)l * N + off;
    stage_in(s, src, len, [](uint64_t v) { return v; });
    __syncthreads();
    fwd_any<CL, LOGN>(s, twiddles(d_tw, p, 0, logn), q, logn);
    uint64_t *dst = out + g * out_gs + (int64_t)l * N + off;
    if (to_mont) {  // x 2^64 mod q: one Shoup product by the constant 2^64 mod q
        const uint64_t r1 = mc[p].r1, r1s = mc[p].r1_shoup;
        for (int k = threadIdx.x; k < len; k += blockDim.x) dst[k] = mul_shoup(s[SIDX(k)], r1, r1s, q);
    } else {
        for (int k = threadIdx.x; k < len; k += blockDim.x) dst[k] = s[SIDX(k)];
    }
}

template <bool CL, int LOGN = 0>
__global__ void ntt_inv_kernel(const uint64_t *__restrict__ in, int64_t in_gs, uint64_t *out, int64_t out_gs, LimbMap map,
                               const uint64_t *__restrict__ d_tw, const ModConst *__restrict__ mc, int logn_rt) {
    HE_GRID_DEP();
    const int logn = LOGN ? LOGN : logn_rt;
    extern __shared__ uint64_t s[];
    const int N = 1 << logn;
    int poly, off, len;
    slice_of<CL>(logn, poly, off, len);
    const int g = poly / map.n, l = poly % map.n;
    const int p = map.prime[l];
    const uint64_t q = mc[p].q;
    tw_prefetch<CL, false>(s, twiddles(d_tw, p, 1, logn), logn);
    const uint64_t *src = in + g * in_gs + (int64_t)l * N + off;
    stage_in(s, src, len, [](uint64_t v) { return v; });
    __syncthreads();
    inv_any<CL, LOGN>(s, twiddles(d_tw, p, 1, logn), q, logn);
    uint64_t *dst = out + g * out_gs + (int64_t)l * N + off;
    const uint64_t ni = mc[p].ninv, nis = mc[p].ninv_shoup;
    for (int k = threadIdx.x; k < len; k += blockDim.x) dst[k] = mul_shoup(s[SIDX(k)], ni, nis, q);
}

// signed int64 coefficients of group g, reduced mod each limb's prime, then forward NTT.
template <bool CL, int LOGN = 0>
__global__ void ntt_from_int64_kernel(const int64_t *__restrict__ in, uint64_t *out, LimbMap map, const uint64_t *__restrict__ d_tw,
                                      const ModConst *__restrict__ mc, int logn_rt, int to_mont) {
    HE_GRID_DEP();
    const int logn = LOGN ? LOGN : logn_rt;
    extern __shared__ uint64_t s[];
    const int N = 1 << logn;
    int poly, off, len;
    slice_of<CL>(logn, poly, off, len);
    const int g = poly / map.n, l = poly % map.n;
    const int p = map.prime[l];
    const uint64_t q = mc[p].q;
    tw_prefetch<CL, true>(s, twiddles(d_tw, p, 0, logn), logn);
    const int64_t *src = in + (int64_t)g * N + off;
    const uint64_t mu = mc[p].mu;
    stage_in(s, src, len, [q, mu](int64_t v) { return reduce_signed(v, q, mu); });
    __syncthreads();
    fwd_any<CL, LOGN>(s, twiddles(d_tw, p, 0, logn), q, logn);
    uint64_t *dst = out + ((int64_t)g * map.n + l) * N + off;
    if (to_mont) {  // x 2^64 mod q: one Shoup product by the constant 2^64 mod q
        const uint64_t r1 = mc[p].r1, r1s = mc[p].r1_shoup;
        for (int k = threadIdx.x; k < len; k += blockDim.x) dst[k] = mul_shoup(s[SIDX(k)], r1, r1s, q);
    } else {
        for (int k = threadIdx.x; k < len; k += blockDim.x) dst[k] = s[SIDX(k)];
    }
}

// ---- pair forms (two CTAs per limb-poly, he_ntt.cuh): the same operations as the kernels above ----
// Launch bounds: pair_threads(LOGN) threads, registers for three CTAs of 256 threads per SM at
// N = 2^13 (at most 85; at 64 the passes spill)
__device__ __forceinline__ int pair_rank() { return (int)cg::this_cluster().block_rank(); }
#define PAIR_BOUNDS(LOGN) __launch_bounds__(pair_threads_c(LOGN), 768 / pair_threads_c(LOGN))

template <int LOGN>
__global__ void PAIR_BOUNDS(LOGN) ntt_fwd_pair_kernel(const uint64_t *__restrict__ in, int64_t in_gs, uint64_t *out, int64_t out_gs, LimbMap map,
                                                           const uint64_t *__restrict__ d_tw, const ModConst *__restrict__ mc, int to_mont) {
    HE_GRID_DEP();
    extern __shared__ uint64_t s[];
    constexpr int N = 1 << LOGN, NS = N / 2;
    const int poly = blockIdx.x / 2, off = pair_rank() * NS;
    const int g = poly / map.n, l = poly % map.n, p = map.prime[l];
    const uint64_t q = mc[p].q;
    stage_in(s, in + g * in_gs + (int64_t)l * N + off, NS, [](uint64_t v) { return v; });
    ntt_fwd_pair<LOGN>(s, twiddles(d_tw, p, 0, LOGN), q);
    uint64_t *dst = out + g * out_gs + (int64_t)l * N + off;
    if (to_mont) {
        const uint64_t r1 = mc[p].r1, r1s = mc[p].r1_shoup;
        for (int k = threadIdx.x; k < NS; k += blockDim.x) dst[k] = mul_shoup(s[SIDX(k)], r1, r1s, q);
    } else {
        for (int k = threadIdx.x; k < NS; k += blockDim.x) dst[k] = s[SIDX(k)];
    }
}

template <int LOGN>
__global__ void PAIR_BOUNDS(LOGN) ntt_inv_pair_kernel(const uint64_t *__restrict__ in, int64_t in_gs, uint64_t *out, int64_t out_gs, LimbMap map,
                                                           const uint64_t *__restrict__ d_tw, const ModConst *__restrict__ mc) {
    HE_GRID_DEP();
    extern __shared__ uint64_t s[];
    constexpr int N = 1 << LOGN, NS = N / 2;
    const int poly = blockIdx.x / 2, off = pair_rank() * NS;
    const int g = poly / map.n, l = poly % map.n, p = map.prime[l];
    const uint64_t q = mc[p].q;
    stage_in(s, in + g * in_gs + (int64_t)l * N + off, NS, [](uint64_t v) { return v; });
    ntt_inv_pair<LOGN>(s, twiddles(d_tw, p, 1, LOGN), q);
    uint64_t *dst = out + g * out_gs + (int64_t)l * N + off;
    const uint64_t ni = mc[p].ninv, nis = mc[p].ninv_shoup;
    for (int k = threadIdx.x; k < NS; k += blockDim.x) dst[k] = mul_shoup(s[SIDX(k)], ni, nis, q);
}

template <int LOGN>
__global__ void PAIR_BOUNDS(LOGN) ntt_from_int64_pair_kernel(const int64_t *__restrict__ in, uint64_t *out, LimbMap map,
                                                                  const uint64_t *__restrict__ d_tw, const ModConst *__restrict__ mc, int to_mont) {
    HE_GRID_DEP();
    extern __shared__ uint64_t s[];
    constexpr int N = 1 << LOGN, NS = N / 2;
    const int poly = blockIdx.x / 2, off = pair_rank() * NS;
    const int g = poly / map.n, l = poly % map.n, p = map.prime[l];
    const uint64_t q = mc[p].q, mu = mc[p].mu;
    stage_in(s, in + (int64_t)g * N + off, NS, [q, mu](int64_t v) { return reduce_signed(v, q, mu); });
    ntt_fwd_pair<LOGN>(s, twiddles(d_tw, p, 0, LOGN), q);
    uint64_t *dst = out + ((int64_t)g * map.n + l) * N + off;
    if (to_mont) {
        const uint64_t r1 = mc[p].r1, r1s = mc[p].r1_shoup;
        for (int k = threadIdx.x; k < NS; k += blockDim.x) dst[k] = mul_shoup(s[SIDX(k)], r1, r1s, q);
    } else {
        for (int k = threadIdx.x; k < NS; k += blockDim.x) dst[k] = s[SIDX(k)];
    }
}

// out = data 2^-64 mod q (Montgomery form back to canonical); grid (blocks, groups, limbs)
// ---- two-phase form (he_set_ntt_form 2): the bodies are in he_ntt.cuh ----
template <int LOGN, bool I64>
__global__ void __launch_bounds__(NTT2_THREADS, 8) ntt2_cols_kernel(const void *__restrict__ in_v, int64_t in_gs, uint64_t *out, int64_t out_gs,
                                                                  LimbMap map, const uint64_t *__restrict__ d_tw, const ModConst *__restrict__ mc,
                                                                  int to_mont) {
    HE_GRID_DEP();
    constexpr int N = 1 << LOGN, TILES = (N >> 6) / NTT2_TC;
    __shared__ uint64_t sm[ntt2_cols_smem_words()];
    const int poly = blockIdx.x / TILES, c0 = (blockIdx.x % TILES) * NTT2_TC;
    const int g = poly / map.n, l = poly % map.n, p = map.prime[l];
    const uint64_t q = mc[p].q, r1 = mc[p].r1, r1s = mc[p].r1_shoup, mu = mc[p].mu;
    uint64_t *dst = out + g * out_gs + (int64_t)l * N;
    if constexpr (I64) {  // int64 coefficients, shared by the limbs of group g, reduced mod q
        const int64_t *src = static_cast<const int64_t *>(in_v) + g * in_gs;
        ntt2_fwd_cols<LOGN>(sm, [=](int64_t x) { return to_mont ? signed_to_mont(src[x], r1, r1s, q) : reduce_signed(src[x], q, mu); }, dst, c0,
                            TwGlobal{twiddles(d_tw, p, 0, LOGN)}, q);
    } else {
        const uint64_t *src = static_cast<const uint64_t *>(in_v) + g * in_gs + (int64_t)l * N;
        ntt2_fwd_cols<LOGN>(sm, [=](int64_t x) { return to_mont ? mul_shoup(src[x], r1, r1s, q) : src[x]; }, dst, c0,
                            TwGlobal{twiddles(d_tw, p, 0, LOGN)}, q);
    }
}

template <int LOGN>
__global__ void __launch_bounds__(NTT2_THREADS, 8) ntt2_rows_kernel(uint64_t *data, int64_t gs, LimbMap map, const uint64_t *__restrict__ d_tw,
                                                                  const ModConst *__restrict__ mc) {
    HE_GRID_DEP();
    constexpr int N = 1 << LOGN, TILES = 64 / NTT2_TR;
    __shared__ uint64_t sm[ntt2_frows_smem_words(LOGN - 6)];
    const int poly = blockIdx.x / TILES, b0 = (blockIdx.x % TILES) * NTT2_TR;
    const int g = poly / map.n, l = poly % map.n, p = map.prime[l];
    ntt2_fwd_rows<LOGN>(sm, data + g * gs + (int64_t)l * N, b0, TwGlobal{twiddles(d_tw, p, 0, LOGN)}, mc[p].q, mc[p].mu);
}

// inverse: rows (in to out), then columns in place with the factor N^-1
template <int LOGN, int NBA>
__global__ void __launch_bounds__(NTT2_THREADS) ntt2_inv_rows_kernel(const uint64_t *__restrict__ in, int64_t in_gs, uint64_t *out, int64_t out_gs,
                                                                   LimbMap map, const uint64_t *__restrict__ d_tw, const ModConst *__restrict__ mc) {
    HE_GRID_DEP();
    constexpr int N = 1 << LOGN, TILES = 64 / NTT2_TR;
    __shared__ uint64_t sm[ntt2_rows_smem_words(LOGN - 6)];
    const int poly = blockIdx.x / TILES, b0 = (blockIdx.x % TILES) * NTT2_TR;
    const int g = poly / map.n, l = poly % map.n, p = map.prime[l];
    ntt2_inv_rows<LOGN, NBA>(sm, in + g * in_gs + (int64_t)l * N, out + g * out_gs + (int64_t)l * N, b0, TwGlobal{twiddles(d_tw, p, 1, LOGN)},
                             mc[p].q);
}

template <int LOGN>
__global__ void __launch_bounds__(NTT2_THREADS, 8) ntt2_inv_cols_kernel(uint64_t *data, int64_t gs, LimbMap map, const uint64_t *__restrict__ d_tw,
                                                                      const ModConst *__restrict__ mc) {
    HE_GRID_DEP();
    constexpr int N = 1 << LOGN, TILES = (N >> 6) / NTT2_TC;
    __shared__ uint64_t sm[ntt2_cols_smem_words()];
    const int poly = blockIdx.x / TILES, c0 = (blockIdx.x % TILES) * NTT2_TC;
    const int g = poly / map.n, l = poly % map.n, p = map.prime[l];
    const uint64_t q = mc[p].q, ni = mc[p].ninv, nis = mc[p].ninv_shoup;
    uint64_t *x = data + g * gs + (int64_t)l * N;
    ntt2_inv_cols<LOGN>(sm, x, c0, TwGlobal{twiddles(d_tw, p, 1, LOGN)}, q, [=](int64_t k, uint64_t v) { x[k] = mul_shoup(v, ni, nis, q); });
}

__global__ void from_mont_kernel(const uint64_t *__restrict__ data, uint64_t *out, LimbMap map, const ModConst *__restrict__ mc, int logn) {
    HE_GRID_DEP();
    const int N = 1 << logn;
    const int g = blockIdx.y, l = blockIdx.z;
    const int p = map.prime[l];
    const int64_t base = ((int64_t)g * map.n + l) * N;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) out[base + k] = mont_mul(data[base + k], 1, mc[p].q, mc[p].qinv);
}

__global__ void to_mont_kernel(uint64_t *data, LimbMap map, const ModConst *__restrict__ mc, int logn) {
    HE_GRID_DEP();
    const int N = 1 << logn;
    const int g = blockIdx.y, l = blockIdx.z;
    const int p = map.prime[l];
    uint64_t *d = data + ((int64_t)g * map.n + l) * N;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) d[k] = mont_mul(d[k], mc[p].r2, mc[p].q, mc[p].qinv);
}

}  // namespace

// One-CTA form: N/16 threads (one radix-16 set each) up to 256, so that two CTAs (two limb-polys)
// share an SM and one's barriers overlap the other's work (the passes use ~110 registers); from
// N = 2^14 a limb-poly's shared memory allows one CTA per SM, which then takes 512 threads.
// (Radix-8 passes need ~72 registers and fit three CTAs per SM at N = 2^13, but the extra pass
// made the N = 2^13 plain step 2% slower on GB300.)
// Threads loop over several sets when there are more sets than threads.
// cluster form for launches of at most this many limb-polys (one CTA each would leave most SMs idle)
#define HE_CL_MAX_POLYS 48

bool use_cluster(int logn, int polys) { return logn >= HE_NTT_CL_MIN_LOGN && polys <= HE_CL_MAX_POLYS; }
int cl_threads(int logn) { return std::min(512, 1 << (logn - 3 - HE_NTT_CL_RADIX_LOG)); }
// the slice's padded data, then its N/8 - 1 twiddle pairs (16-byte aligned: N/8 + N/256 is even)
size_t cl_smem_bytes(int logn) { return ntt_smem_bytes(logn - 3) + ((size_t)16 << (logn - 3)); }

int ntt_threads(int logn) {
    if (logn <= HE_NTT_RADIX_LOG) return 1;
    const int sets = 1 << (logn - HE_NTT_RADIX_LOG);
    const int cap = logn >= 14 ? 512 : 256;
    return sets < cap ? sets : cap;
}

// the pair form instance for a compile-time ring size (nullptr: none, use the one-CTA form)
template <class F>
static auto pair_instance(int logn, F f) {
    using K = decltype(f(std::integral_constant<int, 13>{}));
    switch (logn) {
        case 12: return f(std::integral_constant<int, 12>{});
        case 13: return f(std::integral_constant<int, 13>{});
        case 14: return f(std::integral_constant<int, 14>{});
        default: return (K) nullptr;
    }
}

bool use_pair(const he_ctx *ctx, int polys) { return ctx->ntt_form == 1 && !use_cluster(ctx->log_n, polys) && ctx->log_n >= 12 && ctx->log_n <= 14; }
bool use_two_phase(const he_ctx *ctx, int polys) {
    return ctx->ntt_form == 2 && !use_cluster(ctx->log_n, polys) && ctx->log_n >= 12 && ctx->log_n <= 14;
}

// the two launches of the two-phase forward transform (from int64 coefficients when I64)
template <bool I64>
static void launch_two_phase(he_ctx *ctx, const void *in, int64_t in_gs, uint64_t *out, int64_t out_gs, int polys, const LimbMap &map, int to_mont) {
    const int logn = ctx->log_n, C = ctx->n >> 6;
    const unsigned cols = (unsigned)(polys * (C / NTT2_TC)), rows = (unsigned)(polys * (64 / NTT2_TR));
    const uint64_t *tw = ctx->d_tw;
    const ModConst *mc = ctx->d_mc;
    ctx->launches += 2;
    auto go = [&](auto L, auto NB1) {
        launch_k(ntt2_cols_kernel<decltype(L)::value, I64>, cols, NTT2_THREADS, 0, ctx->stream, in, in_gs, out, out_gs, map, tw, mc, to_mont);
        launch_k(ntt2_rows_kernel<decltype(L)::value>, rows, NTT2_THREADS, 0, ctx->stream, out, out_gs, map, tw, mc);
    };
    if (logn == 12) go(std::integral_constant<int, 12>{}, std::integral_constant<int, 3>{});
    else if (logn == 13) go(std::integral_constant<int, 13>{}, std::integral_constant<int, 4>{});
    else go(std::integral_constant<int, 14>{}, std::integral_constant<int, 4>{});
}

void launch_ntt_fwd_strided(he_ctx *ctx, const uint64_t *in, int64_t in_gs, uint64_t *out, int64_t out_gs, int groups,
                            const LimbMap &map, int to_mont) {
    if (groups * map.n == 0) return;
    if (use_two_phase(ctx, groups * map.n)) {
        launch_two_phase<false>(ctx, in, in_gs, out, out_gs, groups * map.n, map, to_mont);
        return;
    }
    ctx->launches++;
    if (use_pair(ctx, groups * map.n)) {
        launch_cluster_n(pair_instance(ctx->log_n, [](auto L) { return ntt_fwd_pair_kernel<L.value>; }), groups * map.n * 2, pair_threads(ctx->log_n),
                         pair_smem_bytes(ctx->log_n), ctx->stream, 2, in, in_gs, out, out_gs, map, (const uint64_t *)ctx->d_tw,
                         (const ModConst *)ctx->d_mc, to_mont);
        return;
    }
    const int polys = groups * map.n;
    if (use_cluster(ctx->log_n, polys))
        launch_cluster(by_logn(ctx->log_n, [](auto L) { return ntt_fwd_kernel<true, L.value>; }), polys * HE_NTT_CL, cl_threads(ctx->log_n),
                       cl_smem_bytes(ctx->log_n), ctx->stream, in, in_gs, out, out_gs, map, ctx->d_tw, ctx->d_mc, ctx->log_n, to_mont);
    else
        launch_k(by_logn(ctx->log_n, [](auto L) { return ntt_fwd_kernel<false, L.value>; }), polys, ntt_threads(ctx->log_n), ntt_smem_bytes(ctx->log_n),
                 ctx->stream, in, in_gs, out, out_gs, map, ctx->d_tw, ctx->d_mc, ctx->log_n, to_mont);
}

void launch_ntt_inv_strided(he_ctx *ctx, const uint64_t *in, int64_t in_gs, uint64_t *out, int64_t out_gs, int groups, const LimbMap &map) {
    if (groups * map.n == 0) return;
    if (use_two_phase(ctx, groups * map.n)) {
        const int polys = groups * map.n, C = ctx->n >> 6;
        const unsigned cols = (unsigned)(polys * (C / NTT2_TC)), rows = (unsigned)(polys * (64 / NTT2_TR));
        const uint64_t *tw = ctx->d_tw;
        const ModConst *mc = ctx->d_mc;
        ctx->launches += 2;
        auto go = [&](auto L, auto NBA) {
            launch_k(ntt2_inv_rows_kernel<decltype(L)::value, decltype(NBA)::value>, rows, NTT2_THREADS, 0, ctx->stream, in, in_gs, out, out_gs, map, tw,
                     mc);
            launch_k(ntt2_inv_cols_kernel<decltype(L)::value>, cols, NTT2_THREADS, 0, ctx->stream, out, out_gs, map, tw, mc);
        };
        if (ctx->log_n == 12) go(std::integral_constant<int, 12>{}, std::integral_constant<int, 3>{});
        else if (ctx->log_n == 13) go(std::integral_constant<int, 13>{}, std::integral_constant<int, 3>{});
        else go(std::integral_constant<int, 14>{}, std::integral_constant<int, 4>{});
        return;
    }
    ctx->launches++;
    if (use_pair(ctx, groups * map.n)) {
        launch_cluster_n(pair_instance(ctx->log_n, [](auto L) { return ntt_inv_pair_kernel<L.value>; }), groups * map.n * 2, pair_threads(ctx->log_n),
                         pair_smem_bytes(ctx->log_n), ctx->stream, 2, in, in_gs, out, out_gs, map, (const uint64_t *)ctx->d_tw,
                         (const ModConst *)ctx->d_mc);
        return;
    }
    const int polys = groups * map.n;
    if (use_cluster(ctx->log_n, polys))
        launch_cluster(by_logn(ctx->log_n, [](auto L) { return ntt_inv_kernel<true, L.value>; }), polys * HE_NTT_CL, cl_threads(ctx->log_n),
                       cl_smem_bytes(ctx->log_n), ctx->stream, in, in_gs, out, out_gs, map, ctx->d_tw, ctx->d_mc, ctx->log_n);
    else
        launch_k(by_logn(ctx->log_n, [](auto L) { return ntt_inv_kernel<false, L.value>; }), polys, ntt_threads(ctx->log_n), ntt_smem_bytes(ctx->log_n),
                 ctx->stream, in, in_gs, out, out_gs, map, ctx->d_tw, ctx->d_mc, ctx->log_n);
}

void launch_from_mont(he_ctx *ctx, const uint64_t *data, uint64_t *out, int groups, const LimbMap &map) {
    if (groups * map.n == 0) return;
    ctx->launches++;
    launch_k(from_mont_kernel, dim3((unsigned)((ctx->n + 255) / 256), (unsigned)groups, (unsigned)map.n), 256, 0, ctx->stream, data, out, map, ctx->d_mc,
                                                                                                                     ctx->log_n);
}

void launch_ntt_fwd(he_ctx *ctx, const uint64_t *in, uint64_t *out, int groups, const LimbMap &map) {
    int64_t gs = (int64_t)map.n * ctx->n;
    launch_ntt_fwd_strided(ctx, in, gs, out, gs, groups, map, 0);
}

void launch_ntt_inv(he_ctx *ctx, const uint64_t *in, uint64_t *out, int groups, const LimbMap &map) {
    int64_t gs = (int64_t)map.n * ctx->n;
    launch_ntt_inv_strided(ctx, in, gs, out, gs, groups, map);
}

void launch_ntt_from_int64(he_ctx *ctx, const int64_t *in, uint64_t *out, int groups, const LimbMap &map, int to_mont) {
    if (groups * map.n == 0) return;
    const int polys = groups * map.n;
    if (use_two_phase(ctx, polys)) {
        launch_two_phase<true>(ctx, in, ctx->n, out, (int64_t)map.n * ctx->n, polys, map, to_mont);
        return;
    }
    ctx->launches++;
    if (use_pair(ctx, polys)) {
        launch_cluster_n(pair_instance(ctx->log_n, [](auto L) { return ntt_from_int64_pair_kernel<L.value>; }), polys * 2, pair_threads(ctx->log_n),
                         pair_smem_bytes(ctx->log_n), ctx->stream, 2, in, out, map, (const uint64_t *)ctx->d_tw, (const ModConst *)ctx->d_mc, to_mont);
        return;
    }
    if (use_cluster(ctx->log_n, polys))
        launch_cluster(by_logn(ctx->log_n, [](auto L) { return ntt_from_int64_kernel<true, L.value>; }), polys * HE_NTT_CL, cl_threads(ctx->log_n),
                       cl_smem_bytes(ctx->log_n), ctx->stream, in, out, map, ctx->d_tw, ctx->d_mc, ctx->log_n, to_mont);
    else {
        auto k = by_logn(ctx->log_n, [](auto L) { return ntt_from_int64_kernel<false, L.value>; });
        // 72 registers: three CTAs fit on an SM, so in a multi-stream step the other streams'
        // kernels find room beside it (capping it at two per SM made the encoded matrix alone
        // faster, 80 against 95 us, and the benchmark step 3% slower)
        launch_k(k, polys, ntt_threads(ctx->log_n), ntt_smem_bytes(ctx->log_n), ctx->stream, in, out, map, ctx->d_tw, ctx->d_mc, ctx->log_n, to_mont);
    }
}

void launch_to_mont(he_ctx *ctx, uint64_t *data, int groups, const LimbMap &map) {
    if (groups * map.n == 0) return;
    dim3 grid((ctx->n + 255) / 256, groups, map.n);
    ctx->launches++;
    launch_k(to_mont_kernel, grid, 256, 0, ctx->stream, data, map, ctx->d_mc, ctx->log_n);
}

void ntt_set_smem_limits(int max_bytes) {
    // one-CTA forms, and the cluster forms (slice plus its twiddles: above 48 KB from N = 2^14)
    each_logn([max_bytes](auto L) {
        cudaFuncSetAttribute(ntt_fwd_kernel<false, L.value>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
        cudaFuncSetAttribute(ntt_inv_kernel<false, L.value>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
        cudaFuncSetAttribute(ntt_from_int64_kernel<false, L.value>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
        cudaFuncSetAttribute(ntt_fwd_kernel<true, L.value>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
        cudaFuncSetAttribute(ntt_inv_kernel<true, L.value>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
        cudaFuncSetAttribute(ntt_from_int64_kernel<true, L.value>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
    });
    for (int logn : {12, 13, 14}) {
        cudaFuncSetAttribute(pair_instance(logn, [](auto L) { return ntt_fwd_pair_kernel<L.value>; }), cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
        cudaFuncSetAttribute(pair_instance(logn, [](auto L) { return ntt_inv_pair_kernel<L.value>; }), cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
        cudaFuncSetAttribute(pair_instance(logn, [](auto L) { return ntt_from_int64_pair_kernel<L.value>; }), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             max_bytes);
    }
}
