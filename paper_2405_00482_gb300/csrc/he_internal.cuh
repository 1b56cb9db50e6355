// he_internal.cuh -- internal definitions of the GB300 RNS-CKKS / PackVFL library.
//
// Data layout in HBM (all residues uint64, canonical in [0, q)):
//   limb-poly     [N] in NTT form, bit-reversed order: slot k holds a(psi^(2 brv(k) + 1))
//   ciphertext    [2][level+1][N]   (c0, c1)
//   Galois key    [dnum][2][L+K][N] (b_d, a_d), Montgomery form (x * 2^64 mod q)
//   MatMult plaintexts [R][C][m'][level+1+K][N], Montgomery form
// Montgomery form is used for operands that are fixed while a hot loop reads them,
// so that one REDC returns a canonical product.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <memory>
#include <type_traits>
#include <mutex>
#include <vector>

#include "../../include/he.h"

#define HE_MAX_LIMBS 24   // Q primes + P primes
#define HE_MAX_Q 16
#define HE_MAX_P 8
#define HE_MAX_DNUM 8

typedef unsigned __int128 u128;

// ------------------------------------------------------------------------------------------
// modular arithmetic (device)
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t add_mod(uint64_t a, uint64_t b, uint64_t q) {
    uint64_t s = a + b;
    return s >= q ? s - q : s;
}
__device__ __forceinline__ uint64_t sub_mod(uint64_t a, uint64_t b, uint64_t q) { return a >= b ? a - b : a + q - b; }

// Shoup: x * w mod q with wp = floor(w 2^64 / q); valid for any x < 2^64, q < 2^63
__device__ __forceinline__ uint64_t mul_shoup(uint64_t x, uint64_t w, uint64_t wp, uint64_t q) {
    uint64_t hi = __umul64hi(x, wp);
    uint64_t r = x * w - hi * q;
    return r >= q ? r - q : r;
}
// lazy variant, result in [0, 2q)
__device__ __forceinline__ uint64_t mul_shoup_lazy(uint64_t x, uint64_t w, uint64_t wp, uint64_t q) {
    return x * w - __umul64hi(x, wp) * q;
}

// Montgomery reduction of T = hi 2^64 + lo < q 2^64: returns T 2^-64 mod q in [0, q).
// qinv = -q^-1 mod 2^64.
__device__ __forceinline__ uint64_t redc(uint64_t hi, uint64_t lo, uint64_t q, uint64_t qinv) {
    uint64_t m = lo * qinv;
    uint64_t r = hi + __umul64hi(m, q) + (lo != 0);
    return r >= q ? r - q : r;
}
__device__ __forceinline__ uint64_t redc128(u128 t, uint64_t q, uint64_t qinv) {
    return redc((uint64_t)(t >> 64), (uint64_t)t, q, qinv);
}
// How many products of two residues below q a 128-bit sum may take before redc128, whose input
// must stay below q 2^64: 2^(64 - bits(q)) (8 for 61-bit primes, 2^24 for 40-bit ones; capped)
__device__ __forceinline__ int lazy_terms(uint64_t q) {
    const int b = 64 - __clzll((long long)q);
    return 1 << (64 - b < 24 ? 64 - b : 24);
}
// a * bM 2^-64 mod q  (bM in Montgomery form -> canonical product)
__device__ __forceinline__ uint64_t mont_mul(uint64_t a, uint64_t bM, uint64_t q, uint64_t qinv) {
    return redc128((u128)a * bM, q, qinv);
}

// Barrett reduction (Barrett, CRYPTO '86) of x < 2^64 with mu = floor(2^64 / q): the quotient
// estimate hi(x mu) is floor(x / q) or one less, so one conditional subtraction remains.
__device__ __forceinline__ uint64_t reduce_barrett(uint64_t x, uint64_t q, uint64_t mu) {
    const uint64_t r = x - __umul64hi(x, mu) * q;
    return r >= q ? r - q : r;
}
// canonical residue of a signed v in (-2^63, 2^63)
__device__ __forceinline__ uint64_t reduce_signed(int64_t v, uint64_t q, uint64_t mu) {
    if (v >= 0) return reduce_barrett((uint64_t)v, q, mu);
    const uint64_t r = reduce_barrett((uint64_t)(-(v + 1)), q, mu);  // -(v+1) >= 0, no overflow at INT64_MIN
    return q - 1 - r;
}

// position of the NTT-domain slot k after the automorphism X -> X^g (bit-reversed order):
// out[k] = in[automorph_src(k, g)], exponent e_k = 2 brv(k) + 1.
__device__ __forceinline__ uint32_t automorph_src(uint32_t k, uint32_t g, int logn) {
    uint32_t e = 2u * (__brev(k) >> (32 - logn)) + 1u;
    uint32_t e2 = (uint32_t)(((uint64_t)e * g) & ((2ull << logn) - 1));
    return __brev((e2 - 1u) >> 1) >> (32 - logn);
}

// ------------------------------------------------------------------------------------------
// per-prime constants
// ------------------------------------------------------------------------------------------
struct ModConst {
    uint64_t q;
    uint64_t qinv;    // -q^-1 mod 2^64
    uint64_t r2;      // 2^128 mod q (to Montgomery form: redc(x * r2))
    uint64_t ninv, ninv_shoup;  // N^-1 mod q
    uint64_t mu;      // floor(2^64 / q), for reduce_barrett
    uint64_t r1, r1_shoup;  // 2^64 mod q with its Shoup quotient: x -> x 2^64 mod q (Montgomery form)
    uint64_t p40, p40_shoup, p80, p80_shoup;  // 2^40 and 2^80 mod q: recombination of byte-split products (he_bconv.cu)
};

// next start/end event pair of profiled kernel class `kind` (HE_PROF_*), or nullptr when profiling is off
cudaEvent_t *prof_pair(he_ctx *ctx, int kind);

// index map from a batch's limb position to the context's prime index
struct LimbMap {
    int32_t n;                     // limbs per group
    int32_t prime[HE_MAX_LIMBS];   // prime index of each limb
};

// basis-conversion constants for ModUp of one level (digits of c1 -> Q_level U P)
struct ModUpConst {
    int32_t ndig, alpha, ext, nq;       // digits present, primes per digit, limbs of Q_level U P, level+1
    int32_t ext_prime[HE_MAX_LIMBS];    // prime index of each extended limb
    // for digit d, source i (0 <= i < alpha): [(Qd/q_i)^-1]_{q_i} with Shoup companion
    uint64_t inv[HE_MAX_DNUM][4], inv_shoup[HE_MAX_DNUM][4];
    // (Qd/q_i) mod target prime of extended limb u, with Shoup companion
    uint64_t hat[HE_MAX_DNUM][4][HE_MAX_LIMBS], hat_shoup[HE_MAX_DNUM][4][HE_MAX_LIMBS];
};

// constants for ModDown of one level (Q_level U P -> Q_level)
struct ModDownConst {
    int32_t nq, K;                       // level+1, number of P primes
    int32_t q_prime[HE_MAX_Q];           // prime indices of Q_level
    int32_t p_prime[HE_MAX_P];
    uint64_t inv[HE_MAX_P], inv_shoup[HE_MAX_P];                      // [(P/p_i)^-1]_{p_i}
    uint64_t hat[HE_MAX_P][HE_MAX_Q], hat_shoup[HE_MAX_P][HE_MAX_Q];  // (P/p_i) mod q_j
    uint64_t pinv[HE_MAX_Q], pinv_shoup[HE_MAX_Q];                    // P^-1 mod q_j
};

// What the contexts of one family (a context and its forks) share: the device tables, the
// secret, and the Galois keys.  Freed with the last context of the family.
struct he_shared {
    std::mutex mu;                            // guards keys (keygen on one context, lookups on others)
    std::map<uint32_t, uint64_t *> keys;      // Galois element -> [dnum][2][L+K][N]
    int key_fusion = 1;                       // fused key tables of encoded matrices: 0 never, 1 on reuse, 2 always
    size_t fuse_max = (size_t)8 << 30;        // largest fused table built (bytes)
    void *owned[6] = {};                      // device tables: d_mc, d_tw, d_fft, d_sk, d_sk_mont, d_bconv_a
    ~he_shared() {
        for (auto &kv : keys) cudaFree(kv.second);
        for (void *p : owned) cudaFree(p);
    }
    uint64_t *key(uint32_t g) {
        std::lock_guard<std::mutex> lock(mu);
        auto it = keys.find(g);
        return it == keys.end() ? nullptr : it->second;
    }
};

struct he_ctx {
    int log_n, n, L, K, dnum, alpha;
    int device;                       // CUDA device the context was created on (current at he_ctx_create)
    int sms = 1;                      // its multiprocessors
    uint64_t seed;
    cudaStream_t stream;
    std::vector<uint64_t> primes;     // Q then P
    std::vector<ModConst> mc;         // host copy
    ModConst *d_mc;                   // device copy
    uint64_t *d_tw;                   // per prime: [2][N] pairs (w, Shoup(w)), forward psi^brv(k) and inverse psi^-brv(k),
                                      // then [2][15 N/16] stage-ordered copies (he_ntt.cuh, tw_prime_words)
    void *d_fft;                      // encode/decode tables (double-float twiddles, twist, slot positions)
    uint64_t *d_sk_mont;              // [L+K][N] secret in NTT + Montgomery form
    uint64_t *d_sk;                   // [L+K][N] secret in NTT form
    std::shared_ptr<he_shared> sh;   // tables and keys, shared with forks
    std::vector<ModUpConst> modup;    // per level
    std::vector<ModDownConst> moddown;  // per level
    uint64_t cdt[38];
    // scratch (grown on demand, reused across calls on this context's stream)
    uint64_t *scratch;
    size_t scratch_words;
    int batch_variant = 0;            // last variant a batch tuned to (used by serving lanes)
    int bconv = 0;                    // basis extension of ModUp: 0 exact INT64 products, 1 INT8 tensor-core limb split
    int ntt_form = -1;                // NTT launches of many limb-polys: 0 one CTA each, 1 a 2-CTA cluster each, 2 two phases
                                      // (forward only; -1: not yet timed)
    float ntt_form_ms[HE_NTT_FORMS] = {};  // the timed milliseconds of each form (an encoded matrix's transform)
    int ks_variant = -1;              // transform variant of the many-rotation key switch, chosen by timing (-1: not yet)
    float ks_tune_ms[HE_KS_VARIANTS] = {};  // the timed milliseconds of each variant (one full chunk of rotations)
    uint32_t *d_bconv_a = nullptr;    // INT8 engine: tensor-core A fragments of every (level, digit), shared with forks
    std::vector<size_t> bconv_a_off;  // their offsets (uint4 units), [level * dnum + digit]
    // staging of the host-memory entry points (he_host.cu), grown on demand: a device buffer for
    // inputs and results, a page-locked host buffer for copies from or to pageable memory, and
    // an event recorded after the last copy out of the host buffer
    void *stage_dev = nullptr;
    size_t stage_dev_bytes = 0;
    void *stage_host = nullptr;
    size_t stage_host_bytes = 0;
    cudaEvent_t stage_ev = nullptr;
    // kernels launched so far, and CUDA-event timing of the MatMult loop kernel when enabled
    int64_t launches;
    bool prof_on;
    std::vector<cudaEvent_t> prof_events[HE_PROF_KINDS];  // per profiled kernel class: start/end pairs, recorded on `stream`
    size_t prof_used[HE_PROF_KINDS];
};

// Kernels templated on the ring size: LOGN in {12, 13, 14} (the parameter sets in use) has it at
// compile time, 0 reads it at run time.  by_logn(logn, f) calls f with the matching
// std::integral_constant (f returns the kernel instance); each_logn(f) calls f with every one.
template <class F>
inline auto by_logn(int logn, F f) {
    switch (logn) {
        case 12: return f(std::integral_constant<int, 12>{});
        case 13: return f(std::integral_constant<int, 13>{});
        case 14: return f(std::integral_constant<int, 14>{});
        default: return f(std::integral_constant<int, 0>{});
    }
}
template <class F>
inline void each_logn(F f) {
    f(std::integral_constant<int, 0>{});
    f(std::integral_constant<int, 12>{});
    f(std::integral_constant<int, 13>{});
    f(std::integral_constant<int, 14>{});
}

// contexts of one family (a context and its forks) share tables and keys, so plaintext
// matrices made on one serve all
inline bool same_family(const he_ctx *a, const he_ctx *b) { return a == b || (a && b && a->sh && a->sh == b->sh); }

// one MatMult of a batch (device table entry)
struct MMJob {
    const uint64_t *ct;            // input ciphertext [2][level+1][N]
    uint64_t *out;                 // output ciphertext [2][level][N]
    const uint64_t *pts;           // [m'][level+1+K][N], Montgomery form
    const uint64_t *const *keys;   // [m'-1] Galois keys
    const uint32_t *galois;        // [m'-1]
    int32_t m_prime;
};

// one rotation of a batch of rotations (each job its own ciphertext and step)
struct RotJob {
    const uint64_t *ct;   // input [2][level+1][N]
    uint64_t *out;        // output [2][level+1][N], not aliasing any input of the batch
    const uint64_t *key;  // Galois key of the step
    uint32_t g;           // Galois element
    int32_t pad;
};
// up to HE_ROT_CHUNK rotations, passed to the kernels by value (kernel parameters), so a launch
// needs no copy of a job table to the device
#define HE_ROT_CHUNK 64
struct RotTable {
    RotJob j[HE_ROT_CHUNK];
};

// shared geometry and per-job scratch strides of a batch
struct BatchGeom {
    int32_t ndig, ext, nq, L, LK, K, level;
    uint64_t *D, *coef, *acc, *cacc, *sum, *tmp;
    int64_t d_words, coef_words, acc_words, cacc_words, sum_words, tmp_words;
};

struct he_plan {
    int64_t m, n, slots, mp, np, mb, nb, row_blocks, col_blocks, m_prime, blocks;
    int64_t baby;  // 0: the diagonal method's m' - 1 hoisted rotations; else baby steps B of the BSGS schedule
};
// the BSGS MatMult (he_bsgs.cu) of an encoded matrix whose plan has baby steps
int matmult_bsgs(he_ctx *ctx, he_ptmat *pm, const he_ct *ins, he_ct *outs);

struct he_ptmat {
    he_ctx *ctx;
    he_plan plan;
    int level;
    double scale;
    int ext;                 // limbs per plaintext (level + 1 + K)
    uint64_t *data;          // [R][C][m'][ext][N], NTT + Montgomery
    const uint64_t **d_keys; // device array [m'-1] of Galois key pointers (filled at first use)
    std::vector<uint32_t> galois;
    uint32_t *d_galois;      // [m'-1]
    int variant = -1;        // loop-kernel variant chosen by timing (-1: not yet tuned)
    float tune_ms[HE_MM_MAX_VARIANTS] = {};
    // fused key tables [R][C][m'-1][ndig][2][ext][N] (key_i pt_i products, he_set_key_fusion)
    uint64_t *fused = nullptr;
    int fuse_state = 0;      // 0 not tried, 1 built and faster (used), -1 not used for this matrix
    int fvariant = -1;       // staged variant of the fused form chosen by timing
    int fvariant_pin = -1;   // >= 0: fused form with this variant, built without timing
    float fuse_ms[HE_MM_MAX_VARIANTS] = {};
    uint64_t enc_gen = 0;    // bumped by every (re-)encoding of data
    uint64_t fused_gen = 0;  // enc_gen the fused tables were built from
    uint64_t mm_gen = ~0ull; // enc_gen at the last MatMult
};

// a prepared batch of R = C = 1 MatMults at one level (he_batch_create)
struct he_batch {
    he_ctx *ctx;
    int count;
    std::vector<const he_ptmat *> pms;
    MMJob *h_jobs;               // pinned host table, copied to d_jobs at the start of every run
    MMJob *d_jobs;
    int32_t *d_order_v[HE_MM_MAX_VARIANTS] = {};  // work items (job, limb, tile) in issue order, per loop-kernel variant
    int n_items_v[HE_MM_MAX_VARIANTS] = {};
    int ctas_v[HE_MM_MAX_VARIANTS] = {};           // persistent grid per variant (resident CTAs per SM x SMs)
    int variant = -1;            // chosen by timing on the first run (-1: not yet)
    float tune_ms[HE_MM_MAX_VARIANTS] = {};
    int stage_form = 0;          // ModUp / ModDown / rescale stages: 0 one CTA per limb-poly, 1 8-CTA clusters (timed with the variant)
    float stage_ms[2] = {};
    unsigned int *d_counter;     // work-queue head
    BatchGeom bg;
    uint64_t *mem;               // per-job scratch
    cudaStream_t stream;         // capture stream
    cudaEvent_t ev_in, ev_out;
    cudaGraphExec_t exec;
    bool have_graph;
};

int launch_matmult_batch(he_ctx *ctx, he_batch *b, cudaStream_t stream);
// words of scratch per rotation job at `level`, and the launches of `count` jobs (device table)
size_t rotate_many_words(const he_ctx *ctx, int level);
// count <= HE_ROT_CHUNK jobs (host table), scratch of count rotate_many_words
void launch_rotate_many(he_ctx *ctx, const RotJob *jobs, int count, int level, uint64_t *scratch);
// ModUp with the INT8 tensor-core basis extension (he_bconv.cu): for jobs j < count, c1 of job j
// in NTT form (jobs[j].ct + (level+1) N when jobs is given, else c1_ntt) and in coefficient form
// at coef + j coef_w, digits into D + j d_w ([ndig][ext][N], NTT form).  Two launches.
void launch_modup_i8(he_ctx *ctx, const RotTable *jobs, int count, int level, const uint64_t *c1_ntt, const uint64_t *coef, int64_t coef_w,
                     uint64_t *D, int64_t d_w);
// the INT8 engine's A-fragment tables of every level and digit (at context creation)
int bconv_i8_tables(he_ctx *ctx);
// key switch (inner product, ModDown, automorphism of c0) of `count` rotations (host table) whose
// ModUp digits are at D + j d_stride (d_stride 0: one shared decomposition), two (few rotations)
// or four launches per HE_ROT_CHUNK rotations; pc: scratch of keyswitch_many_pc_words(ctx, count)
// words, laid out [min(count, HE_ROT_CHUNK)][2][K][N] then [..][2][level+1][N]
size_t keyswitch_many_pc_words(const he_ctx *ctx, int count);
void launch_keyswitch_many(he_ctx *ctx, const RotJob *jobs, int count, int level, const uint64_t *D, int64_t d_stride, uint64_t *pc);
int mm_variant_count();
int mm_variant_tile(int v);  // coefficients per tile of loop-kernel variant v
void mm_variant_shape(int v, int *vec, int *grp, int *stages, int *ga);
int mm_batch_ctas_per_sm(int v, int ndig);
int tune_matmult_loop(he_ctx *ctx, he_ptmat *pm, const uint64_t *ct, const uint64_t *D, uint64_t *acc, uint64_t *cacc);
int tune_matmult_fused(he_ctx *ctx, he_ptmat *pm, const uint64_t *ct, const uint64_t *D, uint64_t *acc, uint64_t *cacc);
bool capturing(cudaStream_t st);           // st is being captured into a graph
bool mm_variant_fusable(int v, int ndig);  // variant v has a fused-key form for ndig digits
void launch_fuse_keys(he_ctx *ctx, he_ptmat *pm);  // pm->fused from pm->data and the bound Galois keys
// defined in he_api.cu (inside its extern "C" block)
extern "C" {
int batch_create_impl(he_ctx *ctx, int count, int level, const he_ptmat *const *pms, he_batch **out);
int batch_launch(he_ctx *ctx, he_batch *b);
int ptmat_bind_keys(he_ctx *ctx, he_ptmat *pm);
}

// Programmatic dependent launch.  Every kernel is launched with programmatic stream
// serialization and begins with HE_GRID_DEP(): it lets the next kernel in the stream be
// scheduled at once (its blocks start while this grid drains), then waits until the previous
// grid has completed and its writes are visible.  The body therefore runs strictly after its
// predecessor, as with ordinary stream order; only the launch latency between dependent kernels
// overlaps.  (Both instructions are no-ops for a launch without the attribute.)
#define HE_GRID_DEP()                                                      \
    do {                                                                   \
        asm volatile("griddepcontrol.launch_dependents;" ::: "memory");   \
        asm volatile("griddepcontrol.wait;" ::: "memory");                \
    } while (0)
// The two halves, for kernels that start loads before the wait.  Those loads may read only the
// context's tables written at its creation (which synchronises), never data of an earlier launch:
// with every kernel releasing its successor on entry, a kernel's pre-wait code can run while
// kernels two or more launches back are still running.
#define HE_GRID_LAUNCH() asm volatile("griddepcontrol.launch_dependents;" ::: "memory")
#define HE_GRID_WAIT() asm volatile("griddepcontrol.wait;" ::: "memory")

template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// thread-block cluster launch (cluster of cl_size CTAs along x), also programmatically serialized
#define HE_NTT_CL_SIZE 8
template <typename... KArgs, typename... Args>
inline cudaError_t launch_cluster_n(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t st, int cl_size, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cl_size;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}
template <typename... KArgs, typename... Args>
inline cudaError_t launch_cluster(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t st, Args... args) {
    return launch_cluster_n(kernel, grid, block, smem, st, HE_NTT_CL_SIZE, args...);
}

// ------------------------------------------------------------------------------------------
// launchers (all asynchronous on ctx->stream)
// ------------------------------------------------------------------------------------------
int he_check(cudaError_t e);
// Galois element 5^r mod 2N of a left rotation by `step` slots, r = step mod N/2 in [0, N/2)
uint32_t galois_of(const he_ctx *ctx, int64_t step);
uint64_t *ctx_scratch(he_ctx *ctx, size_t words);  // nullptr on allocation failure

// NTT of `groups` x map.n limb-polys; in and out may alias.
void launch_from_mont(he_ctx *ctx, const uint64_t *data, uint64_t *out, int groups, const LimbMap &map);
void launch_ntt_fwd(he_ctx *ctx, const uint64_t *in, uint64_t *out, int groups, const LimbMap &map);
void launch_ntt_inv(he_ctx *ctx, const uint64_t *in, uint64_t *out, int groups, const LimbMap &map);
// strided forms: limb l of group g at base + g * gs + l * N; to_mont stores x 2^64 mod q
void launch_ntt_fwd_strided(he_ctx *ctx, const uint64_t *in, int64_t in_gs, uint64_t *out, int64_t out_gs, int groups,
                            const LimbMap &map, int to_mont);
void launch_ntt_inv_strided(he_ctx *ctx, const uint64_t *in, int64_t in_gs, uint64_t *out, int64_t out_gs, int groups, const LimbMap &map);
int ntt_threads(int logn);
bool use_cluster(int logn, int polys);  // launch in the cluster form (few limb-polys)
bool use_pair(const he_ctx *ctx, int polys);  // launch in the 2-CTA pair form (many limb-polys, when the context chose it)
bool use_two_phase(const he_ctx *ctx, int polys);  // launch in two phases (many limb-polys, NTT form 2, log N = 12..14)
int cl_threads(int logn);
size_t cl_smem_bytes(int logn);
// dynamic shared memory of a CTA that holds one limb-poly for the NTT (padded layout)
inline size_t ntt_smem_bytes(int logn) { return ((size_t)1 << logn) * 8 + ((size_t)1 << logn) / 32 * 8; }
// NTT forward of signed int64 coefficient vectors reduced per limb: in [groups][N] -> out [groups][map.n][N]
void launch_ntt_from_int64(he_ctx *ctx, const int64_t *in, uint64_t *out, int groups, const LimbMap &map, int to_mont);
// x -> x 2^64 mod q in place
void launch_to_mont(he_ctx *ctx, uint64_t *data, int groups, const LimbMap &map);

// elementwise
void launch_add(he_ctx *ctx, const uint64_t *a, const uint64_t *b, uint64_t *out, int groups, const LimbMap &map);
void launch_mul_plain(he_ctx *ctx, const uint64_t *ct, const uint64_t *pt, uint64_t *out, int level);

// key switching
void launch_modup(he_ctx *ctx, const uint64_t *c1_ntt, int level, uint64_t *D, uint64_t *tmp_coeff);
void launch_ks_inner(he_ctx *ctx, const uint64_t *D, int level, uint32_t g, const uint64_t *key, uint64_t *u /*[2][ext][N]*/);
// out_c = add_c (optional, NTT) + ModDown(x_c) for c = 0..ncomp-1 ; x [ncomp][ext][N], tmp [ncomp][K][N]
void launch_moddown(he_ctx *ctx, const uint64_t *x, int level, int ncomp, const uint64_t *add0, const uint64_t *add1, uint64_t *out,
                    uint64_t *tmp);
void launch_automorph(he_ctx *ctx, const uint64_t *in, uint64_t *out, int groups, const LimbMap &map, uint32_t g);
void launch_rescale(he_ctx *ctx, const uint64_t *ct, int level, uint64_t *out, uint64_t *tmp);
// ModDown of [2][level+1+K][N] plus add0/add1 (NTT, [level+1][N] each, may be null), then
// rescale, into out [2][level][N]: one cluster launch when moddown_rescale_fused says so
bool moddown_rescale_fused(const he_ctx *ctx, int level);
void launch_moddown_rescale(he_ctx *ctx, const uint64_t *x, int level, const uint64_t *add0, const uint64_t *add1, uint64_t *out,
                            uint64_t *tmp);  // tmp: 2 (K+1) N words
void launch_matmult_loop(he_ctx *ctx, const he_ptmat *pm, int r, int c, const uint64_t *ct, const uint64_t *D,
                         uint64_t *acc /*[2][ext][N]*/, uint64_t *cacc /*[2][level+1][N]*/, int accumulate);

void launch_matmult_loop_with_tables(he_ctx *ctx, const he_ptmat *pm, int r, int c, const uint64_t *ct, const uint64_t *D,
                                     const uint64_t *const *keys, const uint32_t *galois, uint64_t *acc, uint64_t *cacc, int accumulate);

// encoding, sampling, encryption
void launch_encode(he_ctx *ctx, const double *slots, int64_t n_slots, int64_t stride, int count, double scale, int64_t *coeffs);
// the diagonal layout of X (Eq. 2 after Eq. 3; X given transposed when trans) and its encoding
// in one launch; false (nothing launched) where that form does not apply
bool launch_encode_matrix(he_ctx *ctx, const he_plan &p, const double *X, int trans, int count, double scale, int64_t *coeffs);
// the replicated layout of y (Eq. 3) and its encoding in one launch, count = column blocks; false
// (nothing launched) where that form does not apply
bool launch_encode_vector(he_ctx *ctx, const he_plan &p, const double *y, int count, double scale, int64_t *coeffs);
void launch_decode(he_ctx *ctx, const double *coeffs, int count, double scale, double *slots);
void launch_decrypt_coeffs(he_ctx *ctx, const uint64_t *ct, int level, int count, double *coeffs, uint64_t *tmp);
// decode of `count` decrypted coefficient vectors (the row blocks' output ciphertexts) with the lazy
// rotate-and-sum of the plan in the same launch, into y [m]; false where that form does not apply
bool launch_decode_ras(he_ctx *ctx, const he_plan &p, const double *coeffs, int count, double scale, const double *mask, double *y);
// he_encrypt's five steps as one cluster launch per limb (false: that form does not apply); with
// m_int (integer coefficients, pt null) the plaintext is encoded into the same launch
bool launch_encrypt_fused(he_ctx *ctx, const uint64_t *pt, const int64_t *m_int, int level, uint64_t nonce, const uint64_t *nonce_dev,
                          uint64_t *ct);
void launch_sample_uniform(he_ctx *ctx, uint64_t tag, uint64_t nonce, const LimbMap &map, int limb_offset, uint64_t *out,
                           const uint64_t *nonce_dev = nullptr);
void launch_sample_gauss(he_ctx *ctx, uint64_t tag, uint64_t nonce, int64_t *out, const uint64_t *nonce_dev = nullptr);
void launch_sample_ternary(he_ctx *ctx, int64_t *out);
void launch_encrypt_combine(he_ctx *ctx, const uint64_t *pt, const uint64_t *a, const uint64_t *e, int level, uint64_t *ct);
void launch_keygen_combine(he_ctx *ctx, const uint64_t *a, const uint64_t *e, uint32_t g, int digit, uint64_t *key_d);
void launch_layout_matrix(he_ctx *ctx, const he_plan &p, const double *X, double *slots, int trans = 0);
void launch_layout_vector(he_ctx *ctx, const he_plan &p, const double *y, double *slots);
void launch_lazy_ras(he_ctx *ctx, const he_plan &p, const double *slots, const double *mask, double *y);
void launch_ras_gather(he_ctx *ctx, const he_plan &p, const double *slots, double *y);
