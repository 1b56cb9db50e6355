// he_api.cu -- context, host-side parameter math and the C ABI entry points of he.h.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "he_internal.cuh"

void ntt_set_smem_limits(int max_bytes);
void ops_set_smem_limits(int max_bytes);
void encode_set_smem_limits(int max_bytes);
void cdiag_set_smem_limits(int max_bytes);
void bconv_set_smem_limits(int max_bytes);
void keyswitch_set_smem_limits(int max_bytes);

namespace {

// ---------------------------------------------------------------- host number theory
uint64_t hmul(uint64_t a, uint64_t b, uint64_t m) { return (uint64_t)((u128)a * b % m); }
uint64_t hpow(uint64_t a, uint64_t e, uint64_t m) {
    uint64_t r = 1 % m;
    a %= m;
    for (; e; e >>= 1, a = hmul(a, a, m))
        if (e & 1) r = hmul(r, a, m);
    return r;
}
uint64_t hinv(uint64_t a, uint64_t m) { return hpow(a % m, m - 2, m); }  // m prime

// strong-probable-prime test to the seven bases known to decide all 64-bit integers
bool probable_prime(uint64_t n) {
    if (n < 4) return n >= 2;
    if (!(n & 1)) return false;
    uint64_t d = n - 1;
    int r = 0;
    while (!(d & 1)) d >>= 1, ++r;
    const uint64_t bases[7] = {2, 325, 9375, 28178, 450775, 9780504, 1795265022};
    for (uint64_t b : bases) {
        uint64_t a = b % n;
        if (a == 0) continue;
        uint64_t x = hpow(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool ok = false;
        for (int i = 1; i < r && !ok; ++i) {
            x = hmul(x, x, n);
            ok = (x == n - 1);
        }
        if (!ok) return false;
    }
    return true;
}

// largest unused prime below 2^bits that is 1 mod 2N
int prime_chain(int log_n, const std::vector<int> &bits, std::vector<uint64_t> &out) {
    const uint64_t step = 2ull << log_n;
    out.clear();
    for (int b : bits) {
        if (b < 20 || b > 61) return HE_EINVAL;
        const uint64_t hi = 1ull << b, lo = hi >> 1;
        uint64_t c = (hi - 1) - ((hi - 1 - 1) % step);  // largest value < hi with c = 1 mod step
        bool found = false;
        for (; c > lo; c -= step) {
            if (std::find(out.begin(), out.end(), c) != out.end()) continue;
            if (probable_prime(c)) {
                out.push_back(c);
                found = true;
                break;
            }
        }
        if (!found) return HE_EINVAL;
    }
    return HE_OK;
}

int check_params(const he_params *p) {
    if (!p) return HE_EINVAL;
    if (p->log_n < 4 || p->log_n > 14) return HE_EINVAL;
    if (p->n_q < 1 || p->n_q > HE_MAX_Q || p->n_p < 1 || p->n_p > HE_MAX_P) return HE_EINVAL;
    if (p->dnum < 1 || p->dnum > p->n_q || p->dnum > HE_MAX_DNUM) return HE_EINVAL;
    if ((p->n_q + p->dnum - 1) / p->dnum > 4) return HE_EINVAL;  // at most 4 primes per digit
    return HE_OK;
}

std::vector<int> all_bits(const he_params *p) {
    std::vector<int> b(p->q_bits, p->q_bits + p->n_q);
    b.insert(b.end(), p->p_bits, p->p_bits + p->n_p);
    return b;
}

uint64_t shoup(uint64_t w, uint64_t q) { return (uint64_t)(((u128)w << 64) / q); }

uint64_t brv(uint64_t x, int bits) {
    uint64_t r = 0;
    for (int i = 0; i < bits; ++i, x >>= 1) r = (r << 1) | (x & 1);
    return r;
}

// a primitive 2N-th root: psi = x^((q-1)/2N) for the first odd x >= 3 with psi^N = -1
uint64_t find_psi(uint64_t q, int log_n) {
    const uint64_t n = 1ull << log_n;
    for (uint64_t x = 3;; x += 2) {
        uint64_t psi = hpow(x, (q - 1) / (2 * n), q);
        if (hpow(psi, n, q) == q - 1) return psi;
    }
}

ModConst make_modconst(uint64_t q, int log_n) {
    ModConst m{};
    m.q = q;
    uint64_t inv = q;  // q * q = 1 mod 8: three correct bits, doubled by each Newton step
    for (int i = 0; i < 5; ++i) inv *= 2 - q * inv;
    m.qinv = (uint64_t)0 - inv;
    uint64_t r1 = (uint64_t)(((u128)1 << 64) % q);
    m.r2 = hmul(r1, r1, q);
    m.ninv = hinv((1ull << log_n) % q, q);
    m.ninv_shoup = shoup(m.ninv, q);
    m.mu = (uint64_t)((((u128)1) << 64) / q);
    m.r1 = r1;
    m.r1_shoup = shoup(r1, q);
    m.p40 = hpow(2, 40, q);
    m.p40_shoup = shoup(m.p40, q);
    m.p80 = hpow(2, 80, q);
    m.p80_shoup = shoup(m.p80, q);
    return m;
}

bool cuda_ok(cudaError_t e) { return e == cudaSuccess; }

}  // namespace

int he_check(cudaError_t e) { return e == cudaSuccess ? HE_OK : HE_ECUDA; }

uint64_t *ctx_scratch(he_ctx *ctx, size_t words) {
    if (words <= ctx->scratch_words) return ctx->scratch;
    // previous users of the buffer are ordered on the stream; wait before releasing it
    cudaStreamSynchronize(ctx->stream);
    if (ctx->scratch) cudaFree(ctx->scratch);
    ctx->scratch = nullptr;
    ctx->scratch_words = 0;
    if (cudaMalloc(&ctx->scratch, words * 8) != cudaSuccess) return nullptr;
    ctx->scratch_words = words;
    return ctx->scratch;
}

static int last_launch() { return cudaGetLastError() == cudaSuccess ? HE_OK : HE_ECUDA; }

static LimbMap qmap(int level) {
    LimbMap m{};
    m.n = level + 1;
    for (int l = 0; l <= level; ++l) m.prime[l] = l;
    return m;
}

static LimbMap qpmap(const he_ctx *ctx, int level) {
    LimbMap m{};
    m.n = level + 1 + ctx->K;
    for (int l = 0; l <= level; ++l) m.prime[l] = l;
    for (int i = 0; i < ctx->K; ++i) m.prime[level + 1 + i] = ctx->L + i;
    return m;
}

// The kernels' dynamic shared-memory limits are per function and per process, so they are set
// once per device to the device's opt-in maximum (a context with a smaller ring must not lower
// the limit that another context's launches need); the limit only permits, it reserves nothing.
static int set_smem_limits_once() {
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return HE_ECUDA;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev]) return HE_OK;
    int smem = 0;
    if (cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || smem <= 0) return HE_ECUDA;
    ntt_set_smem_limits(smem);
    ops_set_smem_limits(smem);
    encode_set_smem_limits(smem);
    cdiag_set_smem_limits(smem);
    bconv_set_smem_limits(smem);
    keyswitch_set_smem_limits(smem);
    if (cudaGetLastError() != cudaSuccess) return HE_ECUDA;
    done[dev] = true;
    return HE_OK;
}

uint32_t galois_of(const he_ctx *ctx, int64_t step) {
    const int64_t slots = ctx->n / 2;
    int64_t r = ((step % slots) + slots) % slots;
    return (uint32_t)hpow(5, (uint64_t)r, 2ull * ctx->n);
}

extern "C" {

const char *he_strerror(int s) {
    switch (s) {
        case HE_OK: return "ok";
        case HE_EINVAL: return "invalid argument";
        case HE_ENOMEM: return "out of memory";
        case HE_ECUDA: return "CUDA error";
        case HE_EKEY: return "missing Galois key";
        case HE_ELEVEL: return "level out of range or mismatched";
        case HE_ESCALE: return "scale mismatch";
        case HE_ETIMEOUT: return "device wait timed out";
        case HE_EBUDGET: return "memory budget exceeded";
        default: return "unknown status";
    }
}

int he_params_primes(const he_params *p, uint64_t *out) {
    int rc = check_params(p);
    if (rc != HE_OK || !out) return HE_EINVAL;
    std::vector<uint64_t> pr;
    rc = prime_chain(p->log_n, all_bits(p), pr);
    if (rc != HE_OK) return rc;
    std::copy(pr.begin(), pr.end(), out);
    return HE_OK;
}

int he_cdt_table(uint64_t *out) {
    if (!out) return HE_EINVAL;
    // rho(y) = exp(-y^2 / 20.48) for y = -19..19 (sigma = 3.2); cumulative sums left to right
    double rho[39], total = 0.0;
    for (int i = 0; i < 39; ++i) {
        const double y = (double)(i - 19);
        rho[i] = exp(-(y * y) / 20.48);
    }
    for (int i = 0; i < 39; ++i) total += rho[i];
    double cum = 0.0;
    for (int k = 0; k < 38; ++k) {
        cum += rho[k];
        out[k] = (uint64_t)floor(ldexp(cum / total, 40));
    }
    return HE_OK;
}

void he_ctx_destroy(he_ctx *ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->scratch);  // the tables and keys go with the family's last context (he_shared)
    cudaFree(ctx->stage_dev);
    cudaFreeHost(ctx->stage_host);
    if (ctx->stage_ev) cudaEventDestroy(ctx->stage_ev);
    for (auto &v : ctx->prof_events)
        for (cudaEvent_t e : v) cudaEventDestroy(e);
    delete ctx;
}

int he_ctx_create(const he_params *p, uint64_t seed, void *stream, he_ctx **out) {
    if (!out) return HE_EINVAL;
    *out = nullptr;
    int rc = check_params(p);
    if (rc != HE_OK) return rc;
    he_ctx *ctx = new (std::nothrow) he_ctx();
    if (!ctx) return HE_ENOMEM;
    ctx->sh = std::make_shared<he_shared>();
    ctx->log_n = p->log_n;
    ctx->n = 1 << p->log_n;
    ctx->L = p->n_q;
    ctx->K = p->n_p;
    ctx->dnum = p->dnum;
    ctx->alpha = (p->n_q + p->dnum - 1) / p->dnum;
    ctx->seed = seed;
    ctx->stream = (cudaStream_t)stream;
    if (cudaGetDevice(&ctx->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess) {
        delete ctx;
        return HE_ECUDA;
    }
    rc = prime_chain(p->log_n, all_bits(p), ctx->primes);
    if (rc != HE_OK) {
        delete ctx;
        return rc;
    }
    he_cdt_table(ctx->cdt);
    const int LK = ctx->L + ctx->K, N = ctx->n;
    rc = set_smem_limits_once();
    if (rc != HE_OK) {
        delete ctx;
        return rc;
    }

    // per-prime constants and NTT twiddles
    const size_t t4 = ctx->log_n >= 4 ? (size_t)15 * (N / 16) : 0, prime_words = (size_t)4 * N + 4 * t4;
    std::vector<uint64_t> tw((size_t)LK * prime_words);
    for (int i = 0; i < LK; ++i) {
        const uint64_t q = ctx->primes[i];
        ctx->mc.push_back(make_modconst(q, ctx->log_n));
        const uint64_t psi = find_psi(q, ctx->log_n), ipsi = hinv(psi, q);
        std::vector<uint64_t> pw(N), ipw(N);
        pw[0] = ipw[0] = 1;
        for (int k = 1; k < N; ++k) {
            pw[k] = hmul(pw[k - 1], psi, q);
            ipw[k] = hmul(ipw[k - 1], ipsi, q);
        }
        // [forward pairs (psi^brv(k), Shoup quotient)][inverse pairs (psi^-brv(k), quotient)]
        uint64_t *t = tw.data() + (size_t)i * prime_words;
        for (int k = 0; k < N; ++k) {
            const uint64_t e = brv(k, ctx->log_n);
            t[2 * k] = pw[e];
            t[2 * k + 1] = shoup(pw[e], q);
            t[2 * N + 2 * k] = ipw[e];
            t[2 * N + 2 * k + 1] = shoup(ipw[e], q);
        }
        // stage-ordered copies for the radix-16 pass whose sets are its groups (G = N/16 sets):
        // forward last pass, stage j (m = N/2^(4-j)): entry i < 2^j of set g at ((2^j - 1 + i) G + g)
        // is table entry m + g 2^j + i; inverse first pass, stage j (m = N/2^(j+1)): entry
        // i < 2^(3-j) at ((16 - 2^(4-j) + i) G + g) is entry m + g 2^(3-j) + i
        if (t4) {
            const int G = N / 16;
            uint64_t *f4 = t + 4 * (size_t)N, *i4 = f4 + 2 * t4;
            for (int j = 0; j < 4; ++j)
                for (int g = 0; g < G; ++g) {
                    for (int e = 0; e < (1 << j); ++e) {
                        const size_t dst = 2 * ((size_t)((1 << j) - 1 + e) * G + g), src = 2 * ((size_t)(N >> (4 - j)) + ((size_t)g << j) + e);
                        f4[dst] = t[src];
                        f4[dst + 1] = t[src + 1];
                    }
                    for (int e = 0; e < (8 >> j); ++e) {
                        const size_t dst = 2 * ((size_t)(16 - (16 >> j) + e) * G + g),
                                     src = 2 * N + 2 * ((size_t)(N >> (j + 1)) + ((size_t)g << (3 - j)) + e);
                        i4[dst] = t[src];
                        i4[dst + 1] = t[src + 1];
                    }
                }
        }
    }
    // FFT tables as double-float (hi, lo) pairs: [N/4] exp(-2 pi i k/(N/2)), [N/2] exp(-i pi k / N),
    // then [N/2] int32 slot positions t_j = (5^j mod 2N - 1) / 4
    const int M = N / 2;
    std::vector<float> fft((size_t)4 * (M / 2) + 4 * M + M, 0.0f);
    const double PI = 3.14159265358979323846264338327950288;
    auto put = [](float *dst, double re, double im) {
        const float rh = (float)re, ih = (float)im;
        dst[0] = rh;
        dst[1] = (float)(re - (double)rh);
        dst[2] = ih;
        dst[3] = (float)(im - (double)ih);
    };
    for (int k = 0; k < M / 2; ++k) put(fft.data() + 4 * k, cos(2.0 * PI * k / M), -sin(2.0 * PI * k / M));
    float *twist = fft.data() + 4 * (M / 2);
    for (int k = 0; k < M; ++k) put(twist + 4 * k, cos(PI * k / N), -sin(PI * k / N));
    int32_t *pos = reinterpret_cast<int32_t *>(twist + 4 * M);
    uint64_t e = 1;
    for (int j = 0; j < M; ++j) {
        pos[j] = (int32_t)((e - 1) / 4);
        e = e * 5 % (2ull * N);
    }
    // base-conversion constants per level
    for (int level = 0; level < ctx->L; ++level) {
        ModUpConst mu{};
        mu.alpha = ctx->alpha;
        mu.nq = level + 1;
        mu.ext = level + 1 + ctx->K;
        mu.ndig = (level + 1 + ctx->alpha - 1) / ctx->alpha;
        for (int u = 0; u < mu.ext; ++u) mu.ext_prime[u] = u <= level ? u : ctx->L + (u - level - 1);
        for (int d = 0; d < mu.ndig; ++d) {
            const int lo = d * ctx->alpha, hi = std::min(lo + ctx->alpha, level + 1);
            for (int i = lo; i < hi; ++i) {
                const uint64_t qi = ctx->primes[i];
                uint64_t hat_qi = 1;
                for (int j = lo; j < hi; ++j)
                    if (j != i) hat_qi = hmul(hat_qi, ctx->primes[j] % qi, qi);
                mu.inv[d][i - lo] = hinv(hat_qi, qi);
                mu.inv_shoup[d][i - lo] = shoup(mu.inv[d][i - lo], qi);
                for (int u = 0; u < mu.ext; ++u) {
                    const uint64_t t = ctx->primes[mu.ext_prime[u]];
                    uint64_t h = 1 % t;
                    for (int j = lo; j < hi; ++j)
                        if (j != i) h = hmul(h, ctx->primes[j] % t, t);
                    mu.hat[d][i - lo][u] = h;
                    mu.hat_shoup[d][i - lo][u] = shoup(h, t);
                }
            }
        }
        ctx->modup.push_back(mu);
        ModDownConst md{};
        md.nq = level + 1;
        md.K = ctx->K;
        for (int j = 0; j <= level; ++j) md.q_prime[j] = j;
        for (int i = 0; i < ctx->K; ++i) {
            md.p_prime[i] = ctx->L + i;
            const uint64_t pi = ctx->primes[ctx->L + i];
            uint64_t hat = 1;
            for (int r = 0; r < ctx->K; ++r)
                if (r != i) hat = hmul(hat, ctx->primes[ctx->L + r] % pi, pi);
            md.inv[i] = hinv(hat, pi);
            md.inv_shoup[i] = shoup(md.inv[i], pi);
            for (int j = 0; j <= level; ++j) {
                const uint64_t q = ctx->primes[j];
                uint64_t h = 1 % q;
                for (int r = 0; r < ctx->K; ++r)
                    if (r != i) h = hmul(h, ctx->primes[ctx->L + r] % q, q);
                md.hat[i][j] = h;
                md.hat_shoup[i][j] = shoup(h, q);
            }
        }
        for (int j = 0; j <= level; ++j) {
            const uint64_t q = ctx->primes[j];
            uint64_t P = 1 % q;
            for (int r = 0; r < ctx->K; ++r) P = hmul(P, ctx->primes[ctx->L + r] % q, q);
            md.pinv[j] = hinv(P, q);
            md.pinv_shoup[j] = shoup(md.pinv[j], q);
        }
        ctx->moddown.push_back(md);
    }
    bool ok = cuda_ok(cudaMalloc(&ctx->d_mc, sizeof(ModConst) * LK)) && cuda_ok(cudaMalloc(&ctx->d_tw, tw.size() * 8)) &&
              cuda_ok(cudaMalloc(&ctx->d_fft, fft.size() * 4)) && cuda_ok(cudaMalloc(&ctx->d_sk, (size_t)LK * N * 8)) &&
              cuda_ok(cudaMalloc(&ctx->d_sk_mont, (size_t)LK * N * 8));
    ctx->sh->owned[0] = ctx->d_mc;
    ctx->sh->owned[1] = ctx->d_tw;
    ctx->sh->owned[2] = ctx->d_fft;
    ctx->sh->owned[3] = ctx->d_sk;
    ctx->sh->owned[4] = ctx->d_sk_mont;
    if (!ok) {
        he_ctx_destroy(ctx);
        return HE_ENOMEM;
    }
    ok = cuda_ok(cudaMemcpy(ctx->d_mc, ctx->mc.data(), sizeof(ModConst) * LK, cudaMemcpyHostToDevice)) &&
         cuda_ok(cudaMemcpy(ctx->d_tw, tw.data(), tw.size() * 8, cudaMemcpyHostToDevice)) &&
         cuda_ok(cudaMemcpy(ctx->d_fft, fft.data(), fft.size() * 4, cudaMemcpyHostToDevice));
    // secret key: ternary coefficients -> every prime of Q U P, NTT form (and Montgomery form)
    int64_t *s_int = reinterpret_cast<int64_t *>(ctx_scratch(ctx, N));
    if (!ok || !s_int) {
        he_ctx_destroy(ctx);
        return HE_ECUDA;
    }
    launch_sample_ternary(ctx, s_int);
    LimbMap all{};
    all.n = LK;
    for (int i = 0; i < LK; ++i) all.prime[i] = i;
    launch_ntt_from_int64(ctx, s_int, ctx->d_sk, 1, all, 0);
    cudaMemcpyAsync(ctx->d_sk_mont, ctx->d_sk, (size_t)LK * N * 8, cudaMemcpyDeviceToDevice, ctx->stream);
    launch_to_mont(ctx, ctx->d_sk_mont, 1, all);
    if (last_launch() != HE_OK || cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        he_ctx_destroy(ctx);
        return HE_ECUDA;
    }
    rc = bconv_i8_tables(ctx);
    if (rc != HE_OK) {
        he_ctx_destroy(ctx);
        return rc;
    }
    *out = ctx;
    return HE_OK;
}

size_t he_ct_bytes(const he_ctx *ctx, int level) {
    if (!ctx || level < 0 || level >= ctx->L) return 0;
    return 2 * (size_t)(level + 1) * ctx->n * sizeof(uint64_t);
}

size_t he_pt_bytes(const he_ctx *ctx, int level) {
    if (!ctx || level < 0 || level >= ctx->L) return 0;
    return (size_t)(level + 1) * ctx->n * sizeof(uint64_t);
}

int he_ctx_fork(he_ctx *parent, void *stream, he_ctx **out) {
    if (!parent || !out) return HE_EINVAL;
    *out = nullptr;
    he_ctx *ctx = new (std::nothrow) he_ctx();
    if (!ctx) return HE_ENOMEM;
    // everything read-only is copied or shared; the stream, scratch, counters and profiling are own
    ctx->log_n = parent->log_n;
    ctx->n = parent->n;
    ctx->L = parent->L;
    ctx->K = parent->K;
    ctx->dnum = parent->dnum;
    ctx->alpha = parent->alpha;
    ctx->device = parent->device;
    ctx->sms = parent->sms;
    ctx->seed = parent->seed;
    ctx->stream = (cudaStream_t)stream;
    ctx->primes = parent->primes;
    ctx->mc = parent->mc;
    ctx->d_mc = parent->d_mc;
    ctx->d_tw = parent->d_tw;
    ctx->d_fft = parent->d_fft;
    ctx->d_sk_mont = parent->d_sk_mont;
    ctx->d_sk = parent->d_sk;
    ctx->sh = parent->sh;
    ctx->modup = parent->modup;
    ctx->moddown = parent->moddown;
    memcpy(ctx->cdt, parent->cdt, sizeof(ctx->cdt));
    ctx->batch_variant = parent->batch_variant;
    ctx->bconv = parent->bconv;
    ctx->ntt_form = parent->ntt_form;
    for (int f = 0; f < HE_NTT_FORMS; ++f) ctx->ntt_form_ms[f] = parent->ntt_form_ms[f];
    ctx->d_bconv_a = parent->d_bconv_a;
    ctx->bconv_a_off = parent->bconv_a_off;
    // the parent's pending work (keys, tables) must be complete before the fork's stream uses it
    if (cudaStreamSynchronize(parent->stream) != cudaSuccess) {
        delete ctx;
        return HE_ECUDA;
    }
    *out = ctx;
    return HE_OK;
}

int he_synchronize(he_ctx *ctx) {
    if (!ctx) return HE_EINVAL;
    return he_check(cudaStreamSynchronize(ctx->stream));
}

int he_launch_count(const he_ctx *ctx, int64_t *count) {
    if (!ctx || !count) return HE_EINVAL;
    *count = ctx->launches;
    return HE_OK;
}

int he_profile_enable(he_ctx *ctx, int on) {
    if (!ctx) return HE_EINVAL;
    cudaStreamSynchronize(ctx->stream);
    ctx->prof_on = on != 0;
    for (size_t &u : ctx->prof_used) u = 0;
    return HE_OK;
}

int he_profile_read_kind(he_ctx *ctx, int kind, double *ms_total, int64_t *launches) {
    if (!ctx || !ms_total || !launches || kind < 0 || kind >= HE_PROF_KINDS) return HE_EINVAL;
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return HE_ECUDA;
    double total = 0.0;
    for (size_t i = 0; i + 1 < ctx->prof_used[kind]; i += 2) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, ctx->prof_events[kind][i], ctx->prof_events[kind][i + 1]) != cudaSuccess) return HE_ECUDA;
        total += ms;
    }
    *ms_total = total;
    *launches = (int64_t)(ctx->prof_used[kind] / 2);
    return HE_OK;
}

int he_profile_read(he_ctx *ctx, double *ms_total, int64_t *launches) { return he_profile_read_kind(ctx, HE_PROF_LOOP, ms_total, launches); }

int he_ctx_info(const he_ctx *ctx, int64_t *n, int32_t *n_q, int32_t *n_p) {
    if (!ctx) return HE_EINVAL;
    if (n) *n = ctx->n;
    if (n_q) *n_q = ctx->L;
    if (n_p) *n_p = ctx->K;
    return HE_OK;
}

int he_keygen(he_ctx *ctx, const int32_t *steps, int n_steps) {
    if (!ctx || n_steps < 0 || (n_steps > 0 && !steps)) return HE_EINVAL;
    const int LK = ctx->L + ctx->K, N = ctx->n;
    LimbMap all{};
    all.n = LK;
    for (int i = 0; i < LK; ++i) all.prime[i] = i;
    for (int s = 0; s < n_steps; ++s) {
        const uint32_t g = galois_of(ctx, steps[s]);
        if (ctx->sh->key(g)) continue;
        uint64_t *key = nullptr;
        if (cudaMalloc(&key, (size_t)ctx->dnum * 2 * LK * N * 8) != cudaSuccess) return HE_ENOMEM;
        uint64_t *tmp = ctx_scratch(ctx, (size_t)2 * LK * N + N);
        if (!tmp) {
            cudaFree(key);
            return HE_ENOMEM;
        }
        uint64_t *a = tmp, *e = tmp + (size_t)LK * N;
        int64_t *e_int = reinterpret_cast<int64_t *>(tmp + (size_t)2 * LK * N);
        for (int d = 0; d < ctx->dnum; ++d) {
            const uint64_t nonce = ((uint64_t)g << 8) | (uint64_t)d;
            launch_sample_uniform(ctx, 4, nonce, all, 0, a);
            launch_ntt_fwd(ctx, a, a, 1, all);
            launch_sample_gauss(ctx, 5, nonce, e_int);
            launch_ntt_from_int64(ctx, e_int, e, 1, all, 0);
            launch_keygen_combine(ctx, a, e, g, d, key + (size_t)d * 2 * LK * N);
        }
        if (last_launch() != HE_OK) {
            cudaFree(key);
            return HE_ECUDA;
        }
        {
            std::lock_guard<std::mutex> lock(ctx->sh->mu);
            auto ins = ctx->sh->keys.emplace(g, key);
            if (!ins.second) cudaFree(key);  // another context of the family made it meanwhile
        }
    }
    return HE_OK;
}

int he_encode(he_ctx *ctx, const double *slots, int64_t n_slots, double scale, int level, he_pt *out) {
    if (!ctx || !out || !out->data || (n_slots > 0 && !slots) || n_slots < 0 || n_slots > ctx->n / 2) return HE_EINVAL;
    if (level < 0 || level >= ctx->L) return HE_ELEVEL;
    int64_t *coef = reinterpret_cast<int64_t *>(ctx_scratch(ctx, ctx->n));
    if (!coef) return HE_ENOMEM;
    launch_encode(ctx, slots, n_slots, n_slots, 1, scale, coef);
    launch_ntt_from_int64(ctx, coef, out->data, 1, qmap(level), 0);
    out->level = level;
    out->scale = scale;
    return last_launch();
}

// the encryption as separate launches (sampling, NTTs, combine); tmp: 2 (level+1) N + N words
static void encrypt_steps(he_ctx *ctx, const uint64_t *pt, int level, uint64_t nonce, const uint64_t *nonce_dev, uint64_t *ct, uint64_t *tmp) {
    const size_t N = ctx->n, nl = level + 1;
    uint64_t *a = tmp, *e = tmp + nl * N;
    int64_t *e_int = reinterpret_cast<int64_t *>(tmp + 2 * nl * N);
    const LimbMap m = qmap(level);
    launch_sample_uniform(ctx, 2, nonce, m, 0, a, nonce_dev);
    launch_ntt_fwd(ctx, a, a, 1, m);
    launch_sample_gauss(ctx, 3, nonce, e_int, nonce_dev);
    launch_ntt_from_int64(ctx, e_int, e, 1, m, 0);
    launch_encrypt_combine(ctx, pt, a, e, level, ct);
}

static int encrypt_impl(he_ctx *ctx, const he_pt *pt, uint64_t nonce, const uint64_t *nonce_dev, he_ct *out) {
    if (!ctx || !pt || !out || !pt->data || !out->data) return HE_EINVAL;
    const int level = pt->level;
    if (level < 0 || level >= ctx->L) return HE_ELEVEL;
    const size_t N = ctx->n, nl = level + 1;
    if (launch_encrypt_fused(ctx, pt->data, nullptr, level, nonce, nonce_dev, out->data)) {
        out->level = level;
        out->scale = pt->scale;
        return last_launch();
    }
    uint64_t *tmp = ctx_scratch(ctx, 2 * nl * N + N);
    if (!tmp) return HE_ENOMEM;
    encrypt_steps(ctx, pt->data, level, nonce, nonce_dev, out->data, tmp);
    out->level = level;
    out->scale = pt->scale;
    return last_launch();
}

int he_encrypt(he_ctx *ctx, const he_pt *pt, uint64_t nonce, he_ct *out) { return encrypt_impl(ctx, pt, nonce, nullptr, out); }

int he_encrypt_dnonce(he_ctx *ctx, const he_pt *pt, const uint64_t *nonce_dev, he_ct *out) {
    if (!nonce_dev) return HE_EINVAL;
    return encrypt_impl(ctx, pt, 0, nonce_dev, out);
}

int he_decrypt(he_ctx *ctx, const he_ct *ct, double *slots_out) {
    if (!ctx || !ct || !ct->data || !slots_out) return HE_EINVAL;
    if (ct->level < 0 || ct->level >= ctx->L) return HE_ELEVEL;
    double *coef = reinterpret_cast<double *>(ctx_scratch(ctx, ctx->n));
    if (!coef) return HE_ENOMEM;
    launch_decrypt_coeffs(ctx, ct->data, ct->level, 1, coef, nullptr);
    launch_decode(ctx, coef, 1, ct->scale, slots_out);
    return last_launch();
}

int he_add(he_ctx *ctx, const he_ct *a, const he_ct *b, he_ct *out) {
    if (!ctx || !a || !b || !out || !a->data || !b->data || !out->data) return HE_EINVAL;
    if (a->level != b->level || a->level < 0 || a->level >= ctx->L) return HE_ELEVEL;
    if (fabs(a->scale - b->scale) > 1e-9 * fabs(a->scale)) return HE_ESCALE;
    launch_add(ctx, a->data, b->data, out->data, 2, qmap(a->level));
    out->level = a->level;
    out->scale = a->scale;
    return last_launch();
}

int he_add_plain(he_ctx *ctx, const he_ct *ct, const he_pt *pt, he_ct *out) {
    if (!ctx || !ct || !pt || !out || !ct->data || !pt->data || !out->data) return HE_EINVAL;
    if (ct->level < 0 || ct->level >= ctx->L || pt->level < ct->level) return HE_ELEVEL;
    if (fabs(ct->scale - pt->scale) > 1e-9 * fabs(ct->scale)) return HE_ESCALE;
    const size_t nl = ct->level + 1, N = ctx->n;
    if (out->data != ct->data &&
        cudaMemcpyAsync(out->data + nl * N, ct->data + nl * N, nl * N * sizeof(uint64_t), cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess)
        return HE_ECUDA;
    launch_add(ctx, ct->data, pt->data, out->data, 1, qmap(ct->level));
    out->level = ct->level;
    out->scale = ct->scale;
    return last_launch();
}

int he_mul_plain(he_ctx *ctx, const he_ct *ct, const he_pt *pt, he_ct *out) {
    if (!ctx || !ct || !pt || !out || !ct->data || !pt->data || !out->data) return HE_EINVAL;
    if (ct->level < 0 || ct->level >= ctx->L || pt->level < ct->level) return HE_ELEVEL;
    launch_mul_plain(ctx, ct->data, pt->data, out->data, ct->level);
    out->level = ct->level;
    out->scale = ct->scale * pt->scale;
    return last_launch();
}

int he_rescale(he_ctx *ctx, const he_ct *in, he_ct *out) {
    if (!ctx || !in || !in->data) return HE_EINVAL;
    if (in->level < 1 || in->level >= ctx->L) return HE_ELEVEL;
    if (!out || !out->data) return HE_EINVAL;
    uint64_t *tmp = ctx_scratch(ctx, 2 * (size_t)ctx->n);
    if (!tmp) return HE_ENOMEM;
    const int level = in->level;
    const double scale = in->scale / (double)ctx->primes[level];
    launch_rescale(ctx, in->data, level, out->data, tmp);
    out->level = level - 1;
    out->scale = scale;
    return last_launch();
}

int he_rotate_hoisted(he_ctx *ctx, const he_ct *in, const int32_t *steps, int k, he_ct *outs) {
    if (!ctx || !in || !in->data || k < 0 || (k > 0 && (!steps || !outs))) return HE_EINVAL;
    const int level = in->level;
    if (level < 0 || level >= ctx->L) return HE_ELEVEL;
    const size_t N = ctx->n, nl = level + 1, ct_words = 2 * nl * N;
    std::vector<RotJob> jobs;
    jobs.reserve(k);
    std::vector<int> copies;
    for (int i = 0; i < k; ++i) {
        // an output must not overlap the input, whose c0 every rotation still reads
        if (!outs[i].data || (outs[i].data < in->data + ct_words && in->data < outs[i].data + ct_words)) return HE_EINVAL;
        const int64_t half = ctx->n / 2;
        if (((int64_t)steps[i] % half + half) % half == 0) {  // RotL by a multiple of N/2 is the identity
            copies.push_back(i);
            continue;
        }
        const uint32_t g = galois_of(ctx, steps[i]);
        const uint64_t *key = ctx->sh->key(g);
        if (!key) return HE_EKEY;
        jobs.push_back(RotJob{in->data, outs[i].data, key, g, 0});
    }
    for (int i : copies)
        if (cudaMemcpyAsync(outs[i].data, in->data, ct_words * sizeof(uint64_t), cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess)
            return HE_ECUDA;
    const int n_jobs = (int)jobs.size();
    if (n_jobs > 0) {
        // one ModUp of c1 (O4), then the key switch of every rotation, two launches per 64
        const ModUpConst &mu = ctx->modup[level];
        const size_t wD = (size_t)mu.ndig * mu.ext * N, wc = nl * N, wp = keyswitch_many_pc_words(ctx, n_jobs);
        uint64_t *s = ctx_scratch(ctx, wD + wc + wp);
        if (!s) return HE_ENOMEM;
        uint64_t *D = s, *coef = D + wD, *pc = coef + wc;
        launch_modup(ctx, in->data + nl * N, level, D, coef);
        launch_keyswitch_many(ctx, jobs.data(), n_jobs, level, D, 0, pc);
    }
    for (int i = 0; i < k; ++i) {
        outs[i].level = level;
        outs[i].scale = in->scale;
    }
    return last_launch();
}

int he_rotate(he_ctx *ctx, const he_ct *in, int32_t step, he_ct *out) { return he_rotate_hoisted(ctx, in, &step, 1, out); }

int he_rotate_many(he_ctx *ctx, const he_ct *ins, const int32_t *steps, int count, he_ct *outs) {
    if (!ctx || count < 0 || (count > 0 && (!ins || !steps || !outs))) return HE_EINVAL;
    if (count == 0) return HE_OK;
    const int level = ins[0].level;
    if (level < 0 || level >= ctx->L) return HE_ELEVEL;
    const size_t N = ctx->n, ct_words = 2 * (size_t)(level + 1) * N;
    for (int i = 0; i < count; ++i) {
        if (!ins[i].data || !outs[i].data) return HE_EINVAL;
        if (ins[i].level != level) return HE_ELEVEL;
        for (int j = 0; j < count; ++j)  // outputs are written while later jobs still read inputs
            if (outs[i].data < ins[j].data + ct_words && ins[j].data < outs[i].data + ct_words) return HE_EINVAL;
    }
    std::vector<RotJob> jobs;
    jobs.reserve(count);
    for (int i = 0; i < count; ++i) {
        const int64_t half = ctx->n / 2;
        if (((int64_t)steps[i] % half + half) % half == 0) {  // RotL by a multiple of N/2 is the identity
            if (cudaMemcpyAsync(outs[i].data, ins[i].data, ct_words * sizeof(uint64_t), cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess)
                return HE_ECUDA;
            continue;
        }
        const uint32_t g = galois_of(ctx, steps[i]);
        const uint64_t *key = ctx->sh->key(g);
        if (!key) return HE_EKEY;
        jobs.push_back(RotJob{ins[i].data, outs[i].data, key, g, 0});
    }
    const int n_jobs = (int)jobs.size();
    if (n_jobs > 0) {
        // chunks of HE_ROT_CHUNK rotations, their job tables passed as kernel parameters; the
        // chunks reuse one scratch region in stream order
        const int chunk = n_jobs < HE_ROT_CHUNK ? n_jobs : HE_ROT_CHUNK;
        uint64_t *s = ctx_scratch(ctx, (size_t)chunk * rotate_many_words(ctx, level));
        if (!s) return HE_ENOMEM;
        for (int c0 = 0; c0 < n_jobs; c0 += chunk) launch_rotate_many(ctx, jobs.data() + c0, std::min(chunk, n_jobs - c0), level, s);
    }
    for (int i = 0; i < count; ++i) {
        outs[i].level = level;
        outs[i].scale = ins[i].scale;
    }
    return last_launch();
}

int he_plan_create(int64_t m, int64_t n, int64_t slots, he_plan **out) {
    if (!out) return HE_EINVAL;
    *out = nullptr;
    if (m < 1 || n < 1 || slots < 1 || (slots & (slots - 1)) || m > (1ll << 40) || n > (1ll << 40)) return HE_EINVAL;
    he_plan *p = new (std::nothrow) he_plan();
    if (!p) return HE_ENOMEM;
    auto up = [](int64_t v) {
        int64_t r = 1;
        while (r < v) r <<= 1;
        return r;
    };
    p->m = m;
    p->n = n;
    p->slots = slots;
    p->mp = up(m);
    p->np = up(n);
    p->mb = std::min(p->mp, slots);
    p->nb = std::min(p->np, slots);
    p->row_blocks = p->mp / p->mb;
    p->col_blocks = p->np / p->nb;
    p->m_prime = std::max<int64_t>(1, p->mb * p->nb / slots);
    p->blocks = slots / p->nb;
    p->baby = 0;
    *out = p;
    return HE_OK;
}

int he_plan_set_baby_steps(he_plan *p, int64_t baby) {
    if (!p || baby < 0 || (baby & (baby - 1)) || (baby && p->m_prime % baby)) return HE_EINVAL;
    p->baby = baby;
    return HE_OK;
}

int he_plan_rotation_steps(const he_plan *p, int32_t *steps, int *n_steps) {
    if (!p || !n_steps) return HE_EINVAL;
    std::vector<int32_t> v;
    if (p->baby == 0) {
        for (int64_t i = 1; i < p->m_prime; ++i) v.push_back((int32_t)i);
    } else {
        for (int64_t b = 1; b < p->baby; ++b) v.push_back((int32_t)b);
        for (int64_t g = 1; g < p->m_prime / p->baby; ++g) v.push_back((int32_t)(g * p->baby));
    }
    if (steps) std::copy(v.begin(), v.end(), steps);
    *n_steps = (int)v.size();
    return HE_OK;
}

int he_plan_query(const he_plan *p, int64_t *info) {
    if (!p || !info) return HE_EINVAL;
    const int64_t v[11] = {p->m, p->n, p->slots, p->mp, p->np, p->mb, p->nb, p->row_blocks, p->col_blocks, p->m_prime, p->blocks};
    memcpy(info, v, sizeof(v));
    return HE_OK;
}

void he_plan_free(he_plan *p) { delete p; }

static int ptmat_alloc(he_ctx *ctx, const he_plan *plan, int level, double scale, he_ptmat **out) {
    if (!ctx || !plan || !out) return HE_EINVAL;
    *out = nullptr;
    if (plan->slots != ctx->n / 2) return HE_EINVAL;
    if (level < 1 || level >= ctx->L) return HE_ELEVEL;
    he_ptmat *pm = new (std::nothrow) he_ptmat();
    if (!pm) return HE_ENOMEM;
    pm->ctx = ctx;
    pm->plan = *plan;
    pm->level = level;
    pm->scale = scale;
    pm->ext = level + 1 + ctx->K;
    const size_t count = (size_t)plan->row_blocks * plan->col_blocks * plan->m_prime;
    if (cudaMalloc(&pm->data, count * pm->ext * ctx->n * 8) != cudaSuccess) {
        delete pm;
        return HE_ENOMEM;
    }
    *out = pm;
    return HE_OK;
}

// The first matrix encoded on a context times its transform (one launch of many limb-polys) in
// every NTT form, one CTA or a 2-CTA pair per limb-poly or two phases (the same values: the
// launch is repeated on the same input), and keeps the fastest for every such launch of the
// context; not under stream capture, nor for launches small enough for the cluster form.
// Synchronises the stream.
static void tune_ntt_form(he_ctx *ctx, const int64_t *coef, uint64_t *out, int groups, const LimbMap &map) {
    const int polys = groups * map.n;
    if (use_cluster(ctx->log_n, polys) || ctx->log_n < 12 || ctx->log_n > 14) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(ctx->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return;
    }
    int best = 0;
    for (int f = 0; f < HE_NTT_FORMS; ++f) {
        ctx->ntt_form = f;
        float ms = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {
            cudaEventRecord(e0, ctx->stream);
            launch_ntt_from_int64(ctx, coef, out, groups, map, 1);
            cudaEventRecord(e1, ctx->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) break;
            float t = 0.0f;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0 && t < ms) ms = t;
        }
        ctx->ntt_form_ms[f] = ms;
        if (ms < ctx->ntt_form_ms[best]) best = f;
    }
    ctx->ntt_form = best;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
}

static int ptmat_encode(he_ctx *ctx, he_ptmat *pm, const double *X, int trans) {
    if (!ctx || !pm || !X || !same_family(pm->ctx, ctx)) return HE_EINVAL;
    const he_plan &p = pm->plan;
    const size_t N = ctx->n, count = (size_t)p.row_blocks * p.col_blocks * p.m_prime;
    uint64_t *s = ctx_scratch(ctx, count * (N / 2) + count * N);
    if (!s) return HE_ENOMEM;
    double *slots = reinterpret_cast<double *>(s);
    int64_t *coef = reinterpret_cast<int64_t *>(s + count * (N / 2));
    if (!launch_encode_matrix(ctx, p, X, trans, (int)count, pm->scale, coef)) {
        launch_layout_matrix(ctx, p, X, slots, trans);
        launch_encode(ctx, slots, N / 2, N / 2, (int)count, pm->scale, coef);
    }
    if (ctx->ntt_form < 0) tune_ntt_form(ctx, coef, pm->data, (int)count, qpmap(ctx, pm->level));
    cudaEvent_t *ev = prof_pair(ctx, HE_PROF_MATRIX_NTT);
    if (ev) cudaEventRecord(ev[0], ctx->stream);
    launch_ntt_from_int64(ctx, coef, pm->data, (int)count, qpmap(ctx, pm->level), 1);
    if (ev) cudaEventRecord(ev[1], ctx->stream);
    pm->enc_gen++;
    if (pm->fuse_state == 1 && pm->fused) {  // keep the fused key tables in step with the plaintexts
        launch_fuse_keys(ctx, pm);
        pm->fused_gen = pm->enc_gen;
    }
    return last_launch();
}

int he_ptmat_encode(he_ctx *ctx, he_ptmat *pm, const double *X) { return ptmat_encode(ctx, pm, X, 0); }
int he_ptmat_encode_transposed(he_ctx *ctx, he_ptmat *pm, const double *Xt) { return ptmat_encode(ctx, pm, Xt, 1); }

static int encode_matrix(he_ctx *ctx, const he_plan *plan, const double *X, int level, int trans, he_ptmat **out) {
    if (!ctx || !X) return HE_EINVAL;
    if (level < 1 || level >= ctx->L) return HE_ELEVEL;
    int rc = ptmat_alloc(ctx, plan, level, (double)ctx->primes[level], out);
    if (rc != HE_OK) return rc;
    rc = ptmat_encode(ctx, *out, X, trans);
    if (rc != HE_OK) {
        he_ptmat_free(*out);
        *out = nullptr;
    }
    return rc;
}

int he_encode_matrix(he_ctx *ctx, const he_plan *plan, const double *X, int level, he_ptmat **out) {
    return encode_matrix(ctx, plan, X, level, 0, out);
}
int he_encode_matrix_transposed(he_ctx *ctx, const he_plan *plan, const double *Xt, int level, he_ptmat **out) {
    return encode_matrix(ctx, plan, Xt, level, 1, out);
}

int he_ptmat_export(he_ctx *ctx, const he_ptmat *pm, uint64_t *coeffs_out) {
    if (!ctx || !pm || !coeffs_out || !same_family(pm->ctx, ctx)) return HE_EINVAL;
    const he_plan &p = pm->plan;
    const int count = (int)(p.row_blocks * p.col_blocks * p.m_prime);
    const LimbMap m = qpmap(ctx, pm->level);
    const int64_t gs = (int64_t)m.n * ctx->n;
    launch_from_mont(ctx, pm->data, coeffs_out, count, m);
    launch_ntt_inv_strided(ctx, coeffs_out, gs, coeffs_out, gs, count, m);
    return last_launch();
}

int he_ptmat_import(he_ctx *ctx, const he_plan *plan, const uint64_t *coeffs, int level, double scale, he_ptmat **out) {
    if (!coeffs) return HE_EINVAL;
    int rc = ptmat_alloc(ctx, plan, level, scale, out);
    if (rc != HE_OK) return rc;
    he_ptmat *pm = *out;
    const size_t count = (size_t)plan->row_blocks * plan->col_blocks * plan->m_prime;
    const LimbMap m = qpmap(ctx, level);
    const int64_t gs = (int64_t)m.n * ctx->n;
    launch_ntt_fwd_strided(ctx, coeffs, gs, pm->data, gs, (int)count, m, 1);
    rc = last_launch();
    if (rc != HE_OK) {
        he_ptmat_free(pm);
        *out = nullptr;
    }
    return rc;
}

void he_ptmat_free(he_ptmat *pm) {
    if (!pm) return;
    cudaStreamSynchronize(pm->ctx->stream);
    cudaFree(pm->fused);
    cudaFree(pm->data);
    cudaFree(pm->d_keys);
    cudaFree(pm->d_galois);
    delete pm;
}

int he_encode_vector(he_ctx *ctx, const he_plan *plan, const double *y, double scale, int level, he_pt *outs) {
    if (!ctx || !plan || !y || !outs || plan->slots != ctx->n / 2) return HE_EINVAL;
    if (level < 0 || level >= ctx->L) return HE_ELEVEL;
    const size_t N = ctx->n, C = plan->col_blocks;
    for (size_t c = 0; c < C; ++c)
        if (!outs[c].data) return HE_EINVAL;
    uint64_t *s = ctx_scratch(ctx, C * (N / 2) + C * N);
    if (!s) return HE_ENOMEM;
    double *slots = reinterpret_cast<double *>(s);
    int64_t *coef = reinterpret_cast<int64_t *>(s + C * (N / 2));
    if (!launch_encode_vector(ctx, *plan, y, (int)C, scale, coef)) {
        launch_layout_vector(ctx, *plan, y, slots);
        launch_encode(ctx, slots, N / 2, N / 2, (int)C, scale, coef);
    }
    for (size_t c = 0; c < C; ++c) {
        launch_ntt_from_int64(ctx, coef + c * N, outs[c].data, 1, qmap(level), 0);
        outs[c].level = level;
        outs[c].scale = scale;
    }
    return last_launch();
}

int he_encrypt_vector(he_ctx *ctx, const he_plan *plan, const double *y, double scale, int level, uint64_t nonce, const uint64_t *nonce_dev,
                      he_ct *outs) {
    if (!ctx || !plan || !y || !outs || plan->slots != ctx->n / 2) return HE_EINVAL;
    if (level < 0 || level >= ctx->L) return HE_ELEVEL;
    const size_t N = ctx->n, C = plan->col_blocks, nl = level + 1;
    for (size_t c = 0; c < C; ++c)
        if (!outs[c].data) return HE_EINVAL;
    const bool fused = use_cluster(ctx->log_n, 2 * (int)nl);  // the condition of launch_encrypt_fused
    // slots, integer coefficients, and (separate launches only) one plaintext and the encryption's temporaries
    const size_t w_slots = C * (N / 2), w_coef = C * N, w_pt = fused ? 0 : nl * N, w_tmp = fused ? 0 : 2 * nl * N + N;
    uint64_t *s = ctx_scratch(ctx, w_slots + w_coef + w_pt + w_tmp);
    if (!s) return HE_ENOMEM;
    double *slots = reinterpret_cast<double *>(s);
    int64_t *coef = reinterpret_cast<int64_t *>(s + w_slots);
    if (!launch_encode_vector(ctx, *plan, y, (int)C, scale, coef)) {
        launch_layout_vector(ctx, *plan, y, slots);
        launch_encode(ctx, slots, N / 2, N / 2, (int)C, scale, coef);
    }
    for (size_t c = 0; c < C; ++c) {
        const uint64_t *nd = nonce_dev ? nonce_dev + c : nullptr;
        if (fused) {
            launch_encrypt_fused(ctx, nullptr, coef + c * N, level, nonce + c, nd, outs[c].data);
        } else {
            uint64_t *pt = s + w_slots + w_coef, *tmp = pt + w_pt;
            launch_ntt_from_int64(ctx, coef + c * N, pt, 1, qmap(level), 0);
            encrypt_steps(ctx, pt, level, nonce + c, nd, outs[c].data, tmp);
        }
        outs[c].level = level;
        outs[c].scale = scale;
    }
    return last_launch();
}

// Build pm's fused key tables, time the fused forms against the two-level form's tuned time and
// keep the tables only if faster (he_set_key_fusion).  A table over the size limit or an
// allocation failure leaves the matrix on the two-level form.  Synchronises the stream.
static int fuse_try(he_ctx *ctx, he_ptmat *pm, const uint64_t *ct, const uint64_t *D, uint64_t *acc, uint64_t *cacc) {
    const he_plan &p = pm->plan;
    const size_t bytes =
        (size_t)p.row_blocks * p.col_blocks * (p.m_prime - 1) * 2 * ctx->modup[pm->level].ndig * pm->ext * ctx->n * sizeof(uint64_t);
    pm->fuse_state = -1;
    if (pm->fvariant_pin < 0 && (bytes > ctx->sh->fuse_max || pm->variant < 0)) return HE_OK;
    if (cudaMalloc(&pm->fused, bytes) != cudaSuccess) {
        cudaGetLastError();
        pm->fused = nullptr;
        return HE_OK;
    }
    launch_fuse_keys(ctx, pm);
    pm->fused_gen = pm->enc_gen;
    if (pm->fvariant_pin >= 0) {
        pm->fvariant = pm->fvariant_pin;
        pm->fuse_state = 1;
        return last_launch();
    }
    const int rc = tune_matmult_fused(ctx, pm, ct, D, acc, cacc);
    if (rc != HE_OK) return rc;
    if (pm->fvariant >= 0 && pm->fuse_ms[pm->fvariant] < pm->tune_ms[pm->variant]) {
        pm->fuse_state = 1;
        return HE_OK;
    }
    cudaFree(pm->fused);  // the tuning synchronised the stream
    pm->fused = nullptr;
    return HE_OK;
}

int he_set_key_fusion(he_ctx *ctx, int mode, size_t max_bytes) {
    if (!ctx || mode < 0 || mode > 2) return HE_EINVAL;
    ctx->sh->key_fusion = mode;
    ctx->sh->fuse_max = max_bytes ? max_bytes : ((size_t)8 << 30);
    return HE_OK;
}

int he_ptmat_key_fusion(const he_ptmat *pm, int *state, int *variant, float *ms) {
    if (!pm || !state || !variant) return HE_EINVAL;
    *state = pm->fuse_state;
    *variant = pm->fvariant;
    if (ms)
        for (int v = 0; v < mm_variant_count(); ++v) ms[v] = pm->fuse_ms[v];
    return HE_OK;
}

int he_ptmat_set_key_fusion(he_ptmat *pm, int on, int variant) {
    if (!pm || on < 0 || on > 1 || variant < -1 || variant >= mm_variant_count()) return HE_EINVAL;
    if (on && variant >= 0 && !mm_variant_fusable(variant, pm->ctx->modup[pm->level].ndig)) return HE_EINVAL;
    pm->fvariant_pin = on ? variant : -1;
    if (!on) {
        if (pm->fused) {
            cudaStreamSynchronize(pm->ctx->stream);
            cudaFree(pm->fused);
            pm->fused = nullptr;
        }
        pm->fuse_state = -1;
    } else if (pm->fuse_state < 0) {
        pm->fuse_state = 0;
    } else if (pm->fuse_state == 1 && variant >= 0) {
        pm->fvariant = variant;
    }
    return HE_OK;
}

// resolve the Galois keys of rotation steps 1..m'-1 into a device pointer table, once
int ptmat_bind_keys(he_ctx *ctx, he_ptmat *pm) {
    const int64_t steps = pm->plan.m_prime - 1;
    if (steps <= 0 || pm->d_keys) return HE_OK;
    std::vector<const uint64_t *> ptrs(steps);
    std::vector<uint32_t> gal(steps);
    for (int64_t i = 0; i < steps; ++i) {
        gal[i] = galois_of(ctx, i + 1);
        ptrs[i] = ctx->sh->key(gal[i]);
        if (!ptrs[i]) return HE_EKEY;
    }
    if (cudaMalloc(&pm->d_keys, steps * sizeof(uint64_t *)) != cudaSuccess) return HE_ENOMEM;
    if (cudaMalloc(&pm->d_galois, steps * sizeof(uint32_t)) != cudaSuccess) return HE_ENOMEM;
    if (cudaMemcpy(pm->d_keys, ptrs.data(), steps * sizeof(uint64_t *), cudaMemcpyHostToDevice) != cudaSuccess) return HE_ECUDA;
    if (cudaMemcpy(pm->d_galois, gal.data(), steps * sizeof(uint32_t), cudaMemcpyHostToDevice) != cudaSuccess) return HE_ECUDA;
    pm->galois = gal;
    return HE_OK;
}

int he_matmult_plain_cipher(he_ctx *ctx, const he_plan *plan, const he_ptmat *pm_c, const he_ct *ins, int n_in, he_ct *outs, int n_out) {
    if (!ctx || !plan || !pm_c || !ins || !outs || !same_family(pm_c->ctx, ctx)) return HE_EINVAL;
    he_ptmat *pm = const_cast<he_ptmat *>(pm_c);
    const he_plan &p = pm->plan;
    if (p.m != plan->m || p.n != plan->n || p.slots != plan->slots) return HE_EINVAL;
    if (n_in != p.col_blocks || n_out != p.row_blocks) return HE_EINVAL;
    const int level = pm->level;
    for (int c = 0; c < n_in; ++c) {
        if (!ins[c].data) return HE_EINVAL;
        if (ins[c].level != level) return HE_ELEVEL;
    }
    for (int r = 0; r < n_out; ++r)
        if (!outs[r].data) return HE_EINVAL;
    if (p.baby) return matmult_bsgs(ctx, pm, ins, outs);
    int rc = ptmat_bind_keys(ctx, pm);
    if (rc != HE_OK) return rc;
    const ModUpConst &mu = ctx->modup[level];
    const size_t N = ctx->n, nl = level + 1, ext = mu.ext, C = p.col_blocks;
    const bool rot = p.m_prime > 1;
    const size_t wD = rot ? C * mu.ndig * ext * N : 0, wc = nl * N, wa = 2 * ext * N, wcc = 2 * nl * N, wsum = 2 * nl * N,
                 wt = 2 * (ctx->K > 1 ? ctx->K : 1) * N + 2 * N;
    uint64_t *s = ctx_scratch(ctx, wD + wc + wa + wcc + wsum + wt);
    if (!s) return HE_ENOMEM;
    uint64_t *D = s, *coef = D + wD, *acc = coef + wc, *cacc = acc + wa, *sum = cacc + wcc, *tmp = sum + wsum;
    if (rot)
        for (size_t c = 0; c < C; ++c) launch_modup(ctx, ins[c].data + nl * N, level, D + c * mu.ndig * ext * N, coef);
    if (pm->variant < 0) {
        if (rot) {
            rc = tune_matmult_loop(ctx, pm, ins[0].data, D, acc, cacc);
            if (rc != HE_OK) return rc;
        } else {
            pm->variant = 0;
        }
    }
    if (rot) {
        const bool reused = pm->mm_gen == pm->enc_gen;  // this encoding was multiplied before
        pm->mm_gen = pm->enc_gen;
        const int mode = ctx->sh->key_fusion;
        const bool pinned = pm->fvariant_pin >= 0;
        if (pm->fuse_state == 0 && (pinned || (mode > 0 && (reused || mode == 2))) && mu.ndig <= 3 && !capturing(ctx->stream)) {
            rc = fuse_try(ctx, pm, ins[0].data, D, acc, cacc);
            if (rc != HE_OK) return rc;
        }
    }
    for (int r = 0; r < n_out; ++r) {
        for (size_t c = 0; c < C; ++c)
            launch_matmult_loop(ctx, pm, r, (int)c, ins[c].data, rot ? D + c * mu.ndig * ext * N : nullptr, acc, cacc, c > 0);
        const uint64_t *pre = cacc;
        if (rot && moddown_rescale_fused(ctx, level)) {
            launch_moddown_rescale(ctx, acc, level, cacc, cacc + nl * N, outs[r].data, tmp);
        } else {
            if (rot) {
                launch_moddown(ctx, acc, level, 2, cacc, cacc + nl * N, sum, tmp);
                pre = sum;
            }
            launch_rescale(ctx, pre, level, outs[r].data, tmp);
        }
        outs[r].level = level - 1;
        outs[r].scale = ins[0].scale * pm->scale / (double)ctx->primes[level];
    }
    return last_launch();
}

void he_batch_free(he_batch *b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->have_graph) cudaGraphExecDestroy(b->exec);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->stream) cudaStreamDestroy(b->stream);
    cudaFreeHost(b->h_jobs);
    cudaFree(b->d_jobs);
    for (int v = 0; v < HE_MM_MAX_VARIANTS; ++v) cudaFree(b->d_order_v[v]);
    cudaFree(b->d_counter);
    cudaFree(b->mem);
    delete b;
}

// Allocate a batch of `count` job slots at `level`.  With pms, the slots hold those MatMults
// (work order sorted by decreasing m'); without, they start empty (m' = 0, skipped by every
// kernel) and a scheduler fills them before each launch.
int batch_create_impl(he_ctx *ctx, int count, int level, const he_ptmat *const *pms, he_batch **out) {
    he_batch *b = new (std::nothrow) he_batch();
    if (!b) return HE_ENOMEM;
    b->ctx = ctx;
    b->count = count;
    if (pms) b->pms.assign(pms, pms + count);
    const ModUpConst &mu = ctx->modup[level];
    const int64_t N = ctx->n, nq = level + 1;
    BatchGeom &g = b->bg;
    g.ndig = mu.ndig;
    g.ext = mu.ext;
    g.nq = (int)nq;
    g.L = ctx->L;
    g.LK = ctx->L + ctx->K;
    g.K = ctx->K;
    g.level = level;
    g.d_words = (int64_t)mu.ndig * mu.ext * N;
    g.coef_words = nq * N;
    g.acc_words = 2 * (int64_t)mu.ext * N;
    g.cacc_words = 2 * nq * N;
    g.sum_words = 2 * nq * N;
    g.tmp_words = 2 * (int64_t)ctx->K * N + 2 * N;
    const int64_t per = g.d_words + g.coef_words + g.acc_words + g.cacc_words + g.sum_words + g.tmp_words;
    bool ok = cudaMalloc(&b->mem, (size_t)per * count * 8) == cudaSuccess && cudaMallocHost(&b->h_jobs, sizeof(MMJob) * count) == cudaSuccess &&
              cudaMalloc(&b->d_jobs, sizeof(MMJob) * count) == cudaSuccess && cudaMalloc(&b->d_counter, sizeof(unsigned int)) == cudaSuccess;
    if (!ok) {
        he_batch_free(b);
        return HE_ENOMEM;
    }
    uint64_t *m = b->mem;
    g.D = m;
    m += g.d_words * count;
    g.coef = m;
    m += g.coef_words * count;
    g.acc = m;
    m += g.acc_words * count;
    g.cacc = m;
    m += g.cacc_words * count;
    g.sum = m;
    m += g.sum_words * count;
    g.tmp = m;
    for (int j = 0; j < count; ++j) {
        MMJob &jb = b->h_jobs[j];
        jb = MMJob{};
        if (pms) {
            jb.pts = pms[j]->data;
            jb.keys = pms[j]->d_keys;
            jb.galois = pms[j]->d_galois;
            jb.m_prime = (int32_t)pms[j]->plan.m_prime;
        }
    }
    // issue order, per loop-kernel variant (tile widths differ): tile-major, then limb, then
    // jobs by decreasing m', so the CTAs in flight read the same key tiles (shared by every job)
    // and long jobs start first
    std::vector<int> by_len(count);
    for (int j = 0; j < count; ++j) by_len[j] = j;
    std::stable_sort(by_len.begin(), by_len.end(), [&](int a, int c) { return b->h_jobs[a].m_prime > b->h_jobs[c].m_prime; });
    for (int v = 0; v < mm_variant_count(); ++v) {
        const int tiles = (int)((N + mm_variant_tile(v) - 1) / mm_variant_tile(v));
        std::vector<int32_t> order;
        order.reserve((size_t)tiles * mu.ext * count);
        for (int t = 0; t < tiles; ++t)
            for (int u = 0; u < mu.ext; ++u)
                for (int j : by_len) order.push_back((int32_t)(((int64_t)j * mu.ext + u) * tiles + t));
        b->n_items_v[v] = (int)order.size();
        if (cudaMalloc(&b->d_order_v[v], sizeof(int32_t) * order.size()) != cudaSuccess ||
            cudaMemcpy(b->d_order_v[v], order.data(), sizeof(int32_t) * order.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
            he_batch_free(b);
            return HE_ENOMEM;
        }
    }
    b->variant = pms ? -1 : ctx->batch_variant;
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (int v = 0; v < mm_variant_count(); ++v) b->ctas_v[v] = mm_batch_ctas_per_sm(v, mu.ndig) * (sms > 0 ? sms : 1);
    ok = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        he_batch_free(b);
        return HE_ENOMEM;
    }
    *out = b;
    return HE_OK;
}

// Launch the batch (capturing its graph on first use) on its own stream; the job table must be filled.
int batch_launch(he_ctx *ctx, he_batch *b) {
    if (!b->have_graph) {
        cudaGraph_t graph;
        if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return HE_ECUDA;
        int rc = launch_matmult_batch(ctx, b, b->stream);
        cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
        if (rc != HE_OK || e != cudaSuccess) return HE_ECUDA;
        e = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return HE_ECUDA;
        b->have_graph = true;
    } else {
        ctx->launches += 7;
    }
    if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess) return HE_ECUDA;
    return cudaEventRecord(b->ev_out, b->stream) == cudaSuccess ? HE_OK : HE_ECUDA;
}

int he_batch_create(he_ctx *ctx, int count, const he_plan *const *plans, const he_ptmat *const *pms, he_batch **out) {
    if (!ctx || !out || count < 1 || !plans || !pms) return HE_EINVAL;
    *out = nullptr;
    const int level = pms[0] ? pms[0]->level : -1;
    for (int j = 0; j < count; ++j) {
        if (!plans[j] || !pms[j] || !same_family(pms[j]->ctx, ctx)) return HE_EINVAL;
        const he_plan &p = pms[j]->plan;
        if (p.m != plans[j]->m || p.n != plans[j]->n || p.row_blocks != 1 || p.col_blocks != 1 || p.baby) return HE_EINVAL;
        if (pms[j]->level != level) return HE_ELEVEL;
        int rc = ptmat_bind_keys(ctx, const_cast<he_ptmat *>(pms[j]));
        if (rc != HE_OK) return rc;
    }
    return batch_create_impl(ctx, count, level, pms, out);
}

int he_batch_run(he_ctx *ctx, he_batch *b, const he_ct *ins, he_ct *outs) {
    if (!ctx || !b || b->ctx != ctx || !ins || !outs || b->pms.empty()) return HE_EINVAL;
    const int level = b->bg.level;
    for (int j = 0; j < b->count; ++j) {
        if (!ins[j].data || !outs[j].data) return HE_EINVAL;
        if (ins[j].level != level) return HE_ELEVEL;
    }
    // the previous run's table copy must be done before the host table is rewritten
    if (b->have_graph && cudaEventSynchronize(b->ev_out) != cudaSuccess) return HE_ECUDA;
    for (int j = 0; j < b->count; ++j) {
        b->h_jobs[j].ct = ins[j].data;
        b->h_jobs[j].out = outs[j].data;
    }
    if (cudaEventRecord(b->ev_in, ctx->stream) != cudaSuccess || cudaStreamWaitEvent(b->stream, b->ev_in, 0) != cudaSuccess) return HE_ECUDA;
    if (b->variant < 0) {
        // first run: time the whole batch once per loop-kernel variant (same results), keep the fastest
        cudaEvent_t e0, e1;
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return HE_ECUDA;
        int best = 0;
        float best_ms = 1e30f;
        for (int v = 0; v < mm_variant_count(); ++v) {
            b->variant = v;
            float ms = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {  // one untimed run, then the better of two
                cudaEventRecord(e0, b->stream);
                if (launch_matmult_batch(ctx, b, b->stream) != HE_OK) break;
                cudaEventRecord(e1, b->stream);
                if (cudaEventSynchronize(e1) != cudaSuccess) break;
                float t = 0.0f;
                cudaEventElapsedTime(&t, e0, e1);
                if (rep > 0 && t < ms) ms = t;
            }
            b->tune_ms[v] = ms;
            if (ms < best_ms) {
                best_ms = ms;
                best = v;
            }
        }
        // then the stage form (one-CTA or cluster ModUp / ModDown / rescale) with that variant
        b->variant = best;
        int best_form = 0;
        for (int f = 0; f < 2; ++f) {
            b->stage_form = f;
            float ms = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {
                cudaEventRecord(e0, b->stream);
                if (launch_matmult_batch(ctx, b, b->stream) != HE_OK) break;
                cudaEventRecord(e1, b->stream);
                if (cudaEventSynchronize(e1) != cudaSuccess) break;
                float t = 0.0f;
                cudaEventElapsedTime(&t, e0, e1);
                if (rep > 0 && t < ms) ms = t;
            }
            b->stage_ms[f] = ms;
            if (ms < b->stage_ms[best_form]) best_form = f;
        }
        b->stage_form = best_form;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        ctx->batch_variant = best;
    }
    int rc = batch_launch(ctx, b);
    if (rc != HE_OK) return rc;
    if (cudaStreamWaitEvent(ctx->stream, b->ev_out, 0) != cudaSuccess) return HE_ECUDA;
    for (int j = 0; j < b->count; ++j) {
        outs[j].level = level - 1;
        outs[j].scale = ins[j].scale * b->pms[j]->scale / (double)ctx->primes[level];
    }
    return HE_OK;
}

int he_loop_variant_count(void) { return mm_variant_count(); }

int he_loop_variant_shape(int v, int *vec, int *groups, int *stages, int *gathers) {
    if (v < 0 || v >= mm_variant_count() || !vec || !groups || !stages || !gathers) return HE_EINVAL;
    mm_variant_shape(v, vec, groups, stages, gathers);
    return HE_OK;
}

int he_ptmat_tuning(const he_ptmat *pm, int *variant, float *ms) {
    if (!pm || !variant) return HE_EINVAL;
    *variant = pm->variant;
    if (ms)
        for (int v = 0; v < mm_variant_count(); ++v) ms[v] = pm->tune_ms[v];
    return HE_OK;
}

int he_ptmat_set_variant(he_ptmat *pm, int v) {
    if (!pm || v < -1 || v >= mm_variant_count()) return HE_EINVAL;
    pm->variant = v;
    return HE_OK;
}

int he_batch_set_variant(he_batch *b, int v) {
    if (!b || v < -1 || v >= mm_variant_count()) return HE_EINVAL;
    if (b->have_graph) {
        if (cudaStreamSynchronize(b->stream) != cudaSuccess) return HE_ECUDA;
        cudaGraphExecDestroy(b->exec);
        b->have_graph = false;
    }
    b->variant = v;
    return HE_OK;
}

int he_batch_tuning(const he_batch *b, int *variant, float *ms) {
    if (!b || !variant) return HE_EINVAL;
    *variant = b->variant;
    if (ms)
        for (int v = 0; v < mm_variant_count(); ++v) ms[v] = b->tune_ms[v];
    return HE_OK;
}

int he_batch_stage_form(const he_batch *b, int *form, float *ms) {
    if (!b || !form) return HE_EINVAL;
    *form = b->stage_form;
    if (ms) {
        ms[0] = b->stage_ms[0];
        ms[1] = b->stage_ms[1];
    }
    return HE_OK;
}

int he_batch_set_stage_form(he_batch *b, int form) {
    if (!b || form < 0 || form > 1) return HE_EINVAL;
    if (b->have_graph) {
        if (cudaStreamSynchronize(b->stream) != cudaSuccess) return HE_ECUDA;
        cudaGraphExecDestroy(b->exec);
        b->have_graph = false;
    }
    b->stage_form = form;
    return HE_OK;
}

int he_matmult_decode(he_ctx *ctx, const he_plan *plan, const double *slots, double *y_out) {
    return he_matmult_decode_masked(ctx, plan, slots, nullptr, y_out);
}

int he_matmult_decode_masked(he_ctx *ctx, const he_plan *plan, const double *slots, const double *mask, double *y_out) {
    if (!ctx || !plan || !slots || !y_out || plan->slots != ctx->n / 2) return HE_EINVAL;
    launch_lazy_ras(ctx, *plan, slots, mask, y_out);
    return last_launch();
}

int he_matmult_decrypt(he_ctx *ctx, const he_plan *plan, const he_ct *cts, int n_ct, const double *mask, double *y_out) {
    if (!ctx || !plan || !cts || !y_out || plan->slots != ctx->n / 2 || n_ct != plan->row_blocks) return HE_EINVAL;
    for (int r = 0; r < n_ct; ++r) {
        if (!cts[r].data) return HE_EINVAL;
        if (cts[r].level < 0 || cts[r].level >= ctx->L) return HE_ELEVEL;
        if (cts[r].scale != cts[0].scale) return HE_ESCALE;
    }
    const size_t N = ctx->n;
    uint64_t *s = ctx_scratch(ctx, (size_t)n_ct * N + (size_t)n_ct * (N / 2));
    if (!s) return HE_ENOMEM;
    double *coef = reinterpret_cast<double *>(s), *slots = coef + (size_t)n_ct * N;
    for (int r = 0; r < n_ct; ++r) launch_decrypt_coeffs(ctx, cts[r].data, cts[r].level, 1, coef + (size_t)r * N, nullptr);
    if (!launch_decode_ras(ctx, *plan, coef, n_ct, cts[0].scale, mask, y_out)) {
        launch_decode(ctx, coef, n_ct, cts[0].scale, slots);
        launch_lazy_ras(ctx, *plan, slots, mask, y_out);
    }
    return last_launch();
}

int he_plan_ras_steps(const he_plan *p, int32_t *steps, int *n_steps) {
    if (!p || !n_steps) return HE_EINVAL;
    int n = 0;
    for (int64_t step = p->m_prime; step < p->nb; step *= 2) {
        if (steps) steps[n] = (int32_t)step;
        ++n;
    }
    *n_steps = n;
    return HE_OK;
}

int he_ras(he_ctx *ctx, const he_plan *plan, const he_ct *in, he_ct *out) {
    if (!ctx || !plan || !in || !out || !in->data || !out->data || plan->slots != ctx->n / 2) return HE_EINVAL;
    const int level = in->level;
    if (level < 0 || level >= ctx->L) return HE_ELEVEL;
    int32_t steps[64];
    int ns = 0;
    he_plan_ras_steps(plan, steps, &ns);
    std::vector<const uint64_t *> keys(ns);
    for (int j = 0; j < ns; ++j) {
        keys[j] = ctx->sh->key(galois_of(ctx, steps[j]));
        if (!keys[j]) return HE_EKEY;
    }
    const ModUpConst &mu = ctx->modup[level];
    const size_t N = ctx->n, nl = level + 1, ext = mu.ext;
    const size_t wD = mu.ndig * ext * N, wc = nl * N, wu = 2 * ext * N, wr = nl * N, wt = 2 * ctx->K * N, wrot = 2 * nl * N;
    uint64_t *s = ctx_scratch(ctx, wD + wc + wu + wr + wt + wrot);
    if (!s) return HE_ENOMEM;
    uint64_t *D = s, *coef = D + wD, *u = coef + wc, *rc0 = u + wu, *tmp = rc0 + wr, *rot = tmp + wt;
    if (out->data != in->data &&
        cudaMemcpyAsync(out->data, in->data, 2 * nl * N * sizeof(uint64_t), cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess)
        return HE_ECUDA;
    // x <- x + RotL(x, step) for each step in turn (each rotation depends on the previous sum)
    for (int j = 0; j < ns; ++j) {
        const uint32_t g = galois_of(ctx, steps[j]);
        launch_modup(ctx, out->data + nl * N, level, D, coef);
        launch_ks_inner(ctx, D, level, g, keys[j], u);
        launch_automorph(ctx, out->data, rc0, 1, qmap(level), g);
        launch_moddown(ctx, u, level, 2, rc0, nullptr, rot, tmp);
        launch_add(ctx, out->data, rot, out->data, 2, qmap(level));
    }
    out->level = level;
    out->scale = in->scale;
    return last_launch();
}

int he_ras_decode(he_ctx *ctx, const he_plan *plan, const double *slots, double *y_out) {
    if (!ctx || !plan || !slots || !y_out || plan->slots != ctx->n / 2) return HE_EINVAL;
    launch_ras_gather(ctx, *plan, slots, y_out);
    return last_launch();
}

int he_modup_export(he_ctx *ctx, const he_ct *ct, uint64_t *digits_out) {
    if (!ctx || !ct || !ct->data || !digits_out) return HE_EINVAL;
    const int level = ct->level;
    if (level < 0 || level >= ctx->L) return HE_ELEVEL;
    const ModUpConst &mu = ctx->modup[level];
    const size_t N = ctx->n, nl = level + 1;
    uint64_t *coef = ctx_scratch(ctx, nl * N);
    if (!coef) return HE_ENOMEM;
    launch_modup(ctx, ct->data + nl * N, level, digits_out, coef);
    LimbMap emap{};
    emap.n = mu.ext;
    for (int u = 0; u < mu.ext; ++u) emap.prime[u] = mu.ext_prime[u];
    const int64_t gs = (int64_t)mu.ext * ctx->n;
    launch_ntt_inv_strided(ctx, digits_out, gs, digits_out, gs, mu.ndig, emap);
    return last_launch();
}

int he_ct_export(he_ctx *ctx, const he_ct *ct, uint64_t *coeffs_out) {
    if (!ctx || !ct || !ct->data || !coeffs_out) return HE_EINVAL;
    if (ct->level < 0 || ct->level >= ctx->L) return HE_ELEVEL;
    launch_ntt_inv(ctx, ct->data, coeffs_out, 2, qmap(ct->level));
    return last_launch();
}

int he_ct_import(he_ctx *ctx, const uint64_t *coeffs, int level, double scale, he_ct *out) {
    if (!ctx || !coeffs || !out || !out->data) return HE_EINVAL;
    if (level < 0 || level >= ctx->L) return HE_ELEVEL;
    launch_ntt_fwd(ctx, coeffs, out->data, 2, qmap(level));
    out->level = level;
    out->scale = scale;
    return last_launch();
}

int he_pt_export(he_ctx *ctx, const he_pt *pt, uint64_t *coeffs_out) {
    if (!ctx || !pt || !pt->data || !coeffs_out) return HE_EINVAL;
    if (pt->level < 0 || pt->level >= ctx->L) return HE_ELEVEL;
    launch_ntt_inv(ctx, pt->data, coeffs_out, 1, qmap(pt->level));
    return last_launch();
}

int he_pt_import(he_ctx *ctx, const uint64_t *coeffs, int level, double scale, he_pt *out) {
    if (!ctx || !coeffs || !out || !out->data) return HE_EINVAL;
    if (level < 0 || level >= ctx->L) return HE_ELEVEL;
    launch_ntt_fwd(ctx, coeffs, out->data, 1, qmap(level));
    out->level = level;
    out->scale = scale;
    return last_launch();
}

int he_ntt_form(const he_ctx *ctx, int *form, float *ms) {
    if (!ctx || !form) return HE_EINVAL;
    *form = ctx->ntt_form;
    if (ms)
        for (int f = 0; f < HE_NTT_FORMS; ++f) ms[f] = ctx->ntt_form_ms[f];
    return HE_OK;
}

int he_set_ntt_form(he_ctx *ctx, int form) {
    if (!ctx || form < -1 || form >= HE_NTT_FORMS) return HE_EINVAL;
    ctx->ntt_form = form;
    return HE_OK;
}

}  // extern "C"
