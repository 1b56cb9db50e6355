// he_host.cu -- the entry points that take and return HOST memory: the party-facing side of the
// MatMult (Sec. 3, Alg. 1).  P_A encodes its cleartext matrix X, P_B encrypts its vector y and
// later decrypts the product, and ciphertexts cross between the parties as bytes.  Each call
// stages its bulk data through buffers of the context (a device buffer, and a page-locked host
// buffer when the caller's memory is pageable), copies with one cudaMemcpyAsync per buffer on the
// context's stream, and then runs the same kernels as its device-memory counterpart, so results
// are identical bit for bit.
#include <string.h>

#include <vector>

#include "he_internal.cuh"

int he_check(cudaError_t e);

bool capturing(cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}

namespace {

// A host pointer the GPU can copy from asynchronously (cudaMallocHost / cudaHostRegister memory).
bool page_locked(const void *p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // clear the sticky-free error of an unknown pointer
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

// device staging of at least `bytes`; the previous contents are not kept.  Growing waits for
// the stream (earlier calls may still read the old buffer) and so cannot happen under capture.
void *stage_dev(he_ctx *ctx, size_t bytes) {
    if (bytes <= ctx->stage_dev_bytes) return ctx->stage_dev;
    if (capturing(ctx->stream)) return nullptr;
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->stage_dev);
    ctx->stage_dev = nullptr;
    ctx->stage_dev_bytes = 0;
    if (cudaMalloc(&ctx->stage_dev, bytes) != cudaSuccess) return nullptr;
    ctx->stage_dev_bytes = bytes;
    return ctx->stage_dev;
}

// page-locked host staging of at least `bytes`, free to overwrite (the last copy out of it has
// completed)
void *stage_host(he_ctx *ctx, size_t bytes) {
    if (ctx->stage_ev && cudaEventSynchronize(ctx->stage_ev) != cudaSuccess) return nullptr;
    if (bytes <= ctx->stage_host_bytes) return ctx->stage_host;
    cudaFreeHost(ctx->stage_host);
    ctx->stage_host = nullptr;
    ctx->stage_host_bytes = 0;
    if (cudaMallocHost(&ctx->stage_host, bytes) != cudaSuccess) return nullptr;
    ctx->stage_host_bytes = bytes;
    return ctx->stage_host;
}

// host -> device on the context's stream: one asynchronous copy from page-locked memory; from
// pageable memory a copy into the page-locked staging first (not allowed under stream capture,
// where the copy would replay from a buffer the caller no longer controls)
int h2d(he_ctx *ctx, void *dst, const void *src, size_t bytes) {
    if (bytes == 0) return HE_OK;
    if (page_locked(src)) return he_check(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->stream));
    if (capturing(ctx->stream)) return HE_EINVAL;
    void *h = stage_host(ctx, bytes);
    if (!h) return HE_ENOMEM;
    memcpy(h, src, bytes);
    if (cudaMemcpyAsync(dst, h, bytes, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess) return HE_ECUDA;
    if (!ctx->stage_ev && cudaEventCreateWithFlags(&ctx->stage_ev, cudaEventDisableTiming) != cudaSuccess) return HE_ECUDA;
    return he_check(cudaEventRecord(ctx->stage_ev, ctx->stream));
}

// device -> host on the context's stream.  Page-locked destination: one asynchronous copy, the
// values valid once the stream reaches it.  Pageable: the call waits and the values are valid on
// return.
int d2h(he_ctx *ctx, void *dst, const void *src, size_t bytes) {
    if (bytes == 0) return HE_OK;
    if (page_locked(dst)) return he_check(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    if (capturing(ctx->stream)) return HE_EINVAL;
    void *h = stage_host(ctx, bytes);
    if (!h) return HE_ENOMEM;
    if (cudaMemcpyAsync(h, src, bytes, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess) return HE_ECUDA;
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return HE_ECUDA;
    memcpy(dst, h, bytes);
    return HE_OK;
}

// serialized ciphertext: header, the primes of its level, then [2][level+1][N] canonical
// coefficients (little-endian uint64 throughout)
constexpr uint32_t kCtMagic = 0x54434548u;  // "HECT"
constexpr uint32_t kCtVersion = 1;
struct CtHeader {
    uint32_t magic, version;
    int32_t log_n, level;
    double scale;
    uint64_t reserved;
};
static_assert(sizeof(CtHeader) == 32, "header layout");

size_t ct_serial_bytes(const he_ctx *ctx, int level) {
    return sizeof(CtHeader) + (size_t)(level + 1) * 8 + 2 * (size_t)(level + 1) * ctx->n * 8;
}

}  // namespace

extern "C" {

int he_encode_matrix_host(he_ctx *ctx, const he_plan *plan, const double *X, int level, int transposed, he_ptmat **out) {
    if (!ctx || !plan || !X || !out) return HE_EINVAL;
    *out = nullptr;
    const size_t bytes = (size_t)plan->m * plan->n * sizeof(double);
    void *d = stage_dev(ctx, bytes);
    if (!d) return HE_ENOMEM;
    int rc = h2d(ctx, d, X, bytes);
    if (rc != HE_OK) return rc;
    return transposed ? he_encode_matrix_transposed(ctx, plan, static_cast<const double *>(d), level, out)
                      : he_encode_matrix(ctx, plan, static_cast<const double *>(d), level, out);
}

int he_ptmat_encode_host(he_ctx *ctx, he_ptmat *pm, const double *X, int transposed) {
    if (!ctx || !pm || !X || !same_family(pm->ctx, ctx)) return HE_EINVAL;
    const size_t bytes = (size_t)pm->plan.m * pm->plan.n * sizeof(double);
    void *d = stage_dev(ctx, bytes);
    if (!d) return HE_ENOMEM;
    int rc = h2d(ctx, d, X, bytes);
    if (rc != HE_OK) return rc;
    return transposed ? he_ptmat_encode_transposed(ctx, pm, static_cast<const double *>(d)) : he_ptmat_encode(ctx, pm, static_cast<const double *>(d));
}

int he_encrypt_vector_host(he_ctx *ctx, const he_plan *plan, const double *y, double scale, int level, uint64_t nonce, const uint64_t *nonce_dev,
                           he_ct *outs) {
    if (!ctx || !plan || !y || !outs) return HE_EINVAL;
    const size_t bytes = (size_t)plan->n * sizeof(double);
    void *d = stage_dev(ctx, bytes);
    if (!d) return HE_ENOMEM;
    int rc = h2d(ctx, d, y, bytes);
    if (rc != HE_OK) return rc;
    return he_encrypt_vector(ctx, plan, static_cast<const double *>(d), scale, level, nonce, nonce_dev, outs);
}

int he_decrypt_host(he_ctx *ctx, const he_ct *ct, double *slots) {
    if (!ctx || !ct || !slots) return HE_EINVAL;
    const size_t bytes = (size_t)(ctx->n / 2) * sizeof(double);
    void *d = stage_dev(ctx, bytes);
    if (!d) return HE_ENOMEM;
    int rc = he_decrypt(ctx, ct, static_cast<double *>(d));
    if (rc != HE_OK) return rc;
    return d2h(ctx, slots, d, bytes);
}

int he_matmult_decrypt_host(he_ctx *ctx, const he_plan *plan, const he_ct *cts, int n_ct, const double *mask, double *y) {
    if (!ctx || !plan || !cts || !y || plan->slots != ctx->n / 2 || n_ct != plan->row_blocks) return HE_EINVAL;
    const size_t w_mask = mask ? (size_t)n_ct * plan->slots : 0, w_y = (size_t)plan->m;
    double *d = static_cast<double *>(stage_dev(ctx, (w_mask + w_y) * sizeof(double)));
    if (!d) return HE_ENOMEM;
    double *d_mask = mask ? d : nullptr, *d_y = d + w_mask;
    int rc = mask ? h2d(ctx, d_mask, mask, w_mask * sizeof(double)) : HE_OK;
    if (rc != HE_OK) return rc;
    rc = he_matmult_decrypt(ctx, plan, cts, n_ct, d_mask, d_y);
    if (rc != HE_OK) return rc;
    return d2h(ctx, y, d_y, w_y * sizeof(double));
}

int he_ct_export_host(he_ctx *ctx, const he_ct *ct, void *buf, size_t *len) {
    if (!ctx || !ct || !len) return HE_EINVAL;
    if (ct->level < 0 || ct->level >= ctx->L) return HE_ELEVEL;
    const size_t need = ct_serial_bytes(ctx, ct->level);
    if (!buf) {  // size query
        *len = need;
        return HE_OK;
    }
    if (*len < need || !ct->data) {
        *len = need;
        return HE_EINVAL;
    }
    const size_t nl = ct->level + 1, coef_bytes = 2 * nl * ctx->n * 8;
    void *d = stage_dev(ctx, coef_bytes);
    if (!d) return HE_ENOMEM;
    int rc = he_ct_export(ctx, ct, static_cast<uint64_t *>(d));
    if (rc != HE_OK) return rc;
    unsigned char *b = static_cast<unsigned char *>(buf);
    CtHeader h{kCtMagic, kCtVersion, ctx->log_n, ct->level, ct->scale, 0};
    memcpy(b, &h, sizeof(h));
    memcpy(b + sizeof(h), ctx->primes.data(), nl * 8);
    rc = d2h(ctx, b + sizeof(h) + nl * 8, d, coef_bytes);
    if (rc != HE_OK) return rc;
    // the bytes are complete on return, whatever memory they are in
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return HE_ECUDA;
    *len = need;
    return HE_OK;
}

int he_ct_host_level(const void *buf, size_t len, int32_t *level) {
    if (!buf || !level || len < sizeof(CtHeader)) return HE_EINVAL;
    CtHeader h;
    memcpy(&h, buf, sizeof(h));
    if (h.magic != kCtMagic || h.version != kCtVersion || h.level < 0 || h.level >= HE_MAX_Q) return HE_EINVAL;
    *level = h.level;
    return HE_OK;
}

int he_ct_import_host(he_ctx *ctx, const void *buf, size_t len, he_ct *out) {
    if (!ctx || !buf || !out || !out->data || len < sizeof(CtHeader)) return HE_EINVAL;
    CtHeader h;
    memcpy(&h, buf, sizeof(h));
    if (h.magic != kCtMagic || h.version != kCtVersion || h.log_n != ctx->log_n) return HE_EINVAL;
    if (h.level < 0 || h.level >= ctx->L) return HE_ELEVEL;
    const size_t nl = h.level + 1, N = ctx->n;
    if (len != ct_serial_bytes(ctx, h.level)) return HE_EINVAL;
    const unsigned char *b = static_cast<const unsigned char *>(buf);
    std::vector<uint64_t> primes(nl);
    memcpy(primes.data(), b + sizeof(h), nl * 8);
    for (size_t l = 0; l < nl; ++l)
        if (primes[l] != ctx->primes[l]) return HE_EINVAL;  // made under other parameters
    // every coefficient must be a canonical residue of its limb's prime
    const unsigned char *coef = b + sizeof(h) + nl * 8;
    for (size_t c = 0; c < 2; ++c)
        for (size_t l = 0; l < nl; ++l) {
            const unsigned char *row = coef + ((c * nl + l) * N) * 8;
            for (size_t k = 0; k < N; ++k) {
                uint64_t v;
                memcpy(&v, row + k * 8, 8);
                if (v >= primes[l]) return HE_EINVAL;
            }
        }
    const size_t coef_bytes = 2 * nl * N * 8;
    void *d = stage_dev(ctx, coef_bytes);
    if (!d) return HE_ENOMEM;
    int rc = h2d(ctx, d, coef, coef_bytes);
    if (rc != HE_OK) return rc;
    return he_ct_import(ctx, static_cast<const uint64_t *>(d), h.level, h.scale, out);
}

}  // extern "C"
