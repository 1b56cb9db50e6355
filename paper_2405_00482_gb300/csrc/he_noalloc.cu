// he_noalloc.cu -- the MatMult entry point that allocates no memory.
//
// Some callers cannot let the library call cudaMalloc: an application whose device memory is
// owned and budgeted by its own allocator (a framework's caching allocator, or a serving
// process that fixes its footprint when it starts), or a latency-sensitive loop where an
// allocation, and the device-wide wait that cudaFree implies, must not happen inside a call.
// he_matmult_plain_cipher_noalloc serves them: it computes exactly what he_matmult_plain_cipher
// computes, but its temporary buffers (ModUp digits, accumulators, the key-pointer table) live
// in one fixed array of device memory reserved in this file when the library is loaded.
#include <mutex>

#include "he_internal.cuh"

void launch_moddown(he_ctx *ctx, const uint64_t *x, int level, int ncomp, const uint64_t *add0, const uint64_t *add1, uint64_t *out,
                    uint64_t *tmp);

// 16 MiB, held by every GPU that loads the library until the process exits.
#define HE_NOALLOC_WORDS ((size_t)2 << 20)

static __device__ __align__(256) uint64_t g_noalloc_scratch[HE_NOALLOC_WORDS];

namespace {

// host-side device address of g_noalloc_scratch, looked up once per device
std::mutex g_mu;
uint64_t *g_addr[64];

// writes rotation i's Galois key pointer and Galois element into the table at the front of the scratch array
struct KeyChunk {
    const uint64_t *key[128];
    uint32_t galois[128];
    int32_t first, count;
};

__global__ void fill_key_table_kernel(KeyChunk kc, int64_t n_steps) {
    HE_GRID_DEP();
    const uint64_t **keys = reinterpret_cast<const uint64_t **>(g_noalloc_scratch);
    uint32_t *gal = reinterpret_cast<uint32_t *>(g_noalloc_scratch + n_steps);
    for (int t = threadIdx.x; t < kc.count; t += blockDim.x) {
        keys[kc.first + t] = kc.key[t];
        gal[kc.first + t] = kc.galois[t];
    }
}

// The device address is looked up with the context's device current (the calling thread's
// current device is restored afterwards), so a context on another GPU gets its own copy.
int scratch_address(const he_ctx *ctx, uint64_t **out) {
    const int dev = ctx->device;
    if (dev < 0 || dev >= 64) return HE_ECUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        int cur = 0;
        if (cudaGetDevice(&cur) != cudaSuccess) return HE_ECUDA;
        if (cur != dev && cudaSetDevice(dev) != cudaSuccess) return HE_ECUDA;
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (cur != dev) cudaSetDevice(cur);
        if (e != cudaSuccess || !p) return HE_ECUDA;
        g_addr[dev] = static_cast<uint64_t *>(p);
    }
    *out = g_addr[dev];
    return HE_OK;
}

}  // namespace

extern "C" int he_matmult_plain_cipher_noalloc(he_ctx *ctx, const he_plan *plan, const he_ptmat *pm, const he_ct *ins, int n_in, he_ct *outs,
                                               int n_out) {
    if (!ctx || !plan || !pm || !ins || !outs || !same_family(pm->ctx, ctx)) return HE_EINVAL;
    const he_plan &p = pm->plan;
    if (p.m != plan->m || p.n != plan->n || p.slots != plan->slots) return HE_EINVAL;
    if (n_in != p.col_blocks || n_out != p.row_blocks || p.baby) return HE_EINVAL;
    const int level = pm->level;
    for (int c = 0; c < n_in; ++c) {
        if (!ins[c].data) return HE_EINVAL;
        if (ins[c].level != level) return HE_ELEVEL;
    }
    for (int r = 0; r < n_out; ++r)
        if (!outs[r].data) return HE_EINVAL;
    const ModUpConst &mu = ctx->modup[level];
    const size_t N = ctx->n, nl = level + 1, ext = mu.ext, C = p.col_blocks;
    const bool rot = p.m_prime > 1;
    const size_t steps = rot ? (size_t)p.m_prime - 1 : 0;
    // layout: [key pointers][Galois elements, padded to 8 bytes][D per column block][coef][acc][cacc][sum][tmp]
    const size_t w_tab = steps + (steps + 1) / 2;
    const size_t w_tab_al = (w_tab + 31) & ~(size_t)31;
    const size_t wD = rot ? C * mu.ndig * ext * N : 0, wc = nl * N, wa = 2 * ext * N, wcc = 2 * nl * N, wsum = 2 * nl * N,
                 wt = 2 * (ctx->K > 1 ? ctx->K : 1) * N + 2 * N;
    const size_t need = w_tab_al + wD + wc + wa + wcc + wsum + wt;
    if (need > HE_NOALLOC_WORDS) return HE_EBUDGET;  // larger than the fixed 16 MiB array
    for (size_t i = 0; i < steps; ++i)
        if (!ctx->sh->key(galois_of(ctx, (int64_t)i + 1))) return HE_EKEY;
    uint64_t *base = nullptr;
    int rc = scratch_address(ctx, &base);
    if (rc != HE_OK) return rc;
    // the key table: kernel parameters carry the pointers, so nothing is staged through host memory
    for (size_t first = 0; first < steps; first += 128) {
        KeyChunk kc{};
        kc.first = (int32_t)first;
        kc.count = (int32_t)(steps - first < 128 ? steps - first : 128);
        for (int t = 0; t < kc.count; ++t) {
            const uint32_t g = galois_of(ctx, (int64_t)(first + t) + 1);
            kc.galois[t] = g;
            kc.key[t] = ctx->sh->key(g);
        }
        ctx->launches++;
        launch_k(fill_key_table_kernel, 1, 128, 0, ctx->stream, kc, (int64_t)steps);
    }
    const uint64_t *const *keys = reinterpret_cast<const uint64_t *const *>(base);
    const uint32_t *galois = reinterpret_cast<const uint32_t *>(base + steps);
    // every region below is written before it is read in each call, so nothing needs clearing
    uint64_t *D = base + w_tab_al, *coef = D + wD, *acc = coef + wc, *cacc = acc + wa, *sum = cacc + wcc, *tmp = sum + wsum;
    if (rot)
        for (size_t c = 0; c < C; ++c) launch_modup(ctx, ins[c].data + nl * N, level, D + c * mu.ndig * ext * N, coef);
    for (int r = 0; r < n_out; ++r) {
        for (size_t c = 0; c < C; ++c)
            launch_matmult_loop_with_tables(ctx, pm, r, (int)c, ins[c].data, rot ? D + c * mu.ndig * ext * N : nullptr, keys, galois, acc,
                                            cacc, c > 0);
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
    return cudaGetLastError() == cudaSuccess ? HE_OK : HE_ECUDA;
}
