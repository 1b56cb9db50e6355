// he_bsgs.cu -- the baby-step giant-step schedule of the diagonal MatMult (an extension of the
// PackVFL row of Tab. 2: fewer Galois keys, not fewer products).
//
// With m' = B G diagonals, i = g B + b, and RotL of a slot-wise product equal to the product of
// the RotLs,
//     sum_i e_i (x) RotL(y, i) = sum_g RotL( sum_b RotR(e_{gB+b}, gB) (x) RotL(y, b), gB ).
// The encoded matrix of such a plan already holds the pre-rotated plaintexts (the encoding reads
// slot s of diagonal i from slot s - gB).  Per column block the B - 1 baby rotations of the input
// share one decomposition (O4, he_rotate_hoisted's key switch); per row block one launch forms
// every partial sum s_g = sum_c sum_b pt_{gB+b} (x) x_{c,b} (O2 and O1 on the Q limbs), the G - 1
// giant rotations RotL(s_g, gB) run as one batch of O3 (he_rotate_many's launches), and the sum
// over g is rescaled once.  Galois keys: B - 1 + G - 1 instead of m' - 1.  Every step is the
// exact modular arithmetic of the corresponding O1-O4, so the output is bit-identical to their
// composition in that order.
#include <vector>

#include "he_internal.cuh"

namespace {

struct BsgsGeom {
    const uint64_t *X;   // baby rotations [C][B][2][nl][N]: x_{c,b} = RotL(ct_c, b)
    const uint64_t *pts; // the row block's plaintexts [C][m'][ext][N], Montgomery form
    uint64_t *inner;     // partial sums [G][2][nl][N]
    int32_t B, C, nl, ext;
};

// grid (N / 256, nl, G): inner_g[comp][l][k] = sum_c sum_b ptM[c][gB+b][l][k] x_{c,b}[comp][l][k],
// products accumulated in 128 bits and reduced (REDC, plaintext in Montgomery form) every
// lazy_terms(q) terms
__global__ void __launch_bounds__(256) bsgs_mac_kernel(BsgsGeom bg, const ModConst *__restrict__ mc, int logn) {
    HE_GRID_DEP();
    const int64_t N = (int64_t)1 << logn;
    const int64_t k = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const int l = blockIdx.y, g = blockIdx.z;
    if (k >= N) return;
    const uint64_t q = mc[l].q, qinv = mc[l].qinv;
    const int mp = bg.B * (int)gridDim.z;
    const int64_t ct_w = 2 * (int64_t)bg.nl * N;
    uint64_t r0 = 0, r1 = 0;
    u128 t0 = 0, t1 = 0;
    int pending = 0;
    const int period = lazy_terms(q);
    for (int c = 0; c < bg.C; ++c) {
        for (int b = 0; b < bg.B; ++b) {
            const uint64_t *x = bg.X + ((int64_t)c * bg.B + b) * ct_w + (int64_t)l * N + k;
            const uint64_t p = __ldg(bg.pts + (((int64_t)c * mp + g * bg.B + b) * bg.ext + l) * N + k);
            t0 += (u128)__ldg(x) * p;
            t1 += (u128)__ldg(x + (int64_t)bg.nl * N) * p;
            if (++pending == period) {
                r0 = add_mod(r0, redc128(t0, q, qinv), q);
                r1 = add_mod(r1, redc128(t1, q, qinv), q);
                t0 = t1 = 0;
                pending = 0;
            }
        }
    }
    r0 = add_mod(r0, redc128(t0, q, qinv), q);
    r1 = add_mod(r1, redc128(t1, q, qinv), q);
    uint64_t *o = bg.inner + (int64_t)g * 2 * bg.nl * N + (int64_t)l * N + k;
    o[0] = r0;
    o[(int64_t)bg.nl * N] = r1;
}

// grid (N / 256, nl, 2): acc[comp][l][k] += sum_g rot_g[comp][l][k]
__global__ void __launch_bounds__(256) bsgs_sum_kernel(uint64_t *acc, const uint64_t *__restrict__ rot, int count, int nl,
                                                      const ModConst *__restrict__ mc, int logn) {
    HE_GRID_DEP();
    const int64_t N = (int64_t)1 << logn;
    const int64_t k = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const int l = blockIdx.y, c = blockIdx.z;
    if (k >= N) return;
    const uint64_t q = mc[l].q;
    const int64_t off = ((int64_t)c * nl + l) * N + k, ct_w = 2 * (int64_t)nl * N;
    uint64_t v = acc[off];
    for (int g = 0; g < count; ++g) v = add_mod(v, __ldg(rot + g * ct_w + off), q);
    acc[off] = v;
}

}  // namespace

int matmult_bsgs(he_ctx *ctx, he_ptmat *pm, const he_ct *ins, he_ct *outs) {
    const he_plan &p = pm->plan;
    const int level = pm->level;
    const int B = (int)p.baby, G = (int)(p.m_prime / p.baby), C = (int)p.col_blocks, R = (int)p.row_blocks;
    const size_t N = ctx->n, nl = level + 1, ct_w = 2 * nl * N;
    const ModUpConst &mu = ctx->modup[level];
    // Galois keys of the baby steps b = 1..B-1 and the giant steps g B, g = 1..G-1
    std::vector<const uint64_t *> kb(B), kg(G);
    std::vector<uint32_t> gb(B), gg(G);
    for (int b = 1; b < B; ++b) {
        gb[b] = galois_of(ctx, b);
        if (!(kb[b] = ctx->sh->key(gb[b]))) return HE_EKEY;
    }
    for (int g = 1; g < G; ++g) {
        gg[g] = galois_of(ctx, (int64_t)g * B);
        if (!(kg[g] = ctx->sh->key(gg[g]))) return HE_EKEY;
    }
    // scratch: baby rotations, ModUp digits and c1 coefficients of one input, the key switch's
    // tables, partial sums, giant rotations and their batch scratch, rescale temporaries
    const int gchunk = G - 1 < HE_ROT_CHUNK ? G - 1 : HE_ROT_CHUNK;
    const size_t wX = (size_t)C * B * ct_w, wD = (size_t)mu.ndig * mu.ext * N + nl * N, wpc = B > 1 ? keyswitch_many_pc_words(ctx, B - 1) : 0,
                 wI = (size_t)G * ct_w, wRot = (size_t)(G - 1) * ct_w, wRm = gchunk > 0 ? (size_t)gchunk * rotate_many_words(ctx, level) : 0,
                 wT = 2 * (size_t)(ctx->K > 1 ? ctx->K : 1) * N + 2 * N;
    uint64_t *s = ctx_scratch(ctx, wX + wD + wpc + wI + wRot + wRm + wT);
    if (!s) return HE_ENOMEM;
    uint64_t *X = s, *D = X + wX, *coef = D + (size_t)mu.ndig * mu.ext * N, *pc = D + wD, *inner = pc + wpc, *rot = inner + wI, *rm = rot + wRot,
             *tmp = rm + wRm;
    // baby steps: x_{c,0} = ct_c, x_{c,b} = RotL(ct_c, b) with one decomposition per input
    for (int c = 0; c < C; ++c) {
        uint64_t *Xc = X + (size_t)c * B * ct_w;
        if (cudaMemcpyAsync(Xc, ins[c].data, ct_w * sizeof(uint64_t), cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess) return HE_ECUDA;
        if (B == 1) continue;
        std::vector<RotJob> jobs(B - 1);
        for (int b = 1; b < B; ++b) jobs[b - 1] = RotJob{ins[c].data, Xc + (size_t)b * ct_w, kb[b], gb[b], 0};
        launch_modup(ctx, ins[c].data + nl * N, level, D, coef);
        launch_keyswitch_many(ctx, jobs.data(), B - 1, level, D, 0, pc);
    }
    const unsigned eb = (unsigned)((N + 255) / 256);
    for (int r = 0; r < R; ++r) {
        BsgsGeom bg{};
        bg.X = X;
        bg.pts = pm->data + (size_t)r * C * p.m_prime * pm->ext * N;
        bg.inner = inner;
        bg.B = B;
        bg.C = C;
        bg.nl = (int)nl;
        bg.ext = pm->ext;
        ctx->launches++;
        launch_k(bsgs_mac_kernel, dim3(eb, (unsigned)nl, (unsigned)G), 256, 0, ctx->stream, bg, (const ModConst *)ctx->d_mc, ctx->log_n);
        // giant steps RotL(s_g, g B), g >= 1, as batches of O3 on different ciphertexts
        for (int g0 = 1; g0 < G; g0 += HE_ROT_CHUNK) {
            const int n = G - g0 < HE_ROT_CHUNK ? G - g0 : HE_ROT_CHUNK;
            std::vector<RotJob> jobs(n);
            for (int t = 0; t < n; ++t) {
                const int g = g0 + t;
                jobs[t] = RotJob{inner + (size_t)g * ct_w, rot + (size_t)(g - 1) * ct_w, kg[g], gg[g], 0};
            }
            launch_rotate_many(ctx, jobs.data(), n, level, rm);
        }
        if (G > 1) {
            ctx->launches++;
            launch_k(bsgs_sum_kernel, dim3(eb, (unsigned)nl, 2u), 256, 0, ctx->stream, inner, (const uint64_t *)rot, G - 1, (int)nl,
                     (const ModConst *)ctx->d_mc, ctx->log_n);
        }
        launch_rescale(ctx, inner, level, outs[r].data, tmp);
        outs[r].level = level - 1;
        outs[r].scale = ins[0].scale * pm->scale / (double)ctx->primes[level];
    }
    return cudaGetLastError() == cudaSuccess ? HE_OK : HE_ECUDA;
}
