/*
 * he.h -- C ABI of the GB300 (sm_103a) library for the PackVFL encrypted MatMult.
 *
 * The library computes X [[y]] = [[X y]] (Eq. 1, Sec. 3) between a cleartext matrix X and
 * CKKS/RLWE ciphertexts [[y]] (Sec. 2.2) in PackVFL's hybrid layout: diagonal encoding
 * (Eq. 2, Sec. 4.1), input packing (Eq. 3, Sec. 4.2.1) and partitioning (Sec. 4.2.2),
 * hoisted rotations (O4, Sec. 2.2) and lazy rotate-and-sum (Sec. 4.3).
 *
 * Conventions for every call:
 *  - Return value: HE_OK (0) or a negative HE_E* status; nothing is thrown across the ABI.
 *  - Bulk data (slots, matrices, ciphertexts, plaintexts) live in DEVICE memory owned by
 *    the caller, passed as plain pointers.  Every device call is asynchronous on the
 *    context's CUDA stream (given at creation); the caller orders other work against it.
 *  - Ciphertext and plaintext buffers are in the library's internal form: limbs of
 *    uint64 residues, NTT (evaluation) domain, bit-reversed slot order.  he_ct_export /
 *    he_ct_import convert from / to the canonical coefficient form.
 *  - Keys, tables, plans and encoded matrices are owned by the library and released by
 *    the matching *_free / he_ctx_destroy.
 *  - Rotation direction: RotL(x, r)[j] = x[(j + r) mod N/2] (Sec. 3.1.1), realised by the
 *    automorphism X -> X^(5^r mod 2N).
 */
#ifndef HE_H
#define HE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    HE_OK = 0,
    HE_EINVAL = -1,   /* bad argument (null pointer, size out of range, mismatched plan) */
    HE_ENOMEM = -2,   /* device or host allocation failed */
    HE_ECUDA = -3,    /* a CUDA call failed (no device, launch error) */
    HE_EKEY = -4,     /* a rotation needs a Galois key that he_keygen did not make */
    HE_ELEVEL = -5,   /* level out of range or operands at different levels */
    HE_ESCALE = -6,   /* operand scales do not match */
    HE_ETIMEOUT = -7, /* a bounded device wait gave up */
    HE_EBUDGET = -8   /* request exceeds the configured memory budget */
};

typedef struct he_ctx he_ctx;       /* parameters, NTT tables, secret key, Galois keys */
typedef struct he_plan he_plan;     /* MatMult layout plan (host only) */
typedef struct he_ptmat he_ptmat;   /* encoded diagonal plaintext matrix (device) */

/* RNS-CKKS parameters.  The ring is Z_q[X]/(X^N+1) with N = 2^log_n (Sec. 2.2), N/2 slots.
 * Primes: for each bit size in q_bits then p_bits, the largest prime q < 2^bits with
 * q = 1 mod 2N not already chosen.  Key switching splits the q primes into dnum digits of
 * ceil(n_q / dnum) consecutive primes.  Secret ternary, noise discrete Gaussian sigma 3.2. */
typedef struct he_params {
    int32_t log_n;        /* 4 <= log_n <= 14 */
    int32_t n_q;          /* ciphertext primes, 1..16 (levels 0..n_q-1) */
    int32_t n_p;          /* special primes, 1..8 */
    int32_t dnum;         /* 1..n_q */
    int32_t q_bits[16];   /* each 20..61 */
    int32_t p_bits[8];
} he_params;

/* A ciphertext [[x]] = (c0, c1) at `level` (level+1 primes) and scale.  data: device,
 * 2*(level+1)*N uint64, caller-owned. */
typedef struct he_ct {
    uint64_t *data;
    int32_t level;
    double scale;
} he_ct;

/* A plaintext polynomial at `level`, data: device, (level+1)*N uint64, caller-owned. */
typedef struct he_pt {
    uint64_t *data;
    int32_t level;
    double scale;
} he_pt;

/* Human-readable text of a status code (static string). */
const char *he_strerror(int status);

/* Host only (no GPU): the prime chain of `p` into out[n_q + n_p] (q primes then p primes). */
int he_params_primes(const he_params *p, uint64_t *out);

/* Host only: the 38 thresholds of the Gaussian sampler's cumulative table (40-bit). */
int he_cdt_table(uint64_t *out38);

/* Create a context on the current CUDA device: tables, secret key s from `seed`
 * (Philox-4x64-10 stream), all on `cuda_stream` (a cudaStream_t; NULL = legacy stream). */
int he_ctx_create(const he_params *p, uint64_t seed, void *cuda_stream, he_ctx **out);
void he_ctx_destroy(he_ctx *ctx);
/* A context on another stream that shares parent's tables, secret and Galois keys (keys made on
 * any context of the family are seen by all), with its own scratch, so calls on the two streams
 * can run concurrently.  Plaintext matrices and weight matrices made on one context of the
 * family may be encoded into and used on any other; the caller orders the streams (a matrix
 * encoded on one stream and used on another needs an event between them), makes no two calls on
 * one matrix from two host threads at once (a call may tune the matrix or build its fused key
 * tables) and frees a matrix before the context that made it.  The family's tables and keys are freed with its last
 * context; forks and parent may be destroyed in any order.  he_keygen on one context may run
 * while the others work (the key table is guarded).  Waits for the parent's stream once. */
int he_ctx_fork(he_ctx *parent, void *cuda_stream, he_ctx **out);
/* Wait for every call issued on the context's stream. */
int he_synchronize(he_ctx *ctx);
/* N of the ring and the prime count; any out pointer may be NULL. */
int he_ctx_info(const he_ctx *ctx, int64_t *n, int32_t *n_q, int32_t *n_p);

/* Number of kernels this context has launched so far (all calls). */
int he_launch_count(const he_ctx *ctx, int64_t *count);
/* Per-launch CUDA-event timing, on the context's stream, of some kernel classes: the MatMult's
 * key-switch / multiply-accumulate loop kernel (HE_PROF_LOOP), the transform of an encoded
 * matrix's limb-polys (HE_PROF_MATRIX_NTT), and the many-rotation key switch's transform-only
 * kernels (HE_PROF_KS_TRANSFORM: inverse NTT of the P limbs, conversion and NTT of the Q limbs) and
 * its elementwise kernels (HE_PROF_KS_ELEMENTWISE: inner products, ModDown's combination).
 * Enabling (on != 0) or disabling clears every record. */
#define HE_PROF_LOOP 0
#define HE_PROF_MATRIX_NTT 1
#define HE_PROF_KS_TRANSFORM 2
#define HE_PROF_KS_ELEMENTWISE 3
#define HE_PROF_KINDS 4
int he_profile_enable(he_ctx *ctx, int on);
/* Synchronises the stream; total milliseconds and number of timed launches of the loop kernel
 * since enabling (he_profile_read_kind with HE_PROF_LOOP). */
int he_profile_read(he_ctx *ctx, double *ms_total, int64_t *launches);
int he_profile_read_kind(he_ctx *ctx, int kind, double *ms_total, int64_t *launches);

/* Bytes of a caller-owned ciphertext ([2][level+1][N] uint64 residues) or plaintext
 * ([level+1][N]) buffer at `level`; 0 for a NULL context or a level outside 0 .. L-1. */
size_t he_ct_bytes(const he_ctx *ctx, int level);
size_t he_pt_bytes(const he_ctx *ctx, int level);

/* Galois keys for left rotations by each of steps[0..n_steps) (O3/O4, Sec. 2.2). Keys
 * already present are kept.  Device memory: dnum*2*(n_q+n_p)*N*8 bytes per key. */
int he_keygen(he_ctx *ctx, const int32_t *steps, int n_steps);

/* Encode n_slots <= N/2 real slot values (device doubles) at `scale` into a plaintext at
 * `level` (Sec. 2.2 encoding: slot j at root zeta^(5^j), zeta = exp(i pi / N)). */
int he_encode(he_ctx *ctx, const double *slots, int64_t n_slots, double scale, int level, he_pt *out);

/* Symmetric RLWE encryption (Sec. 2.2): c0 = m - a s + e, c1 = a, at the plaintext's level;
 * a and e are drawn from the Philox stream selected by `nonce`. */
int he_encrypt(he_ctx *ctx, const he_pt *pt, uint64_t nonce, he_ct *out);

/* he_encrypt with the nonce read from device memory (one uint64_t at nonce_dev, 8-byte
 * aligned) when the sampling kernels run, not when the call is made: a CUDA graph captured
 * around this call encrypts under whatever nonce the buffer holds at each replay, so the
 * caller writes a fresh nonce before each replay (never reuse one under the same key).
 * Same ciphertext as he_encrypt with that nonce. */
int he_encrypt_dnonce(he_ctx *ctx, const he_pt *pt, const uint64_t *nonce_dev, he_ct *out);

/* Decryption (Sec. 2.2) at the first prime and decoding: N/2 real slot values (device) of
 * c0 + c1 s divided by the ciphertext's scale. */
int he_decrypt(he_ctx *ctx, const he_ct *ct, double *slots_out);

/* O1 (Sec. 2.2): out = a + b (same level and scale). out may alias a or b. */
int he_add(he_ctx *ctx, const he_ct *a, const he_ct *b, he_ct *out);
/* O1 with a plaintext operand (Sec. 2.2; the replicated d = u_A + (u_B - y) and the random
 * masks of Alg. 1): out = (c0 + pt, c1).  pt at a level >= ct's and at the ct's scale
 * (HE_ESCALE otherwise).  out may alias ct. */
int he_add_plain(he_ctx *ctx, const he_ct *ct, const he_pt *pt, he_ct *out);
/* O2 (Sec. 2.2): out = pt (x) ct slot-wise, scale multiplies; pt at a level >= ct's. */
int he_mul_plain(he_ctx *ctx, const he_ct *ct, const he_pt *pt, he_ct *out);
/* Rescale by the last prime: level -> level-1, scale / q_level (rounding division). */
int he_rescale(he_ctx *ctx, const he_ct *in, he_ct *out);

/* O3 (Sec. 2.2): out = RotL(in, step).  Needs the key for `step` (HE_EKEY otherwise). */
int he_rotate(he_ctx *ctx, const he_ct *in, int32_t step, he_ct *out);
/* O4 (Sec. 2.2): outs[i] = RotL(in, steps[i]) for i < k, sharing one decomposition of c1. */
int he_rotate_hoisted(he_ctx *ctx, const he_ct *in, const int32_t *steps, int k, he_ct *outs);
/* O3 on many different ciphertexts, each by its own step (outs[i] = RotL(ins[i], steps[i]),
 * bit-identical to he_rotate per pair), as one launch per stage over all of them (in chunks of
 * 64): ModUp, key-switch inner product, ModDown.  All inputs at one level; outputs must not
 * overlap any input (HE_EINVAL); a missing Galois key gives HE_EKEY; steps that are multiples
 * of N/2 copy. */
int he_rotate_many(he_ctx *ctx, const he_ct *ins, const int32_t *steps, int count, he_ct *outs);

/* Host only: plan the MatMult of an m x n matrix with n-vectors in `slots` (= N/2) slots:
 * zero padding to powers of two (Sec. 3), input packing with m' = ceil(m n / N') (Eq. 3),
 * row/column partitioning when m or n exceed N' (Sec. 4.2.2, Tab. 3). */
int he_plan_create(int64_t m, int64_t n, int64_t slots, he_plan **out);
/* info[0..10] = m, n, slots, m_pad, n_pad, m_block, n_block, row_blocks (output cts),
 * col_blocks (input cts), m_prime (diagonals per block), packed groups per ct. */
int he_plan_query(const he_plan *plan, int64_t *info);
void he_plan_free(he_plan *plan);
/* Baby-step giant-step schedule of the diagonal method (an extension of Tab. 2's PackVFL row,
 * not in the paper): with baby = B > 0 (a power of two dividing m') the plan's MatMult computes
 * sum_g RotL( sum_b RotR(e_{gB+b}, gB) (x) RotL(y, b), gB ) over g < m'/B, b < B, which equals
 * sum_i e_i (x) RotL(y, i).  Matrices encoded under the plan hold the pre-rotated plaintexts;
 * he_matmult_plain_cipher then runs B - 1 hoisted baby rotations per input, one
 * multiply-accumulate launch per output and m'/B - 1 giant rotations, with B - 1 + m'/B - 1
 * Galois keys instead of m' - 1 (fewer key bytes, more key-switching launches).  baby = 0 (the
 * default) restores the diagonal method.  Set it before encoding a matrix with the plan; batches,
 * the batched server lanes and he_matmult_plain_cipher_noalloc take only baby = 0 plans
 * (HE_EINVAL).  HE_EINVAL if baby is not 0 or a power of two dividing m'. */
int he_plan_set_baby_steps(he_plan *plan, int64_t baby);
/* The left-rotation steps whose Galois keys the plan's MatMult needs (1..m'-1, or the baby
 * steps 1..B-1 then the giant steps g B), into steps (may be NULL to count them). */
int he_plan_rotation_steps(const he_plan *plan, int32_t *steps, int *n_steps);

/* Encode X (device, row-major m x n doubles) into its diagonal plaintexts (Eq. 2 after Eq. 3):
 * e_{r,c,i}[b nb + j] = X[r mb + b m' + (j mod m'), c nb + (i + j) mod nb], at scale
 * q_level so that the MatMult's rescale returns the input ciphertext's scale. */
int he_encode_matrix(he_ctx *ctx, const he_plan *plan, const double *X, int level, he_ptmat **out);
/* Re-encode a new matrix X (same shape, device) into an existing encoded matrix, in place:
 * no allocation, asynchronous on the stream (a VFL iteration's next batch). */
int he_ptmat_encode(he_ctx *ctx, he_ptmat *pm, const double *X);
/* he_encode_matrix / he_ptmat_encode of the matrix X = Xt^T given its transpose Xt (device,
 * row-major n x m): the same plaintexts, bit for bit, without a transposed copy (a VFL party
 * holding its features X_A multiplies by X_A^T for the gradient and by X_A for the forward pass). */
int he_encode_matrix_transposed(he_ctx *ctx, const he_plan *plan, const double *Xt, int level, he_ptmat **out);
int he_ptmat_encode_transposed(he_ctx *ctx, he_ptmat *pm, const double *Xt);
/* Same object from integer plaintexts already encoded elsewhere: coeffs (device) holds
 * [R][C][m'][level+1+n_p][N] canonical residues in coefficient form over q_0..q_level, p_*. */
int he_ptmat_import(he_ctx *ctx, const he_plan *plan, const uint64_t *coeffs, int level, double scale, he_ptmat **out);
/* The inverse of he_ptmat_import: the encoded matrix's plaintexts in canonical coefficient form,
 * [R][C][m'][level+1+K][N] words, into caller-owned device memory (for parity checks and
 * transport). */
int he_ptmat_export(he_ctx *ctx, const he_ptmat *pm, uint64_t *coeffs_out);
void he_ptmat_free(he_ptmat *pm);

/* P_B's side: replicate piece c of y (device, n doubles) N'/nb times and encode it into
 * outs[c] for c < col_blocks (Sec. 4.2.1, "[[d]] is expanded by replicating its pattern"). */
int he_encode_vector(he_ctx *ctx, const he_plan *plan, const double *y, double scale, int level, he_pt *outs);
/* he_encode_vector then he_encrypt of each column block c, under nonce + c, or under the device
 * nonce nonce_dev[c] (read when the kernels run, as he_encrypt_dnonce) when nonce_dev is not
 * NULL: outs[0..col_blocks) ciphertexts at `level`.  The encoded coefficients join the error
 * before its NTT (NTT(m) + NTT(e) = NTT(m + e) mod q), so the ciphertexts equal those of the
 * separate calls bit for bit, in two launches for a single block. */
int he_encrypt_vector(he_ctx *ctx, const he_plan *plan, const double *y, double scale, int level, uint64_t nonce, const uint64_t *nonce_dev,
                      he_ct *outs);

/* The hot path: outs[r] = Rescale( sum_c sum_{i<m'} e_{r,c,i} (x) HstRotL(ins[c], i) ) for
 * r < row_blocks, with ins[c] for c < col_blocks at the ptmat's level (Tab. 2 PackVFL row,
 * Tab. 3).  Rotations stay in the extended basis and are divided by P once per output.
 * outs[r].data must hold 2*level*N words (one level is consumed). */
int he_matmult_plain_cipher(he_ctx *ctx, const he_plan *plan, const he_ptmat *pm, const he_ct *ins, int n_in,
                            he_ct *outs, int n_out);

/* he_matmult_plain_cipher without any memory allocation.  The paper has no counterpart: this
 * is a deployment variant of the same computation.  It is for callers that cannot let the
 * library call cudaMalloc or cudaFree: applications whose device memory belongs to their own
 * allocator and budget, and loops that must not pay, inside a call, the device-wide wait that
 * cudaFree implies.  Same arguments and bit-identical results as he_matmult_plain_cipher.
 * Its temporaries (ModUp digits, accumulators, the Galois-key table) live in one 16 MiB array
 * of device memory that the library reserves on every GPU it is loaded on, until the process
 * exits; a product that needs more returns HE_EBUDGET and computes nothing.  The first call on
 * each device looks up the array's device address (this can load the library's device code),
 * so make that first call before any stream capture.  Every call uses the same array: calls
 * that overlap on the GPU (other streams, other contexts, other threads) race and corrupt each
 * other's results, so serialise them.  Nothing in the array has to start at zero: each call
 * writes every word before reading it.  Plans with baby steps (he_plan_set_baby_steps) are
 * refused with HE_EINVAL. */
int he_matmult_plain_cipher_noalloc(he_ctx *ctx, const he_plan *plan, const he_ptmat *pm, const he_ct *ins, int n_in, he_ct *outs,
                                    int n_out);

/* The key switch of many rotations (he_rotate_hoisted, he_rotate_many with at least 32 of them)
 * runs its transforms as one CTA per limb-poly with the usual thread count (variant 0), with
 * 512 threads and at most 64 registers (variant 1), or in two phases of small CTAs per transform
 * (variant 2, log N = 12..14: the NTT form 2 split into rows and columns, see he_ntt_form).  The
 * first such call on a context times them on its first chunk (synchronising the stream; not
 * under stream capture) and keeps the fastest: variant (-1 before) and ms[0..HE_KS_VARIANTS-1]
 * (may be NULL) report the choice and the timings.  Every variant gives the same residues. */
#define HE_KS_VARIANTS 3
int he_keyswitch_tuning(const he_ctx *ctx, int *variant, float *ms);
/* Pin the key switch's transform variant for this context (0 .. HE_KS_VARIANTS-1; variant 2 only
 * at log N = 12..14, HE_EINVAL otherwise), or -1 to time them again on the next call. */
int he_set_keyswitch_variant(he_ctx *ctx, int variant);

/* NTT launches of many limb-polys (an encoded matrix's 4 x m' transforms, import and export of
 * plaintext batches) run as one CTA per limb-poly (form 0), as a 2-CTA cluster per limb-poly
 * (form 1: each CTA holds half of the coefficients, the one stage that pairs the halves goes
 * through distributed shared memory), or in two phases (form 2, log N = 12..14: with N = 64 C,
 * the forward transform's stages 0-5 as 64-point transforms of the C columns x = l C + c, then
 * the remaining stages as C-point transforms of the 64 rows, each phase one launch of many small
 * CTAs, the intermediate values in global memory; the inverse transform rows first; the ModUp of
 * he_rotate_many takes this form too).  The first matrix a
 * context encodes times the forms on its transform (synchronising the stream; not under stream
 * capture) and keeps the fastest for the context; he_ntt_form reports the choice (-1 before) and
 * ms[0..HE_NTT_FORMS-1] (may be NULL), he_set_ntt_form pins one (0 .. HE_NTT_FORMS-1, or -1 to
 * time again).  Results are the same in every form.  A fork starts with its parent's choice. */
#define HE_NTT_FORMS 3
int he_ntt_form(const he_ctx *ctx, int *form, float *ms);
int he_set_ntt_form(he_ctx *ctx, int form);

/* Basis extension engine of ModUp (the fast base conversion inside hybrid key switching, O3/O4
 * of Sec. 2.2) for this context's later calls: HE_BCONV_INT64 (default) sums the products
 * v_i (Q_d/q_i mod t) with exact 64-bit modular arithmetic; HE_BCONV_INT8_TC cuts v_i and the
 * constants into bytes, forms the byte products' 32-bit sums on the tensor cores (mma.sync
 * m16n8k32 u8 x u8 -> s32) and recombines them exactly mod t.  Both give the same residues bit
 * for bit (results never depend on the engine).  Used by he_rotate, he_rotate_hoisted,
 * he_rotate_many (he_cdiag_transpose) and he_matmult_plain_cipher; the batch and serving kernels
 * keep the INT64 form.  A fork starts with its parent's engine. */
#define HE_BCONV_INT64 0
#define HE_BCONV_INT8_TC 1
int he_set_basis_extension(he_ctx *ctx, int engine);
int he_get_basis_extension(const he_ctx *ctx, int *engine);
/* Host only: sum_i v[i] h[i] mod t for i < alpha (1..4, any 64-bit v[i], h[i], 3 <= t < 2^62)
 * computed as HE_BCONV_INT8_TC computes it (byte products, 32-bit partial sums, recombination),
 * for checking that arithmetic on the CPU. */
int he_bconv_i8_host(int alpha, const uint64_t *v, const uint64_t *h, uint64_t t, uint64_t *out);
/* ModUp (Sec. 2.2) of ct's c1 with the context's engine, exported in canonical coefficient form:
 * digits_out (device) [ndig][level+1+n_p][N] words, ndig = ceil((level+1) / alpha), alpha =
 * ceil(n_q / dnum): digit d's primes copied, every other limb of Q_level U P the fast base
 * conversion of the digit (for parity checks). */
int he_modup_export(he_ctx *ctx, const he_ct *ct, uint64_t *digits_out);

/* Batched form of the hot path for many independent MatMults of uneven shapes (one input
 * and one output ciphertext each, i.e. m, n <= N/2) at one level.  he_batch_create binds the
 * plans, encoded matrices and Galois keys and allocates the batch's scratch; he_batch_run
 * computes outs[j] = MatMult(pms[j], ins[j]) for every j with one persistent work-queue kernel
 * for all rotation steps of all jobs (keys shared across jobs), the whole sequence captured
 * once into a CUDA graph and replayed on later runs.  Results are bit-identical to
 * he_matmult_plain_cipher on each job.  Asynchronous on the context's stream. */
typedef struct he_batch he_batch;
int he_batch_create(he_ctx *ctx, int count, const he_plan *const *plans, const he_ptmat *const *pms, he_batch **out);
int he_batch_run(he_ctx *ctx, he_batch *batch, const he_ct *ins, he_ct *outs);
void he_batch_free(he_batch *batch);

/* Autotuning of the key-switch / multiply-accumulate loop kernel.  Its variants give identical
 * results and differ in coefficients per thread (1 or 2), rotation groups per block (4 or 8)
 * and how each rotation step's operands are prefetched: in registers one step ahead, or S
 * steps ahead through a per-thread cp.async pipeline in shared memory that carries the key and
 * plaintext streams and, in the "gathers" variants, the automorphism gathers of the ModUp
 * digits and c0 too.  The first he_matmult_plain_cipher call with an encoded matrix, and the
 * first he_batch_run of a batch, time each variant (best of a few runs, synchronising the
 * stream) and keep the fastest.  he_loop_variant_count gives the number of variants (at most HE_MM_MAX_VARIANTS);
 * he_loop_variant_shape the (vec, groups, stages, gathers) of variant v (HE_EINVAL if v is out
 * of range).  The tuning queries report the choice (-1 before the first call) and write the
 * timed milliseconds of every variant to ms[0 .. count-1] (ms may be NULL; else it holds
 * HE_MM_MAX_VARIANTS floats). */
#define HE_MM_MAX_VARIANTS 8
int he_loop_variant_count(void);
int he_loop_variant_shape(int v, int *vec, int *groups, int *stages, int *gathers);
int he_ptmat_tuning(const he_ptmat *pm, int *variant, float *ms);
int he_batch_tuning(const he_batch *batch, int *variant, float *ms);
/* Pin the loop-kernel variant of an encoded matrix or a batch (0 .. count-1), or with -1 let
 * the next call tune again.  HE_EINVAL for NULL or v out of range.  A batch re-captures its
 * graph on its next run (this call waits for the batch's previous run to finish). */
int he_ptmat_set_variant(he_ptmat *pm, int v);
int he_batch_set_variant(he_batch *batch, int v);
/* Fused key tables (Sec. 2.2 O4 with the plaintext product of Sec. 4.2 folded in): for an encoded
 * matrix that is multiplied more than once, the MatMult can read, for every rotation step i,
 * digit d and component c, the products F_i[d][c] = ksk_i[d][c] (x) pt_i (Montgomery form, built
 * once on the GPU from the bound Galois keys) instead of the key and the plaintext, so that the
 * loop accumulates sum_i sum_d D_d(src_i) F_i[d][c] with one product per operand pair and no
 * per-step reduction.  The residues, and so the outputs, are the same as without the tables.
 * Memory: (m' - 1) ndig 2 (l+1+K) N 8 bytes per plaintext block, owned by the encoded matrix.
 * he_set_key_fusion sets the context family's policy: mode 0 never; 1 (default) when an encoding
 * is multiplied a second time without being re-encoded; 2 at the first MatMult; tables above
 * max_bytes (0: 8 GiB) are never built.  When built, both forms are timed on that call (which
 * then synchronises the stream) and the tables kept only if faster.  Re-encoding a matrix that
 * holds tables rebuilds them in stream order.  Only for 1 to 3 digits, not under stream
 * capture (a captured MatMult uses the tables if they exist), not on the batched, BSGS and
 * allocation-free paths.  he_ptmat_key_fusion reports state (0 not tried, 1 in use, -1 not
 * used), the fused form's variant and, when ms is not NULL, its timed ms per variant
 * (HE_MM_MAX_VARIANTS entries, 0 for variants without a fused form);
 * he_ptmat_set_key_fusion(pm, 0, -1) frees the tables (after pm's context's stream: no graph
 * captured with them may be replayed afterwards) and keeps them off for pm;
 * (pm, 1, -1) makes pm eligible again; (pm, 1, v) pins the fused form with loop-kernel variant v
 * (one with cp.async stages, he_loop_variant_shape) for pm whatever the context's mode: the
 * tables are built at pm's next MatMult (not under capture) and used without timing.  HE_EINVAL
 * for NULL, a mode out of range or a variant without a fused form. */
int he_set_key_fusion(he_ctx *ctx, int mode, size_t max_bytes);
int he_ptmat_key_fusion(const he_ptmat *pm, int *state, int *variant, float *ms);
int he_ptmat_set_key_fusion(he_ptmat *pm, int on, int variant);
/* A batch's ModUp, ModDown and rescale run as one CTA per limb-poly (form 0) or as 8-CTA clusters
 * per limb-poly (form 1: fewer, shorter launches, for batches of few jobs); the results are the
 * same.  The first he_batch_run times both forms with the chosen loop variant and keeps the faster;
 * he_batch_stage_form reports it (form, and ms[0..1] when ms is not NULL), he_batch_set_stage_form
 * pins one (0 or 1; re-captures the graph on the next run).  A server's batch lanes use form 1. */
int he_batch_stage_form(const he_batch *batch, int *form, float *ms);
int he_batch_set_stage_form(he_batch *batch, int form);

/* Serving loop with continuous batching (requests of differing shapes, m, n <= N/2, at one
 * level).  A scheduler thread admits requests in arrival order while the device bytes they pin
 * (encoded matrix, input and output ciphertext) fit hbm_budget_bytes, packs admitted requests
 * into up to `slots` slots of one of two batch lanes and launches that lane's captured batch
 * graph; requests arriving while a lane runs join the other lane's next launch, so their work
 * overlaps.  A request that arrives alone while nothing of its ring runs is served by one
 * he_matmult_plain_cipher call on the context's stream instead (no batch of one).  plain != 0 serves one request per he_matmult_plain_cipher call instead (the
 * one-request-per-launch baseline).  While a server runs it owns the context's stream and
 * scratch: make no other calls on the context until he_server_free.  Completion is observed
 * with CUDA events; no kernel waits on another. */
typedef struct he_server he_server;
int he_server_create(he_ctx *ctx, int slots, int level, size_t hbm_budget_bytes, int plain, he_server **out);
/* Serve a further ring: requests whose encoded matrix belongs to ctx's family at `level` (another
 * ring size or parameter set, e.g. an N = 4096 context beside an N = 8192 one) get lanes of their
 * own on ctx's stream, under the same budget and in the same arrival order.  Only before the first
 * submit (HE_EINVAL after, for a ring already served, or beyond 8 rings).  The server owns every
 * ring's context while it runs, as it owns the first. */
int he_server_add_ring(he_server *s, he_ctx *ctx, int level);
/* Queue outs = MatMult(pm, in); in must be ready on its ring context's stream when this is called.
 * HE_EBUDGET if the request alone exceeds the budget; HE_EINVAL for a matrix of no served ring
 * (HE_ELEVEL for a served family at another level), or a baby-step plan on batch lanes.  *out's
 * level and scale are set now, its data when the request completes. */
int he_server_submit(he_server *s, const he_plan *plan, const he_ptmat *pm, const he_ct *in, he_ct *out, int64_t *request_id);
/* Block until the request completes (its output is then ready for any stream) or timeout_us
 * passes (HE_ETIMEOUT); latency_s (optional) = completion - submission, host clock.  Once it
 * has returned the request's status, the server forgets the request: a second wait on the same
 * id returns HE_EINVAL.  After HE_ETIMEOUT the request is still known and can be waited for again. */
int he_server_wait(he_server *s, int64_t request_id, int64_t timeout_us, double *latency_s);
int he_server_stats(he_server *s, int64_t *completed, int64_t *launches, size_t *bytes_in_use);
/* Finishes every queued request, stops the scheduler and releases the lanes. */
void he_server_free(he_server *s);

/* VFL-NN forward pass with the encrypted operand diagonally encoded (Alg. 3, Sec. 5.3).
 * P_A encrypts its activation matrix A (m x n, powers of two, max(m, n) <= N/2) as its
 * min(m, n) diagonals e_i[j] = A[j mod m, (i + j) mod n] (Eq. 2), each repeated over the N/2
 * slots (he_cdiag_encode_matrix, then he_encrypt of each).  P_B holds W (n x K, row-major,
 * device); he_cdiag_encode_weights encodes each column, repeated with period n, at scale
 * q_level.  he_cdiag_matmult then gives, for every column k,
 *   outs[k] = Rescale( sum_i RotL(w_k, i) (x) [[e_i]] ),
 * with the plaintext rotation done as the automorphism X -> X^(5^i) of w_k's plaintext (no
 * key switching: "eliminate all O4").  After decryption, he_cdiag_decode turns the K slot
 * vectors (device [K][N/2]) into Z = A W (device, m x K row-major), summing the n/m slot
 * groups when m < n (lazy rotate-and-sum, Sec. 4.3).  n_ct <= 1024 per call. */
typedef struct he_cdmat he_cdmat;
int he_cdiag_encode_weights(he_ctx *ctx, const double *W, int64_t n, int64_t K, int level, he_cdmat **out);
void he_cdmat_free(he_cdmat *W);
int he_cdiag_encode_matrix(he_ctx *ctx, const double *A, int64_t m, int64_t n, double scale, int level, he_pt *outs);
int he_cdiag_matmult(he_ctx *ctx, const he_cdmat *W, const he_ct *cts, int n_ct, he_ct *outs);
int he_cdiag_decode(he_ctx *ctx, int64_t m, int64_t n, int64_t K, const double *slots, double *Z);
/* Transposed matrices' diagonal conversion (Sec. 5.3, Eq. 5): from the min(m, n) diagonal
 * ciphertexts of A (m x n), the diagonal ciphertexts of A^T (n x m) for the backward pass
 * (Alg. 4), each a rotation outs[i] = RotL(cts[k], r) with k = (-i) mod min(m, n) and r = i
 * when m >= n, r = (-k) mod n when m < n (the printed RotR form does not give A^T's diagonals).
 * Needs the Galois keys of those steps (HE_EKEY otherwise); outs must not alias cts. */
int he_cdiag_transpose(he_ctx *ctx, const he_ct *cts, int64_t m, int64_t n, he_ct *outs);
/* Host only: the distinct nonzero rotation steps he_cdiag_transpose uses for an m x n matrix
 * (the Galois keys to make first), ascending; steps may be NULL to count them (at most
 * min(m, n) - 1). */
int he_cdiag_transpose_steps(int64_t m, int64_t n, int32_t *steps, int *n_steps);

/* P_B's side after decryption: lazy rotate-and-sum (Sec. 4.3).  slots: device
 * [row_blocks][N/2] doubles (he_decrypt of each output), y_out: device m doubles. */
/* Decryption, decoding and the lazy rotate-and-sum of a MatMult's outputs in one call:
 * cts[0..row_blocks) (one scale), mask as he_matmult_decode_masked (device [row_blocks][N/2],
 * may be NULL), y_out (device, m doubles).  The same doubles as he_decrypt of each ciphertext
 * then he_matmult_decode(_masked), without the slot array (the sums run in the decoding launch). */
int he_matmult_decrypt(he_ctx *ctx, const he_plan *plan, const he_ct *cts, int n_ct, const double *mask, double *y_out);
int he_matmult_decode(he_ctx *ctx, const he_plan *plan, const double *slots, double *y_out);
/* Alg. 1's last step: remove a slot mask (device [row_blocks][N/2] doubles, the values that
 * were encoded and added with he_add_plain before decryption; NULL = none) and apply the lazy
 * rotate-and-sum: y = lazyRaS(slots - mask). */
int he_matmult_decode_masked(he_ctx *ctx, const he_plan *plan, const double *slots, const double *mask, double *y_out);

/* The ciphertext rotate-and-sum that the lazy RaS replaces (Sec. 3, Sec. 4.3), for consumers
 * that need the sums inside the ciphertext: for each step m' 2^j, j < log2(nb / m'), in turn,
 * x <- x + RotL(x, step).  Afterwards slot b nb + t of row block r's ciphertext holds output
 * row r mb + b m' + t.  he_plan_ras_steps lists the steps (steps may be NULL to count them;
 * at most 40); he_ras needs their Galois keys (HE_EKEY) and runs on one row block's output
 * ciphertext (out may alias in).  he_ras_decode gathers y from the decrypted slots [R][N/2]. */
int he_plan_ras_steps(const he_plan *plan, int32_t *steps, int *n_steps);
int he_ras(he_ctx *ctx, const he_plan *plan, const he_ct *in, he_ct *out);
int he_ras_decode(he_ctx *ctx, const he_plan *plan, const double *slots, double *y_out);

/* Host-memory forms of the party-facing calls (the problem statement of Sec. 3 and Alg. 1: P_A
 * holds the cleartext X, P_B encrypts y and decrypts the product, ciphertexts travel between the
 * parties as bytes).  Each takes its bulk inputs from and writes its results to HOST memory and
 * otherwise equals its device-memory counterpart above, bit for bit.  Inputs are copied on the
 * context's stream with one copy per buffer: from page-locked memory (cudaMallocHost,
 * cudaHostRegister) the copy is asynchronous, so the buffer must stay unchanged until the stream
 * has passed it; from pageable memory the library first copies into its own page-locked staging
 * (a stream capture of such a call returns HE_EINVAL).  Results: into page-locked memory the copy
 * is queued and the values are valid once the stream reaches it (he_synchronize); into pageable
 * memory the call waits and the values are valid on return.  The staging buffers belong to the
 * context (a fork has its own) and grow on demand.
 *
 * he_encode_matrix_host / he_ptmat_encode_host: X host row-major m x n doubles (its transpose,
 * n x m, when transposed != 0), as he_encode_matrix(_transposed) / he_ptmat_encode(_transposed).
 * he_encrypt_vector_host: y host, n doubles, as he_encrypt_vector.
 * he_decrypt_host: N/2 slot values into host memory, as he_decrypt.
 * he_matmult_decrypt_host: mask host [row_blocks][N/2] doubles or NULL, y host m doubles, as
 * he_matmult_decrypt. */
int he_encode_matrix_host(he_ctx *ctx, const he_plan *plan, const double *X, int level, int transposed, he_ptmat **out);
int he_ptmat_encode_host(he_ctx *ctx, he_ptmat *pm, const double *X, int transposed);
int he_encrypt_vector_host(he_ctx *ctx, const he_plan *plan, const double *y, double scale, int level, uint64_t nonce,
                           const uint64_t *nonce_dev, he_ct *outs);
int he_decrypt_host(he_ctx *ctx, const he_ct *ct, double *slots);
int he_matmult_decrypt_host(he_ctx *ctx, const he_plan *plan, const he_ct *cts, int n_ct, const double *mask, double *y);

/* A ciphertext as bytes in host memory, for transport between parties (Alg. 1: [[d]] and the
 * masked gradients cross the network).  Layout, little-endian: a 32-byte header (uint32 magic
 * "HECT", uint32 version 1, int32 log_n, int32 level, double scale, 8 reserved bytes), the
 * level+1 primes q_0..q_level (uint64), then [2][level+1][N] uint64 canonical coefficients
 * (coefficient form, so the bytes do not depend on the NTT ordering).
 * he_ct_export_host: with buf == NULL writes the byte count to *len; else *len is buf's capacity
 * (HE_EINVAL, with the needed count in *len, if too small) and on return holds the bytes written.
 * Synchronises: the bytes are complete on return.
 * he_ct_host_level: the level stored in a buffer (to size the import's device buffer).
 * he_ct_import_host: checks the header, that log_n and the primes are this context's and that
 * every coefficient is canonical (HE_EINVAL otherwise, HE_ELEVEL for a level the context lacks);
 * out->data (device) must hold he_ct_bytes(level) bytes; sets out's level and scale. */
int he_ct_export_host(he_ctx *ctx, const he_ct *ct, void *buf, size_t *len);
int he_ct_host_level(const void *buf, size_t len, int32_t *level);
int he_ct_import_host(he_ctx *ctx, const void *buf, size_t len, he_ct *out);

/* Canonical coefficient form (device, [2][level+1][N]) of a ciphertext, and back. */
int he_ct_export(he_ctx *ctx, const he_ct *ct, uint64_t *coeffs_out);
int he_ct_import(he_ctx *ctx, const uint64_t *coeffs, int level, double scale, he_ct *out);
/* Same for plaintexts ([level+1][N]). */
int he_pt_export(he_ctx *ctx, const he_pt *pt, uint64_t *coeffs_out);
int he_pt_import(he_ctx *ctx, const uint64_t *coeffs, int level, double scale, he_pt *out);

#ifdef __cplusplus
}
#endif
#endif /* HE_H */
