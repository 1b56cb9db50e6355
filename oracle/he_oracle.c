/*
 * he_oracle.c -- plain, slow CPU oracle for RNS-CKKS and the PackVFL MatMult.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this file.  The GPU library shares no code,
 * header, table or constant generator with it.
 *
 * Everything here works on polynomials of Z_q[X]/(X^N + 1) in the COEFFICIENT
 * domain (Sec. 2.2: RLWE ciphertexts (x - a s + e, a) over that ring).  Residues
 * are canonical, in [0, q).  Products use unsigned __int128 and the C `%`
 * operator; a number-theoretic transform is used only inside poly_mul, as a
 * tool to multiply two polynomials (it is pinned against a schoolbook product).
 *
 * Layouts (row-major, uint64 residues):
 *   RNS poly   [limbs][N]
 *   ciphertext [2][limbs][N]          (c0, c1)
 *   Galois key [dnum][2][L+K][N]      (b_d, a_d) over Q then P primes
 *   extended digits (ModUp) [ndig][limbs+K][N]
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------ */
/* scalar modular arithmetic                                            */
/* ------------------------------------------------------------------ */
static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)(((u128)a * b) % q); }
static uint64_t addmod(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)(((u128)a + b) % q); }
static uint64_t submod(uint64_t a, uint64_t b, uint64_t q) { a %= q; b %= q; return a >= b ? a - b : a + (q - b); }

uint64_t or_powmod(uint64_t a, uint64_t e, uint64_t q) {
    uint64_t r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = mulmod(r, a, q);
        a = mulmod(a, a, q);
        e >>= 1;
    }
    return r;
}

/* Threads of the OpenMP loops below (1 when built without OpenMP).  Only loops whose
 * iterations are independent, or whose partial results are combined by exact modular sums,
 * are parallel, so results do not depend on the thread count. */
int or_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* inverse modulo a prime q (Fermat) */
uint64_t or_invmod(uint64_t a, uint64_t q) { return or_powmod(a, q - 2, q); }

/* signed integer -> residue in [0, q) */
static uint64_t from_signed(int64_t v, uint64_t q) {
    int64_t r = v % (int64_t)q;
    if (r < 0) r += (int64_t)q;
    return (uint64_t)r;
}

/* Miller-Rabin; the first twelve primes as bases decide every n < 3.3e24. */
int or_is_prime(uint64_t n) {
    static const uint64_t bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; ++i) {
        if (n == bases[i]) return 1;
        if (n % bases[i] == 0) return 0;
    }
    uint64_t d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; ++s; }
    for (int i = 0; i < 12; ++i) {
        uint64_t x = or_powmod(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int composite = 1;
        for (int r = 1; r < s; ++r) {
            x = mulmod(x, x, n);
            if (x == n - 1) { composite = 0; break; }
        }
        if (composite) return 0;
    }
    return 1;
}

/*
 * Prime chain.  For each requested bit size b, in order, take the largest prime
 * q < 2^b with q = 1 (mod 2N) that is not already in the chain.  The congruence
 * makes X^N + 1 split into linear factors mod q (needed for the RNS ring of
 * Sec. 2.2).  Returns 0, or -1 when no such prime above 2^(b-1) exists.
 */
int or_gen_primes(int log_n, int count, const int *bits, uint64_t *out) {
    uint64_t m = 2ull << log_n; /* 2N */
    for (int i = 0; i < count; ++i) {
        int b = bits[i];
        if (b < 2 || b > 62) return -1;
        uint64_t top = 1ull << b;
        uint64_t c = ((top - 1) / m) * m + 1;
        if (c >= top) c -= m;
        int found = 0;
        while (c > (top >> 1)) {
            int used = 0;
            for (int j = 0; j < i; ++j) used |= (out[j] == c);
            if (!used && or_is_prime(c)) { out[i] = c; found = 1; break; }
            c -= m;
        }
        if (!found) return -1;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* ring Z_q[X]/(X^N+1), one limb                                        */
/* ------------------------------------------------------------------ */

/* schoolbook negacyclic product: X^N = -1 (the ring of Sec. 2.2) */
void or_negacyclic_schoolbook(int n, uint64_t q, const uint64_t *a, const uint64_t *b, uint64_t *out) {
    for (int k = 0; k < n; ++k) out[k] = 0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            uint64_t p = mulmod(a[i], b[j], q);
            int k = i + j;
            if (k < n) out[k] = addmod(out[k], p, q);
            else out[k - n] = submod(out[k - n], p, q);
        }
}

/* a primitive 2N-th root of unity mod q: x^((q-1)/2N) for the first x >= 2 that is a non-residue */
static uint64_t root_2n(int n, uint64_t q) {
    for (uint64_t x = 2;; ++x) {
        if (or_powmod(x, (q - 1) / 2, q) == q - 1) return or_powmod(x, (q - 1) / (2 * (uint64_t)n), q);
    }
}

static unsigned bitrev(unsigned x, int bits) {
    unsigned r = 0;
    for (int i = 0; i < bits; ++i) { r = (r << 1) | (x & 1); x >>= 1; }
    return r;
}

/* cyclic DFT over Z_q of length n with root w (radix-2, decimation in time). */
static void cyclic_ntt(int n, uint64_t q, uint64_t w, uint64_t *a) {
    int logn = 0;
    while ((1 << logn) < n) ++logn;
    for (int i = 0; i < n; ++i) {
        int j = (int)bitrev((unsigned)i, logn);
        if (j > i) { uint64_t t = a[i]; a[i] = a[j]; a[j] = t; }
    }
    for (int len = 2; len <= n; len <<= 1) {
        uint64_t wl = or_powmod(w, (uint64_t)(n / len), q);
        for (int s = 0; s < n; s += len) {
            uint64_t wk = 1;
            for (int j = 0; j < len / 2; ++j) {
                uint64_t u = a[s + j], v = mulmod(a[s + j + len / 2], wk, q);
                a[s + j] = addmod(u, v, q);
                a[s + j + len / 2] = submod(u, v, q);
                wk = mulmod(wk, wl, q);
            }
        }
    }
}

/* a -> (a(psi^(2k+1)))_k : twist by psi^j, then cyclic DFT with omega = psi^2 */
void or_ntt_forward(int n, uint64_t q, uint64_t *a) {
    uint64_t psi = root_2n(n, q), p = 1;
    for (int j = 0; j < n; ++j) { a[j] = mulmod(a[j], p, q); p = mulmod(p, psi, q); }
    cyclic_ntt(n, q, mulmod(psi, psi, q), a);
}

void or_ntt_inverse(int n, uint64_t q, uint64_t *a) {
    uint64_t psi = root_2n(n, q);
    uint64_t ipsi = or_invmod(psi, q);
    cyclic_ntt(n, q, mulmod(ipsi, ipsi, q), a);
    uint64_t ninv = or_invmod((uint64_t)n % q, q), p = ninv;
    for (int j = 0; j < n; ++j) { a[j] = mulmod(a[j], p, q); p = mulmod(p, ipsi, q); }
}

/* negacyclic product through the transform (checked against the schoolbook one) */
void or_poly_mul(int n, uint64_t q, const uint64_t *a, const uint64_t *b, uint64_t *out) {
    uint64_t *fa = malloc(sizeof(uint64_t) * n), *fb = malloc(sizeof(uint64_t) * n);
    for (int i = 0; i < n; ++i) { fa[i] = a[i] % q; fb[i] = b[i] % q; }
    or_ntt_forward(n, q, fa);
    or_ntt_forward(n, q, fb);
    for (int i = 0; i < n; ++i) fa[i] = mulmod(fa[i], fb[i], q);
    or_ntt_inverse(n, q, fa);
    memcpy(out, fa, sizeof(uint64_t) * n);
    free(fa);
    free(fb);
}

/* Galois automorphism a(X) -> a(X^g), g odd: coefficient k moves to k*g mod 2N, negated past N. */
void or_automorph(int n, uint64_t q, uint64_t g, const uint64_t *a, uint64_t *out) {
    uint64_t two_n = 2 * (uint64_t)n;
    for (int k = 0; k < n; ++k) {
        uint64_t t = ((uint64_t)k * g) % two_n;
        if (t < (uint64_t)n) out[t] = a[k] % q;
        else out[t - n] = submod(0, a[k], q);
    }
}

/* ------------------------------------------------------------------ */
/* Philox-4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11) and samplers      */
/* ------------------------------------------------------------------ */
void or_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3], k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        u128 p0 = (u128)0xD2E7470EE14C6C93ull * c0;
        u128 p1 = (u128)0xCA5A826395121157ull * c2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B97F4A7C15ull;
        k1 += 0xBB67AE8584CAA73Bull;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* stream tags (Philox key word 1) */
enum { TAG_SECRET = 1, TAG_ENC_A = 2, TAG_ENC_E = 3, TAG_EVK_A = 4, TAG_EVK_E = 5 };

static void block(uint64_t seed, uint64_t tag, uint64_t b, uint64_t limb, uint64_t nonce, uint64_t out[4]) {
    uint64_t ctr[4] = {b, limb, nonce, 0}, key[2] = {seed, tag};
    or_philox4x64(ctr, key, out);
}

/* ternary secret: s_j = (w mod 3) - 1, w = word (j mod 4) of block j/4 */
void or_sample_ternary(int n, uint64_t seed, int64_t *s) {
    uint64_t w[4];
    for (int j = 0; j < n; ++j) {
        if ((j & 3) == 0) block(seed, TAG_SECRET, (uint64_t)j >> 2, 0, 0, w);
        s[j] = (int64_t)(w[j & 3] % 3) - 1;
    }
}

/* uniform mod q: the 128-bit integer (word 2(j&1)+1 : word 2(j&1)) of block j/2, reduced mod q */
void or_sample_uniform(int n, uint64_t seed, uint64_t tag, uint64_t nonce, int limb, uint64_t q, uint64_t *out) {
    uint64_t w[4];
    for (int j = 0; j < n; ++j) {
        if ((j & 1) == 0) block(seed, tag, (uint64_t)j >> 1, (uint64_t)limb, nonce, w);
        u128 v = ((u128)w[2 * (j & 1) + 1] << 64) | w[2 * (j & 1)];
        out[j] = (uint64_t)(v % q);
    }
}

/*
 * Discrete Gaussian, sigma = 3.2, support |x| <= 19, by cumulative table.
 * rho(y) = exp(-y^2 / 20.48); cum_k = rho(-19) + ... + rho(-19+k), summed left to right;
 * T_k = floor(2^40 * cum_k / total), k = 0..37.  A 40-bit draw r gives x = -19 + #{k : r >= T_k}.
 */
void or_cdt_table(uint64_t *t) {
    double rho[39], total = 0.0, cum = 0.0;
    for (int i = 0; i < 39; ++i) {
        double y = (double)(i - 19);
        rho[i] = exp(-(y * y) / 20.48);
    }
    for (int i = 0; i < 39; ++i) total += rho[i];
    for (int k = 0; k < 38; ++k) {
        cum += rho[k];
        t[k] = (uint64_t)floor(ldexp(cum / total, 40));
    }
}

void or_sample_gauss(int n, uint64_t seed, uint64_t tag, uint64_t nonce, int64_t *out) {
    uint64_t t[38], w[4];
    or_cdt_table(t);
    for (int j = 0; j < n; ++j) {
        if ((j & 3) == 0) block(seed, tag, (uint64_t)j >> 2, 0, nonce, w);
        uint64_t r = w[j & 3] >> 24;
        int64_t x = -19;
        for (int k = 0; k < 38; ++k) x += (r >= t[k]);
        out[j] = x;
    }
}

/* ------------------------------------------------------------------ */
/* RNS-CKKS scheme                                                      */
/* ------------------------------------------------------------------ */
typedef struct {
    int32_t n;    /* ring degree N */
    int32_t L;    /* number of ciphertext primes q_0..q_{L-1} */
    int32_t K;    /* number of special primes p_0..p_{K-1} */
    int32_t dnum; /* key-switching digits */
    uint64_t primes[64]; /* q_0..q_{L-1}, p_0..p_{K-1} */
} or_params;

static int alpha_of(const or_params *p) { return (p->L + p->dnum - 1) / p->dnum; }
static int ndigits_at(const or_params *p, int level) { int a = alpha_of(p); return (level + 1 + a - 1) / a; }
/* prime of limb u in the basis Q_level U P */
static uint64_t qp_prime(const or_params *p, int level, int u) { return u <= level ? p->primes[u] : p->primes[p->L + (u - level - 1)]; }
/* index of that limb inside a top-level key (Q primes, then P primes) */
static int key_limb(const or_params *p, int level, int u) { return u <= level ? u : p->L + (u - level - 1); }

static void mul_into(int n, uint64_t q, const uint64_t *a, const uint64_t *b, uint64_t *acc, uint64_t *tmp) {
    or_poly_mul(n, q, a, b, tmp);
    for (int k = 0; k < n; ++k) acc[k] = addmod(acc[k], tmp[k], q);
}

void or_keygen_secret(const or_params *p, uint64_t seed, int64_t *s) { or_sample_ternary(p->n, seed, s); }

/*
 * Galois (rotation) key for automorphism X -> X^g, hybrid key switching with dnum digits.
 * Digit d holds primes q_{d*alpha} .. q_{min((d+1)alpha, L)-1}.  Over every prime of Q U P:
 *   b_d = -a_d s + e_d + P * T_d * phi_g(s),   a_d uniform,
 * where T_d = 1 mod the digit's primes and 0 mod the other Q primes (P*T_d vanishes mod P).
 */
void or_galois_key(const or_params *p, uint64_t seed, const int64_t *s, uint64_t g, uint64_t *evk) {
    int n = p->n, L = p->L, K = p->K, al = alpha_of(p);
    uint64_t *a = malloc(sizeof(uint64_t) * n), *sl = malloc(sizeof(uint64_t) * n), *tmp = malloc(sizeof(uint64_t) * n);
    uint64_t *sg = malloc(sizeof(uint64_t) * n), *sgl = malloc(sizeof(uint64_t) * n);
    int64_t *e = malloc(sizeof(int64_t) * n);
    for (int d = 0; d < p->dnum; ++d) {
        uint64_t nonce = (g << 8) | (uint64_t)d;
        or_sample_gauss(n, seed, TAG_EVK_E, nonce, e);
        for (int l = 0; l < L + K; ++l) {
            uint64_t q = p->primes[l];
            uint64_t *b_out = evk + ((size_t)(d * 2 + 0) * (L + K) + l) * n;
            uint64_t *a_out = evk + ((size_t)(d * 2 + 1) * (L + K) + l) * n;
            or_sample_uniform(n, seed, TAG_EVK_A, nonce, l, q, a);
            for (int k = 0; k < n; ++k) sl[k] = from_signed(s[k], q);
            or_poly_mul(n, q, a, sl, tmp);
            for (int k = 0; k < n; ++k) b_out[k] = submod(from_signed(e[k], q), tmp[k], q);
            if (l < L && l >= d * al && l < (d + 1) * al) {
                uint64_t pmod = 1 % q;
                for (int j = 0; j < K; ++j) pmod = mulmod(pmod, p->primes[L + j] % q, q);
                or_automorph(n, q, g, sl, sg);
                for (int k = 0; k < n; ++k) b_out[k] = addmod(b_out[k], mulmod(pmod, sg[k], q), q);
            }
            memcpy(a_out, a, sizeof(uint64_t) * n);
        }
    }
    (void)sgl;
    free(a); free(sl); free(tmp); free(sg); free(sgl); free(e);
}

/* symmetric RLWE encryption (Sec. 2.2): c0 = m - a s + e, c1 = a, at the given level */
void or_encrypt(const or_params *p, uint64_t seed, const int64_t *s, uint64_t nonce, int level, const uint64_t *m, uint64_t *ct) {
    int n = p->n, nl = level + 1;
    uint64_t *a = malloc(sizeof(uint64_t) * n), *sl = malloc(sizeof(uint64_t) * n), *tmp = malloc(sizeof(uint64_t) * n);
    int64_t *e = malloc(sizeof(int64_t) * n);
    or_sample_gauss(n, seed, TAG_ENC_E, nonce, e);
    for (int l = 0; l < nl; ++l) {
        uint64_t q = p->primes[l];
        or_sample_uniform(n, seed, TAG_ENC_A, nonce, l, q, a);
        for (int k = 0; k < n; ++k) sl[k] = from_signed(s[k], q);
        or_poly_mul(n, q, a, sl, tmp);
        uint64_t *c0 = ct + (size_t)l * n, *c1 = ct + (size_t)(nl + l) * n;
        for (int k = 0; k < n; ++k) c0[k] = addmod(submod(m[(size_t)l * n + k], tmp[k], q), from_signed(e[k], q), q);
        memcpy(c1, a, sizeof(uint64_t) * n);
    }
    free(a); free(sl); free(tmp); free(e);
}

/* decryption (Sec. 2.2): c0 + c1 s = m + e, per limb */
void or_decrypt(const or_params *p, const int64_t *s, int level, const uint64_t *ct, uint64_t *m) {
    int n = p->n, nl = level + 1;
    uint64_t *sl = malloc(sizeof(uint64_t) * n), *tmp = malloc(sizeof(uint64_t) * n);
    for (int l = 0; l < nl; ++l) {
        uint64_t q = p->primes[l];
        for (int k = 0; k < n; ++k) sl[k] = from_signed(s[k], q);
        or_poly_mul(n, q, ct + (size_t)(nl + l) * n, sl, tmp);
        for (int k = 0; k < n; ++k) m[(size_t)l * n + k] = addmod(ct[(size_t)l * n + k], tmp[k], q);
    }
    free(sl); free(tmp);
}

/* O1: slot-wise addition of two ciphertexts at one level */
void or_add(const or_params *p, int level, const uint64_t *x, const uint64_t *y, uint64_t *out) {
    int n = p->n, nl = level + 1;
    for (int c = 0; c < 2; ++c)
        for (int l = 0; l < nl; ++l) {
            uint64_t q = p->primes[l];
            size_t o = ((size_t)c * nl + l) * n;
            for (int k = 0; k < n; ++k) out[o + k] = addmod(x[o + k], y[o + k], q);
        }
}

/* O1 with a plaintext operand: (c0 + m, c1) (the decryption c0 + c1 s gains m) */
void or_add_plain(const or_params *p, int level, const uint64_t *ct, const uint64_t *pt, uint64_t *out) {
    int n = p->n, nl = level + 1;
    for (int l = 0; l < nl; ++l) {
        uint64_t q = p->primes[l];
        for (int k = 0; k < n; ++k) {
            out[(size_t)l * n + k] = addmod(ct[(size_t)l * n + k], pt[(size_t)l * n + k], q);
            out[((size_t)nl + l) * n + k] = ct[((size_t)nl + l) * n + k];
        }
    }
}

/* O2: plaintext x ciphertext (each component times the plaintext polynomial) */
void or_mul_plain(const or_params *p, int level, const uint64_t *ct, const uint64_t *pt, uint64_t *out) {
    int n = p->n, nl = level + 1;
    for (int c = 0; c < 2; ++c)
        for (int l = 0; l < nl; ++l)
            or_poly_mul(n, p->primes[l], ct + ((size_t)c * nl + l) * n, pt + (size_t)l * n, out + ((size_t)c * nl + l) * n);
}

/*
 * ModUp (basis extension of each digit of c1 to Q_level U P), exact fast base conversion:
 *   y_t = sum_{i in d} [x_i * (Qd/q_i)^{-1}]_{q_i} * (Qd/q_i mod t)  mod t,
 * and the digit's own primes are copied.  Output [ndig][level+1+K][N].
 */
void or_modup(const or_params *p, int level, const uint64_t *c1, uint64_t *D) {
    int n = p->n, al = alpha_of(p), nd = ndigits_at(p, level), nl = level + 1, ext = nl + p->K;
    for (int d = 0; d < nd; ++d) {
        int lo = d * al, hi = (d + 1) * al < nl ? (d + 1) * al : nl;
        for (int u = 0; u < ext; ++u) {
            uint64_t t = qp_prime(p, level, u);
            uint64_t *out = D + ((size_t)d * ext + u) * n;
            if (u >= lo && u < hi) { memcpy(out, c1 + (size_t)u * n, sizeof(uint64_t) * n); continue; }
            for (int k = 0; k < n; ++k) out[k] = 0;
            for (int i = lo; i < hi; ++i) {
                uint64_t qi = p->primes[i];
                uint64_t hat_qi = 1, hat_t = 1 % t; /* Qd/q_i mod q_i and mod t */
                for (int j = lo; j < hi; ++j)
                    if (j != i) { hat_qi = mulmod(hat_qi, p->primes[j] % qi, qi); hat_t = mulmod(hat_t, p->primes[j] % t, t); }
                uint64_t inv = or_invmod(hat_qi, qi);
                for (int k = 0; k < n; ++k) {
                    uint64_t v = mulmod(c1[(size_t)i * n + k], inv, qi);
                    out[k] = addmod(out[k], mulmod(v % t, hat_t, t), t);
                }
            }
        }
    }
}

/*
 * ModDown (Q_level U P -> Q_level), divide by P with the exact fast base conversion of the P part:
 *   out_j = (x_j - sum_i [x_{p_i} (P/p_i)^{-1}]_{p_i} (P/p_i mod q_j)) * P^{-1}  mod q_j.
 */
void or_moddown(const or_params *p, int level, const uint64_t *x, uint64_t *out) {
    int n = p->n, nl = level + 1, K = p->K, L = p->L;
    for (int j = 0; j < nl; ++j) {
        uint64_t q = p->primes[j];
        uint64_t pinv = 1 % q;
        for (int i = 0; i < K; ++i) pinv = mulmod(pinv, p->primes[L + i] % q, q);
        pinv = or_invmod(pinv, q);
        for (int k = 0; k < n; ++k) out[(size_t)j * n + k] = x[(size_t)j * n + k];
        for (int i = 0; i < K; ++i) {
            uint64_t pi = p->primes[L + i];
            uint64_t hat_pi = 1, hat_q = 1 % q;
            for (int r = 0; r < K; ++r)
                if (r != i) { hat_pi = mulmod(hat_pi, p->primes[L + r] % pi, pi); hat_q = mulmod(hat_q, p->primes[L + r] % q, q); }
            uint64_t inv = or_invmod(hat_pi, pi);
            const uint64_t *xp = x + (size_t)(nl + i) * n;
            for (int k = 0; k < n; ++k) {
                uint64_t v = mulmod(xp[k], inv, pi);
                out[(size_t)j * n + k] = submod(out[(size_t)j * n + k], mulmod(v % q, hat_q, q), q);
            }
        }
        for (int k = 0; k < n; ++k) out[(size_t)j * n + k] = mulmod(out[(size_t)j * n + k], pinv, q);
    }
}

/* sum_d phi_g(D_d) * evk_d over Q_level U P, both key components (the key-switch inner product) */
static void ks_inner(const or_params *p, int level, const uint64_t *D, uint64_t g, const uint64_t *evk, uint64_t *u0, uint64_t *u1) {
    int n = p->n, nd = ndigits_at(p, level), ext = level + 1 + p->K, LK = p->L + p->K;
    uint64_t *dg = malloc(sizeof(uint64_t) * n), *tmp = malloc(sizeof(uint64_t) * n);
    memset(u0, 0, sizeof(uint64_t) * (size_t)ext * n);
    memset(u1, 0, sizeof(uint64_t) * (size_t)ext * n);
    for (int d = 0; d < nd; ++d)
        for (int u = 0; u < ext; ++u) {
            uint64_t t = qp_prime(p, level, u);
            int kl = key_limb(p, level, u);
            or_automorph(n, t, g, D + ((size_t)d * ext + u) * n, dg);
            mul_into(n, t, dg, evk + ((size_t)(d * 2 + 0) * LK + kl) * n, u0 + (size_t)u * n, tmp);
            mul_into(n, t, dg, evk + ((size_t)(d * 2 + 1) * LK + kl) * n, u1 + (size_t)u * n, tmp);
        }
    free(dg); free(tmp);
}

/*
 * O4 (HstRot, Sec. 2.2): rotations of one ciphertext that share one decomposition.
 * D = ModUp(c1) once; for each Galois element g:
 *   (phi_g(c0) + ModDown(sum_d phi_g(D_d) b_{g,d}),  ModDown(sum_d phi_g(D_d) a_{g,d})).
 * A single rotation is this with one element.  evks: [n_steps][dnum][2][L+K][N]; outs [n_steps][2][level+1][N].
 */
void or_rotate_hoisted(const or_params *p, int level, const uint64_t *ct, int n_steps, const uint64_t *galois, const uint64_t *evks, uint64_t *outs) {
    int n = p->n, nl = level + 1, ext = nl + p->K, nd = ndigits_at(p, level);
    size_t key_words = (size_t)p->dnum * 2 * (p->L + p->K) * n;
    uint64_t *D = malloc(sizeof(uint64_t) * (size_t)nd * ext * n);
    uint64_t *u0 = malloc(sizeof(uint64_t) * (size_t)ext * n), *u1 = malloc(sizeof(uint64_t) * (size_t)ext * n);
    uint64_t *v = malloc(sizeof(uint64_t) * (size_t)nl * n), *tmp = malloc(sizeof(uint64_t) * n);
    or_modup(p, level, ct + (size_t)nl * n, D);
    for (int s = 0; s < n_steps; ++s) {
        uint64_t g = galois[s];
        uint64_t *out = outs + (size_t)s * 2 * nl * n;
        ks_inner(p, level, D, g, evks + (size_t)s * key_words, u0, u1);
        or_moddown(p, level, u0, v);
        for (int l = 0; l < nl; ++l) {
            uint64_t q = p->primes[l];
            or_automorph(n, q, g, ct + (size_t)l * n, tmp);
            for (int k = 0; k < n; ++k) out[(size_t)l * n + k] = addmod(tmp[k], v[(size_t)l * n + k], q);
        }
        or_moddown(p, level, u1, out + (size_t)nl * n);
    }
    free(D); free(u0); free(u1); free(v); free(tmp);
}

/*
 * The diagonal MatMult sum_i pt_i (x) HstRotL(ct, i) (Eq. 2/3, Tab. 2), with the rotation
 * outputs kept in the extended basis Q U P and divided by P once at the end ("double hoisting").
 * pts_qp: [n_pt][level+1+K][N] plaintexts over Q_level U P; pt_i's Q limbs serve the c0 terms.
 * Rotation i (1 <= i < n_pt) uses galois[i-1] and key evks[i-1].  out: [2][level+1][N].
 */
void or_matmult_double(const or_params *p, int level, const uint64_t *ct, int n_pt, const uint64_t *pts_qp, const uint64_t *galois, const uint64_t *evks, uint64_t *out) {
    int n = p->n, nl = level + 1, ext = nl + p->K, nd = ndigits_at(p, level);
    size_t key_words = (size_t)p->dnum * 2 * (p->L + p->K) * n;
    uint64_t *D = malloc(sizeof(uint64_t) * (size_t)nd * ext * n);
    uint64_t *acc0 = calloc((size_t)ext * n, sizeof(uint64_t)), *acc1 = calloc((size_t)ext * n, sizeof(uint64_t));
    uint64_t *v = malloc(sizeof(uint64_t) * (size_t)nl * n), *tmp = malloc(sizeof(uint64_t) * n);
    const uint64_t *c0 = ct, *c1 = ct + (size_t)nl * n;
    uint64_t *o0 = out, *o1 = out + (size_t)nl * n;
    memset(out, 0, sizeof(uint64_t) * 2 * (size_t)nl * n);
    /* i = 0: no rotation */
    for (int l = 0; l < nl; ++l) {
        uint64_t q = p->primes[l];
        mul_into(n, q, c0 + (size_t)l * n, pts_qp + (size_t)l * n, o0 + (size_t)l * n, tmp);
        mul_into(n, q, c1 + (size_t)l * n, pts_qp + (size_t)l * n, o1 + (size_t)l * n, tmp);
    }
    if (n_pt > 1) or_modup(p, level, c1, D);
    /* i >= 1: each thread sums its diagonals into its own accumulators, which are then added
     * (modular sums: the result does not depend on the split) */
#pragma omp parallel
    {
        uint64_t *u0 = malloc(sizeof(uint64_t) * (size_t)ext * n), *u1 = malloc(sizeof(uint64_t) * (size_t)ext * n);
        uint64_t *a0 = calloc((size_t)ext * n, sizeof(uint64_t)), *a1 = calloc((size_t)ext * n, sizeof(uint64_t));
        uint64_t *b0 = calloc((size_t)nl * n, sizeof(uint64_t));
        uint64_t *t = malloc(sizeof(uint64_t) * n), *rc = malloc(sizeof(uint64_t) * n);
#pragma omp for schedule(dynamic, 1)
        for (int i = 1; i < n_pt; ++i) {
            uint64_t g = galois[i - 1];
            const uint64_t *pt = pts_qp + (size_t)i * ext * n;
            ks_inner(p, level, D, g, evks + (size_t)(i - 1) * key_words, u0, u1);
            for (int u = 0; u < ext; ++u) {
                uint64_t tq = qp_prime(p, level, u);
                mul_into(n, tq, u0 + (size_t)u * n, pt + (size_t)u * n, a0 + (size_t)u * n, t);
                mul_into(n, tq, u1 + (size_t)u * n, pt + (size_t)u * n, a1 + (size_t)u * n, t);
            }
            for (int l = 0; l < nl; ++l) {
                uint64_t q = p->primes[l];
                or_automorph(n, q, g, c0 + (size_t)l * n, rc);
                mul_into(n, q, rc, pt + (size_t)l * n, b0 + (size_t)l * n, t);
            }
        }
#pragma omp critical
        {
            for (size_t w = 0; w < (size_t)ext * n; ++w) {
                uint64_t tq = qp_prime(p, level, (int)(w / n));
                acc0[w] = addmod(acc0[w], a0[w], tq);
                acc1[w] = addmod(acc1[w], a1[w], tq);
            }
            for (size_t w = 0; w < (size_t)nl * n; ++w) o0[w] = addmod(o0[w], b0[w], p->primes[w / n]);
        }
        free(u0); free(u1); free(a0); free(a1); free(b0); free(t); free(rc);
    }
    if (n_pt > 1) {
        or_moddown(p, level, acc0, v);
        for (size_t w = 0; w < (size_t)nl * n; ++w) o0[w] = addmod(o0[w], v[w], p->primes[w / n]);
        or_moddown(p, level, acc1, v);
        for (size_t w = 0; w < (size_t)nl * n; ++w) o1[w] = addmod(o1[w], v[w], p->primes[w / n]);
    }
    free(D); free(acc0); free(acc1); free(v); free(tmp);
}

/*
 * Rescale by the last prime q_l (level l -> l-1): with h = floor(q_l/2), r = [c_l + h]_{q_l},
 * c'_j = (c_j - (r - h)) * q_l^{-1} mod q_j, i.e. c/q_l rounded to nearest, per component.
 */
void or_rescale(const or_params *p, int level, const uint64_t *ct, uint64_t *out) {
    int n = p->n, nl = level + 1, no = level;
    uint64_t ql = p->primes[level], h = ql / 2;
    for (int c = 0; c < 2; ++c) {
        const uint64_t *last = ct + ((size_t)c * nl + level) * n;
        for (int j = 0; j < no; ++j) {
            uint64_t q = p->primes[j], inv = or_invmod(ql % q, q);
            const uint64_t *cj = ct + ((size_t)c * nl + j) * n;
            uint64_t *oj = out + ((size_t)c * no + j) * n;
            for (int k = 0; k < n; ++k) {
                uint64_t r = (last[k] + h) % ql;
                int64_t centred = (int64_t)r - (int64_t)h;
                oj[k] = mulmod(submod(cj[k], from_signed(centred, q), q), inv, q);
            }
        }
    }
}
