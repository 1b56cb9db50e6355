// he_encode.cu -- CKKS encoding/decoding (double-float FFT), Philox-4x64-10 sampling, encryption.
//
// Encoding (Sec. 2.2): the real polynomial m with m(zeta^(5^j)) = z_j, zeta = exp(i pi/N).
// Since 5^j = 1 mod 4, the N/2 slot roots are zeta^(4t+1), and with c_k = m_k + i m_{k+N/2}
//   z at t  =  sum_{k<N/2} (c_k zeta^k) w^(t k),  w = exp(2 pi i / (N/2)),
// so encoding is an inverse length-N/2 DFT followed by a twist by zeta^-k, and decoding the
// forward one.  Slot j sits at t_j = (5^j mod 2N - 1) / 4.
#include <climits>

#include "he_internal.cuh"
#include "he_ntt.cuh"

namespace {

// ---- double-float arithmetic ----
// GB300's FP64 pipe issues a small fraction of its FP32 rate, so the FFTs run on pairs of
// floats (value = hi + lo, ~48-bit significand) built from error-free transforms: Knuth's
// two-sum for additions and an FMA-based two-product for multiplications.
struct df {
    float hi, lo;
};
__device__ __forceinline__ df quick_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ df df_add(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    const df t = two_sum(a.lo, b.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = quick_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df df_mul(df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return quick_two_sum(p, e);
}
// hi = x rounded to float, lo = the remainder x - hi rounded to float.  GB300's FP64 pipe is
// about 1.7 lanes per clock per SM with a 64-cycle dependent latency, so for 2^-60 <= |x| < 2^101
// both come from the significand with integer operations: hi is its top 24 bits rounded to
// nearest (ties to even; a carry out raises the exponent), and the remainder, at most 2^28 units
// of x's last place, is rounded by the int -> float conversion and scaled by that place's value
// (a normal float in this range).  Bit-identical to the two FP64 conversions, which serve the rest.
__device__ __forceinline__ df df_from(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7FF);
    if (E >= 1023 - 60 && E <= 1023 + 100) {
        const unsigned long long M = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
        unsigned long long Mh = M >> 29;
        const unsigned long long r = M & ((1ull << 29) - 1);
        Mh += (r > (1ull << 28)) || (r == (1ull << 28) && (Mh & 1));
        const int rem = (int)((long long)M - (long long)(Mh << 29));
        const unsigned sgn = (unsigned)(b >> 63) << 31;
        const float hi = __uint_as_float(sgn | ((unsigned)(E - 896 + (int)(Mh >> 24)) << 23) | (unsigned)(Mh & 0x7FFFFF));
        const float lo = __fmul_rn(__int2float_rn(sgn ? -rem : rem), __uint_as_float((unsigned)(E - 1075 + 127) << 23));
        return {hi, lo};
    }
    const float h = __double2float_rn(x);
    return {h, __double2float_rn(x - (double)h)};
}
// u as a double, rounded to nearest (ties to even), with integer operations only: the leading
// bit's position is the exponent, the 53 bits from it the significand
__device__ __forceinline__ double u64_to_double_rn(unsigned long long u, bool negative) {
    if (!u) return 0.0;
    int e = 63 - __clzll((long long)u);
    unsigned long long mant;
    if (e <= 52) {
        mant = u << (52 - e);
    } else {
        const int sh = e - 52;
        mant = u >> sh;
        const unsigned long long rem = u & ((1ull << sh) - 1), half = 1ull << (sh - 1);
        mant += (rem > half) || (rem == half && (mant & 1));
        if (mant >> 53) {
            mant >>= 1;
            ++e;
        }
    }
    return __longlong_as_double((long long)(((unsigned long long)negative << 63) | ((unsigned long long)(e + 1023) << 52) | (mant & 0xFFFFFFFFFFFFFull)));
}
// a float as a double, exactly: for normal floats the exponent re-biased and the significand
// widened with integer operations (no FP64-pipe conversion); zero, subnormals, inf and NaN by the cast
__device__ __forceinline__ double f2d_exact(float f) {
    const unsigned b = __float_as_uint(f), e = (b >> 23) & 0xFFu;
    if (e == 0u || e == 0xFFu) return (double)f;
    return __longlong_as_double((long long)(((unsigned long long)(b >> 31) << 63) | ((unsigned long long)(e + 896u) << 52) |
                                            ((unsigned long long)(b & 0x7FFFFFu) << 29)));
}
__device__ __forceinline__ double df_to(df a) { return f2d_exact(a.hi) + f2d_exact(a.lo); }

// Rounding to an integer without the FP64 pipe (on GB300 a small fraction of the FP32 rate, and
// the encoders round every coefficient).  rint_f: nearest integer, ties to even (below 2^23 by
// adding and removing 2^23, which leaves units in the last place; above it x is an integer).
__device__ __forceinline__ float rint_f(float x) {
    const float m = copysignf(8388608.0f, x);
    return fabsf(x) < 8388608.0f ? __fsub_rn(__fadd_rn(x, m), m) : x;
}
// an integral float as int64, from its exponent and significand (saturating beyond 2^63)
__device__ __forceinline__ long long f2ll_integral(float f) {
    const unsigned b = __float_as_uint(f);
    const int e = (int)((b >> 23) & 0xFFu) - 150;  // |f| = significand * 2^e
    if (e > 39) return (int)b < 0 ? LLONG_MIN : LLONG_MAX;
    const long long m = (long long)((b & 0x7FFFFFu) | 0x800000u);
    const long long v = e >= 0 ? m << e : (e > -24 ? m >> -e : 0);  // e < 0: the low bits are zero
    return (int)b < 0 ? -v : v;
}
// nearest integer to the double-float value hi + lo: rint(hi) plus the rounded remainder
// (hi - rint(hi), exact, plus lo).  Above 2^24 hi is even and the remainder is lo itself, so ties go
// to even as in exact rounding; below, the float remainder can pick the other neighbour within
// 2^-24 of a half-integer, far inside the transform's own error (relative ~2^-44).
__device__ __forceinline__ long long df_round_ll(df a) {
    const float rh = rint_f(a.hi);
    return f2ll_integral(rh) + f2ll_integral(rint_f(__fadd_rn(__fsub_rn(a.hi, rh), a.lo)));
}

// complex value in shared memory: (re.hi, re.lo, im.hi, im.lo)
// a c + b d in double-float: the two leading products exact as FMA two-products, their sum by
// two-sum, then the products' errors and the four cross terms accumulated in float and added to
// the low part before one renormalisation (19 operations against 34 for two df_mul and a df_add;
// the same ~2^-46 relative accuracy)
__device__ __forceinline__ df df_dot2(df a, df c, df b, df d) {
    const float p1 = __fmul_rn(a.hi, c.hi), e1 = __fmaf_rn(a.hi, c.hi, -p1);
    const float p2 = __fmul_rn(b.hi, d.hi), e2 = __fmaf_rn(b.hi, d.hi, -p2);
    const df s = two_sum(p1, p2);
    float t = __fadd_rn(e1, e2);
    t = __fmaf_rn(a.hi, c.lo, t);
    t = __fmaf_rn(a.lo, c.hi, t);
    t = __fmaf_rn(b.hi, d.lo, t);
    t = __fmaf_rn(b.lo, d.hi, t);
    return quick_two_sum(s.hi, __fadd_rn(s.lo, t));
}
__device__ __forceinline__ void cmul(float4 v, float4 w, float4 &out) {
    const df vr{v.x, v.y}, vi{v.z, v.w}, wr{w.x, w.y}, wi{w.z, w.w};
    const df re = df_dot2(vr, wr, df_neg(vi), wi);
    const df im = df_dot2(vr, wi, vi, wr);
    out = make_float4(re.hi, re.lo, im.hi, im.lo);
}

// one radix-2 butterfly (u, v) <- (u + v w, u - v w) in double-float
__device__ __forceinline__ void fft_bfly(float4 &u4, float4 &v4, float4 w) {
    float4 v;
    cmul(v4, w, v);
    const float4 u = u4;
    const df ur{u.x, u.y}, ui{u.z, u.w}, vr{v.x, v.y}, vi{v.z, v.w};
    const df s0r = df_add(ur, vr), s0i = df_add(ui, vi), d0r = df_add(ur, df_neg(vr)), d0i = df_add(ui, df_neg(vi));
    u4 = make_float4(s0r.hi, s0r.lo, s0i.hi, s0i.lo);
    v4 = make_float4(d0r.hi, d0r.lo, d0i.hi, d0i.lo);
}

__device__ __forceinline__ float4 shfl4_xor(float4 v) {
    return make_float4(__shfl_xor_sync(0xffffffffu, v.x, 1), __shfl_xor_sync(0xffffffffu, v.y, 1), __shfl_xor_sync(0xffffffffu, v.z, 1),
                       __shfl_xor_sync(0xffffffffu, v.w, 1));
}
__device__ __forceinline__ float4 shfl4(float4 v, int src) {
    return make_float4(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src), __shfl_sync(0xffffffffu, v.z, src),
                       __shfl_sync(0xffffffffu, v.w, src));
}

// Radix-2 decimation-in-time FFT of M = N/2 complex values in shared memory, input in
// bit-reversed order: stage lg (1..log M) combines a[i1], a[i2 = i1 + 2^(lg-1)] with
// w = tw[(i1 mod 2^(lg-1)) * M / 2^lg], tw[k] = exp(-2 pi i k / M) (its conjugate for
// sign = +1), as (u + v w, u - v w).  The stages are grouped into passes of up to three: a
// thread loads the 8 elements that interact over a pass into registers, runs those butterflies
// there (the same operations on the same values as one stage at a time, so the result does not
// depend on the grouping) and writes them back, so a 4096-point transform makes 4 trips through
// shared memory and block barriers instead of 12, with 4 independent butterflies per stage.
// Twiddle of a butterfly at stage lg whose element sits at pos = x mod 2^(lg-1): tw[pos 2^(log M - lg)].
// TwFftGlobal reads the table; TwFftLocal a shared-memory copy of the entries the slice-local
// stages of the cluster form read, stw[j] = tw[j 2^(log M - lg_ms)] for j < 2^(lg_ms - 1).
struct TwFftGlobal {
    const float4 *tw;
    int logm;
    __device__ __forceinline__ float4 at(int pos, int lg) const { return tw[pos << (logm - lg)]; }
};
struct TwFftLocal {
    const float4 *stw;
    int lg_ms;
    __device__ __forceinline__ float4 at(int pos, int lg) const { return stw[pos << (lg_ms - lg)]; }
};

template <int NB, class TWA = TwFftGlobal>
__device__ __forceinline__ void fft_pass(float4 *a, TWA tw, int logm, int s0, int sign, int set0 = 0, int set1 = -1, int off = 0) {
    constexpr int E = 1 << NB;
    if (set1 < 0) set1 = 1 << (logm - NB);
    a -= off;  // element x at a[x] (a slice holds [off, off + its length))
    for (int set = set0 + threadIdx.x; set < set1; set += blockDim.x) {
        const int g = set >> s0, low = set & ((1 << s0) - 1);
        const int base = (g << (s0 + NB)) + low;
        float4 r[E];
#pragma unroll
        for (int k = 0; k < E; ++k) r[k] = a[base + (k << s0)];
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            const int h = 1 << j, lg = s0 + j + 1;
#pragma unroll
            for (int k = 0; k < E; ++k) {
                if ((k & (2 * h - 1)) < h) {
                    const int pos = (base + (k << s0)) & ((1 << (lg - 1)) - 1);
                    float4 w = tw.at(pos, lg);
                    if (sign > 0) w = make_float4(w.x, w.y, -w.z, -w.w);
                    fft_bfly(r[k], r[k + h], w);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < E; ++k) a[base + (k << s0)] = r[k];
    }
    __syncthreads();
}

// Stages s0 and s0 + 1 over sets [set0, set1) of four elements base + k 2^s0 (k < 4), two lanes
// per set: at stage s0 lane p holds k = 2p, 2p + 1 (one butterfly, twiddle position low); then
// the lanes swap one element by shuffle (lane 0 gives k = 1 for k = 2) and lane p holds k = p,
// p + 2 for stage s0 + 1 (twiddle position low + p 2^s0).  The same butterflies as two radix-2
// passes, one trip through shared memory and one barrier instead of two.  2 (set1 - set0) is a
// multiple of blockDim.x, so whole warps run each iteration.
template <class TWA>
__device__ __forceinline__ void fft_pass_pair(float4 *a, TWA tw, int s0, int sign, int set0, int set1, int off) {
    a -= off;
    const int p = threadIdx.x & 1, d = 1 << s0;
    for (int t = 2 * set0 + (int)threadIdx.x; t < 2 * set1; t += blockDim.x) {
        const int set = t >> 1, g = set >> s0, low = set & (d - 1);
        const int base = (g << (s0 + 2)) + low;
        float4 x0 = a[base + 2 * p * d], x1 = a[base + (2 * p + 1) * d];
        float4 w = tw.at(low, s0 + 1);
        if (sign > 0) w = make_float4(w.x, w.y, -w.z, -w.w);
        fft_bfly(x0, x1, w);
        const float4 got = shfl4_xor(p ? x0 : x1);
        float4 y0 = p ? got : x0, y1 = p ? x1 : got;
        w = tw.at(low + p * d, s0 + 2);
        if (sign > 0) w = make_float4(w.x, w.y, -w.z, -w.w);
        fft_bfly(y0, y1, w);
        a[base + p * d] = y0;
        a[base + (p + 2) * d] = y1;
    }
    __syncthreads();
}

__device__ void fft_smem(float4 *a, const float4 *__restrict__ tw, int logm, int sign) {
    int s0 = 0;
    while (s0 < logm) {
        const int nb = logm - s0 < 3 ? logm - s0 : 3;
        switch (nb) {
            case 3: fft_pass<3>(a, TwFftGlobal{tw, logm}, logm, s0, sign); break;
            case 2: fft_pass<2>(a, TwFftGlobal{tw, logm}, logm, s0, sign); break;
            default: fft_pass<1>(a, TwFftGlobal{tw, logm}, logm, s0, sign); break;
        }
        s0 += nb;
    }
}

// one CTA per plaintext: slots [count][stride] (first n_slots used) -> coeffs int64 [count][N]
__global__ void encode_kernel(const double *__restrict__ slots, int64_t n_slots, int64_t stride, double scale,
                              const float4 *__restrict__ tw, const float4 *__restrict__ twist, const int32_t *__restrict__ slot_pos,
                              int64_t *out, int logn) {
    HE_GRID_DEP();
    extern __shared__ float4 a[];
    const int logm = logn - 1, M = 1 << logm, N = 1 << logn;
    const double *z = slots + (int64_t)blockIdx.x * stride;
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
        const int t = slot_pos[j];
        const int bt = __brev(t) >> (32 - logm);
        const df v = df_from(j < n_slots ? z[j] : 0.0);
        a[bt] = make_float4(v.hi, v.lo, 0.f, 0.f);
    }
    __syncthreads();
    fft_smem(a, tw, logm, -1);
    const df f = df_from(2.0 / (double)N * scale);  // exact: a power of two times the scale
    int64_t *o = out + (int64_t)blockIdx.x * N;
    for (int k = threadIdx.x; k < M; k += blockDim.x) {
        float4 c;
        cmul(a[k], twist[k], c);  // times zeta^-k
        o[k] = df_round_ll(df_mul(df{c.x, c.y}, f));
        o[k + M] = df_round_ll(df_mul(df{c.z, c.w}, f));
    }
}

// one CTA per polynomial: real coefficients [count][N] -> slot values [count][N/2] / scale
__global__ void decode_kernel(const double *__restrict__ coeffs, double scale, const float4 *__restrict__ tw,
                              const float4 *__restrict__ twist, const int32_t *__restrict__ slot_pos, double *out, int logn) {
    HE_GRID_DEP();
    extern __shared__ float4 a[];
    const int logm = logn - 1, M = 1 << logm, N = 1 << logn;
    const double *m = coeffs + (int64_t)blockIdx.x * N;
    for (int k = threadIdx.x; k < M; k += blockDim.x) {
        const float4 w = twist[k];  // zeta^-k; use its conjugate zeta^k
        const df re = df_from(m[k]), im = df_from(m[k + M]);
        float4 c;
        cmul(make_float4(re.hi, re.lo, im.hi, im.lo), make_float4(w.x, w.y, -w.z, -w.w), c);
        a[__brev(k) >> (32 - logm)] = c;
    }
    __syncthreads();
    fft_smem(a, tw, logm, +1);
    double *o = out + (int64_t)blockIdx.x * M;
    const double inv = 1.0 / scale;
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
        const float4 v = a[slot_pos[j]];
        o[j] = df_to(df{v.x, v.y}) * inv;
    }
}

// ---- cluster form: CL = 2^CLG CTAs (one thread-block cluster) share one transform ----
// CTA `rank` holds positions [rank MS, (rank+1) MS) of the array (MS = M / CL).  The first
// log M - CLG stages pair elements of one slice and run as register passes on it; the last CLG
// stages pair the CL elements j + c MS (c < CL), which lie in different CTAs, and run as one
// radix-CL step through distributed shared memory, each CTA taking MS / CL of the offsets j.
// The butterflies and their order per element are those of fft_smem, so the output is
// bit-identical to the one-CTA form.  Used when a launch has few transforms, which would leave
// most SMs idle with one CTA each.
// local passes of the cluster form: radix 2, one butterfly per thread per stage (MS/2 threads, at
// most 512), since a cluster transform is latency-bound and on GB300 the most warps with the
// shortest chains finished it soonest (radix 8 > radix 4 > radix 2 in time)
// RL: local passes of radix 2^RL (MS >> RL threads).  RL = 1 throughout: on GB300 radix 4 and 8
// (and 2 CTAs per transform with radix 8, or one CTA) were slower even for the 64 transforms of
// an encoded matrix, where the launch is throughput- rather than latency-bound
// The slice-local stages read their twiddles from a shared-memory copy placed right after the
// slice (a + MS), which the kernel starts with fft_tw_issue before it loads its data; the copy is
// the same for every CTA (those stages' twiddles do not depend on the slice).
template <int CLG>
__device__ __forceinline__ void fft_tw_issue(float4 *a, const float4 *__restrict__ tw, int logm) {
    const int MS = 1 << (logm - CLG);
    float4 *stw = a + MS;
    for (int j = threadIdx.x; j < MS / 2; j += blockDim.x) {
        const unsigned sa = (unsigned)__cvta_generic_to_shared(stw + j);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(tw + (j << CLG)) : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// LOGM > 0: log M at compile time (logm == LOGM), so the pass loop unrolls and indices fold
template <int CLG, int RL, int LOGM = 0>
__device__ __forceinline__ void fft_cluster(float4 *a, const float4 *__restrict__ tw, int logm, int sign) {
    constexpr int CL = 1 << CLG;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int lg_ms = logm - CLG, MS = 1 << lg_ms, off = rank * MS;
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");  // the twiddle copy of fft_tw_issue
    __syncthreads();
    const TwFftLocal tloc{a + MS, lg_ms};
    if constexpr (RL == 1) {
        // radix-2 stages two at a time, lane pairs swapping one element by shuffle in between
#pragma unroll(LOGM > 0 ? 16 : 1)
        for (int s0 = 0; s0 + 1 < (LOGM > 0 ? LOGM - CLG : 16); s0 += 2) {
            if (s0 + 1 >= lg_ms) break;
            fft_pass_pair(a, tloc, s0, sign, rank * (MS / 4), (rank + 1) * (MS / 4), off);
        }
        if (lg_ms & 1) fft_pass<1>(a, tloc, logm, lg_ms - 1, sign, rank * (MS / 2), (rank + 1) * (MS / 2), off);
    } else {
#pragma unroll(LOGM > 0 ? 16 : 1)
        for (int s0 = 0; s0 < (LOGM > 0 ? LOGM - CLG : 16); s0 += RL) {
            if (s0 >= lg_ms) break;
            const int nb = lg_ms - s0 < RL ? lg_ms - s0 : RL;
            const int E = 1 << nb;
            switch (nb) {
                case 3: fft_pass<3>(a, tloc, logm, s0, sign, rank * (MS / E), (rank + 1) * (MS / E), off); break;
                case 2: fft_pass<2>(a, tloc, logm, s0, sign, rank * (MS / E), (rank + 1) * (MS / E), off); break;
                default: fft_pass<1>(a, tloc, logm, s0, sign, rank * (MS / E), (rank + 1) * (MS / E), off); break;
            }
        }
    }
    // The cross-CTA stages: the CL elements j + c MS of an offset j go through CLG radix-2
    // stages, stage st pairing c and c + 2^st.  2^(CLG-1) adjacent lanes share an offset, each
    // holding the pair of one butterfly per stage: lane p holds c = ins(p, st) and c + 2^st (bit st
    // inserted into p), and between stages the lanes swap elements by warp shuffles, so every
    // thread of the CTA takes part (MS / 2 butterflies per stage).  The butterfly of c uses twiddle
    // position j + g MS with g = c mod 2^st = p mod 2^st; the thread's twiddles of its first offset
    // are loaded before the cluster barrier, their latency overlapping the wait.
    constexpr int T = CL > 1 ? CL / 2 : 1;
    const int per = MS >> CLG, p = threadIdx.x & (T - 1), lane_base = (threadIdx.x & 31) & ~(T - 1);
    auto ins = [](int v, int st) { return (v & ((1 << st) - 1)) | ((v >> st) << (st + 1)); };
    float4 wc[CLG > 0 ? CLG : 1];
    auto cross_tw = [&](int j) {
#pragma unroll
        for (int st = 0; st < CLG; ++st) wc[st] = tw[(j + ((p & ((1 << st) - 1)) << lg_ms)) << (logm - lg_ms - st - 1)];
    };
    // MS / 2 is a multiple of 32 and of blockDim.x (MS >= 64 for the rings that use clusters), so
    // whole warps run each iteration and the shuffles see every lane
    if ((int)threadIdx.x < per * T) cross_tw(rank * per + (int)(threadIdx.x / T));
    cl.sync();
    for (int t = threadIdx.x; t < per * T; t += blockDim.x) {
        const int j = rank * per + t / T;
        if (t != (int)threadIdx.x) cross_tw(j);
        int c_lo = ins(p, 0);
        float4 x0 = cl.map_shared_rank(a, c_lo)[j], x1 = cl.map_shared_rank(a, c_lo | 1)[j];
#pragma unroll
        for (int st = 0; st < CLG; ++st) {
            if (st > 0) {
                // this lane's new pair from the lanes holding them at stage st - 1 (element c sits
                // at lane c with bit st - 1 removed, in slot bit st - 1 of c)
                const int lo = ins(p, st), hi = lo | (1 << st);
                const int src_lo = lane_base + ((lo & ((1 << (st - 1)) - 1)) | ((lo >> st) << (st - 1)));
                const int src_hi = lane_base + ((hi & ((1 << (st - 1)) - 1)) | ((hi >> st) << (st - 1)));
                const float4 a0 = shfl4(x0, src_lo), a1 = shfl4(x1, src_lo), b0 = shfl4(x0, src_hi), b1 = shfl4(x1, src_hi);
                x0 = (lo >> (st - 1)) & 1 ? a1 : a0;
                x1 = (hi >> (st - 1)) & 1 ? b1 : b0;
                c_lo = lo;
            }
            float4 w = wc[st];
            if (sign > 0) w = make_float4(w.x, w.y, -w.z, -w.w);
            fft_bfly(x0, x1, w);
        }
        cl.map_shared_rank(a, c_lo)[j] = x0;
        cl.map_shared_rank(a, c_lo | (1 << (CLG > 0 ? CLG - 1 : 0)))[j] = x1;
    }
    cl.sync();
}

// Slot value j of plaintext `item`: from a slot array ([count][stride], first n_slots used), or
// straight from a cleartext matrix in the diagonal layout of Eq. 2 after Eq. 3 (item = (r C + c) m'
// + i, the order of an encoded matrix; the values layout_matrix_kernel writes), or from a vector
// replicated per Eq. 3 (item = column block c; the values layout_vector_kernel writes).
struct SlotsSrc {
    const double *z;
    int64_t n_slots, stride;
    __device__ __forceinline__ double operator()(int item, int j) const { return j < n_slots ? z[(int64_t)item * stride + j] : 0.0; }
};
struct MatrixSrc {
    he_plan p;
    const double *X;  // m x n row-major, or its n x m transpose when trans
    int trans, lm, lc, lnb, lmb;  // log2 of m', column blocks, nb, mb
    __device__ __forceinline__ double operator()(int item, int j0) const {
        const int64_t i = item & (p.m_prime - 1), rest = item >> lm;
        const int64_t c = rest & (p.col_blocks - 1), r = rest >> lc;
        // BSGS schedule: diagonal i = g B + b pre-rotated right by g B slots
        const int64_t j = p.baby ? (j0 - (i - (i & (p.baby - 1)))) & (p.slots - 1) : j0;
        const int64_t b = j >> lnb, jj = j & (p.nb - 1);
        const int64_t row = (r << lmb) + (b << lm) + (jj & (p.m_prime - 1));
        const int64_t col = (c << lnb) + ((i + jj) & (p.nb - 1));
        return (row < p.m && col < p.n) ? X[trans ? col * p.m + row : row * p.n + col] : 0.0;
    }
};
struct VectorSrc {
    const double *y;
    int64_t n, nb;
    int lnb;  // log2 nb
    __device__ __forceinline__ double operator()(int item, int j) const {
        const int64_t col = ((int64_t)item << lnb) + (j & (nb - 1));
        return col < n ? y[col] : 0.0;
    }
};

// cluster per plaintext: the slot values go straight to their bit-reversed positions in the
// owning CTAs; each CTA then twists and rounds the coefficients of its slice
template <int CLG, int RL, int LOGN, class SRC>
__global__ void encode_cl_kernel(SRC src, double scale, const float4 *__restrict__ tw, const float4 *__restrict__ twist,
                                 const int32_t *__restrict__ slot_pos, int64_t *out, int logn_rt) {
    HE_GRID_LAUNCH();
    const int logn = LOGN ? LOGN : logn_rt;
    extern __shared__ float4 a[];
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank(), item = blockIdx.x >> CLG;
    const int logm = logn - 1, M = 1 << logm, N = 1 << logn, lg_ms = logm - CLG, MS = 1 << lg_ms, off = rank * MS;
    const int per = M >> CLG;
    // the context's tables before the wait: the twiddle copy and the first two slot positions
    fft_tw_issue<CLG>(a, tw, logm);
    int pos_pre[2];
    float4 tw_pre[2];  // the epilogue's twist factors
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        if ((int)threadIdx.x + r * (int)blockDim.x < per) pos_pre[r] = slot_pos[rank * per + threadIdx.x + r * blockDim.x];
        if ((int)threadIdx.x + r * (int)blockDim.x < MS) tw_pre[r] = twist[off + threadIdx.x + r * blockDim.x];
    }
    cl.sync();  // every CTA of the cluster has started before its shared memory is written (no data of an earlier launch)
    HE_GRID_WAIT();
    int r = 0;
    for (int j = rank * per + threadIdx.x; j < (rank + 1) * per; j += blockDim.x, ++r) {
        const int bt = __brev(r == 0 ? pos_pre[0] : (r == 1 ? pos_pre[1] : slot_pos[j])) >> (32 - logm);
        const df v = df_from(src(item, j));
        cl.map_shared_rank(a, bt >> lg_ms)[bt & (MS - 1)] = make_float4(v.hi, v.lo, 0.f, 0.f);
    }
    cl.sync();
    fft_cluster<CLG, RL, LOGN ? LOGN - 1 : 0>(a, tw, logm, -1);
    const df f = df_from(2.0 / (double)N * scale);
    int64_t *o = out + (int64_t)item * N;
    r = 0;
    for (int i = threadIdx.x; i < MS; i += blockDim.x, ++r) {
        const int k = off + i;
        float4 c;
        cmul(a[i], r == 0 ? tw_pre[0] : (r == 1 ? tw_pre[1] : twist[k]), c);
        o[k] = df_round_ll(df_mul(df{c.x, c.y}, f));
        o[k + M] = df_round_ll(df_mul(df{c.z, c.w}, f));
    }
}

// Two real inputs per transform: the slot vectors x (item 2p) and y (item 2p+1) go in as the real
// and imaginary parts of one sequence, so a cluster runs one length-M FFT for two plaintexts.
// The DFT is linear and maps a real sequence to a Hermitian one, so with Z = DFT(x + i y):
// DFT(x)[k] = (Z[k] + conj Z[-k]) / 2 and DFT(y)[k] = -i (Z[k] - conj Z[-k]) / 2 (indices mod M);
// each CTA reads Z[-k] of its slice from the CTA holding it.  Then the twist and rounding of
// encode_cl_kernel for each (the 1/2 folded into the power-of-two factor).  An odd last item
// pairs with zeros and writes one plaintext.
template <int CLG, int RL, int LOGN, class SRC>
__global__ void encode_pair_cl_kernel(SRC src, int count, double scale, const float4 *__restrict__ tw, const float4 *__restrict__ twist,
                                      const int32_t *__restrict__ slot_pos, int64_t *out, int logn_rt) {
    HE_GRID_LAUNCH();
    const int logn = LOGN ? LOGN : logn_rt;
    extern __shared__ float4 a[];
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank(), pair = blockIdx.x >> CLG;
    const int logm = logn - 1, M = 1 << logm, N = 1 << logn, lg_ms = logm - CLG, MS = 1 << lg_ms, off = rank * MS;
    const int ix = 2 * pair, iy = 2 * pair + 1;
    const bool has_y = iy < count;
    const int per = M >> CLG;
    fft_tw_issue<CLG>(a, tw, logm);  // the context's tables before the wait, as in encode_cl_kernel
    int pos_pre[2];
#pragma unroll
    for (int r = 0; r < 2; ++r)
        if ((int)threadIdx.x + r * (int)blockDim.x < per) pos_pre[r] = slot_pos[rank * per + threadIdx.x + r * blockDim.x];
    cl.sync();  // every CTA of the cluster has started before its shared memory is written (no data of an earlier launch)
    HE_GRID_WAIT();
    int r = 0;
    for (int j = rank * per + threadIdx.x; j < (rank + 1) * per; j += blockDim.x, ++r) {
        const int bt = __brev(r == 0 ? pos_pre[0] : (r == 1 ? pos_pre[1] : slot_pos[j])) >> (32 - logm);
        const df vx = df_from(src(ix, j)), vy = df_from(has_y ? src(iy, j) : 0.0);
        cl.map_shared_rank(a, bt >> lg_ms)[bt & (MS - 1)] = make_float4(vx.hi, vx.lo, vy.hi, vy.lo);
    }
    cl.sync();
    fft_cluster<CLG, RL, LOGN ? LOGN - 1 : 0>(a, tw, logm, -1);  // ends with a cluster barrier
    const df f = df_from(1.0 / (double)N * scale);  // 2/N times the 1/2 of the separation
    int64_t *ox = out + (int64_t)ix * N, *oy = out + (int64_t)iy * N;
    for (int i = threadIdx.x; i < MS; i += blockDim.x) {
        const int k = off + i, km = (M - k) & (M - 1);
        const float4 zk = a[i], zm = cl.map_shared_rank(a, km >> lg_ms)[km & (MS - 1)];
        const df zr{zk.x, zk.y}, zi{zk.z, zk.w}, mr{zm.x, zm.y}, mi{zm.z, zm.w};
        // 2 DFT(x)[k] = (zr + mr) + i (zi - mi);  2 DFT(y)[k] = (zi + mi) - i (zr - mr)
        const df xr = df_add(zr, mr), xi = df_add(zi, df_neg(mi));
        const df yr = df_add(zi, mi), yi = df_add(mr, df_neg(zr));
        float4 c;
        cmul(make_float4(xr.hi, xr.lo, xi.hi, xi.lo), twist[k], c);
        ox[k] = df_round_ll(df_mul(df{c.x, c.y}, f));
        ox[k + M] = df_round_ll(df_mul(df{c.z, c.w}, f));
        if (has_y) {
            cmul(make_float4(yr.hi, yr.lo, yi.hi, yi.lo), twist[k], c);
            oy[k] = df_round_ll(df_mul(df{c.x, c.y}, f));
            oy[k + M] = df_round_ll(df_mul(df{c.z, c.w}, f));
        }
    }
    cl.sync();  // the other CTAs read this one's shared memory until here
}

// cluster per polynomial: each CTA loads the coefficients whose bit-reversed positions it holds;
// the slot values are read from the owning CTAs
// What the decode writes once the slot values are in the cluster's shared memory.  DecodeSlots:
// slot j of plaintext `item` to out[item][j].  DecodeRas: the lazy rotate-and-sum of the rows of
// row block `item` (Sec. 4.3), y[row] = sum over s < nb/m' of slot[b nb + t + s m'] (minus the
// mask), each row by one thread in the order s = 0, 1, ... of lazy_ras_kernel, over the same
// slot values, so the same doubles without the slot array.
// Each epilogue's slot positions of its first two iterations are read by prefetch() before the
// kernel waits for its predecessor.
struct EpiPre {
    int pos[2];
};
struct DecodeSlots {
    double *out;
    __device__ __forceinline__ EpiPre prefetch(int, int rank, int clg, int M, int, const int32_t *__restrict__ slot_pos) const {
        EpiPre pre;
        const int per = M >> clg;
#pragma unroll
        for (int r = 0; r < 2; ++r)
            if ((int)threadIdx.x + r * (int)blockDim.x < per) pre.pos[r] = slot_pos[rank * per + threadIdx.x + r * blockDim.x];
        return pre;
    }
    __device__ __forceinline__ void operator()(cg::cluster_group &cl, const float4 *a, int item, int rank, int clg, int M, int lg_ms,
                                               const int32_t *__restrict__ slot_pos, double inv, double *, const EpiPre &pre) const {
        double *o = out + (int64_t)item * M;
        const int per = M >> clg, MS = 1 << lg_ms;
        int r = 0;
        for (int j = rank * per + threadIdx.x; j < (rank + 1) * per; j += blockDim.x, ++r) {
            const int pos = r == 0 ? pre.pos[0] : (r == 1 ? pre.pos[1] : slot_pos[j]);
            const float4 v = cl.map_shared_rank(a, pos >> lg_ms)[pos & (MS - 1)];
            o[j] = df_to(df{v.x, v.y}) * inv;
        }
        cl.barrier_arrive();  // done with the other CTAs' shared memory (the kernel waits at its end)
    }
};
struct DecodeRas {
    he_plan p;
    const double *mask;  // [row blocks][slots] or null
    double *y;
    int lm, lnb, ls, lmb;  // log2 of m', nb, slots, mb
    // Row rem of the block goes to CTA rem mod CL.  A CTA first forms every term of its rows, term
    // s of its i-th row (slot value, minus the mask) into vals[i terms + s], all threads taking
    // some so that the FP64 work (a pipe of about 1.7 lanes per clock per SM) is spread over the
    // CTA's warps and its load latencies overlap; then each row's terms are summed in the order
    // s = 0, 1, ... by one thread (rows spread over four warps, one per scheduler).  vals is the
    // CTA's twiddle copy, free after the transform: MS doubles, which the terms fit whenever the
    // block's rows hold each slot at most once; otherwise each thread forms and sums a row itself.
    // slot of term q (row i = q / terms, term s = q mod terms) of this CTA's rows
    __device__ __forceinline__ int64_t slot_of(int64_t q, int lt, int rank, int clg) const {
        const int64_t rem = ((q >> lt) << clg) + rank;
        return ((rem >> lm) << lnb) + (rem & (p.m_prime - 1)) + ((q & ((1ll << lt) - 1)) << lm);
    }
    __device__ __forceinline__ EpiPre prefetch(int, int rank, int clg, int, int lg_ms, const int32_t *__restrict__ slot_pos) const {
        EpiPre pre;
        const int64_t terms = p.nb >> lm, rows = rank < p.mb ? ((p.mb - 1 - rank) >> clg) + 1 : 0;
        const int lt = terms ? lnb - lm : 0;
        if (rows * terms <= (1 << lg_ms)) {
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int64_t q = threadIdx.x + (int64_t)r * blockDim.x;
                if (q < rows * terms) pre.pos[r] = slot_pos[slot_of(q, lt, rank, clg)];
            }
        }
        return pre;
    }
    __device__ __forceinline__ void operator()(cg::cluster_group &cl, const float4 *a, int item, int rank, int clg, int, int lg_ms,
                                               const int32_t *__restrict__ slot_pos, double inv, double *vals, const EpiPre &pre) const {
        const int MS = 1 << lg_ms;
        const int64_t terms = p.nb >> lm, row0 = (int64_t)item << lmb;
        const int lt = terms ? lnb - lm : 0;
        const int64_t rows = rank < p.mb ? ((p.mb - 1 - rank) >> clg) + 1 : 0;
        auto term_at = [&](int64_t j, int pos) {
            const float4 v = cl.map_shared_rank(a, pos >> lg_ms)[pos & (MS - 1)];
            const double val = df_to(df{v.x, v.y}) * inv;
            return mask ? val - mask[((int64_t)item << ls) + j] : val;
        };
        auto term = [&](int64_t rem, int64_t s) {
            const int64_t j = ((rem >> lm) << lnb) + (rem & (p.m_prime - 1)) + (s << lm);
            return term_at(j, slot_pos[j]);
        };
        if (rows * terms <= MS) {
            int r = 0;
#pragma unroll 2
            for (int64_t q = threadIdx.x; q < rows * terms; q += blockDim.x, ++r) {
                const int64_t rem = ((q >> lt) << clg) + rank, j = slot_of(q, lt, rank, clg);
                if (row0 + rem < p.m) vals[q] = term_at(j, r == 0 ? pre.pos[0] : (r == 1 ? pre.pos[1] : slot_pos[j]));
            }
            cl.barrier_arrive();  // done with the other CTAs' shared memory: the row sums overlap the barrier
            __syncthreads();
            const int nw = blockDim.x >= 128 ? 4 : (int)(blockDim.x >> 5);
            if ((int)threadIdx.x < 32 * nw) {
                for (int64_t i = ((threadIdx.x & 31) * nw) + (threadIdx.x >> 5); i < rows; i += 32 * nw) {
                    const int64_t row = row0 + (i << clg) + rank;
                    if (row >= p.m) break;
                    double acc = 0.0;
#pragma unroll 4
                    for (int64_t s = 0; s < terms; ++s) acc += vals[(i << lt) + s];
                    y[row] = acc;
                }
            }
            return;
        }
        for (int64_t i = threadIdx.x; i < rows; i += blockDim.x) {
            const int64_t rem = (i << clg) + rank;
            if (row0 + rem >= p.m) break;
            double acc = 0.0;
            for (int64_t s = 0; s < terms; ++s) acc += term(rem, s);
            y[row0 + rem] = acc;
        }
        cl.barrier_arrive();
    }
};

template <int CLG, int RL, int LOGN, class EPI>
__global__ void decode_cl_kernel(const double *__restrict__ coeffs, double scale, const float4 *__restrict__ tw,
                                 const float4 *__restrict__ twist, const int32_t *__restrict__ slot_pos, EPI epi, int logn_rt) {
    HE_GRID_LAUNCH();
    const int logn = LOGN ? LOGN : logn_rt;
    extern __shared__ float4 a[];
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank(), item = blockIdx.x >> CLG;
    const int logm = logn - 1, M = 1 << logm, N = 1 << logn, lg_ms = logm - CLG, MS = 1 << lg_ms, off = rank * MS;
    // the context's tables before the wait: the twiddle copy, the twist factors of the first two
    // iterations and the epilogue's first slot positions
    fft_tw_issue<CLG>(a, tw, logm);
    float4 w_pre[2];
#pragma unroll
    for (int r = 0; r < 2; ++r)
        if ((int)threadIdx.x + r * (int)blockDim.x < MS) w_pre[r] = twist[__brev(off + threadIdx.x + r * blockDim.x) >> (32 - logm)];
    const EpiPre pre = epi.prefetch(item, rank, CLG, M, lg_ms, slot_pos);
    HE_GRID_WAIT();
    const double *m = coeffs + (int64_t)item * N;
    int r = 0;
    for (int i = threadIdx.x; i < MS; i += blockDim.x, ++r) {
        const int k = __brev(off + i) >> (32 - logm);
        const float4 w = r == 0 ? w_pre[0] : (r == 1 ? w_pre[1] : twist[k]);
        const df re = df_from(m[k]), im = df_from(m[k + M]);
        float4 c;
        cmul(make_float4(re.hi, re.lo, im.hi, im.lo), make_float4(w.x, w.y, -w.z, -w.w), c);
        a[i] = c;
    }
    __syncthreads();
    fft_cluster<CLG, RL, LOGN ? LOGN - 1 : 0>(a, tw, logm, +1);
    epi(cl, a, item, rank, CLG, M, lg_ms, slot_pos, 1.0 / scale, reinterpret_cast<double *>(a + MS), pre);  // the twiddle copy as scratch
    cl.barrier_wait();  // the epilogue arrived once the other CTAs' shared memory was last read
}

// decrypt limb 0: m = c0 + c1 s (NTT), inverse NTT, centred, as doubles.  One CTA per
// ciphertext, or (CL) one cluster per ciphertext with each CTA on a slice.
template <bool CL, int LOGN = 0>
__global__ void decrypt_kernel(const uint64_t *__restrict__ ct, int64_t ct_words, int nl, const uint64_t *__restrict__ sk_mont,
                               double *coeffs, const uint64_t *__restrict__ d_tw, const ModConst *__restrict__ mc, int logn_rt) {
    HE_GRID_LAUNCH();
    const int logn = LOGN ? LOGN : logn_rt;
    extern __shared__ uint64_t s[];
    const int N = 1 << logn;
    int item, off, len;
    slice_of<CL>(logn, item, off, len);
    const uint64_t q = mc[0].q, qinv = mc[0].qinv;
    tw_prefetch<CL, false>(s, twiddles(d_tw, 0, 1, logn), logn);  // context tables, before the wait
    HE_GRID_WAIT();
    const uint64_t *c0 = ct + item * ct_words + off, *c1 = ct + item * ct_words + (int64_t)nl * N + off;
    for (int k = threadIdx.x; k < len; k += blockDim.x) s[SIDX(k)] = add_mod(c0[k], mont_mul(c1[k], sk_mont[off + k], q, qinv), q);
    __syncthreads();
    inv_any<CL, LOGN>(s, twiddles(d_tw, 0, 1, logn), q, logn);
    double *o = coeffs + (int64_t)item * N + off;
    const uint64_t half = q >> 1;
    for (int k = threadIdx.x; k < len; k += blockDim.x) {
        const uint64_t v = mul_shoup(s[SIDX(k)], mc[0].ninv, mc[0].ninv_shoup, q);
        o[k] = v > half ? u64_to_double_rn(q - v, true) : u64_to_double_rn(v, false);
    }
}

// ---- Philox-4x64-10 (Salmon et al., SC'11) ----
__device__ __forceinline__ void philox4x64(uint64_t c[4], uint64_t k0, uint64_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t lo0 = 0xD2E7470EE14C6C93ull * c[0], hi0 = __umul64hi(0xD2E7470EE14C6C93ull, c[0]);
        const uint64_t lo1 = 0xCA5A826395121157ull * c[2], hi1 = __umul64hi(0xCA5A826395121157ull, c[2]);
        const uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += 0x9E3779B97F4A7C15ull;
        k1 += 0xBB67AE8584CAA73Bull;
    }
}

// uniform residues: coefficient j of limb l (prime index map.prime[l]) from the 128-bit
// integer (word 2(j&1)+1 : word 2(j&1)) of block (j/2, prime index, nonce, 0), key (seed, tag)
// (nonce_dev, when given, holds the nonce in device memory: read when the kernel runs, so a
// captured graph draws fresh randomness on every replay)
// (hi 2^64 + lo) mod q without a 128-bit division: hi reduced by Barrett, then Montgomery
// reduction gives the value times 2^-64 mod q and a Montgomery product by 2^128 mod q restores the
// factor; exact and canonical, so the same residue as the division
__device__ __forceinline__ uint64_t mod128(uint64_t hi, uint64_t lo, const ModConst &m) {
    return mont_mul(redc(reduce_barrett(hi, m.q, m.mu), lo, m.q, m.qinv), m.r2, m.q, m.qinv);
}

__global__ void sample_uniform_kernel(uint64_t seed, uint64_t tag, uint64_t nonce, const uint64_t *nonce_dev, LimbMap map,
                                      uint64_t *out, const ModConst *__restrict__ mc, int logn) {
    HE_GRID_DEP();
    if (nonce_dev) nonce = *nonce_dev;
    const int N = 1 << logn;
    const int l = blockIdx.y;
    const int p = map.prime[l];
    const ModConst m = mc[p];
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < N / 2; b += gridDim.x * blockDim.x) {
        uint64_t c[4] = {(uint64_t)b, (uint64_t)p, nonce, 0};
        philox4x64(c, seed, tag);
        out[(int64_t)l * N + 2 * b] = mod128(c[1], c[0], m);
        out[(int64_t)l * N + 2 * b + 1] = mod128(c[3], c[2], m);
    }
}

struct Cdt {
    uint64_t t[38];
};

// discrete Gaussian by cumulative table: r = word >> 24, x = -19 + #{k : r >= T_k}
__global__ void sample_gauss_kernel(uint64_t seed, uint64_t tag, uint64_t nonce, const uint64_t *nonce_dev, Cdt cdt, int64_t *out,
                                    int logn) {
    HE_GRID_DEP();
    if (nonce_dev) nonce = *nonce_dev;
    const int N = 1 << logn;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < N / 4; b += gridDim.x * blockDim.x) {
        uint64_t c[4] = {(uint64_t)b, 0, nonce, 0};
        philox4x64(c, seed, tag);
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const uint64_t r = c[w] >> 24;
            int64_t x = -19;
            for (int k = 0; k < 38; ++k) x += (r >= cdt.t[k]);
            out[4 * b + w] = x;
        }
    }
}

// ternary secret: (word mod 3) - 1, block (j/4, 0, 0, 0), key (seed, 1)
__global__ void sample_ternary_kernel(uint64_t seed, int64_t *out, int logn) {
    HE_GRID_DEP();
    const int N = 1 << logn;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < N / 4; b += gridDim.x * blockDim.x) {
        uint64_t c[4] = {(uint64_t)b, 0, 0, 0};
        philox4x64(c, seed, 1);
#pragma unroll
        for (int w = 0; w < 4; ++w) out[4 * b + w] = (int64_t)(c[w] % 3) - 1;
    }
}

// c0 = m - a s + e, c1 = a (NTT domain, limbs 0..level)
// Encryption as two launches: the steps of sample_uniform_kernel (tag 2) and the forward NTT,
// and of sample_gauss_kernel (tag 3) and ntt_from_int64_kernel, for every limb at once (item
// (limb l, which): which 0 gives c1 = NTT(a) in place, which 1 NTT(e) in the c0 slot), then
// encrypt_finish_kernel's c0 = pt - c1 s + e elementwise.  The same values, so the same
// ciphertext as the five separate kernels, one cluster transform deep instead of two.  With m_int
// (the plaintext's integer coefficients, pt null) the error becomes m + e before its NTT and
// c0 = NTT(m + e) - c1 s: NTT(m) + NTT(e) = NTT(m + e) mod q, so the ciphertext equals that of
// encoding m to a plaintext and encrypting it.
template <int LOGN = 0>
__global__ void __launch_bounds__(512) encrypt_ntt_cl_kernel(const int64_t *__restrict__ m_int, int nl, uint64_t seed, uint64_t nonce,
                                                             const uint64_t *nonce_dev, Cdt cdt, uint64_t *ct, const uint64_t *__restrict__ d_tw,
                                                             const ModConst *__restrict__ mc, int logn_rt) {
    HE_GRID_LAUNCH();
    const int logn = LOGN ? LOGN : logn_rt;
    extern __shared__ uint64_t s[];
    const int N = 1 << logn;
    int item, off, len;
    slice_of<true>(logn, item, off, len);
    const int l = item >> 1, which = item & 1;
    const uint64_t q = mc[l].q, mu = mc[l].mu;
    const ulonglong2 *tw = twiddles(d_tw, l, 0, logn);
    tw_prefetch<true, true>(s, tw, logn);  // context tables, before the wait (the nonce comes after it)
    HE_GRID_WAIT();
    if (nonce_dev) nonce = *nonce_dev;
    if (which == 0) {  // uniform residues of limb l, two per Philox block
        for (int b = (off >> 1) + threadIdx.x; b < ((off + len) >> 1); b += blockDim.x) {
            uint64_t c[4] = {(uint64_t)b, (uint64_t)l, nonce, 0};
            philox4x64(c, seed, 2);
            s[SIDX(2 * b - off)] = mod128(c[1], c[0], mc[l]);
            s[SIDX(2 * b + 1 - off)] = mod128(c[3], c[2], mc[l]);
        }
    } else {  // the error (plus m), four per Philox block
        for (int b = (off >> 2) + threadIdx.x; b < ((off + len) >> 2); b += blockDim.x) {
            uint64_t c[4] = {(uint64_t)b, 0, nonce, 0};
            philox4x64(c, seed, 3);
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                const uint64_t r = c[w] >> 24;
                int64_t x = -19;
                for (int k = 0; k < 38; ++k) x += (r >= cdt.t[k]);
                if (m_int) x += m_int[4 * b + w];
                s[SIDX(4 * b + w - off)] = reduce_signed(x, q, mu);
            }
        }
    }
    __syncthreads();
    ntt_fwd_cluster<LOGN>(s, tw, q, logn);
    uint64_t *o = ct + ((int64_t)(which == 0 ? nl : 0) + l) * N + off;
    for (int k = threadIdx.x; k < len; k += blockDim.x) o[k] = s[SIDX(k)];
}

// c0 = pt - c1 s + e (pt null: c0 = (m + e) - c1 s), e (or m + e) read from the c0 slot
__global__ void encrypt_finish_kernel(const uint64_t *__restrict__ pt, const uint64_t *__restrict__ sk_mont, int nl, uint64_t *ct,
                                      const ModConst *__restrict__ mc, int logn) {
    HE_GRID_DEP();
    const int N = 1 << logn;
    const int l = blockIdx.y;
    const uint64_t q = mc[l].q, qinv = mc[l].qinv;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
        const int64_t i = (int64_t)l * N + k;
        const uint64_t as = mont_mul(ct[(int64_t)nl * N + i], sk_mont[i], q, qinv);
        ct[i] = pt ? add_mod(sub_mod(pt[i], as, q), ct[i], q) : sub_mod(ct[i], as, q);
    }
}

__global__ void encrypt_combine_kernel(const uint64_t *__restrict__ pt, const uint64_t *__restrict__ a, const uint64_t *__restrict__ e,
                                       const uint64_t *__restrict__ sk_mont, int nl, uint64_t *ct, const ModConst *__restrict__ mc, int logn) {
    HE_GRID_DEP();
    const int N = 1 << logn;
    const int l = blockIdx.y;
    const uint64_t q = mc[l].q, qinv = mc[l].qinv;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
        const int64_t i = (int64_t)l * N + k;
        const uint64_t as = mont_mul(a[i], sk_mont[i], q, qinv);
        ct[i] = add_mod(sub_mod(pt[i], as, q), e[i], q);
        ct[(int64_t)nl * N + i] = a[i];
    }
}

struct PmodQ {
    uint64_t v[HE_MAX_LIMBS];  // P mod q_l for Q limbs
};

// Galois key digit d over Q U P (NTT): b = -a s + e + [l in digit d] (P mod q_l) s(X^g); stored (b, a) in Montgomery form
__global__ void keygen_combine_kernel(const uint64_t *__restrict__ a, const uint64_t *__restrict__ e, const uint64_t *__restrict__ sk,
                                      const uint64_t *__restrict__ sk_mont, uint32_t g, int d_lo, int d_hi, PmodQ pm, int LK,
                                      uint64_t *key_d, const ModConst *__restrict__ mc, int logn) {
    HE_GRID_DEP();
    const int N = 1 << logn;
    const int l = blockIdx.y;
    const ModConst m = mc[l];
    const bool in_digit = l >= d_lo && l < d_hi;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
        const int64_t i = (int64_t)l * N + k;
        uint64_t b = sub_mod(e[i], mont_mul(a[i], sk_mont[i], m.q, m.qinv), m.q);
        if (in_digit) {
            const uint64_t sg = sk[(int64_t)l * N + automorph_src(k, g, logn)];
            b = add_mod(b, (uint64_t)((u128)sg * pm.v[l] % m.q), m.q);
        }
        key_d[i] = mont_mul(b, m.r2, m.q, m.qinv);
        key_d[(int64_t)LK * N + i] = mont_mul(a[i], m.r2, m.q, m.qinv);
    }
}

}  // namespace

static size_t fft_smem_bytes(int logn) { return (size_t)8 << logn; }  // N/2 float4
#define FFT_THREADS 512

// FFT tables in ctx->d_fft: [N/4] float4 twiddles, [N/2] float4 twist, [N/2] int32 slot positions
// Cluster size for a launch of `count` transforms: 8, 4 or 2 CTAs per transform while the
// launch stays within two CTAs per SM, else one (rings below 2^10 always one).
static int fft_cluster_log(int logn, int count) {
    if (logn < 10) return 0;
    for (int clg = 3; clg >= 1; --clg)
        if (count << clg <= 2 * 152) return clg;
    return 0;
}

template <int CLG, int RL, typename... KArgs, typename... Args>
static void launch_fft_cl(void (*kernel)(KArgs...), he_ctx *ctx, int count, Args... args) {
    const int MS = ctx->n / 2 >> CLG;
    int threads = MS >> RL;
    threads = threads < 32 ? 32 : (threads > 512 ? 512 : threads);
    launch_cluster_n(kernel, count << CLG, threads, (size_t)MS * sizeof(float4) * 3 / 2, ctx->stream, 1 << CLG, args...);  // slice + twiddles
}

// the pair kernel for `count` plaintexts from src; false (nothing launched) below rings of 2^10
template <class SRC>
static bool launch_encode_pairs(he_ctx *ctx, SRC src, int count, double scale, int64_t *coeffs) {
    if (ctx->log_n < 10) return false;
    const float4 *tw = reinterpret_cast<const float4 *>(ctx->d_fft);
    const float4 *twist = tw + ctx->n / 4;
    const int32_t *pos = reinterpret_cast<const int32_t *>(twist + ctx->n / 2);
    const int pairs = (count + 1) / 2;
    switch (fft_cluster_log(ctx->log_n, pairs)) {
        case 3:
            launch_fft_cl<3, 1>(by_logn(ctx->log_n, [](auto L) { return encode_pair_cl_kernel<3, 1, L.value, SRC>; }), ctx, pairs, src, count, scale, tw,
                                twist, pos, coeffs, ctx->log_n);
            return true;
        case 2:
            launch_fft_cl<2, 1>(by_logn(ctx->log_n, [](auto L) { return encode_pair_cl_kernel<2, 1, L.value, SRC>; }), ctx, pairs, src, count, scale, tw,
                                twist, pos, coeffs, ctx->log_n);
            return true;
        case 1:
            launch_fft_cl<1, 1>(by_logn(ctx->log_n, [](auto L) { return encode_pair_cl_kernel<1, 1, L.value, SRC>; }), ctx, pairs, src, count, scale, tw,
                                twist, pos, coeffs, ctx->log_n);
            return true;
        default: return false;
    }
}

bool launch_encode_matrix(he_ctx *ctx, const he_plan &p, const double *X, int trans, int count, double scale, int64_t *coeffs) {
    if (count < 2) return false;
    auto lg = [](int64_t v) { return __builtin_ctzll((unsigned long long)v); };
    const MatrixSrc src{p, X, trans, lg(p.m_prime), lg(p.col_blocks), lg(p.nb), lg(p.mb)};
    if (!launch_encode_pairs(ctx, src, count, scale, coeffs)) return false;
    ctx->launches++;
    return true;
}

bool launch_encode_vector(he_ctx *ctx, const he_plan &p, const double *y, int count, double scale, int64_t *coeffs) {
    const VectorSrc src{y, p.n, p.nb, __builtin_ctzll((unsigned long long)p.nb)};
    if (count >= 2) {
        if (!launch_encode_pairs(ctx, src, count, scale, coeffs)) return false;
        ctx->launches++;
        return true;
    }
    const float4 *tw = reinterpret_cast<const float4 *>(ctx->d_fft);
    const float4 *twist = tw + ctx->n / 4;
    const int32_t *pos = reinterpret_cast<const int32_t *>(twist + ctx->n / 2);
    switch (fft_cluster_log(ctx->log_n, count)) {
        case 3:
            launch_fft_cl<3, 1>(by_logn(ctx->log_n, [](auto L) { return encode_cl_kernel<3, 1, L.value, VectorSrc>; }), ctx, count, src, scale, tw, twist,
                                pos, coeffs, ctx->log_n);
            break;
        case 2:
            launch_fft_cl<2, 1>(by_logn(ctx->log_n, [](auto L) { return encode_cl_kernel<2, 1, L.value, VectorSrc>; }), ctx, count, src, scale, tw, twist,
                                pos, coeffs, ctx->log_n);
            break;
        case 1:
            launch_fft_cl<1, 1>(by_logn(ctx->log_n, [](auto L) { return encode_cl_kernel<1, 1, L.value, VectorSrc>; }), ctx, count, src, scale, tw, twist,
                                pos, coeffs, ctx->log_n);
            break;
        default: return false;
    }
    ctx->launches++;
    return true;
}

void launch_encode(he_ctx *ctx, const double *slots, int64_t n_slots, int64_t stride, int count, double scale, int64_t *coeffs) {
    if (count == 0) return;
    const float4 *tw = reinterpret_cast<const float4 *>(ctx->d_fft);
    const float4 *twist = tw + ctx->n / 4;
    const int32_t *pos = reinterpret_cast<const int32_t *>(twist + ctx->n / 2);
    ctx->launches++;
    if (count >= 2 && launch_encode_pairs(ctx, SlotsSrc{slots, n_slots, stride}, count, scale, coeffs)) return;
    switch (fft_cluster_log(ctx->log_n, count)) {
        case 3:
            launch_fft_cl<3, 1>(by_logn(ctx->log_n, [](auto L) { return encode_cl_kernel<3, 1, L.value, SlotsSrc>; }), ctx, count,
                                SlotsSrc{slots, n_slots, stride}, scale, tw, twist, pos, coeffs, ctx->log_n);
            return;
        case 2:
            launch_fft_cl<2, 1>(by_logn(ctx->log_n, [](auto L) { return encode_cl_kernel<2, 1, L.value, SlotsSrc>; }), ctx, count,
                                SlotsSrc{slots, n_slots, stride}, scale, tw, twist, pos, coeffs, ctx->log_n);
            return;
        case 1:
            launch_fft_cl<1, 1>(by_logn(ctx->log_n, [](auto L) { return encode_cl_kernel<1, 1, L.value, SlotsSrc>; }), ctx, count,
                                SlotsSrc{slots, n_slots, stride}, scale, tw, twist, pos, coeffs, ctx->log_n);
            return;
        default: break;
    }
    launch_k(encode_kernel, count, FFT_THREADS, fft_smem_bytes(ctx->log_n), ctx->stream, slots, n_slots, stride, scale, tw, twist, pos, coeffs, ctx->log_n);
}

void launch_decode(he_ctx *ctx, const double *coeffs, int count, double scale, double *slots) {
    if (count == 0) return;
    const float4 *tw = reinterpret_cast<const float4 *>(ctx->d_fft);
    const float4 *twist = tw + ctx->n / 4;
    const int32_t *pos = reinterpret_cast<const int32_t *>(twist + ctx->n / 2);
    ctx->launches++;
    switch (fft_cluster_log(ctx->log_n, count)) {
        case 3:
            launch_fft_cl<3, 1>(by_logn(ctx->log_n, [](auto L) { return decode_cl_kernel<3, 1, L.value, DecodeSlots>; }), ctx, count, coeffs, scale, tw,
                                twist, pos, DecodeSlots{slots}, ctx->log_n);
            return;
        case 2:
            launch_fft_cl<2, 1>(by_logn(ctx->log_n, [](auto L) { return decode_cl_kernel<2, 1, L.value, DecodeSlots>; }), ctx, count, coeffs, scale, tw,
                                twist, pos, DecodeSlots{slots}, ctx->log_n);
            return;
        case 1:
            launch_fft_cl<1, 1>(by_logn(ctx->log_n, [](auto L) { return decode_cl_kernel<1, 1, L.value, DecodeSlots>; }), ctx, count, coeffs, scale, tw,
                                twist, pos, DecodeSlots{slots}, ctx->log_n);
            return;
        default: break;
    }
    launch_k(decode_kernel, count, FFT_THREADS, fft_smem_bytes(ctx->log_n), ctx->stream, coeffs, scale, tw, twist, pos, slots, ctx->log_n);
}

bool launch_decode_ras(he_ctx *ctx, const he_plan &p, const double *coeffs, int count, double scale, const double *mask, double *y) {
    const float4 *tw = reinterpret_cast<const float4 *>(ctx->d_fft);
    const float4 *twist = tw + ctx->n / 4;
    const int32_t *pos = reinterpret_cast<const int32_t *>(twist + ctx->n / 2);
    auto lg = [](int64_t v) { return __builtin_ctzll((unsigned long long)v); };
    const DecodeRas epi{p, mask, y, lg(p.m_prime), lg(p.nb), lg(p.slots), lg(p.mb)};
    switch (fft_cluster_log(ctx->log_n, count)) {
        case 3:
            launch_fft_cl<3, 1>(by_logn(ctx->log_n, [](auto L) { return decode_cl_kernel<3, 1, L.value, DecodeRas>; }), ctx, count, coeffs, scale, tw, twist,
                                pos, epi, ctx->log_n);
            break;
        case 2:
            launch_fft_cl<2, 1>(by_logn(ctx->log_n, [](auto L) { return decode_cl_kernel<2, 1, L.value, DecodeRas>; }), ctx, count, coeffs, scale, tw, twist,
                                pos, epi, ctx->log_n);
            break;
        case 1:
            launch_fft_cl<1, 1>(by_logn(ctx->log_n, [](auto L) { return decode_cl_kernel<1, 1, L.value, DecodeRas>; }), ctx, count, coeffs, scale, tw, twist,
                                pos, epi, ctx->log_n);
            break;
        default: return false;
    }
    ctx->launches++;
    return true;
}

void launch_decrypt_coeffs(he_ctx *ctx, const uint64_t *ct, int level, int count, double *coeffs, uint64_t *) {
    const int64_t words = 2 * (int64_t)(level + 1) * ctx->n;
    ctx->launches++;
    if (use_cluster(ctx->log_n, count)) {
        launch_cluster(by_logn(ctx->log_n, [](auto L) { return decrypt_kernel<true, L.value>; }), count * HE_NTT_CL_SIZE, cl_threads(ctx->log_n), cl_smem_bytes(ctx->log_n), ctx->stream, ct, words,
                       level + 1, (const uint64_t *)ctx->d_sk_mont, coeffs, (const uint64_t *)ctx->d_tw, (const ModConst *)ctx->d_mc, ctx->log_n);
        return;
    }
    launch_k(by_logn(ctx->log_n, [](auto L) { return decrypt_kernel<false, L.value>; }), count, ntt_threads(ctx->log_n), ntt_smem_bytes(ctx->log_n), ctx->stream, ct, words, level + 1, ctx->d_sk_mont, coeffs, ctx->d_tw, ctx->d_mc,
                                                                    ctx->log_n);
}

void launch_sample_uniform(he_ctx *ctx, uint64_t tag, uint64_t nonce, const LimbMap &map, int, uint64_t *out, const uint64_t *nonce_dev) {
    dim3 grid((ctx->n / 2 + 255) / 256, map.n);
    ctx->launches++;
    launch_k(sample_uniform_kernel, grid, 256, 0, ctx->stream, ctx->seed, tag, nonce, nonce_dev, map, out, ctx->d_mc, ctx->log_n);
}

void launch_sample_gauss(he_ctx *ctx, uint64_t tag, uint64_t nonce, int64_t *out, const uint64_t *nonce_dev) {
    Cdt c;
    for (int k = 0; k < 38; ++k) c.t[k] = ctx->cdt[k];
    ctx->launches++;
    launch_k(sample_gauss_kernel, (ctx->n / 4 + 255) / 256, 256, 0, ctx->stream, ctx->seed, tag, nonce, nonce_dev, c, out, ctx->log_n);
}

void launch_sample_ternary(he_ctx *ctx, int64_t *out) {
    ctx->launches++;
    launch_k(sample_ternary_kernel, (ctx->n / 4 + 255) / 256, 256, 0, ctx->stream, ctx->seed, out, ctx->log_n);
}

bool launch_encrypt_fused(he_ctx *ctx, const uint64_t *pt, const int64_t *m_int, int level, uint64_t nonce, const uint64_t *nonce_dev,
                          uint64_t *ct) {
    if (!use_cluster(ctx->log_n, 2 * (level + 1))) return false;
    Cdt c;
    for (int k = 0; k < 38; ++k) c.t[k] = ctx->cdt[k];
    ctx->launches += 2;
    launch_cluster(by_logn(ctx->log_n, [](auto L) { return encrypt_ntt_cl_kernel<L.value>; }), 2 * (level + 1) * HE_NTT_CL_SIZE,
                   cl_threads(ctx->log_n), cl_smem_bytes(ctx->log_n), ctx->stream, m_int, level + 1, ctx->seed, nonce, nonce_dev, c, ct,
                   (const uint64_t *)ctx->d_tw, (const ModConst *)ctx->d_mc, ctx->log_n);
    launch_k(encrypt_finish_kernel, dim3((ctx->n + 255) / 256, level + 1), 256, 0, ctx->stream, pt, (const uint64_t *)ctx->d_sk_mont, level + 1, ct,
             (const ModConst *)ctx->d_mc, ctx->log_n);
    return true;
}

void launch_encrypt_combine(he_ctx *ctx, const uint64_t *pt, const uint64_t *a, const uint64_t *e, int level, uint64_t *ct) {
    dim3 grid((ctx->n + 255) / 256, level + 1);
    ctx->launches++;
    launch_k(encrypt_combine_kernel, grid, 256, 0, ctx->stream, pt, a, e, ctx->d_sk_mont, level + 1, ct, ctx->d_mc, ctx->log_n);
}

void launch_keygen_combine(he_ctx *ctx, const uint64_t *a, const uint64_t *e, uint32_t g, int digit, uint64_t *key_d) {
    PmodQ pm{};
    for (int l = 0; l < ctx->L; ++l) {
        uint64_t q = ctx->primes[l], v = 1 % q;
        for (int j = 0; j < ctx->K; ++j) v = (uint64_t)((u128)v * (ctx->primes[ctx->L + j] % q) % q);
        pm.v[l] = v;
    }
    const int lo = digit * ctx->alpha, hi = lo + ctx->alpha < ctx->L ? lo + ctx->alpha : ctx->L;
    dim3 grid((ctx->n + 255) / 256, ctx->L + ctx->K);
    ctx->launches++;
    launch_k(keygen_combine_kernel, grid, 256, 0, ctx->stream, a, e, ctx->d_sk, ctx->d_sk_mont, g, lo, hi, pm, ctx->L + ctx->K, key_d, ctx->d_mc,
                                                         ctx->log_n);
}

void encode_set_smem_limits(int max_bytes) {
    cudaFuncSetAttribute(encode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
    cudaFuncSetAttribute(decode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
    each_logn([max_bytes](auto L) {
        cudaFuncSetAttribute(decrypt_kernel<false, L.value>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
        cudaFuncSetAttribute(decrypt_kernel<true, L.value>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
        cudaFuncSetAttribute(encrypt_ntt_cl_kernel<L.value>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
        // cluster FFTs: the slice and the local stages' twiddles (1.5 MS float4)
        cudaFuncSetAttribute(encode_cl_kernel<1, 1, L.value, SlotsSrc>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
        cudaFuncSetAttribute(encode_cl_kernel<1, 1, L.value, VectorSrc>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
        cudaFuncSetAttribute(decode_cl_kernel<1, 1, L.value, DecodeSlots>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
        cudaFuncSetAttribute(decode_cl_kernel<1, 1, L.value, DecodeRas>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
        cudaFuncSetAttribute(encode_cl_kernel<2, 1, L.value, SlotsSrc>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
        cudaFuncSetAttribute(encode_cl_kernel<2, 1, L.value, VectorSrc>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
        cudaFuncSetAttribute(decode_cl_kernel<2, 1, L.value, DecodeSlots>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
        cudaFuncSetAttribute(decode_cl_kernel<2, 1, L.value, DecodeRas>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
        cudaFuncSetAttribute(encode_cl_kernel<3, 1, L.value, SlotsSrc>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
        cudaFuncSetAttribute(encode_cl_kernel<3, 1, L.value, VectorSrc>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
        cudaFuncSetAttribute(encode_pair_cl_kernel<1, 1, L.value, SlotsSrc>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
        cudaFuncSetAttribute(encode_pair_cl_kernel<2, 1, L.value, SlotsSrc>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
        cudaFuncSetAttribute(encode_pair_cl_kernel<3, 1, L.value, SlotsSrc>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
        cudaFuncSetAttribute(encode_pair_cl_kernel<1, 1, L.value, MatrixSrc>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
        cudaFuncSetAttribute(encode_pair_cl_kernel<2, 1, L.value, MatrixSrc>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
        cudaFuncSetAttribute(encode_pair_cl_kernel<3, 1, L.value, MatrixSrc>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
        cudaFuncSetAttribute(encode_pair_cl_kernel<1, 1, L.value, VectorSrc>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
        cudaFuncSetAttribute(encode_pair_cl_kernel<2, 1, L.value, VectorSrc>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
        cudaFuncSetAttribute(encode_pair_cl_kernel<3, 1, L.value, VectorSrc>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
        cudaFuncSetAttribute(decode_cl_kernel<3, 1, L.value, DecodeSlots>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
        cudaFuncSetAttribute(decode_cl_kernel<3, 1, L.value, DecodeRas>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_bytes);
    });
}
