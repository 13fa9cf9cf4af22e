// Device building blocks shared by the single-state kernels (qs_apply.cu) and
// the batched persistent kernel (qs_batch.cu), so both run the same arithmetic.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "qs_internal.h"

namespace qsd {

template <typename R> struct cplx;
template <> struct cplx<double> { using t = double2; };
template <> struct cplx<float> { using t = float2; };

struct Targets {
    int q[QS_MAX_K];   // ascending
};

// Insert a zero bit at each (ascending) target position: group id -> index of
// the group's x = 0 member (Sec. 3.2: the c bits fill the non-target positions).
template <int K>
__device__ __forceinline__ uint64_t group_base(uint64_t g, const Targets &t)
{
#pragma unroll
    for (int j = 0; j < K; j++) {
        uint64_t lo = g & ((1ULL << t.q[j]) - 1);
        g = ((g ^ lo) << 1) | lo;
    }
    return g;
}

template <int K>
__device__ __forceinline__ uint64_t member_offset(int x, const Targets &t)
{
    uint64_t o = 0;
#pragma unroll
    for (int j = 0; j < K; j++)
        if ((x >> j) & 1) o |= 1ULL << t.q[j];
    return o;
}

template <bool CG, typename C>
__device__ __forceinline__ C ld(const C *p)
{
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

// One group of a dense k-qubit cluster (Sec. 3.2): the 2^K amplitudes at
// strides 2^{q_j} are gathered into registers, v <- U v, and scattered back.
// Each complex multiply-accumulate is the pair of real FMA updates of
// Eqs. (2)-(3): acc += (v_R m_R, v_I m_R) then acc += (-v_I m_I, v_R m_I).
// CG: loads bypass L1 (the batched kernel shares states between the CTAs of a
// cluster).
template <typename R, int K, bool CG>
__device__ __forceinline__ void dense_group(typename cplx<R>::t *p, const Targets &t,
                                            const typename cplx<R>::t *Us)
{
    using C = typename cplx<R>::t;
    constexpr int D = 1 << K;
    C v[D];
#pragma unroll
    for (int x = 0; x < D; x++) v[x] = ld<CG>(p + member_offset<K>(x, t));
    // rows of U one at a time (kept rolled so v[] stays in registers)
#pragma unroll 1
    for (int l = 0; l < D; l++) {
        R ar = 0, ai = 0;
        const C *row = Us + l * D;
#pragma unroll
        for (int x = 0; x < D; x++) {
            C m = row[x];
            ar = fma(v[x].x, m.x, ar);
            ai = fma(v[x].y, m.x, ai);
            ar = fma(-v[x].y, m.y, ar);
            ai = fma(v[x].x, m.y, ai);
        }
        C o;
        o.x = ar;
        o.y = ai;
        p[member_offset<K>(l, t)] = o;
    }
}

// Multiply by e^{i pi m / 4}: an odd m first takes one factor
// e^{i pi/4} = (1 + i)/sqrt(2); the remaining quarter turn i^{m >> 1} only swaps
// and negates, done on the bit patterns (sign-bit flips) so complex128 spends
// no FP64 instruction on it.
__device__ __forceinline__ float flip(float x, bool f) { return __int_as_float(__float_as_int(x) ^ (f ? 0x80000000 : 0)); }
__device__ __forceinline__ double flip(double x, bool f)
{
    return __longlong_as_double(__double_as_longlong(x) ^ (f ? (long long)0x8000000000000000ULL : 0LL));
}

template <typename C, typename R>
__device__ __forceinline__ C rotate8(C a, int m)
{
    if (m & 1) {
        const R r = (R)0.70710678118654752440;
        C b;
        b.x = (a.x - a.y) * r;
        b.y = (a.x + a.y) * r;
        a = b;
    }
    const int q = (m >> 1) & 3;                  // i^q: 0 (x, y), 1 (-y, x), 2 (-x, -y), 3 (y, -x)
    const bool sw = q & 1;
    C o;
    o.x = flip(sw ? a.y : a.x, q == 1 || q == 2);
    o.y = flip(sw ? a.x : a.y, q >= 2);
    return o;
}

// Phase products (Sec. 2, Sec. 3.5): amplitude i gets e^{i pi m(i)/4},
// m(i) = sum_q c_q i_q + 4 sum_a i_a popc(i & P_a) mod 8, with P_a the CZ
// partners b > a of qubit a.  With i = h | l (l: the low L bits) this is
// m_lo(l) + m_hi(h) + 4 popc(l & M_h): m_lo is a table over the low bits,
// m_hi and the mask M_h (low qubits whose partner set meets h an odd number of
// times) are fixed for a chunk of 2^L amplitudes.
__device__ __forceinline__ uint8_t phase_low(uint64_t x, const uint64_t *cm, const int *act,
                                             const uint64_t *part, int n_act, int L)
{
    const uint64_t lowmask = (1ULL << L) - 1;
    int m = __popcll(x & cm[0]) + 2 * __popcll(x & cm[1]) + 4 * __popcll(x & cm[2]);
    int par = 0;
    for (int t = 0; t < n_act; t++)
        if (act[t] < L && ((x >> act[t]) & 1)) par ^= __popcll(x & part[t] & lowmask);
    return (uint8_t)((m + 4 * (par & 1)) & 7);
}

__device__ __forceinline__ int phase_high(uint64_t h, const uint64_t *cm, const int *act, const uint64_t *part,
                                          int n_act, int L, uint64_t &Mh)
{
    int mh = __popcll(h & cm[0]) + 2 * __popcll(h & cm[1]) + 4 * __popcll(h & cm[2]);
    int parh = 0;
    Mh = 0;
    for (int t = 0; t < n_act; t++) {
        const int a = act[t];
        const int odd = __popcll(h & part[t]) & 1;
        if (a >= L) parh ^= (int)((h >> a) & 1) & odd;
        else Mh |= (uint64_t)odd << a;
    }
    return (mh + 4 * parh) & 7;
}

// p = fl(fl(re^2) + fl(im^2)) in FP64 (no contraction into an FMA).
__device__ __forceinline__ double prob(double2 a)
{
    return __dadd_rn(__dmul_rn(a.x, a.x), __dmul_rn(a.y, a.y));
}
// x^2 of a float as a double, exact: the 24-bit significand squared fits in
// 48 bits, so the product is assembled from integer operations (the same value
// as the FP64 multiplication of x by itself, without the FP64 pipe, which runs
// at 1/64 of the FP32 rate on this part).  |x| = m 2^E; m^2 has its leading
// one at bit t <= 47, so x^2 = 1.f 2^(t + 2E) with f the bits below it; every
// such square, subnormal x included, is a normal double.
__device__ __forceinline__ double sq_exact(float x)
{
    const uint32_t b = __float_as_uint(x) & 0x7fffffffu;
    const uint32_t e = b >> 23;
    if (e == 0xffu) {                                  // inf, nan: the FP64 unit
        const double d = x;
        return __dmul_rn(d, d);
    }
    const uint32_t m = e ? ((b & 0x7fffffu) | 0x800000u) : b;
    if (m == 0) return 0.0;
    const int E = e ? (int)e - 150 : -149;
    const uint64_t q = (uint64_t)m * m;
    const int lz = __clzll((long long)q);             // leading one at bit 63 - lz
    const uint64_t frac = ((q << lz) << 1) >> 12;     // the 52 bits below it
    const uint64_t bexp = (uint64_t)(63 - lz + 2 * E + 1023);
    return __longlong_as_double((long long)((bexp << 52) | frac));
}
// p = fl(x^2 + y^2) with exact squares: fl(fl(x^2) + fl(y^2)) in FP64.
__device__ __forceinline__ double prob(float2 a)
{
    return __dadd_rn(sq_exact(a.x), sq_exact(a.y));
}

// Natural logarithm of a positive normal double, table-driven (P. T. P. Tang,
// "Table-driven implementation of the logarithm function in IEEE floating-point
// arithmetic", ACM TOMS 16(4), 1990): p = 2^e m, m in [1, 2); c_j is the centre
// of the mantissa interval [1 + j/1024, 1 + (j+1)/1024) picked by the top ten
// mantissa bits, r = m / c_j - 1 (|r| <= 2^-11) and
//   ln p = e ln 2 + ln c_j + ln(1 + r),  ln(1 + r) = r - r^2/2 + r^3/3 - r^4/4,
// truncation error below r^5/5 < 2^-57.  ln c_j and 1/c_j come from the CUDA
// math library once per block (shared-memory table, 16 KB).
constexpr int kLogBits = 10;
struct LogTable {
    double inv[1 << kLogBits], ln[1 << kLogBits];
};

__device__ __forceinline__ void log_table_init(LogTable &t)
{
    for (int j = threadIdx.x; j < (1 << kLogBits); j += blockDim.x) {
        const double c = 1.0 + (j + 0.5) / (double)(1 << kLogBits);
        t.inv[j] = 1.0 / c;
        t.ln[j] = log(c);
    }
}

__device__ __forceinline__ double log_tab(const LogTable &t, double p)
{
    const long long bits = __double_as_longlong(p);
    const int e = (int)(bits >> 52) - 1023;
    const int j = (int)((bits >> (52 - kLogBits)) & ((1 << kLogBits) - 1));
    const double m = __longlong_as_double((bits & 0xFFFFFFFFFFFFFLL) | 0x3FF0000000000000LL);
    const double r = fma(m, t.inv[j], -1.0);
    double q = -0.25;
    q = fma(q, r, 1.0 / 3.0);
    q = fma(q, r, -0.5);
    q = fma(q, r, 1.0);
    return fma((double)e, 0.69314718055994530942, fma(q, r, t.ln[j]));
}

// ---------------------------------------------------------------------------
// Float-float ("double-float") arithmetic: a value is hi + lo with |lo| at most
// half an ulp of hi, about 48 significant bits.  Error-free transforms after
// Knuth (two-sum), Dekker (fast two-sum) and the FMA product error; GB300's
// FP32 pipe is ~64x its FP64 pipe, so 10-20 FP32 operations per emulated
// operation still run far faster than FP64.
struct ff {
    float hi, lo;
};
__device__ __forceinline__ ff ff_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
    return ff{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ ff ff_fast_two_sum(float a, float b)   // |a| >= |b| or a = 0
{
    const float s = __fadd_rn(a, b);
    return ff{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_add(ff a, ff b)
{
    ff s = ff_two_sum(a.hi, b.hi);
    s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return ff_fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ff ff_add_f(ff a, float b)
{
    ff s = ff_two_sum(a.hi, b);
    return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
__device__ __forceinline__ ff ff_mul(ff a, ff b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return ff_fast_two_sum(p, e);
}
// x^2 exactly as hi + lo (the FMA gives the rounding error of the product)
__device__ __forceinline__ ff ff_sqr_f(float x)
{
    const float p = __fmul_rn(x, x);
    return ff{p, fmaf(x, x, -p)};
}
// The top 48 bits of a double d with |d| in [2^-126, 2^128), by bit
// manipulation only: hi = its top 24 significant bits, lo = the next 24
// (0 when they fall below the normal float range).  Relative error < 2^-47.
__device__ __forceinline__ ff ff_from_double(double d)
{
    const uint32_t hw = (uint32_t)__double2hiint(d), lw = (uint32_t)__double2loint(d);
    const int E = (int)((hw >> 20) & 0x7FFu) - 1023;
    const uint32_t sign = hw & 0x80000000u;
    const float hi = __uint_as_float(sign | ((uint32_t)(E + 127) << 23) | ((hw & 0xFFFFFu) << 3) | (lw >> 29));
    const float scale = __uint_as_float((uint32_t)max(E - 47 + 127, 0) << 23);   // 2^(E-47) or 0
    const float lo = __uint2float_rn((lw >> 5) & 0xFFFFFFu) * scale;
    return ff{hi, sign ? -lo : lo};
}

// p ln p for p in [2^-79, 2^100] in float-float, table-driven after Tang
// (ACM TOMS 16(4), 1990): p = 2^e m, c_j the centre of the mantissa interval
// picked by the top ten bits, r = m / c_j - 1 (|r| < 2^-10), and
//   ln p = e ln 2 + ln c_j + r - r^2/2 + r^3/3 - r^4/4,
// with e ln 2, ln c_j and 1/c_j as float-float table entries.  The error of
// ln p is about 2^-48 of |e ln 2| + |ln c_j| plus 2^-55 (float-float
// rounding), so each term p ln p carries a relative error near 2^-47.
constexpr int kFFLogBits = 10;
struct FFLogTable {
    ff inv[1 << kFFLogBits], ln[1 << kFFLogBits];
    ff eln2[255];   // e ln 2 for e = -127 .. 127
};
__device__ __forceinline__ void ff_log_table_init(FFLogTable &t)
{
    for (int j = threadIdx.x; j < (1 << kFFLogBits); j += blockDim.x) {
        const double c = 1.0 + (j + 0.5) / (double)(1 << kFFLogBits);
        t.inv[j] = ff_from_double(1.0 / c);
        t.ln[j] = ff_from_double(log(c));
    }
    for (int e = threadIdx.x; e < 255; e += blockDim.x)
        t.eln2[e] = e == 127 ? ff{0.0f, 0.0f} : ff_from_double((double)(e - 127) * 0.69314718055994530942);
}
__device__ __forceinline__ ff ff_p_ln_p(const FFLogTable &t, ff p)
{
    const uint32_t b = __float_as_uint(p.hi);
    const int e = (int)((b >> 23) & 0xFFu) - 127;
    const int j = (int)((b >> (23 - kFFLogBits)) & ((1u << kFFLogBits) - 1));
    // m = p 2^-e: the exponent of hi replaced, lo scaled by the same power of two
    const ff m = ff{__uint_as_float((b & 0x807FFFFFu) | (127u << 23)), p.lo * __uint_as_float((uint32_t)(127 - e) << 23)};
    ff r = ff_mul(m, t.inv[j]);
    r = ff_two_sum(__fsub_rn(r.hi, 1.0f), r.lo);            // hi - 1 is exact (hi within 2^-10 of 1)
    // ln(1 + r) = r - r^2/2 + r^3/3 - r^4/4: -x^2/2 (x = r.hi) exactly as
    // float-float, the rest (below 2^-32) in FP32, -x r.lo for the cross term
    const float x = r.hi;
    const ff sq = ff_sqr_f(x);
    const ff half = ff{-0.5f * sq.hi, -0.5f * sq.lo};
    const float tail = fmaf(x * x * x, fmaf(x, -0.25f, 0.33333334f), -x * r.lo);
    const ff lnp = ff_add(ff_add(t.eln2[e + 127], t.ln[j]), ff_add(ff_add_f(r, tail), half));
    return ff_mul(p, lnp);
}

}  // namespace qsd
