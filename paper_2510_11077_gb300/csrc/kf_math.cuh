// Arithmetic helpers of the filter kernels, written for a part whose FP64
// pipe issues 2 FMA per clock per SM while its FP32 and integer pipes issue
// 64-128: everything that does not need FP64 runs on the other pipes.
//
//  * phase_sincos: sin and cos of 2 pi x for a phase x in cycles.  The
//    fraction of x is taken exactly as a 64-bit fixed-point number with
//    integer instructions; its top 8 bits index a 256-entry table of
//    sin/cos(2 pi j / 256); the remainder (|a| <= pi/256 rad) goes through
//    Taylor polynomials in double-float arithmetic (a value as an unevaluated
//    sum of two floats, ~48-bit significand), then the angle-addition formula.
//    Error-free transformations: Knuth's two-sum, Dekker's fast two-sum and
//    the FMA two-product (as in the double-float arithmetic of Hida, Li &
//    Bailey 2001).  The table node plus the correction is then summed exactly
//    in 2^-62 fixed point and rounded once to a double, all on the integer
//    pipe: no FP64 instruction at all.
//  * rcp_nr: 1/S from a double-float seed formed on the FP32 and integer
//    pipes, refined by one FP64 Newton-Raphson step (two FMAs).
//  * LogProd: sum of ln S_k as a running product kept in [1, 2), in
//    double-float arithmetic on the FP32 pipe, with its binary exponent
//    accumulated in an integer (one log per lane at the end).
#pragma once

#include <cstdint>

namespace argus {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

__device__ __forceinline__ df fast_two_sum(float a, float b) {   // needs |a| >= |b|
    const float s = a + b;
    return {s, b - (s - a)};
}

__device__ __forceinline__ df df_mul(df a, df b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    return fast_two_sum(p, e);
}

__device__ __forceinline__ df df_add(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    const df t = two_sum(a.lo, b.lo);
    s = fast_two_sum(s.hi, s.lo + t.hi);
    return fast_two_sum(s.hi, s.lo + t.lo);
}

__device__ __forceinline__ df df_add_f(df a, float b) {          // a + b, b a float
    const df s = two_sum(a.hi, b);
    return fast_two_sum(s.hi, s.lo + a.lo);
}

__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }

// frac(x) * 2^64 for a finite double x (exact, integer instructions only).
__device__ __forceinline__ uint64_t frac_cycles_u64(double x) {
    const long long b = __double_as_longlong(x);
    const int ef = int((b >> 52) & 0x7ff);
    const unsigned long long m =
        (static_cast<unsigned long long>(b) & 0xFFFFFFFFFFFFFull) | (ef ? (1ull << 52) : 0ull);
    const int s = ef - 1075 + 64;   // x = m 2^(ef - 1075)
    unsigned long long F = 0ull;
    if (s >= 0 && s < 64) F = m << s;
    else if (s < 0 && s > -64) F = m >> (-s);
    return (b < 0) ? (0ull - F) : F;
}

// x 2^62 rounded to an integer (half away from zero) for a float |x| < 2;
// zero and subnormal floats give 0.  Integer instructions only.
__device__ __forceinline__ long long f2fix62(float x) {
    const unsigned u = __float_as_uint(x);
    const int e = int((u >> 23) & 0xffu);
    const long long m = e ? (long long)((u & 0x7fffffu) | 0x800000u) : 0ll;   // x = m 2^(e - 150)
    const int sh = e - 88;                                                  // x 2^62 = m 2^sh
    long long v = 0;
    if (sh >= 0) v = m << sh;                            // sh <= 38 for |x| < 2
    else if (sh > -63) v = (m + (1ll << (-sh - 1))) >> (-sh);
    return (u >> 31) ? -v : v;
}

// The double nearest to v 2^-62 (ties to even), for |v| < 2^63 (|value| < 2).
// Integer instructions only.
__device__ __forceinline__ double fix62_to_double(long long v) {
    const unsigned long long neg = v < 0 ? 1ull : 0ull;
    const unsigned long long a = neg ? 0ull - static_cast<unsigned long long>(v)
                                     : static_cast<unsigned long long>(v);
    const int lz = __clzll(static_cast<long long>(a));
    const unsigned long long u = a << (lz & 63);          // leading 1 at bit 63
    unsigned long long m = u >> 11;                       // 53 bits, leading 1 at bit 52
    const unsigned r = unsigned(u & 0x7ffu);
    m += (r > 0x400u || (r == 0x400u && (m & 1ull))) ? 1ull : 0ull;
    // the leading bit of a 2^-62 is 2^(1 - lz); a carry out of m bumps the exponent
    const unsigned long long bits =
        (static_cast<unsigned long long>(1024 - lz) << 52) + m - (1ull << 52);
    return a ? __longlong_as_double(static_cast<long long>(bits | (neg << 63))) : 0.0;
}

// Table of sin/cos(2 pi j / 256): the nodes in 2^-62 fixed point (exact:
// every nonzero node is above 2^-6 in magnitude, so its ulp is at least
// 2^-58) for the final sums, and as double-float pairs for the corrections.
constexpr int kPhaseTable = 256;

struct PhaseTable {
    longlong2* d;   // {sin, cos} 2^62
    float4* f;      // {sin.hi, sin.lo, cos.hi, cos.lo}
};

constexpr size_t kPhaseTableBytes = kPhaseTable * (sizeof(longlong2) + sizeof(float4));

__device__ __forceinline__ void fill_phase_table(PhaseTable tab) {
    for (int j = threadIdx.x; j < kPhaseTable; j += blockDim.x) {
        double s, c;
        sincospi(double(j) / (kPhaseTable / 2), &s, &c);
        const float sh = __double2float_rn(s), ch = __double2float_rn(c);
        tab.d[j] = make_longlong2(__double2ll_rn(s * 0x1p62), __double2ll_rn(c * 0x1p62));
        tab.f[j] = make_float4(sh, __double2float_rn(s - double(sh)), ch,
                               __double2float_rn(c - double(ch)));
    }
}

// sin(2 pi x), cos(2 pi x) for x in cycles, given F = frac(x) 2^64 (so that a
// caller may keep the 8-byte F and form sin/cos again later, on the integer
// and FP32 pipes only).  With x = j/256 + a/(2 pi):
//   sin = S_j + [S_j (cos a - 1) + C_j sin a],  cos = C_j + [C_j (cos a - 1) - S_j sin a],
// the brackets (|.| <= 0.013) in double-float; each node + bracket summed in
// 2^-62 fixed point (the bracket's two floats each rounded to 2^-63) and
// rounded once to a double: within 0.5 ulp + 2^-62 of node + bracket.  (A
// result below ~2^-40 in magnitude keeps its absolute, not its relative,
// accuracy.)
__device__ __forceinline__ void sincos_frac(uint64_t F, PhaseTable tab, double& sn, double& cs) {
    const uint64_t j = (F + (1ull << 55)) >> 56;                 // nearest table node
    const long long d = static_cast<long long>(F - (j << 56));   // |d| <= 2^55
    // d exactly as a sum of three floats, then to radians: a = 2 pi 2^-64 d
    const float d2 = float(int(d >> 32)) * 4294967296.0f;        // exact (|d>>32| <= 2^23)
    const unsigned dl = unsigned(d & 0xffffffffll);
    df dd = two_sum(d2, float(dl >> 8) * 256.0f);
    dd = df_add_f(dd, float(dl & 0xffu));
    const df k2pi = {6.28318548202514648e+00f * 5.42101086242752217e-20f,
                     -1.7484556025237907e-07f * 5.42101086242752217e-20f};   // 2 pi * 2^-64
    const df a = df_mul(dd, k2pi);
    const df a2 = df_mul(a, a);
    const float q = a2.hi;
    // sin a = a + a c,  c = -a^2/6 + a^4/120 - a^6/5040
    const df m6 = {-1.66666671633720398e-01f, 4.967053740534411e-09f};             // -1/6
    df c = df_mul(a2, m6);
    c = df_add_f(c, q * q * fmaf(-q, 1.0f / 5040.0f, 1.0f / 120.0f));
    const df sa = df_add(a, df_mul(a, c));
    // cos a - 1 = -a^2/2 + a^4/24 - a^6/720
    const df cm1 = df_add_f(df{-0.5f * a2.hi, -0.5f * a2.lo},
                            q * q * fmaf(-q, 1.0f / 720.0f, 1.0f / 24.0f));
    const int jj = int(j & (kPhaseTable - 1));
    const float4 t = tab.f[jj];
    const longlong2 td = tab.d[jj];
    const df S = {t.x, t.y}, C = {t.z, t.w};
    const df corr_s = df_add(df_mul(S, cm1), df_mul(C, sa));
    const df corr_c = df_add(df_mul(C, cm1), df_neg(df_mul(S, sa)));
    sn = fix62_to_double(td.x + f2fix62(corr_s.hi) + f2fix62(corr_s.lo));
    cs = fix62_to_double(td.y + f2fix62(corr_c.hi) + f2fix62(corr_c.lo));
}

// The same from the phase itself: F = frac(x) 2^64, then sincos_frac.
__device__ __forceinline__ void phase_sincos(double x, PhaseTable tab, double& sn, double& cs) {
    sincos_frac(frac_cycles_u64(x), tab, sn, cs);
}

// 1/S: a seed formed off the FP64 pipe, then one Newton-Raphson step in FP64
// (two FMAs).  S = m 2^E with m in [1, 2).  The seed is 1/m in double-float
// arithmetic on the FP32 pipe: the FP32 approximate reciprocal y0 of m's top
// 24 bits, then one Newton-Raphson step y0 + y0 (1 - m y0), with 1 - m y0
// formed from the FMA two-product of m's top bits and y0 (1 - m_hi y0 is
// exact by Sterbenz's lemma) and m's low bits' product; relative error about
// 2^-44.  The two floats are summed in 2^-62 fixed point and rounded once to
// a double on the integer pipe, and E goes into the exponent field.  The FP64
// step r = y (1 + e), e = 1 - S y, then leaves (1/S)(1 - e^2), e^2 < 2^-86:
// only the last rounding remains.  A seed below the normal range (S above
// 2^1022) is flushed to zero.  S zero, subnormal, infinite or NaN (never a
// valid innovation variance; the log-determinant flags it) takes the
// division.
// rcp_nr3 below is the short-latency form for the paths that are latency
// bound (the time-parallel scan, the joint filter's per-pulsar terms).
__device__ __forceinline__ double rcp_nr(double S) {
    const unsigned hs = unsigned(__double2hiint(S)), ls = unsigned(__double2loint(S));
    const int ef = int((hs >> 20) & 0x7ffu);
    if (ef == 0 || ef == 0x7ff) return 1.0 / S;
    // m = 1.f: its top 24 bits, and the other 29 rounded to a float
    const float mh = __uint_as_float(0x3f800000u | ((hs & 0x000fffffu) << 3) | (ls >> 29));
    const float ml = __uint2float_rn(ls & 0x1fffffffu) * 0x1p-52f;
    float y0;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(mh));
    const float ph = mh * y0;
    const float pl = fmaf(mh, y0, -ph);                       // mh y0 = ph + pl exactly
    const float e = fmaf(-ml, y0, (1.0f - ph) - pl);          // 1 - m y0
    const long long v = f2fix62(y0) + f2fix62(y0 * e);        // y0 + y0 e in 2^-62 fixed point
    const long long yb = __double_as_longlong(fix62_to_double(v));   // in (0.5, 1]: field 1022 or 1023
    const int fe = int((yb >> 52) & 0x7ff) - (ef - 1023);     // 2^-E
    const long long rb = fe > 0 ? (yb & 0x000fffffffffffffll) | (static_cast<long long>(fe) << 52) : 0ll;
    const double y = __longlong_as_double(rb | (static_cast<long long>(hs >> 31) << 63));
    const double r = fma(-S, y, 1.0);
    return fma(y, r, y);
}

// 1/S with a short dependency chain: the FP64 approximate reciprocal
// (measured within 2^-19.9) refined by one third-order step r (1 + e + e^2),
// e = 1 - S r, whose exact result is (1/S)(1 - e^3): three FMAs, for the
// paths where one thread's chain of steps, not the FP64 issue rate, sets the
// time.
__device__ __forceinline__ double rcp_nr3(double S) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(S));
    const double e = fma(-S, r, 1.0);
    return fma(r, fma(e, e, e), r);
}

// Running sum of ln S_k: a mantissa product kept in [1, 2) and an integer
// exponent, with one log per lane at the end.  S_k's own exponent goes to the
// integer first and only its mantissa m in [1, 2) is multiplied in, so the
// product (in [1, 4) before it is halved back) can neither overflow nor
// underflow for any normal S_k.  The product is a double-float (an unevaluated
// sum of two floats, as in the sin/cos above) on the FP32 pipe, not an FP64
// multiply: m enters as its top 24 significant bits plus its other 29 bits
// rounded to a float, and the product by the FMA two-product and the cross
// terms, so each step's relative error is below 2^-46 (over 10^5 TOAs at
// most ~1.4e-9 in the log-determinant, absolute).
struct LogProd {
    float ph = 1.0f, pl = 0.0f;   // the running product ph + pl, ph in [1, 2)
    int ex = 0;
    unsigned bad = 0u;   // set if some S_k was not a positive, normal, finite number
    __device__ __forceinline__ void add(double S) {
        const unsigned hs = unsigned(__double2hiint(S)), ls = unsigned(__double2loint(S));
        bad |= (hs - 0x00100000u) >= (0x7ff00000u - 0x00100000u) ? 1u : 0u;
        // m = 1.f, f the 52 fraction bits: 1 and f's top 23 bits, then f's low 29 bits
        const float mh = __uint_as_float(0x3f800000u | ((hs & 0x000fffffu) << 3) | (ls >> 29));
        const float ml = __uint2float_rn(ls & 0x1fffffffu) * 0x1p-52f;
        const float p = ph * mh;
        float e = fmaf(ph, mh, -p);
        e = fmaf(ph, ml, fmaf(pl, mh, e));
        const float sh = p + e;            // fast two-sum: |p| >= |e|
        const float sl = e - (sh - p);
        const int k = int(__float_as_uint(sh) >> 23) - 127;     // 0 or 1: sh in [1, 4)
        const float sc = __uint_as_float(unsigned(127 - k) << 23);   // 2^-k, exact scaling
        ph = sh * sc;
        pl = sl * sc;
        ex += int((hs >> 20) & 0x7ffu) - 1023 + k;
    }
    __device__ __forceinline__ double value() const {
        return log(double(ph) + double(pl)) + double(ex) * 0.69314718055994530942;
    }
};

}  // namespace argus
