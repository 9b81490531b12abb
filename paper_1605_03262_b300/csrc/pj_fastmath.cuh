// FP64 exp and log with fewer FP64-pipe operations than the library versions, for a GPU whose FP64
// rate is the binding limit. Both follow P. T. P. Tang's table-driven methods, written here from
// the methods' description:
//   exp: "Table-driven implementation of the exponential function in IEEE floating-point
//        arithmetic", ACM TOMS 15(2), 1989. x = (512 m + j) ln2/512 + r with |r| <= ln2/1024;
//        exp(x) = 2^m 2^(j/512) exp(r), exp(r) - 1 by a degree-4 polynomial.
//   log: "Table-driven implementation of the logarithm function in IEEE floating-point
//        arithmetic", ACM TOMS 16(4), 1990. x = 2^m y, F = 1 + j/256 nearest to y,
//        log x = m ln2 + log F + log(1 + (y - F)/F), the last by a degree-6 polynomial; the leading
//        parts of m ln2 and log F are rounded to multiples of 2^-42 so that their sum is exact.
// The tables and split constants are computed on the host in long double (build_math_tables).
// Arguments outside the fast range (non-finite values, |x| > 700 for exp, non-positive or subnormal
// values for log) go to the CUDA library functions. Accuracy against CUDA's exp/log is checked by
// the test suite.
#pragma once

#ifndef __CUDACC_RTC__
#include <cmath>
#include <cstdint>
#endif

namespace pj {

constexpr int kExpTableSize = 512;   // 2^(j/512), j = 0..511
constexpr int kLogTableSize = 257;   // F = 1 + j/256, j = 0..256

struct MathTables {
    double exp2j[kExpTableSize];
    double logF_hi[kLogTableSize];   // log F rounded to a multiple of 2^-42
    double logF_lo[kLogTableSize];   // log F - logF_hi
    double invF[kLogTableSize];      // 1/F rounded
    double exp_invL;                 // 512 / ln 2
    double exp_L1;                   // ln2/512 with its low bits cleared (exact k * L1 for |k| < 2^20)
    double exp_L2;                   // ln2/512 - exp_L1
    double ln2_hi;                   // ln 2 rounded to a multiple of 2^-42
    double ln2_lo;                   // ln 2 - ln2_hi
    double pad;
};

#ifndef __CUDACC_RTC__
inline void build_math_tables(MathTables &t) {
    const long double ln2 = logl(2.0L);
    for (int j = 0; j < kExpTableSize; ++j) t.exp2j[j] = double(exp2l((long double)j / 512.0L));
    const long double q42 = ldexpl(1.0L, 42);
    for (int j = 0; j < kLogTableSize; ++j) {
        const long double F = 1.0L + (long double)j / 256.0L;
        const long double lf = logl(F);
        const long double hi = roundl(lf * q42) / q42;
        t.logF_hi[j] = double(hi);
        t.logF_lo[j] = double(lf - hi);
        t.invF[j] = double(1.0L / F);
    }
    const long double L = ln2 / 512.0L;
    t.exp_invL = double(1.0L / L);
    const long double q = ldexpl(1.0L, 42);            // L < 2^-9: 33 significant bits, k * L1 exact for |k| < 2^20
    const long double l1 = roundl(L * q) / q;
    t.exp_L1 = double(l1);
    t.exp_L2 = double(L - l1);
    const long double h = roundl(ln2 * q42) / q42;
    t.ln2_hi = double(h);
    t.ln2_lo = double(ln2 - h);
    t.pad = 0.0;
}
#endif

#ifdef __CUDACC__

// exp(x): 9 FP64 operations on |x| <= 700.
__device__ __forceinline__ double fast_exp(double x, const MathTables *__restrict__ tb) {
    const int hi = __double2hiint(x) & 0x7fffffff;
    if (hi >= 0x4085e000) return exp(x);           // |x| >= 700, inf or NaN: library path
    constexpr double kShift = 6755399441055744.0;  // 1.5 * 2^52: x * 512/ln2 + kShift rounds to an integer
    const double t = fma(x, __ldg(&tb->exp_invL), kShift);
    const int k = __double2loint(t);
    const double kd = t - kShift;
    double r = fma(-kd, __ldg(&tb->exp_L1), x);
    r = fma(-kd, __ldg(&tb->exp_L2), r);
    // exp(r) - 1, |r| <= 6.8e-4: the r^5 term is below 2e-18
    double q = fma(r, 1.0 / 24.0, 1.0 / 6.0);
    q = fma(q, r, 0.5);
    const double p = fma(q, r * r, r);
    const double tj = __ldg(&tb->exp2j[k & (kExpTableSize - 1)]);
    const double v = fma(tj, p, tj);               // 2^(j/512) exp(r), in [1, 2.01)
    const long long m = static_cast<long long>(k >> 9);
    return __longlong_as_double(__double_as_longlong(v) + (m << 52));
}

// log(x): 12 FP64 operations on positive normal finite x.
__device__ __forceinline__ double fast_log(double x, const MathTables *__restrict__ tb) {
    const long long bits = __double_as_longlong(x);
    const int hi = static_cast<int>(bits >> 32);
    if (hi < 0x00100000 || hi >= 0x7ff00000) return log(x);   // zero, negative, subnormal, inf, NaN
    const int m = (hi >> 20) - 1023;
    const long long mant = bits & 0x000fffffffffffffLL;
    const double y = __longlong_as_double(mant | 0x3ff0000000000000LL);      // in [1, 2)
    const int j = static_cast<int>(((mant >> 43) + 1) >> 1);                 // nearest 1/256 step, 0..256
    const double F = __longlong_as_double(0x3ff0000000000000LL + (static_cast<long long>(j) << 44));
    const double u = (y - F) * __ldg(&tb->invF[j]);                          // y - F exact, |u| <= 1/512
    // log(1 + u), |u| <= 1.96e-3: the u^7 term is below 1e-20
    double q = fma(u, -1.0 / 6.0, 0.2);
    q = fma(q, u, -0.25);
    q = fma(q, u, 1.0 / 3.0);
    q = fma(q, u, -0.5);
    const double poly = fma(q, u * u, u);
    const double md = static_cast<double>(m);
    const double lead = fma(md, __ldg(&tb->ln2_hi), __ldg(&tb->logF_hi[j]));   // exact
    const double trail = fma(md, __ldg(&tb->ln2_lo), __ldg(&tb->logF_lo[j])) + poly;
    return lead + trail;
}

#endif

}  // namespace pj
