// FP64 elementary functions with few FP64 instructions.
//
// GB300 issues FP64 arithmetic at 2 operations per clock per SM, while integer
// and FP32 instructions run at up to 64-128 per clock.  The routines below keep
// every FP64 instruction that the result's accuracy needs and move the rest
// (choosing the reduction integer, building doubles from integers, scaling by
// powers of two) to the integer and FP32 pipes.
//
// Methods (textbook, constants derived for this code from pi and ln 2 in
// 300-bit arithmetic):
//   sin/cos  Cody & Waite (1980) additive range reduction by pi/512 with a
//            three-part constant, then the angle-addition formula around a table
//            point j*pi/512 (the "accurate table" approach of Tang and Gal) with
//            Taylor polynomials for sin r and cos r - 1, |r| <= ~3 pi/1024.
//            13 FP64 instructions + one 16-byte table load.
//   exp      Tang (1989) table-driven method: x = (64 m + j) ln2/64 + r,
//            exp(x) = 2^m 2^(j/64) exp(r), degree-5 Taylor polynomial for
//            exp(r) - 1, |r| <= ~ln2/128.  8 FP64 instructions.
//   1/d      FP32 hardware reciprocal as the seed, then two Newton steps
//            y <- y + y (1 - d y) in FP64.  4 FP64 instructions, error <= 1 ulp.
// Accuracy (checked on the GPU against the C library, see the tests): within a
// few ulp over the argument ranges used here; arguments outside them fall back
// to the CUDA library routine.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace simk {

// Tables (host-filled at handle creation; see sim_api.cu).
constexpr int kSinTab = 1024;  // sin/cos(j pi/512), j in [0, 1024)
constexpr int kExpTab = 64;    // 2^(j/64), j in [0, 64)

struct MathTables {
    const double2 *sincos; // (sin, cos) of j*pi/512
    const double *exp2j;   // 2^(j/64)
};

// |x| as a float by truncating the mantissa (integer instructions; |x| must be
// inside the float exponent range, which every caller checks first).
__device__ __forceinline__ float dbl_to_flt_trunc(double x)
{
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const uint32_t hi = (uint32_t)(b >> 32);
    const int e = (int)((hi >> 20) & 0x7FF);
    if (e < 1023 - 126) return 0.0f;
    if (e > 1023 + 127) return __uint_as_float((hi & 0x80000000u) | 0x7F800000u); // Inf (also for NaN)
    const uint32_t mant = ((hi & 0xFFFFFu) << 3) | (uint32_t)((b >> 29) & 7u);
    return __uint_as_float((hi & 0x80000000u) | ((uint32_t)(e - 1023 + 127) << 23) | mant);
}

// Exact double of a 32-bit integer (integer instructions only).
__device__ __forceinline__ double int_to_dbl(int k)
{
    if (k == 0) return 0.0;
    const uint64_t sign = k < 0 ? (1ull << 63) : 0ull;
    const uint32_t a = (uint32_t)(k < 0 ? -k : k);
    const int lz = __clz((int)a);
    const uint64_t mant = ((uint64_t)a << (lz + 21)) & 0xFFFFFFFFFFFFFull; // drop the leading one
    const uint64_t ex = (uint64_t)(1023 + 31 - lz);
    return __longlong_as_double((long long)(sign | (ex << 52) | mant));
}

// Nearest integer to xf * scale in FP32 (1.5 * 2^23 rounding constant).
__device__ __forceinline__ int round_scaled(float xf, float scale)
{
    const float t = fmaf(xf, scale, 12582912.0f);
    return __float_as_int(t) - 0x4B400000;
}

// pi/512 = C1 + C2 + C3 to about 150 bits (C1, C2 rounded to 32 significant
// bits).  Each reduction step is one FMA, whose product is exact, so
// r = x - k pi/512 is accurate to about one ulp of r.
constexpr double kPio512_1 = 0x1.921fb544p-8;
constexpr double kPio512_2 = 0x1.0b4611a6p-42;
constexpr double kPio512_3 = 0x1.3198a2e037073p-77;
constexpr float k512oPi = 162.974655f;

__device__ __forceinline__ void fast_sincos(double x, const MathTables &T, double &s, double &c)
{
    const float xf = dbl_to_flt_trunc(x);
    if (!(fabsf(xf) < 16384.0f)) { // large, Inf or NaN: library routine
        sincos(x, &s, &c);
        return;
    }
    const int k = round_scaled(xf, k512oPi);
    const double dk = int_to_dbl(k);
    double r = fma(-dk, kPio512_1, x);
    r = fma(-dk, kPio512_2, r);
    r = fma(-dk, kPio512_3, r);
    const double z = r * r;
    // sin r = r + r^3 (-1/6 + r^2/120)           (|r| <= 0.01: next term < 2^-59 |r|)
    const double sr = fma(r * z, fma(z, 1.0 / 120.0, -1.0 / 6.0), r);
    // cos r - 1 = z (-1/2 + z (1/24 - z/720))
    const double cm1 = z * fma(z, fma(z, -1.0 / 720.0, 1.0 / 24.0), -0.5);
    const double2 t = __ldg(T.sincos + (k & (kSinTab - 1)));
    s = fma(t.x, cm1, fma(t.y, sr, t.x));
    c = fma(t.y, cm1, fma(-t.x, sr, t.y));
}

// ln2/64 = L1 + L2 + L3 (L1, L2 rounded to 32 significant bits; two parts are
// enough here because |k| < 2^16).
constexpr double kLn2o64_1 = 0x1.62e42ffp-7;
constexpr double kLn2o64_2 = -0x1.718432a2p-41;
constexpr double kLn2o64_3 = 0x1.3c7673007e5edp-75;
constexpr float k64oLn2 = 92.3324814f;

__device__ __forceinline__ double fast_exp(double x, const MathTables &T)
{
    const float xf = dbl_to_flt_trunc(x);
    if (!(fabsf(xf) < 700.0f)) return exp(x);
    const int k = round_scaled(xf, k64oLn2);
    const double dk = int_to_dbl(k);
    double r = fma(-dk, kLn2o64_1, x);
    r = fma(-dk, kLn2o64_2, r);
    // exp(r) - 1 = r + r^2 (1/2 + r (1/6 + r (1/24 + r/120)))   (|r| <= 0.0055)
    double q = fma(r, 1.0 / 120.0, 1.0 / 24.0);
    q = fma(r, q, 1.0 / 6.0);
    q = fma(r, q, 0.5);
    const double em1 = fma(r * r, q, r);
    const double tj = __ldg(T.exp2j + (k & (kExpTab - 1)));
    const double v = fma(tj, em1, tj);
    // times 2^m, m = floor(k / 64): add m to the exponent field
    const int m = k >> 6;
    return __longlong_as_double(__double_as_longlong(v) + ((long long)m << 52));
}

// 1/d for finite d with |d| in [2^-120, 2^120] (else the IEEE division).
__device__ __forceinline__ double fast_rcp(double d)
{
    const float df = dbl_to_flt_trunc(d);
    const float af = fabsf(df);
    if (!(af > 1e-36f && af < 1e36f)) return 1.0 / d;
    float yf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(df));
    // the seed as a double: float bits widened by integer instructions
    const uint32_t fb = __float_as_uint(yf);
    const uint64_t db = ((uint64_t)(fb & 0x80000000u) << 32) |
                        ((uint64_t)(((fb >> 23) & 0xFFu) - 127 + 1023) << 52) | ((uint64_t)(fb & 0x7FFFFFu) << 29);
    double y = __longlong_as_double((long long)db);
    double e = fma(-d, y, 1.0);
    y = fma(y, e, y);
    e = fma(-d, y, 1.0);
    return fma(y, e, y);
}

// x / (1 - exp(-x)), with its limit 1 at x = 0 (the Hodgkin-Huxley rate form).
// |x| < 0.1: the series 1 + x/2 + x^2/12 - x^4/720 + x^6/30240 - x^8/1209600
// (Bernoulli numbers; the next term is below 2^-58).  Otherwise x * (1/(1 - e^-x)).
__device__ __forceinline__ double fast_x_over_1mexp(double x, const MathTables &T)
{
    const float xf = dbl_to_flt_trunc(x);
    if (fabsf(xf) < 0.1f) {
        const double z = x * x;
        const double p = fma(z, fma(z, fma(z, -1.0 / 1209600.0, 1.0 / 30240.0), -1.0 / 720.0), 1.0 / 12.0);
        return fma(x, 0.5, fma(z, p, 1.0));
    }
    return x * fast_rcp(1.0 - fast_exp(-x, T));
}

} // namespace simk
