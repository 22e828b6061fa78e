// Elementary functions of the node right-hand sides with few FP64 instructions.
//
// GB300 retires about 2 FP64 lanes per clock per SM, against 64 lanes of 32-bit
// integer arithmetic and 128 of FP32.  The routines below keep every FP64
// instruction that the result's accuracy needs and move the rest to the
// integer and FP32 pipes; sin and cos need none at all.
//
// Methods (textbook; constants derived for this code from pi and ln 2 in
// high-precision arithmetic):
//   sin/cos  fixed_sincos, in 64-bit integer arithmetic only: additive range
//            reduction by pi/512 (Cody & Waite 1980) done exactly, as
//            t = |x| * 512/pi with 64 fractional bits from the 117-bit product of
//            x's significand and 512/pi rounded to 64 bits (relative error
//            2^-69.4); k = nearest integer to t, r = (t - k) pi/512 with
//            |r| <= pi/1024; Taylor polynomials sin r = r - r^3 (1/6 - r^2/120)
//            and cos r - 1 = -r^2/2 + r^4/24 (first omitted terms below 2^-70
//            and 2^-59); the angle-addition formula around the table point
//            j pi/512, j = k mod 1024 (the "accurate table" approach of Tang and
//            Gal): sin x = S_j + C_j sin r + S_j (cos r - 1) and
//            cos x = C_j - S_j sin r + C_j (cos r - 1), (S_j, C_j) rounded to
//            2^-62.  Every product is a signed 64 x 64 -> high-64 multiply on
//            scaled operands (each quantity's scale is in its name).  The result
//            is sin and cos on the grid 2^-62, within about 2^-59 of the true
//            values for |x| < 256 (a host model of the same integer steps was
//            checked against long double sinl/cosl over 2 * 10^7 arguments:
//            worst error 8.25 * 2^-62); that grid is what the exact window sums
//            consume.  |x| >= 256, Inf and NaN use the library routine.
//   exp      Tang (1989) table-driven method: x = (64 m + j) ln2/64 + r,
//            exp(x) = 2^m 2^(j/64) exp(r), degree-5 Taylor polynomial for
//            exp(r) - 1, |r| <= ~ln2/128.  8 FP64 instructions.
//   1/d      FP32 hardware reciprocal as the seed, then two Newton steps
//            y <- y + y (1 - d y) in FP64.  4 FP64 instructions, error <= 1 ulp.
// Accuracy is checked on the GPU against the C library (see the tests).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace simk {

// Tables (host-filled at handle creation; see sim_api.cu).
constexpr int kSinTab = 1024;  // sin/cos(j pi/512), j in [0, 1024)
constexpr int kExpTab = 64;    // 2^(j/64), j in [0, 64)

struct MathTables {
    const double2 *sincos;     // (sin, cos) of j*pi/512
    const double *exp2j;       // 2^(j/64)
    const longlong2 *sincos_q; // (sin, cos) of j*pi/512 rounded onto the grid 2^-62
};

// The tables as one block of 64-bit words (host-filled in long double, uploaded
// once per network or device): sincos (2 kSinTab doubles), exp2j (kExpTab
// doubles), sincos_q (2 kSinTab int64).
constexpr int kMathTableWords = 2 * kSinTab + kExpTab + 2 * kSinTab;
__host__ __device__ inline MathTables math_tables_at(const void *block)
{
    const double *d = static_cast<const double *>(block);
    return MathTables{reinterpret_cast<const double2 *>(d), d + 2 * kSinTab,
                      reinterpret_cast<const longlong2 *>(d + 2 * kSinTab + kExpTab)};
}

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

// Constants of fixed_sincos (derived from pi in 80-digit arithmetic).
constexpr uint64_t kPio512Inv56 = 0xa2f9836e4e44152aull; // round(512/pi * 2^56)
constexpr int64_t kPio512Q69 = 3622009729038561421ll;    // round(pi/512 * 2^69)
constexpr int64_t kSixthQ65 = 6148914691236517205ll;     // round(2^65 / 6)
constexpr int64_t kInv120Q55 = 300239975158033ll;        // round(2^55 / 120)
constexpr int64_t kInv24Q55 = 1501199875790165ll;        // round(2^55 / 24)

// sin x and cos x rounded onto the grid 2^-62 (s62, c62 in [-2^62, 2^62]).
// Integer instructions only on the fast path |x| < 256; beyond it, and for Inf
// and NaN, the library routine (ok = false for a non-finite x).
__device__ __forceinline__ void fixed_sincos(double x, const MathTables &T, int64_t &s62, int64_t &c62, bool &ok)
{
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FF);
    if (e >= 1023 + 8) {
        double s, c;
        sincos(x, &s, &c);
        s62 = to_fixed(s, 62, 1, ok);
        c62 = to_fixed(c, 62, 1, ok);
        return;
    }
    int64_t k = 0, f = 0; // x * 512/pi = k + f 2^-64
    if (e >= 1023 - 60) { // below that, x is 0 on this grid
        const uint64_t m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
        const uint64_t lo = m * kPio512Inv56, hi = __umul64hi(m, kPio512Inv56);
        const int sh = 1067 - e; // the product times 2^-sh has 64 fractional bits; sh in [37, 104]
        uint64_t th, tl;
        if (sh < 64) {
            th = hi >> sh;
            tl = (lo >> sh) | (hi << (64 - sh));
        } else {
            th = 0;
            tl = hi >> (sh - 64);
        }
        if (b >> 63) { // negative x: negate the 128-bit value
            tl = ~tl + 1ull;
            th = ~th + (tl == 0ull ? 1ull : 0ull);
        }
        k = (int64_t)th + (int64_t)(tl >> 63); // round to the nearest integer
        f = (int64_t)tl;                       // t - k in [-1/2, 1/2) times 2^64
    }
    const int64_t r69 = __mul64hi(f, kPio512Q69);               // r 2^69
    const int64_t z74 = __mul64hi(r69, r69);                    // r^2 2^74
    const int64_t u65 = kSixthQ65 - __mul64hi(z74, kInv120Q55); // (1/6 - r^2/120) 2^65
    const int64_t v79 = __mul64hi(r69, z74);                    // r^3 2^79
    const int64_t sr69 = r69 - (__mul64hi(v79, u65) >> 11);    // sin r 2^69
    const int64_t zz84 = __mul64hi(z74, z74);                   // r^4 2^84
    const int64_t cm75 = __mul64hi(zz84, kInv24Q55) - z74;      // (cos r - 1) 2^75
    const longlong2 t = __ldg(T.sincos_q + (k & (kSinTab - 1)));
    s62 = t.x + (__mul64hi(t.y, sr69) >> 5) + (__mul64hi(t.x, cm75) >> 11);
    c62 = t.y - (__mul64hi(t.x, sr69) >> 5) + (__mul64hi(t.y, cm75) >> 11);
}

// v 2^-62 rounded onto the coarser grid 2^-F (F <= 61), half up.
__device__ __forceinline__ int64_t q62_to(int64_t v, int F)
{
    const int sh = 62 - F;
    return (v + (1ll << (sh - 1))) >> sh;
}

// sin and cos as doubles, correctly rounded from fixed_sincos's values on the
// grid 2^-62 (NaN for an infinite or NaN x).
__device__ __forceinline__ void fast_sincos(double x, const MathTables &T, double &s, double &c)
{
    int64_t s62, c62;
    bool ok = true;
    fixed_sincos(x, T, s62, c62, ok);
    if (!ok) {
        s = c = x - x;
        return;
    }
    s = fixed_to_double(s62, 62);
    c = fixed_to_double(c62, 62);
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
