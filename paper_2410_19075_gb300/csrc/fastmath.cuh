// Elementary functions of the node right-hand sides with few FP64 instructions.
//
// GB300 retires about 2 FP64 lanes per clock per SM, against 64 lanes of 32-bit
// integer arithmetic and 128 of FP32.  The routines below keep every FP64
// instruction that the result's accuracy needs and move the rest to the
// integer and FP32 pipes; sin and cos need none at all.
//
// Methods (textbook; constants derived for this code from pi and ln 2 in
// high-precision arithmetic):
//   sin/cos  fixed_sincos, in integer arithmetic only: additive range
//            reduction by pi/512 (Cody & Waite 1980), t = |x| * 512/pi from one
//            unsigned 64 x 64 high product of |x| 2^55 and 512/pi 2^56 (grid
//            2^-47); k = nearest integer to t, r = (t - k) pi/512 with
//            |r| <= pi/1024; Taylor polynomials sin r = r - r^3 (1/6 - r^2/120)
//            and cos r - 1 = -r^2/2 + r^4/24 (first omitted terms below 2^-73
//            and 2^-59), whose small terms take 32 x 32 products; the
//            angle-addition formula around the table point j pi/512,
//            j = k mod 1024 (the "accurate table" approach of Tang and Gal):
//            sin x = S_j + C_j sin r + S_j (cos r - 1) and
//            cos x = C_j - S_j sin r + C_j (cos r - 1), (S_j, C_j) rounded to
//            2^-62.  The result is sin and cos on the grid 2^-62 within 2^-53.4
//            of the true values for |x| < 256 (a host model of the same integer
//            steps was checked against long double sinl/cosl over 2 * 10^7
//            arguments and every reduction edge: worst error 7.7e-17, set by the
//            grid 2^-47 of t); that grid is what the exact window sums consume.
//            |x| >= 256, Inf and NaN use the library routine.
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

// Constants of fixed_sincos (derived from pi in 60-digit arithmetic).
constexpr uint64_t kPio512Inv56 = 0xa2f9836e4e44152aull; // round(512/pi * 2^56)
constexpr uint64_t kPio512Q71 = 0xc90fdaa22168c235ull;   // round(pi/512 * 2^71)
constexpr uint32_t kSixthQ34 = 2863311531u;               // round(2^34 / 6)
constexpr uint32_t kInv120Q32 = 35791394u;                // round(2^32 / 120)
constexpr uint32_t kInv24Q36 = 2863311531u;               // round(2^36 / 24)

// floor(a b / 2^64) for signed a and unsigned b: the unsigned high product of
// a's two's-complement bits, less b when a is negative.
__device__ __forceinline__ int64_t mulhi_su(int64_t a, uint64_t b)
{
    return (int64_t)(__umul64hi((uint64_t)a, b) - (a < 0 ? b : 0ull));
}

// floor(a b / 2^64) for signed a and b, from the unsigned high product.
__device__ __forceinline__ int64_t mulhi_ss(int64_t a, int64_t b)
{
    uint64_t h = __umul64hi((uint64_t)a, (uint64_t)b);
    h -= a < 0 ? (uint64_t)b : 0ull;
    h -= b < 0 ? (uint64_t)a : 0ull;
    return (int64_t)h;
}

// sin x and cos x on the grid 2^-62 (s62, c62 in [-2^62, 2^62]), absolute
// error below 2^-53.4.  Integer instructions only on the fast path |x| < 256;
// beyond it, and for Inf and NaN, the library routine (ok = false for a
// non-finite x).  Every 64 x 64 product is unsigned (on GB300 the signed
// high product costs about 1.7 unsigned ones):
//   X = |x| 2^55 (truncated), t = X (512/pi) 2^-64 on the grid 2^-47,
//   k = nearest integer to t, f = t - k in [-1/2, 1/2), r = f pi/512;
//   sin|r| = |r| - |r|^3 (1/6 - r^2/120) and 1 - cos r = r^2/2 - r^4/24, the
//   small terms from 32 x 32 products of the top words;
//   the angle-addition formula around the table point j pi/512, j = k mod 1024:
//   sin = S_j - S_j (1 - cos r) + C_j sin r, cos = C_j - C_j (1 - cos r) - S_j sin r.
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
    const uint64_t m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const uint64_t X = e >= 1020 ? m << (e - 1020) : m >> min(1020 - e, 63); // |x| 2^55 < 2^63
    const uint64_t t = __umul64hi(X, kPio512Inv56);                          // |x| 512/pi 2^47
    const uint64_t k = (t + (1ull << 46)) >> 47;
    const int64_t f47 = (int64_t)(t - (k << 47)); // f 2^47, |f| <= 1/2
    const bool rneg = f47 < 0;
    const uint64_t R = __umul64hi((uint64_t)(rneg ? -f47 : f47) << 17, kPio512Q71); // |r| 2^71
    const uint64_t z = __umul64hi(R, R);                                             // r^2 2^78
    const uint32_t zh = (uint32_t)(z >> 32);                                         // r^2 2^46
    const uint32_t v57 = (uint32_t)(((uint64_t)(uint32_t)(R >> 32) * zh) >> 28);    // |r|^3 2^57
    const uint32_t u34 = kSixthQ34 - __umulhi((uint32_t)(z >> 44), kInv120Q32);     // (1/6 - r^2/120) 2^34
    const uint64_t sr = (R >> 7) - (((uint64_t)v57 * u34) >> 27);                   // sin|r| 2^64
    const uint32_t w = (uint32_t)(((uint64_t)zh * zh) >> 32);                       // r^4 2^60
    const uint64_t cm = (z >> 15) - (((uint64_t)w * kInv24Q36) >> 32);              // (1 - cos r) 2^64
    const longlong2 tq = __ldg(T.sincos_q + (k & (kSinTab - 1)));                   // (S_j, C_j) 2^62
    const int64_t p1 = mulhi_su(tq.y, sr), p3 = mulhi_su(tq.x, sr);
    const int64_t s = tq.x - mulhi_su(tq.x, cm) + (rneg ? -p1 : p1);
    const int64_t c = tq.y - mulhi_su(tq.y, cm) - (rneg ? -p3 : p3);
    s62 = (b >> 63) ? -s : s;
    c62 = c;
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
