// Device helpers shared by the stage kernels: fixed-point conversions, warp
// scans of 64-bit integers, and the exact cross-CTA prefix of tile sums.
//
// Why fixed point: GB300 executes FP64 at about 1/68 of its FP32 rate, while
// 64-bit integer adds run on the integer pipes.  A coupled quantity f (sin/cos
// of a phase, u/v, or V) is rounded once onto a grid of 2^-F, chosen so that one
// grid step is at most about one double ulp of f's typical magnitude.  From
// there on, every window sum is exact integer arithmetic: it does not depend on
// summation order, tile size or look-back timing, it has no cancellation error
// however far the prefix has grown (the "re-anchoring" the prefix-sum method
// needs in FP64), and it costs no FP64 instruction.  One correctly rounded
// conversion turns a window sum back into a double.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace simk {

typedef __int128 i128;
typedef unsigned __int128 u128;

// Device error word bits (mapped to sim_status on the host).
enum : unsigned { ERR_TIMEOUT = 1u, ERR_RANGE = 2u };

__device__ __forceinline__ void raise_error(unsigned *err, unsigned bit)
{
    atomicOr(err, bit);
}

// round(x * 2^F) as int64, ties away from zero.  Sets ok = false when x is not
// finite or |x| >= 2^lim (the range the caller's sums are sized for; lim + F
// must stay below 62).  Integer instructions only.
__device__ __forceinline__ int64_t to_fixed(double x, int F, int lim, bool &ok)
{
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FF);
    const uint64_t m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = e - 1075 + F; // x * 2^F = m * 2^sh
    uint64_t r;
    if (e == 0) {
        r = 0; // zero or subnormal: far below any grid step used here
    } else if (e - 1023 >= lim) {
        ok = false; // out of range, Inf or NaN
        r = 0;
    } else if (sh >= 0) {
        r = m << sh;
    } else {
        const int rs = -sh;
        r = rs > 53 ? 0ull : (m + (1ull << (rs - 1))) >> rs;
    }
    return (b >> 63) ? -(int64_t)r : (int64_t)r;
}

// Correctly rounded (to nearest, ties to even) double of x * 2^-F.
// Integer instructions only.
__device__ __forceinline__ double fixed_to_double(i128 x, int F)
{
    if (x == 0) return 0.0;
    uint64_t sign = 0;
    u128 u;
    if (x < 0) {
        sign = 1ull << 63;
        u = (u128)(-x);
    } else {
        u = (u128)x;
    }
    uint64_t hi = (uint64_t)(u >> 64), lo = (uint64_t)u;
    const int lz = hi ? __clzll((long long)hi) : 64 + __clzll((long long)lo);
    u <<= lz; // leading one at bit 127
    hi = (uint64_t)(u >> 64);
    lo = (uint64_t)u;
    uint64_t mant = hi >> 11; // 53 bits
    const uint64_t rbit = (hi >> 10) & 1ull;
    const bool sticky = ((hi & 0x3FFull) | lo) != 0;
    if (rbit && (sticky || (mant & 1ull))) mant += 1;
    int ex = 127 - lz - F;
    if (mant >> 53) {
        mant >>= 1;
        ex += 1;
    }
    const uint64_t bits = sign | ((uint64_t)(ex + 1023) << 52) | (mant & 0xFFFFFFFFFFFFFull);
    return __longlong_as_double((long long)bits);
}

// int64 version (no 128-bit shifts).
__device__ __forceinline__ double fixed_to_double(int64_t x, int F)
{
    if (x == 0) return 0.0;
    const uint64_t sign = (uint64_t)x & (1ull << 63);
    uint64_t u = x < 0 ? (uint64_t)(-x) : (uint64_t)x;
    const int lz = __clzll((long long)u);
    u <<= lz; // leading one at bit 63
    uint64_t mant = u >> 11;
    const uint64_t rbit = (u >> 10) & 1ull;
    const bool sticky = (u & 0x3FFull) != 0;
    if (rbit && (sticky || (mant & 1ull))) mant += 1;
    int ex = 63 - lz - F;
    if (mant >> 53) {
        mant >>= 1;
        ex += 1;
    }
    return __longlong_as_double((long long)(sign | ((uint64_t)(ex + 1023) << 52) | (mant & 0xFFFFFFFFFFFFFull)));
}

// Correctly rounded double of x * 2^-F for 128-bit x, with 64-bit shifts only.
__device__ __forceinline__ double fixed_to_double_wide(i128 x, int F)
{
    const int64_t hi_s = (int64_t)(x >> 64);
    const uint64_t lo_s = (uint64_t)x;
    if (hi_s == ((int64_t)lo_s >> 63)) return fixed_to_double((int64_t)lo_s, F); // fits in int64
    const uint64_t sign = (uint64_t)hi_s & (1ull << 63);
    const u128 ua = x < 0 ? (u128)(-x) : (u128)x; // |x| >= 2^63 here
    const uint64_t hi = (uint64_t)(ua >> 64), lo = (uint64_t)ua;
    int lz;
    uint64_t top; // the top 64 bits of |x|, leading one at bit 63
    bool low_rest;
    if (hi == 0) { // 2^63 <= |x| < 2^64
        lz = 64;
        top = lo;
        low_rest = false;
    } else {
        lz = __clzll((long long)hi);
        top = lz ? (hi << lz) | (lo >> (64 - lz)) : hi;
        low_rest = lz ? (lo << lz) != 0 : lo != 0;
    }
    uint64_t mant = top >> 11;
    const uint64_t rbit = (top >> 10) & 1ull;
    const bool sticky = ((top & 0x3FFull) != 0) || low_rest;
    if (rbit && (sticky || (mant & 1ull))) mant += 1;
    int ex = 127 - lz - F;
    if (mant >> 53) {
        mant >>= 1;
        ex += 1;
    }
    return __longlong_as_double((long long)(sign | ((uint64_t)(ex + 1023) << 52) | (mant & 0xFFFFFFFFFFFFFull)));
}

// Inclusive warp scan of int64 (Hillis-Steele over shuffles).
__device__ __forceinline__ int64_t warp_incl_scan(int64_t v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// ---------------------------------------------------------------------------
// Cross-CTA prefix without waiting: every CTA publishes its sub-tile totals,
// and the last CTA of the launch to finish (a monotonically increasing done
// counter, taken modulo the grid size, so it never needs resetting) scans
// them.  No CTA ever waits for another, so nothing can hang.

__device__ __forceinline__ i128 ld_cg_i128(const i128 *p)
{
    const longlong2 v = __ldcg(reinterpret_cast<const longlong2 *>(p));
    return (i128)(u128)(unsigned long long)v.x | ((i128)v.y << 64);
}

__device__ __forceinline__ i128 ld_cg(const int64_t *p) { return (i128)__ldcg(p); }
__device__ __forceinline__ i128 ld_cg(const i128 *p) { return ld_cg_i128(p); }

__device__ __forceinline__ void st_i128(i128 *p, i128 v)
{
    longlong2 w;
    w.x = (long long)(unsigned long long)(u128)v;
    w.y = (long long)(v >> 64);
    *reinterpret_cast<longlong2 *>(p) = w;
}

__device__ __forceinline__ i128 shfl_up_i128(i128 v, int o)
{
    const long long lo = (long long)(unsigned long long)(u128)v, hi = (long long)(v >> 64);
    const long long l2 = __shfl_up_sync(0xffffffffu, lo, o), h2 = __shfl_up_sync(0xffffffffu, hi, o);
    return (i128)(u128)(unsigned long long)l2 | ((i128)h2 << 64);
}

// Sum over the 32 lanes of a warp (every lane gets the total; exact).
__device__ __forceinline__ i128 warp_sum_i128(i128 v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long lo = (unsigned long long)(u128)v;
        const unsigned long long hi = (unsigned long long)(u128)(v >> 64);
        const unsigned long long l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        const unsigned long long h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        v += (i128)(((u128)h2 << 64) | (u128)l2);
    }
    return v;
}

// Called by every thread of one CTA (blockDim.x a multiple of 32).  Writes the
// exclusive prefix of in[0..n) to out[0..n] (out[n] = total) and returns the
// total.  in is read through L2 (it was written by other CTAs of this launch).
template <int E, typename T>
__device__ i128 block_exclusive_scan(const T *in, i128 *out, int64_t n)
{
    __shared__ i128 s_w[32];
    __shared__ i128 s_carry;
    const int t = threadIdx.x, nt = blockDim.x, lane = t & 31, warp = t >> 5, nw = nt >> 5;
    if (t == 0) s_carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < n; base += (int64_t)nt * E) {
        const int64_t b0 = base + (int64_t)t * E;
        i128 v[E];
        i128 run = 0;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            v[e] = (b0 + e < n) ? ld_cg(in + b0 + e) : (i128)0;
            run += v[e];
        }
        i128 x = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const i128 y = shfl_up_i128(x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_w[warp] = x;
        __syncthreads();
        if (warp == 0) {
            i128 w = lane < nw ? s_w[lane] : (i128)0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const i128 y = shfl_up_i128(w, o);
                if (lane >= o) w += y;
            }
            if (lane < nw) s_w[lane] = w;
        }
        __syncthreads();
        i128 acc = s_carry + (warp ? s_w[warp - 1] : (i128)0) + (x - run);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            if (b0 + e < n) st_i128(out + b0 + e, acc);
            acc += v[e];
        }
        __syncthreads();
        if (t == 0) s_carry += s_w[nw - 1];
        __syncthreads();
    }
    const i128 total = s_carry;
    if (t == 0) st_i128(out + n, total);
    return total;
}

// Called by one thread after it made its global writes visible (__threadfence).
// Returns true for the last of `count` arrivals on a monotonically increasing
// counter; the counter never needs resetting because every launch adds exactly
// `count` arrivals to it.
__device__ __forceinline__ bool last_arrival(unsigned long long *ctr, unsigned long long count)
{
    const unsigned long long done = atomicAdd(ctr, 1ull);
    const bool last = ((done + 1ull) % count) == 0ull;
    if (last) __threadfence();
    return last;
}

} // namespace simk
