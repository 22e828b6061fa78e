// Device helpers shared by the stage kernels: fixed-point conversions, warp
// scans of 64-bit integers, and the single-pass decoupled look-back over exact
// 128-bit tile sums (Merrill & Garland, "Single-pass Parallel Prefix Scan with
// Decoupled Look-back", NVIDIA TR 2016).
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

// Bound on spin iterations of any cross-CTA wait (~1 s with the back-off).
constexpr int kSpinLimit = 1 << 22;

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

__device__ __forceinline__ double fixed_to_double(int64_t x, int F)
{
    return fixed_to_double((i128)x, F);
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
// Decoupled look-back over CTA tiles with exact 128-bit payloads.
//
// Tickets: every CTA of a launch draws ticket = atomicAdd(counter, 1); with
// exactly nctas CTAs per launch, tile = ticket % nctas and the launch epoch is
// ticket / nctas + 1.  Tiles are therefore processed in ticket order (a CTA only
// waits for tiles whose CTAs have already started), and flags carry the epoch,
// so the slots never need resetting between launches.
struct LookbackSlot {
    unsigned long long flag; // epoch * 4 + status (1 = aggregate, 2 = inclusive)
    unsigned long long pad;
    i128 agg[2];
    i128 inc[2];
};

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ i128 ld_cg_i128(const i128 *p)
{
    const longlong2 v = __ldcg(reinterpret_cast<const longlong2 *>(p));
    return (i128)(u128)(unsigned long long)v.x | ((i128)v.y << 64);
}

__device__ __forceinline__ void st_i128(i128 *p, i128 v)
{
    longlong2 w;
    w.x = (long long)(unsigned long long)(u128)v;
    w.y = (long long)(v >> 64);
    *reinterpret_cast<longlong2 *>(p) = w;
}

// Called by one thread.  Publishes this tile's aggregate, looks back for the
// exclusive prefix, publishes the inclusive prefix, and returns the exclusive
// prefix in excl[0..NQ).  On a wait that exceeds kSpinLimit it raises
// ERR_TIMEOUT and carries on with what it has (results are then invalid, but
// every CTA terminates).
template <int NQ>
__device__ void lookback(LookbackSlot *slots, long long tile, unsigned long long epoch,
                         const i128 (&agg)[NQ], i128 (&excl)[NQ], unsigned *err)
{
#pragma unroll
    for (int c = 0; c < NQ; ++c) excl[c] = 0;
    LookbackSlot *me = slots + tile;
    if (tile > 0) {
#pragma unroll
        for (int c = 0; c < NQ; ++c) st_i128(&me->agg[c], agg[c]);
        __threadfence();
        st_release(&me->flag, epoch * 4ull + 1ull);
        for (long long p = tile - 1; p >= 0; --p) {
            const LookbackSlot *s = slots + p;
            unsigned long long f = ld_acquire(&s->flag);
            int spins = 0;
            while ((f >> 2) != epoch || (f & 3ull) == 0ull) {
                if (++spins > kSpinLimit) {
                    raise_error(err, ERR_TIMEOUT);
                    break;
                }
                __nanosleep(spins < 64 ? 20 : 200);
                f = ld_acquire(&s->flag);
            }
            if ((f >> 2) != epoch) break; // timed out
            if ((f & 3ull) == 2ull) {
#pragma unroll
                for (int c = 0; c < NQ; ++c) excl[c] += ld_cg_i128(&s->inc[c]);
                break;
            }
#pragma unroll
            for (int c = 0; c < NQ; ++c) excl[c] += ld_cg_i128(&s->agg[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < NQ; ++c) st_i128(&me->inc[c], excl[c] + agg[c]);
    __threadfence();
    st_release(&me->flag, epoch * 4ull + 2ull);
}

} // namespace simk
