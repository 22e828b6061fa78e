// Building blocks of the ring stage kernels (RK4 in ring.cu, Dormand-Prince in
// dp5.cu): one CTA works on one 256-node sub-tile of a ring.
//
//   ring_load_bases   per-CTA window bases: the exact prefix at the start of
//                     every piece (split at sub-tile starts and at N) that the
//                     window ends of this CTA's nodes fall in;
//   ring_window       one node's exact window sums W = P(i+R+1) - P(i-R) and its
//                     own fixed-point coupled quantity, from the prefix arrays the
//                     previous kernel wrote (two shifted in-sub-tile reads);
//   ring_prefix_tail  the exact prefix of the next coupled quantity inside the
//                     sub-tile and, without any CTA waiting for another, at every
//                     sub-tile start: the last CTA to finish in each group of 64
//                     sub-tiles scans that group, and the last group scans the
//                     groups (and may record the Kuramoto order parameter);
//   one-pass prefix   (RingPlan::flat, the plain RK4 kernels of rings of at most
//                     128 groups) no scan at the end of a launch at all: each CTA
//                     stores its sub-tile total and adds its 18-bit chunks into
//                     its group's 32-bit accumulators; two warps of each CTA of
//                     the next launch sum the group totals and the sub-tile
//                     totals in front of its window ends (ring_flat_bases).  The last CTA of a launch
//                     used to run two dependent scans after everyone else had
//                     finished, about 4 us each on GB300;
//   stage_body        one fused RK4 stage around a gather of the window sums
//                     (ring windows here, general link matrices in graph.cu).
#pragma once
#include "internal.h"

namespace simk {

__device__ __forceinline__ i128 ldg_i128(const i128 *p)
{
    const longlong2 v = __ldg(reinterpret_cast<const longlong2 *>(p));
    return (i128)(u128)(unsigned long long)v.x | ((i128)v.y << 64);
}

__device__ __forceinline__ i128 warp_incl_scan_i128(i128 v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const i128 t = shfl_up_i128(v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Resident CTAs per SM the register allocation is sized for (256 threads each).
#ifndef SIM_RING_MIN_BLOCKS
#define SIM_RING_MIN_BLOCKS 5
#endif
template <int M> struct MinBlocks { static constexpr int value = SIM_RING_MIN_BLOCKS; };
template <> struct MinBlocks<2> { static constexpr int value = 2; };

// Window bases of one CTA: the right ends b = i+R+1 (side 0) and left ends
// a = i-R (side 1) of its nodes are consecutive, and each side covers at most
// three pieces (split at a sub-tile start and at N).  Per piece: its first
// position on the periodic extension, the multiple of N to subtract, and the
// exact prefix at its sub-tile's start (+ q * total).  Then every node needs one
// in-sub-tile prefix load per end.
template <int NQ> struct RingBases {
    i128 base[2][3][NQ];
    int64_t start[2][3], qn[2][3];
};

// Threads 0 and 1 write the bases; the caller makes them visible with a barrier.
template <int NQ>
__device__ __forceinline__ void ring_compute_bases(const RingPlan &P, const i128 *ingrp_in, const i128 *grpofs_in,
                                                   int64_t sub, RingBases<NQ> &B)
{
    const int tid = threadIdx.x;
    const int64_t N = P.N, nsub = P.nsub, ngroups = P.ngroups;
    if (tid < 2) {
        const int side = tid;
        const int64_t nvalid = N - sub * kSubTile < kSubTile ? N - sub * kSubTile : kSubTile;
        const int64_t p0 = side == 0 ? sub * kSubTile + P.R + 1 : sub * kSubTile - P.R;
        const int64_t p1 = p0 + nvalid - 1; // in [-N, 2N)
        int64_t p = p0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (p > p1) {
                B.start[side][k] = INT64_MAX;
                B.qn[side][k] = 0;
                continue;
            }
            const int q = p < 0 ? -1 : (p >= N ? 1 : 0);
            const int64_t qn = q * N, pp = p - qn;
            const int64_t st = pp >> kSubLog2;
            int64_t end = ((st + 1) << kSubLog2) - 1;
            if (end > N - 1) end = N - 1;
#pragma unroll
            for (int c = 0; c < NQ; ++c) {
                const i128 *grpofs = grpofs_in + c * (ngroups + 1);
                const i128 tot = ldg_i128(grpofs + ngroups);
                B.base[side][k][c] = ldg_i128(grpofs + (st >> kGroupLog2)) + ldg_i128(ingrp_in + c * nsub + st) +
                                     (q < 0 ? -tot : (q > 0 ? tot : (i128)0));
            }
            B.start[side][k] = p;
            B.qn[side][k] = qn;
            p = end + qn + 1;
        }
    }
}

// Chunks of a sub-tile total (|t| < 2^62) for the one-pass accumulators:
// t = c0 + c1 2^18 + c2 2^36 + c3 2^54 with c0..c2 in [0, 2^18) and
// c3 = floor(t / 2^54) in [-2^8, 2^8).  Over at most 8192 sub-tiles every chunk
// sum stays below 2^31, so 32-bit words hold them exactly.
__device__ __forceinline__ unsigned flat_chunk(int64_t t, int k)
{
    return k < 3 ? (unsigned)((t >> (18 * k)) & 0x3ffff) : (unsigned)(int)(t >> 54);
}

// The exact value of four chunk sums (the last one signed).
__device__ __forceinline__ i128 flat_value(unsigned s0, unsigned s1, unsigned s2, unsigned s3)
{
    return (i128)s0 + ((i128)s1 << 18) + ((i128)s2 << 36) + ((i128)(int)s3 << 54);
}

// Per-lane chunk sums of group g: all groups into tk, those in front of group
// g0 into pk.
__device__ __forceinline__ void flat_group_add(const unsigned *acc, int g, int g0, unsigned (&pk)[4], unsigned (&tk)[4])
{
    const uint4 a = __ldg(reinterpret_cast<const uint4 *>(acc) + g);
    const unsigned m = g < g0 ? 0xffffffffu : 0u;
    tk[0] += a.x;
    tk[1] += a.y;
    tk[2] += a.z;
    tk[3] += a.w;
    pk[0] += a.x & m;
    pk[1] += a.y & m;
    pk[2] += a.z & m;
    pk[3] += a.w & m;
}

// One-pass window bases (RingPlan::flat), the counterpart of ring_compute_bases:
// warp `side` (0, 1) finds the exact prefix at the start of its first piece's
// sub-tile st0 as the group totals in front of st0's group plus the sub-tile
// totals in front of st0 inside that group, and the ring total: every lane adds
// the chunks of up to four groups and two sub-tiles, and each chunk sum is one
// redux.sync over the warp.  A later piece starts one sub-tile on (its prefix
// grows by that sub-tile's total) or at sub-tile 0 of the next copy of the ring
// (prefix 0).  These rings have at most 2^21 nodes, so positions and indices
// are 32-bit.  Lane 0 writes the bases; the caller's barrier makes them visible.
template <int NQ>
__device__ __forceinline__ void ring_flat_bases(const RingPlan &P, const int64_t *fsub_in, const unsigned *facc_in,
                                                int64_t sub, RingBases<NQ> &B)
{
    const int lane = threadIdx.x & 31, side = threadIdx.x >> 5;
    if (side > 1) return;
    const int N = (int)P.N, R = (int)P.R, ngroups = (int)P.ngroups, nsub = (int)P.nsub;
    const int s0 = (int)sub * kSubTile;
    const int nvalid = N - s0 < kSubTile ? N - s0 : kSubTile;
    const int p0 = side == 0 ? s0 + R + 1 : s0 - R; // in [-N, 2N)
    const int p1 = p0 + nvalid - 1;
    // the pieces, split at sub-tile starts and at 0 and N (as in ring_compute_bases)
    int start[3], st[3], q[3];
    bool have[3];
    int p = p0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        have[k] = p <= p1;
        const int qq = p < 0 ? -1 : (p >= N ? 1 : 0);
        const int sp = (p - qq * N) >> kSubLog2;
        start[k] = p;
        st[k] = sp;
        q[k] = qq;
        int end = ((sp + 1) << kSubLog2) - 1;
        end = end > N - 1 ? N - 1 : end;
        p = end + qq * N + 1;
    }
    const int g0 = st[0] >> kGroupLog2;
#pragma unroll
    for (int c = 0; c < NQ; ++c) {
        const unsigned *acc = facc_in + c * ngroups * 4;
        const int64_t *fs = fsub_in + c * nsub;
        // the totals of the sub-tiles the later pieces follow (broadcast loads)
        const int64_t f0 = have[1] ? __ldg(fs + st[0]) : 0, f1 = have[2] ? __ldg(fs + st[1]) : 0;
        unsigned pk[4] = {0, 0, 0, 0}, tk[4] = {0, 0, 0, 0};
        // groups lane and lane + 32 with the sub-tiles of the same offsets in
        // st0's group (this fixed, interleaved form measured fastest), then
        // groups 64..127 on rings that have them
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int g = lane + 32 * e;
            if (g < ngroups) flat_group_add(acc, g, g0, pk, tk);
            const int sp = (g0 << kGroupLog2) + g;
            if (sp < st[0]) {
                const int64_t t = __ldg(fs + sp);
#pragma unroll
                for (int k = 0; k < 4; ++k) pk[k] += flat_chunk(t, k);
            }
        }
        if (ngroups > 64) {
#pragma unroll
            for (int e = 2; e < kFlatMaxGroups / 32; ++e) {
                const int g = lane + 32 * e;
                if (g < ngroups) flat_group_add(acc, g, g0, pk, tk);
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            pk[k] = __reduce_add_sync(0xffffffffu, pk[k]);
            tk[k] = __reduce_add_sync(0xffffffffu, tk[k]);
        }
        if (lane == 0) {
            const i128 T = flat_value(tk[0], tk[1], tk[2], tk[3]);
            i128 pre = flat_value(pk[0], pk[1], pk[2], pk[3]); // exact prefix at the start of st[k]
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                if (!have[k]) break;
                if (k > 0) pre = st[k] == 0 ? (i128)0 : pre + (i128)(k == 1 ? f0 : f1);
                B.base[side][k][c] = pre + (q[k] < 0 ? -T : (q[k] > 0 ? T : (i128)0));
            }
        }
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            B.start[side][k] = have[k] ? (int64_t)start[k] : INT64_MAX;
            B.qn[side][k] = have[k] ? (int64_t)q[k] * N : 0;
        }
    }
}

// Called by every thread of the CTA (contains a __syncthreads).
template <int NQ>
__device__ __forceinline__ void ring_load_bases(const RingPlan &P, const i128 *ingrp_in, const i128 *grpofs_in,
                                                int64_t sub, RingBases<NQ> &B)
{
    ring_compute_bases<NQ>(P, ingrp_in, grpofs_in, sub, B);
    __syncthreads();
}

// Node i (position tid in its sub-tile): its own coupled quantity (fixed point
// qo and its double fo) and the exact window sums W of every coupled quantity.
template <int NQ>
__device__ __forceinline__ void ring_window(const RingPlan &P, const int64_t *lam_in, const RingBases<NQ> &B, int tid,
                                            int64_t i, int64_t (&qo)[NQ], double (&fo)[NQ], i128 (&W)[NQ])
{
    const int64_t N = P.N;
    const int64_t b = i + P.R + 1, am = i - P.R;
    const int kb = (b >= B.start[0][1]) + (b >= B.start[0][2]);
    const int ka = (am >= B.start[1][1]) + (am >= B.start[1][2]);
    const int64_t bp = b - B.qn[0][kb], ap = am - B.qn[1][ka];
#pragma unroll
    for (int c = 0; c < NQ; ++c) {
        const int64_t *lam = lam_in + c * N;
        const int64_t l = __ldg(lam + i);
        qo[c] = tid ? l - __ldg(lam + i - 1) : l;
        fo[c] = fixed_to_double(qo[c], P.F);
        const int64_t lb = (bp & (kSubTile - 1)) ? __ldg(lam + bp - 1) : 0;
        const int64_t la = (ap & (kSubTile - 1)) ? __ldg(lam + ap - 1) : 0;
        W[c] = (B.base[0][kb][c] - B.base[1][ka][c]) + (i128)(lb - la);
    }
}

// Exact prefix of the fixed-point values qv (one per node, 0 past the ring's
// end) into lam_out / ingrp_out / grpofs_out.  RECORD: the last CTA records the
// Kuramoto order parameter from the totals (if P.obs is set); DEC_STEPS: it also
// decrements the step budget.  Called by every thread of the CTA.
template <int NQ, bool RECORD, bool DEC_STEPS>
__device__ __forceinline__ void ring_prefix_tail(const RingPlan &P, int64_t *lam_out, i128 *ingrp_out,
                                                 i128 *grpofs_out, int64_t sub, int64_t i, int64_t (&qv)[NQ])
{
    constexpr int NW = kRingThreads / 32;
    __shared__ int64_t s_wtot[NW][NQ];
    __shared__ int s_last;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t N = P.N, nsub = P.nsub, ngroups = P.ngroups;

    // Exact inclusive prefix inside the sub-tile (warp scans + preceding warps).
#pragma unroll
    for (int c = 0; c < NQ; ++c) {
        qv[c] = warp_incl_scan(qv[c]);
        if (lane == 31) s_wtot[warp][c] = qv[c];
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NQ; ++c) {
        int64_t off = 0;
        for (int w = 0; w < warp; ++w) off += s_wtot[w][c];
        if (i < N) lam_out[c * N + i] = off + qv[c];
    }

    // Level 1: the last CTA of each group of 64 sub-tiles scans the group.
    const int64_t g = sub >> kGroupLog2, s0 = g << kGroupLog2;
    const int64_t gsize = nsub - s0 < kGroup ? nsub - s0 : kGroup;
    if (tid == 0) {
#pragma unroll
        for (int c = 0; c < NQ; ++c) {
            int64_t t = 0;
            for (int w = 0; w < NW; ++w) t += s_wtot[w][c];
            P.subtot[c * nsub + sub] = t;
        }
        __threadfence();
        s_last = last_arrival(P.grp_ctr + g, (unsigned long long)gsize);
    }
    __syncthreads();
    if (!s_last) return;
    if (warp == 0) {
#pragma unroll
        for (int c = 0; c < NQ; ++c) {
            const int64_t *st = P.subtot + c * nsub + s0;
            const i128 v0 = 2 * lane < gsize ? (i128)__ldcg(st + 2 * lane) : (i128)0;
            const i128 v1 = 2 * lane + 1 < gsize ? (i128)__ldcg(st + 2 * lane + 1) : (i128)0;
            const i128 x = warp_incl_scan_i128(v0 + v1);
            const i128 ex = x - v0 - v1;
            i128 *ig = ingrp_out + c * nsub + s0;
            if (2 * lane < gsize) st_i128(ig + 2 * lane, ex);
            if (2 * lane + 1 < gsize) st_i128(ig + 2 * lane + 1, ex + v0);
            if (lane == 31) st_i128(P.grptot + c * ngroups + g, x);
        }
        __threadfence();
    }
    __syncthreads();
    if (tid == 0) s_last = last_arrival(P.top_ctr, (unsigned long long)ngroups);
    __syncthreads();
    if (!s_last) return;

    // Level 2: the last group scans the group totals (and records the totals).
    i128 total[NQ];
#pragma unroll
    for (int c = 0; c < NQ; ++c)
        total[c] = block_exclusive_scan<8>(P.grptot + c * ngroups, grpofs_out + c * (ngroups + 1), ngroups);
    if (RECORD && tid == 0 && P.obs) {
        const double S = fixed_to_double(total[0], P.F);
        const double C = fixed_to_double(total[NQ - 1], P.F);
        const unsigned long long n = *P.obs_ctr;
        P.obs[n % (unsigned long long)P.obs_cap] = sqrt(S * S + C * C) / (double)N;
        *P.obs_ctr = n + 1;
    }
    if (DEC_STEPS && tid == 0 && P.steps_left) *P.steps_left -= 1;
}

// As ring_prefix_tail, with NPT adjacent nodes per thread (kSubTile / NPT
// threads per CTA): node i0 + u of the thread holds qv[c][u].
//
// One-pass output (flat): the sub-tile totals into fsub_out, their chunks into
// the group accumulators facc_out, and CTA 0 clears facc_zero (the accumulators the next
// launch adds into).  tree: the two-level scan above as well (both only in the
// prologue, whose output any later kernel may read).
template <int NQ, int NPT, bool RECORD, bool DEC_STEPS>
__device__ __forceinline__ void ring_prefix_tail_n(const RingPlan &P, int64_t *lam_out, i128 *ingrp_out,
                                                   i128 *grpofs_out, int64_t sub, int64_t i0,
                                                   const int64_t (&qv)[NQ][NPT], bool flat, bool tree,
                                                   int64_t *fsub_out, unsigned *facc_out, unsigned *facc_zero)
{
    constexpr int NW = kSubTile / NPT / 32;
    __shared__ int64_t s_wtot[NW][NQ];
    __shared__ int s_last;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t N = P.N, nsub = P.nsub, ngroups = P.ngroups;

    // Exact inclusive prefix inside the sub-tile: the thread's running sums, a
    // warp scan of the thread totals and the preceding warps' totals.
    int64_t run[NQ][NPT], ex[NQ];
#pragma unroll
    for (int c = 0; c < NQ; ++c) {
        run[c][0] = qv[c][0];
#pragma unroll
        for (int u = 1; u < NPT; ++u) run[c][u] = run[c][u - 1] + qv[c][u];
        const int64_t incl = warp_incl_scan(run[c][NPT - 1]);
        ex[c] = incl - run[c][NPT - 1];
        if (lane == 31) s_wtot[warp][c] = incl;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NQ; ++c) {
        int64_t off = ex[c];
        for (int w = 0; w < warp; ++w) off += s_wtot[w][c];
#pragma unroll
        for (int u = 0; u < NPT; ++u)
            if (i0 + u < N) lam_out[c * N + i0 + u] = off + run[c][u];
    }

    if (flat) {
        const int64_t g = sub >> kGroupLog2;
        if (tid == 0) {
#pragma unroll
            for (int c = 0; c < NQ; ++c) {
                int64_t t = 0;
                for (int w = 0; w < NW; ++w) t += s_wtot[w][c];
                fsub_out[c * nsub + sub] = t;
                unsigned *a = facc_out + (c * ngroups + g) * 4;
#pragma unroll
                for (int k = 0; k < 4; ++k) atomicAdd(a + k, flat_chunk(t, k));
            }
        }
        if (sub == 0)
            for (int64_t w = tid; w < NQ * ngroups * 4; w += blockDim.x) facc_zero[w] = 0u;
        if (!tree) {
            if ((RECORD && P.obs) || (DEC_STEPS && P.steps_left)) {
                // the last CTA of the launch: totals from the accumulators
                if (tid == 0) {
                    __threadfence();
                    s_last = last_arrival(P.flat_ctr, (unsigned long long)nsub);
                }
                __syncthreads();
                if (s_last && warp == 0) {
                    i128 total[NQ];
#pragma unroll
                    for (int c = 0; c < NQ; ++c) {
                        unsigned tk[4] = {0, 0, 0, 0};
                        for (int64_t gg = lane; gg < ngroups; gg += 32)
#pragma unroll
                            for (int k = 0; k < 4; ++k) tk[k] += __ldcg(facc_out + (c * ngroups + gg) * 4 + k);
#pragma unroll
                        for (int k = 0; k < 4; ++k) tk[k] = __reduce_add_sync(0xffffffffu, tk[k]);
                        total[c] = flat_value(tk[0], tk[1], tk[2], tk[3]);
                    }
                    if (RECORD && lane == 0 && P.obs) {
                        const double S = fixed_to_double(total[0], P.F);
                        const double C = fixed_to_double(total[NQ - 1], P.F);
                        const unsigned long long n = *P.obs_ctr;
                        P.obs[n % (unsigned long long)P.obs_cap] = sqrt(S * S + C * C) / (double)N;
                        *P.obs_ctr = n + 1;
                    }
                    if (DEC_STEPS && lane == 0 && P.steps_left) *P.steps_left -= 1;
                }
            }
            return;
        }
    }

    // Level 1: the last CTA of each group of 64 sub-tiles scans the group.
    const int64_t g = sub >> kGroupLog2, s0 = g << kGroupLog2;
    const int64_t gsize = nsub - s0 < kGroup ? nsub - s0 : kGroup;
    if (tid == 0) {
#pragma unroll
        for (int c = 0; c < NQ; ++c) {
            int64_t t = 0;
            for (int w = 0; w < NW; ++w) t += s_wtot[w][c];
            P.subtot[c * nsub + sub] = t;
        }
        __threadfence();
        s_last = last_arrival(P.grp_ctr + g, (unsigned long long)gsize);
    }
    __syncthreads();
    if (!s_last) return;
    if (warp == 0) {
#pragma unroll
        for (int c = 0; c < NQ; ++c) {
            const int64_t *st = P.subtot + c * nsub + s0;
            const i128 v0 = 2 * lane < gsize ? (i128)__ldcg(st + 2 * lane) : (i128)0;
            const i128 v1 = 2 * lane + 1 < gsize ? (i128)__ldcg(st + 2 * lane + 1) : (i128)0;
            const i128 x = warp_incl_scan_i128(v0 + v1);
            const i128 e = x - v0 - v1;
            i128 *ig = ingrp_out + c * nsub + s0;
            if (2 * lane < gsize) st_i128(ig + 2 * lane, e);
            if (2 * lane + 1 < gsize) st_i128(ig + 2 * lane + 1, e + v0);
            if (lane == 31) st_i128(P.grptot + c * ngroups + g, x);
        }
        __threadfence();
    }
    __syncthreads();
    if (tid == 0) s_last = last_arrival(P.top_ctr, (unsigned long long)ngroups);
    __syncthreads();
    if (!s_last) return;

    // Level 2: the last group scans the group totals (and records the totals).
    i128 total[NQ];
#pragma unroll
    for (int c = 0; c < NQ; ++c)
        total[c] = block_exclusive_scan<8>(P.grptot + c * ngroups, grpofs_out + c * (ngroups + 1), ngroups);
    if (RECORD && tid == 0 && P.obs) {
        const double S = fixed_to_double(total[0], P.F);
        const double C = fixed_to_double(total[NQ - 1], P.F);
        const unsigned long long n = *P.obs_ctr;
        P.obs[n % (unsigned long long)P.obs_cap] = sqrt(S * S + C * C) / (double)N;
        *P.obs_ctr = n + 1;
    }
    if (DEC_STEPS && tid == 0 && P.steps_left) *P.steps_left -= 1;
}

// Buffers one stage reads and writes (chosen by the stage's parity).
struct RingStageIO {
    const int64_t *lam_in;
    const i128 *ingrp_in, *grpofs_in;
    int64_t *lam_out;
    i128 *ingrp_out, *grpofs_out;
    const int64_t *fsub_in; // one-pass prefix (RingPlan::flat)
    const unsigned *facc_in;
    int64_t *fsub_out;
    unsigned *facc_out, *facc_zero;
    const double *x_in; // local stage-input variables of this stage (HH gates)
    double *x_out;      // local stage-input variables of the next stage
};

// Stage 0 (prologue) writes buffer 0; stage s reads buffer (s+1)&1 and writes
// s&1, so stage 4 leaves f(y_{n+1}) in buffer 0 for the next step.  The
// one-pass group accumulators rotate over four slots: stage s reads slot
// (s-1)&3, adds into s&3 and clears (s+1)&3, which stage s-2 read last.
template <int M, int STAGE>
__host__ __device__ __forceinline__ RingStageIO stage_io(const RingPlan &p)
{
    constexpr int D = Model<M>::D, NX = Model<M>::NX;
    constexpr int in = (STAGE + 1) & 1, out = STAGE == 0 ? 0 : (STAGE & 1);
    RingStageIO a;
    a.lam_in = STAGE ? p.lam[in] : nullptr;
    a.ingrp_in = STAGE ? p.ingrp[in] : nullptr;
    a.grpofs_in = STAGE ? p.grpofs[in] : nullptr;
    a.lam_out = p.lam[out];
    a.ingrp_out = p.ingrp[out];
    a.grpofs_out = p.grpofs[out];
    a.fsub_in = STAGE ? p.fsub[in] : nullptr;
    a.facc_in = STAGE ? p.facc[(STAGE - 1) & 3] : nullptr;
    a.fsub_out = p.fsub[out];
    a.facc_out = p.facc[STAGE & 3];
    a.facc_zero = p.facc[(STAGE + 1) & 3];
    a.x_in = nullptr;
    a.x_out = nullptr;
    if (NX > 0) {
        a.x_in = STAGE == 1 ? p.y + (int64_t)(D - NX) * p.N : STAGE == 3 ? p.xg[1] : STAGE ? p.xg[0] : nullptr;
        a.x_out = STAGE == 1 || STAGE == 3 ? p.xg[0] : STAGE == 2 ? p.xg[1] : nullptr;
    }
    return a;
}

// RK4 stage s of node-parallel networks whose coupling is a sum over exact
// prefixes of the coupled quantity in node order (rings and general link
// matrices): one 256-node sub-tile `sub` per CTA, one node per thread.  The
// gather works in three phases: load() issues the node's own global loads (they
// need nothing shared), sync() makes the CTA's shared window bases visible (a
// barrier every thread reaches), finish() combines them into the node's own
// fixed-point coupled quantity, its window sums W, its link count and coupling
// scale (see models.cuh).  The node's state loads are issued before the barrier
// as well, so the CTA's start latency overlaps the bases' computation.
template <int M, int STAGE, class Gather, bool FLAT_OK = false>
__device__ __forceinline__ void stage_body(const RingPlan &P, const RingStageIO &a, const StepSize &h, int64_t sub,
                                           const Gather &gather)
{
    using Mo = Model<M>;
    constexpr int D = Mo::D, NQ = Mo::NQ, NX = Mo::NX;
    constexpr int XOFF = D - NX; // first local (non-coupled) state variable
    const int tid = threadIdx.x;
    const int64_t N = P.N;
    const int64_t i = sub * kSubTile + tid;

    int64_t qv[NQ];
    bool ok = true;
#pragma unroll
    for (int c = 0; c < NQ; ++c) qv[c] = 0;
    double yv[D], av[D], X[NX > 0 ? NX : 1];
    double Iext = 0.0;
    typename Gather::Pre pre;
    if (STAGE > 0) {
        if (i < N) {
            gather.load(tid, i, pre);
#pragma unroll
            for (int v = 0; v < D; ++v) {
                yv[v] = P.y[v * N + i];
                av[v] = STAGE >= 2 ? P.acc[v * N + i] : 0.0;
            }
#pragma unroll
            for (int g = 0; g < NX; ++g) X[g] = a.x_in[g * N + i];
            if (M == 2 && P.node_param) Iext = P.node_param[i];
        }
        gather.sync();
    }
    if (i < N) {
        double xn[D];
        if (STAGE == 0) {
#pragma unroll
            for (int v = 0; v < D; ++v) xn[v] = P.y[v * N + i];
        } else {
            int64_t qo[NQ];
            double fo[NQ];
            i128 W[NQ];
            int64_t wsize;
            double cs;
            gather.finish(tid, i, pre, qo, fo, W, wsize, cs);
            double k[D];
            Mo::rhs(P.mp, P.F, fo, qo, W, X, Iext, k, wsize, cs);
#pragma unroll
            for (int v = 0; v < D; ++v) {
                if (STAGE == 1) {
                    P.acc[v * N + i] = k[v];
                    xn[v] = yv[v] + h.half * k[v];
                } else if (STAGE == 2) {
                    P.acc[v * N + i] = av[v] + 2.0 * k[v];
                    xn[v] = yv[v] + h.half * k[v];
                } else if (STAGE == 3) {
                    P.acc[v * N + i] = av[v] + 2.0 * k[v];
                    xn[v] = yv[v] + h.dt * k[v];
                } else {
                    const double yn = yv[v] + h.sixth * (av[v] + k[v]);
                    P.y[v * N + i] = yn;
                    xn[v] = yn;
                }
            }
            if (NX > 0 && STAGE >= 1 && STAGE <= 3) {
#pragma unroll
                for (int g = 0; g < NX; ++g) a.x_out[g * N + i] = xn[XOFF + g];
            }
        }
        // a2: coupled quantity of the next stage input on the fixed-point grid
        Mo::coupled_q(P.mp, xn, P.F, P.lim, ok, qv);
    }
    if (!ok) raise_error(P.err, ERR_RANGE);
    constexpr bool RECORD = (M == 0 || M == 3) && (STAGE == 0 || STAGE == 4);
    if constexpr (FLAT_OK) {
        if (P.flat) { // the one-pass prefix (both forms in the prologue)
            int64_t qv1[NQ][1];
#pragma unroll
            for (int c = 0; c < NQ; ++c) qv1[c][0] = qv[c];
            ring_prefix_tail_n<NQ, 1, RECORD, STAGE == 4>(P, a.lam_out, a.ingrp_out, a.grpofs_out, sub, i, qv1, true,
                                                          STAGE == 0, a.fsub_out, a.facc_out, a.facc_zero);
            return;
        }
    }
    ring_prefix_tail<NQ, RECORD, STAGE == 4>(P, a.lam_out, a.ingrp_out, a.grpofs_out, sub, i, qv);
}

} // namespace simk
