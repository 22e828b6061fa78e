// Periodic lattices of Kuramoto nodes (with or without inertia), Section IV:
//   cube  N1^3 nodes, index k N1^2 + j N1 + i, the (2P+1)^3 box around a node;
//   ball  N1^3 nodes, the sphere dx^2 + dy^2 + dz^2 <= P^2 (3D networks);
//   disk  N1^2 nodes, index j N1 + i, the circle dx^2 + dy^2 <= P^2 (2D networks).
// f = (sin, cos) of the stage-input phase, rounded onto the grid 2^-F (F chosen
// so that a full window sum fits in int64), so every window sum is exact
// integer arithmetic and the node's right-hand side needs one cross product of
// the sums with its own (sin, cos).  The ball and disk rotate every node's
// quantity by -alpha in the x pass (lattice_rotated_q); the cube keeps its sums
// unrotated and turns the node's own phase by +alpha (own_phase_turned).
//
// Cube, per RK4 stage (the box is separable):
//   x pass  SX(i,j,k)  = sum_{|dx|<=P} Q(f(i+dx,j,k))      (row prefix in shared memory)
//   y pass  SXY(i,j,k) = sum_{|dy|<=P} SX(i,j+dy,k)        (column prefix in a tile)
//   z pass  W(i,j,k)   = sum_{|dz|<=P} SXY(i,j,k+dz)       (column prefix in a tile)
//           and the coupling term; the node pass then runs the right-hand side,
//           the RK4 update, the next (sin, cos) and the next stage's x pass.
//           Batched cubes use sliding windows along j and k instead, the z pass
//           fused with the node update.
// Ball and disk, per RK4 stage:
//   x pass  for every half-width w = 0..P the x-window sums S_w(i) of Q(f) along
//           every row, sin and cos interleaved; or, when those P+1 arrays would
//           exceed the memory budget (or SIM_FLAG_LOW_MEMORY), the inclusive row
//           prefix E(x) extended periodically by P + 1 entries on the left and P
//           on the right (wrapping int64);
//   gather  W = sum over the chords of the window, one per (dy, dz) (ball) or dy
//           (disk): the row segment |dx| <= w = floor(sqrt(P^2 - dy^2 - dz^2)),
//           read as S_w (one 16-byte load) or E(i + w) - E(i - w - 1) (two),
//           O(P^2) resp. O(P) reads per node, fused with the right-hand side and
//           RK4 update.
#include <algorithm>

#include "internal.h"

namespace simk {

constexpr int kRowWarpsMax = 8;       // x pass: one warp per row
constexpr int kColThreads = 128;      // cube y and z passes: threads per CTA along i
constexpr int64_t kColTarget = 152 * 1024; // cube y and z passes: columns are split into
                                           // segments until about this many threads run
constexpr int kGatherThreads = 256;   // ball/disk gather: one node per thread
constexpr size_t kRowSmemMax = 220 * 1024;

// i-columns per tile: shared memory 2 (N1 + 1) BI 8 bytes stays below ~76 KB
// (two or three CTAs per SM) and every row segment of a load is BI * 8 bytes.
__host__ __device__ inline int cube_tile_lg(int64_t N1) { return N1 <= 297 ? 4 : N1 <= 594 ? 3 : 2; }
__host__ __device__ inline int cube_tile_bi(int64_t N1) { return 1 << cube_tile_lg(N1); }

// Component stride of the tiled cube's xy-window sums in their i-block-major
// layout [i-block][j][k][ii]: every i-block padded to BI columns.
__host__ __device__ inline int64_t cube_sxy_cstride(int64_t N1)
{
    const int BI = cube_tile_bi(N1);
    return ((N1 + BI - 1) / BI) * BI * N1 * N1;
}

static int row_warps(int64_t N1)
{
    const size_t per_warp = 2 * (size_t)(N1 + 1) * sizeof(int64_t);
    int w = (int)(kRowSmemMax / per_warp);
    return w < 1 ? 1 : (w > kRowWarpsMax ? kRowWarpsMax : w);
}

// The cube's fused node pass: smaller CTAs than the x pass, so that the shared
// prefix rows of a CTA round up to less of the SM (seven CTAs of four 464-node
// rows, against three of eight).
constexpr int kNodexWarpsMax = 4;
// CTAs per SM the fused node pass is compiled for: six for Kuramoto (at most 80
// registers, so stage 4 fits six too), five for the model with inertia.
template <int M> constexpr int kNodexBlocks = M == 0 ? 6 : 5;
static int nodex_warps(int64_t N1)
{
    const int w = row_warps(N1);
    return w > kNodexWarpsMax ? kNodexWarpsMax : w;
}

// The coupled quantity a ball's or disk's window sums add up: the node's (sin,
// cos) on the grid 2^-62 rotated by -alpha = -(rot_q pi/2 + alpha0),
//   e^{-i alpha0} (c + i s) = (c cos a0 + s sin a0) + i (s cos a0 - c sin a0),
// four high products with cos alpha0 and sin alpha0 (non-negative, grid 2^-63),
// which land on the grid 2^-61 (so their truncation leaves no bias that a
// window of millions of terms could accumulate), rounded to nearest onto the
// grid 2^-F, then rot_q quarter turns.  The right-hand side then needs only the
// node's own unrotated (sin, cos) (lattice_coupling).
__device__ __forceinline__ void lattice_rotated_q(const LatticePlan &p, int64_t s62, int64_t c62, int64_t &qs,
                                                  int64_t &qc)
{
    const int sh = 61 - p.F;
    const int64_t h = int64_t(1) << (sh - 1);
    const int64_t c1 = (mulhi_su(c62, p.rot_c) + mulhi_su(s62, p.rot_s) + h) >> sh;
    const int64_t s1 = (mulhi_su(s62, p.rot_c) - mulhi_su(c62, p.rot_s) + h) >> sh;
    switch (p.rot_q) { // e^{-i q pi/2}: 1, -i, -1, i
    case 0: qc = c1; qs = s1; break;
    case 1: qc = s1; qs = -c1; break;
    case 2: qc = -c1; qs = -s1; break;
    default: qc = -s1; qs = c1; break;
    }
}

// x pass: one warp per row.  pre(p) = sum_{m<p} Q'(f(m)) for p in [0, N1] is built
// in shared memory (stride N1 + 1 per component).  With Pe(p) = pre(p mod N1) +
// floor(p / N1) pre(N1) the periodic extension:
//   MODE 0 (cube)        SX(i) = Pe(i+P+1) - Pe(i-P), sin and cos in two arrays;
//   MODE 1 (ball, disk,  the extended inclusive prefix E(x) = Pe(x+1),
//           low memory)  x in [-P-1, N1+P-1], (sin, cos) pairs, modulo 2^64;
//   MODE 2 (ball, disk)  for every half-width w = 0..P the window sums
//                        S_w(i) = Pe(i+w+1) - Pe(i-w), (sin, cos) pairs, one
//                        array of nodes pairs per w.
// One row of the x pass (one warp; pre0/pre1 its shared prefix rows).
// IBLK (cube, the tiled passes): SX in the plane-wise i-block-major layout
// [k][i-block][j][ii] (cube_sx_index), which each y tile reads as one
// contiguous block; otherwise node order (the batched sliding passes).
// The row's own part: pre0/pre1[m + 1] = Q'(f(m)) for m < N1 from the stored
// (sin, cos).
template <int MODE>
__device__ __forceinline__ void lattice_x_fill(const LatticePlan &p, int64_t row, int64_t *pre0, int64_t *pre1)
{
    const int lane = threadIdx.x & 31;
    const int64_t N1 = p.N1, nodes = p.nodes;
    const longlong2 *__restrict__ fr = reinterpret_cast<const longlong2 *>(p.f) + row * N1; // (sin, cos) pairs
    for (int64_t mb = lane; mb < N1; mb += 32 * 8) { // coalesced, 8 loads in flight per lane
        int64_t vs[8], vc[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t m = mb + 32 * u;
            const longlong2 v = m < N1 ? __ldg(fr + m) : make_longlong2(0, 0);
            vs[u] = v.x;
            vc[u] = v.y;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t m = mb + 32 * u;
            if (m < N1) {
                if (MODE == 0) { // cube: the node's own phase is turned instead
                    pre0[m + 1] = q62_to(vs[u], p.F);
                    pre1[m + 1] = q62_to(vc[u], p.F);
                } else {
                    lattice_rotated_q(p, vs[u], vc[u], pre0[m + 1], pre1[m + 1]);
                }
            }
        }
    }
}

// The row's prefix and window sums from pre0/pre1[1..N1] (filled by the warp).
template <int MODE, bool IBLK>
__device__ __forceinline__ void lattice_x_scan_out(const LatticePlan &p, int64_t row, int64_t *pre0, int64_t *pre1)
{
    const int lane = threadIdx.x & 31;
    const int64_t N1 = p.N1, P = p.P, nodes = p.nodes;
    const int n1 = (int)N1, per = (n1 + 31) >> 5;
    __syncwarp();
    // lane l owns the prefix slots m0 .. m1 - 1: its part's total, the warp's
    // exclusive scan of the totals, then the part's prefix written once
    const int m0 = min(lane * per, n1) + 1, m1 = min(m0 + per, n1 + 1);
    uint64_t r0 = 0, r1 = 0; // wrapping sums
    for (int m = m0; m < m1; ++m) {
        r0 += (uint64_t)pre0[m];
        r1 += (uint64_t)pre1[m];
    }
    uint64_t e0 = (uint64_t)warp_incl_scan((int64_t)r0) - r0;
    uint64_t e1 = (uint64_t)warp_incl_scan((int64_t)r1) - r1;
    for (int m = m0; m < m1; ++m) {
        e0 += (uint64_t)pre0[m];
        e1 += (uint64_t)pre1[m];
        pre0[m] = (int64_t)e0;
        pre1[m] = (int64_t)e1;
    }
    if (lane == 0) {
        pre0[0] = 0;
        pre1[0] = 0;
    }
    __syncwarp();
    if (MODE == 2) {
        const int64_t t0 = pre0[N1], t1 = pre1[N1];
        longlong2 *__restrict__ o = reinterpret_cast<longlong2 *>(p.sx) + row * N1;
        for (int64_t w = 0; w <= P; ++w, o += nodes) {
            for (int64_t i = lane; i < N1; i += 32) {
                int64_t b = i + w + 1, a = i - w;
                int64_t s0 = 0, s1 = 0;
                if (b > N1) { b -= N1; s0 += t0; s1 += t1; }
                if (a < 0) { a += N1; s0 += t0; s1 += t1; } // Pe(a) = pre(a+N1) - total
                o[i] = make_longlong2(s0 + pre0[b] - pre0[a], s1 + pre1[b] - pre1[a]);
            }
        }
    } else if (MODE == 1) {
        // E(x) = Pe(x + 1) for x in [-P-1, N1+P-1], at slot x + P + 1
        const uint64_t t0 = (uint64_t)pre0[N1], t1 = (uint64_t)pre1[N1];
        longlong2 *__restrict__ o = reinterpret_cast<longlong2 *>(p.sx) + row * p.rs;
        for (int64_t e = lane; e < p.rs; e += 32) {
            int64_t q = e - P; // = x + 1, in [-P, N1 + P]
            uint64_t v0, v1;
            if (q < 0) {
                v0 = (uint64_t)pre0[q + N1] - t0;
                v1 = (uint64_t)pre1[q + N1] - t1;
            } else if (q > N1) {
                v0 = (uint64_t)pre0[q - N1] + t0;
                v1 = (uint64_t)pre1[q - N1] + t1;
            } else {
                v0 = (uint64_t)pre0[q];
                v1 = (uint64_t)pre1[q];
            }
            o[e] = make_longlong2((long long)v0, (long long)v1);
        }
    } else {
        const int64_t t0 = pre0[N1], t1 = pre1[N1];
        if (IBLK) {
            // row = k N1 + j; element i at ((k tiles + i / BI) N1 + j) BI + i % BI.
            // BI divides 32, so lane's column within its i-block stays fixed and
            // every 32 columns move 32 / BI i-blocks further.
            const int lg = cube_tile_lg(N1), BI = 1 << lg, p1 = (int)P;
            const int64_t k = row / N1, j = row - k * N1, tiles = (N1 + BI - 1) >> lg;
            const int64_t bstep = N1 * BI; // one i-block further
            int64_t *__restrict__ o0 = p.sx + (k * tiles * N1 + j) * BI;
            int64_t *__restrict__ o1 = o0 + cube_sxy_cstride(N1);
            const unsigned ostep = (unsigned)bstep << (5 - lg);
            unsigned o = (unsigned)((lane >> lg) * bstep) + (lane & (BI - 1));
#pragma unroll 2
            for (int i = lane; i < n1; i += 32, o += ostep) {
                // 2P + 1 <= N1: at most one end of the window wraps, adding the total
                const int b = i + p1 + 1, a = i - p1;
                const bool hi = b > n1, lo = a < 0;
                const int bb = hi ? b - n1 : b, aa = lo ? a + n1 : a;
                const int64_t s0 = (hi || lo) ? t0 : 0, s1 = (hi || lo) ? t1 : 0;
                o0[o] = s0 + pre0[bb] - pre0[aa];
                o1[o] = s1 + pre1[bb] - pre1[aa];
            }
            // the last i-block's columns past the cube's edge read as zeros
            const int64_t pad = tiles * BI - N1;
            if (lane < pad) {
                const int64_t o = (tiles - 1) * bstep + (BI - pad + lane);
                o0[o] = 0;
                o1[o] = 0;
            }
        } else {
            int64_t *__restrict__ o0 = p.sx + row * N1;
            int64_t *__restrict__ o1 = p.sx + nodes + row * N1;
            for (int64_t i = lane; i < N1; i += 32) {
                int64_t b = i + P + 1, a = i - P;
                int64_t s0 = 0, s1 = 0;
                if (b > N1) { b -= N1; s0 += t0; s1 += t1; }
                if (a < 0) { a += N1; s0 += t0; s1 += t1; } // Pe(a) = pre(a+N1) - total
                o0[i] = s0 + pre0[b] - pre0[a];
                o1[i] = s1 + pre1[b] - pre1[a];
            }
        }
    }
    __syncwarp();
}

template <int MODE, bool IBLK = false>
__device__ __forceinline__ void lattice_x_row(const LatticePlan &p, int64_t row, int64_t *pre0, int64_t *pre1,
                                              bool &)
{
    lattice_x_fill<MODE>(p, row, pre0, pre1);
    lattice_x_scan_out<MODE, IBLK>(p, row, pre0, pre1);
}

template <int MODE>
__global__ void __launch_bounds__(32 * kRowWarpsMax) lattice_x_kernel(LatticePlan p)
{
    if (p.skip && *(const volatile int *)p.skip) return;
    extern __shared__ int64_t smem[];
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int64_t stride = p.N1 + 1, rows = p.nodes / p.N1;
    int64_t *pre0 = smem + (int64_t)warp * 2 * stride;
    int64_t *pre1 = pre0 + stride;
    bool ok = true;
    for (int64_t row = (int64_t)blockIdx.x * nwarps + warp; row < rows; row += (int64_t)gridDim.x * nwarps)
        lattice_x_row<MODE, MODE == 0>(p, row, pre0, pre1, ok);
    if (!ok) raise_error(p.err, ERR_RANGE);
}

// Batched cube x pass: CTA b works on rows (b - x_base[m]) * warps + warp of
// member m = x_item[b]; shared memory is sized for the group's largest edge.
__global__ void __launch_bounds__(32 * kRowWarpsMax)
    cube_batch_x_kernel(const LatticePlan *__restrict__ plans, const int *__restrict__ x_item,
                        const int64_t *__restrict__ x_base)
{
    const int inst = x_item[blockIdx.x];
    const LatticePlan &p = plans[inst];
    extern __shared__ int64_t smem[];
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int64_t stride = p.N1 + 1, rows = p.nodes / p.N1;
    int64_t *pre0 = smem + (int64_t)warp * 2 * stride;
    int64_t *pre1 = pre0 + stride;
    const int64_t row = ((int64_t)blockIdx.x - x_base[inst]) * nwarps + warp;
    bool ok = true;
    if (row < rows) lattice_x_row<0, true>(p, row, pre0, pre1, ok); // uniform over the warp
    if (!ok) raise_error(p.err, ERR_RANGE);
}

// Columns of the y and z passes are split into gridDim.z segments of
// col_seg_len() nodes (small cubes would otherwise run a few thousand threads,
// each walking its column serially); every segment starts its own sliding
// window, so the window sums, being exact, do not depend on the split.
__host__ __device__ inline int64_t col_segments(int64_t N1)
{
    const int64_t cols = N1 * N1;
    int64_t nseg = (kColTarget + cols - 1) / cols;
    if (nseg > N1) nseg = N1;
    return nseg < 1 ? 1 : nseg;
}

__host__ __device__ inline int64_t col_seg_len(int64_t N1)
{
    const int64_t nseg = col_segments(N1);
    return (N1 + nseg - 1) / nseg;
}

// cube y pass: one thread per segment of an (i, k) column, sliding window along
// j (exact int64), 8 rows of window loads issued together; writes the window
// sums.
__device__ __forceinline__ void cube_y_col(const LatticePlan &p, int64_t i, int64_t k, int64_t seg)
{
    constexpr int U = 8;
    const int64_t N1 = p.N1, P = p.P, nodes = p.nodes;
    const int64_t len = col_seg_len(N1), jb = seg * len;
    const int64_t je = jb + len < N1 ? jb + len : N1;
    if (i >= N1 || jb >= N1) return;
    const int64_t col = k * N1 * N1 + i; // + j * N1
    // the x sums in the plane-wise i-block-major layout: (i, j, k) at
    // ((k tiles + i / BI) N1 + j) BI + i % BI, so consecutive j are BI apart
    const int lg = cube_tile_lg(N1), BI = 1 << lg;
    const int64_t tiles = (N1 + BI - 1) >> lg;
    const int64_t *__restrict__ a0 = p.sx + ((k * tiles + (i >> lg)) * N1) * BI + (i & (BI - 1));
    const int64_t *__restrict__ a1 = a0 + cube_sxy_cstride(N1);
    int64_t *__restrict__ o0 = p.sxy + col;
    int64_t *__restrict__ o1 = p.sxy + nodes + col;
    int64_t s0 = 0, s1 = 0;
    for (int64_t d = -P; d <= P; ++d) {
        int64_t j = jb + d;
        j += j < 0 ? N1 : 0;
        j -= j >= N1 ? N1 : 0;
        s0 += __ldg(a0 + j * BI);
        s1 += __ldg(a1 + j * BI);
    }
    for (int64_t j0 = jb; j0 < je; j0 += U) {
        int64_t in0[U], out0[U], in1[U], out1[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t j = j0 + u;
            int64_t jin = j + P + 1, jout = j - P;
            if (jin >= N1) jin -= N1;
            if (jout < 0) jout += N1;
            const bool live = j < je;
            in0[u] = live ? __ldg(a0 + jin * BI) : 0;
            out0[u] = live ? __ldg(a0 + jout * BI) : 0;
            in1[u] = live ? __ldg(a1 + jin * BI) : 0;
            out1[u] = live ? __ldg(a1 + jout * BI) : 0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t j = j0 + u;
            if (j < je) {
                o0[j * N1] = s0;
                o1[j * N1] = s1;
            }
            s0 += in0[u] - out0[u];
            s1 += in1[u] - out1[u];
        }
    }
}

// The (column block, plane, segment) of CTA b of a batched y or z pass: the
// member's CTAs in the order of the single-network grid (x fastest).
__device__ __forceinline__ void cube_col_item(const LatticePlan &p, int64_t lb, int64_t &bx, int64_t &plane,
                                              int64_t &seg)
{
    const int64_t nbx = (p.N1 + kColThreads - 1) / kColThreads;
    bx = lb % nbx;
    plane = (lb / nbx) % p.N1;
    seg = lb / (nbx * p.N1);
}

__global__ void __launch_bounds__(kColThreads)
    cube_batch_y_kernel(const LatticePlan *__restrict__ plans, const int *__restrict__ yz_item,
                        const int64_t *__restrict__ yz_base)
{
    const int inst = yz_item[blockIdx.x];
    const LatticePlan &p = plans[inst];
    int64_t bx, k, seg;
    cube_col_item(p, (int64_t)blockIdx.x - yz_base[inst], bx, k, seg);
    cube_y_col(p, bx * kColThreads + threadIdx.x, k, seg);
}

// Deterministic order parameter of the new state: per-CTA partial sums of the
// fixed-point (sin, cos) (exact i128, so the reduction order does not matter),
// and the last CTA to finish sums every partial and records R.  bid / nblk: the
// CTA's index among the network's CTAs of this launch and their number.
// (ps, pc) summed over the CTA, valid in thread 0; every thread of the CTA calls it.
__device__ __forceinline__ void cta_sum_pair(i128 &ps, i128 &pc)
{
    __shared__ i128 s_ws[32], s_wc[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    ps = warp_sum_i128(ps);
    pc = warp_sum_i128(pc);
    __syncthreads(); // an earlier use of s_ws / s_wc is over
    if (lane == 0) {
        s_ws[warp] = ps;
        s_wc[warp] = pc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ps = 0;
        pc = 0;
        for (int w = 0; w < nw; ++w) {
            ps += s_ws[w];
            pc += s_wc[w];
        }
    }
}

// The order parameter R = |sum_n e^{i theta_n}| / nodes from the exact sums of
// the n partial pairs at part (p.partial or beyond), by one CTA; recorded in p.obs.
__device__ __forceinline__ void lattice_order_total(const LatticePlan &p, const i128 *part, unsigned n)
{
    i128 ts = 0, tc = 0;
    for (unsigned b = threadIdx.x; b < n; b += blockDim.x) {
        ts += ld_cg_i128(part + 2 * b);
        tc += ld_cg_i128(part + 2 * b + 1);
    }
    cta_sum_pair(ts, tc);
    if (threadIdx.x == 0) {
        const double S = fixed_to_double(ts, p.F), C = fixed_to_double(tc, p.F);
        if (p.obs) {
            const unsigned long long n_rec = *p.obs_ctr;
            p.obs[n_rec % (unsigned long long)p.obs_cap] = sqrt(S * S + C * C) / (double)p.nodes;
            *p.obs_ctr = n_rec + 1;
        }
    }
}

// The CTA's partial sums to p.partial[2 bid, 2 bid + 1]; the last CTA of nblk
// to arrive at *ctr adds them all up and records the order parameter.
__device__ void lattice_record_order(const LatticePlan &p, i128 ps, i128 pc, unsigned bid, unsigned nblk,
                                     unsigned long long *ctr)
{
    __shared__ bool s_last;
    cta_sum_pair(ps, pc);
    if (threadIdx.x == 0) {
        st_i128(p.partial + 2 * bid, ps);
        st_i128(p.partial + 2 * bid + 1, pc);
        __threadfence();
        s_last = last_arrival(ctr, nblk);
    }
    __syncthreads();
    if (!s_last) return;
    lattice_order_total(p, p.partial, nblk);
}

// The order parameter from the partials of a previous launch of nblk CTAs (the
// cube's fused node pass, whose CTAs only store their partials): CTA g adds up
// its slice of them into the pair nblk + g, and the last of the kOrderCtas CTAs
// to finish (arrival counter tile_ctr) adds those up.
constexpr int kOrderCtas = 128, kOrderThreads = 256;
__global__ void __launch_bounds__(kOrderThreads) lattice_order_kernel(LatticePlan p, unsigned nblk)
{
    if (p.skip && *(const volatile int *)p.skip) return;
    __shared__ bool s_last;
    const unsigned per = (nblk + gridDim.x - 1) / gridDim.x, b0 = blockIdx.x * per, b1 = min(nblk, b0 + per);
    i128 ts = 0, tc = 0;
    for (unsigned b = b0 + threadIdx.x; b < b1; b += blockDim.x) {
        ts += ld_cg_i128(p.partial + 2 * b);
        tc += ld_cg_i128(p.partial + 2 * b + 1);
    }
    cta_sum_pair(ts, tc);
    if (threadIdx.x == 0) {
        st_i128(p.partial + 2 * (nblk + blockIdx.x), ts);
        st_i128(p.partial + 2 * (nblk + blockIdx.x) + 1, tc);
        __threadfence();
        s_last = last_arrival(p.tile_ctr, gridDim.x);
    }
    __syncthreads();
    if (!s_last) return;
    lattice_order_total(p, p.partial + 2 * nblk, gridDim.x);
}

// One node's RK4 stage: right-hand side from the window sums (W0, W1) and its own
// stage input, the RK4 update, the next stage input's local variables and (sin,
// cos).  STAGE 0 (prologue) only computes (sin, cos) of y.  In two parts, so
// that a thread can issue the loads of its next node before it computes this
// one: lattice_node_load reads what the node needs, lattice_node_finish
// computes and writes; lattice_node is the two in a row.
template <int M> struct LatNodeIn {
    int64_t f62[2];                                // (sin, cos) of the stage input, grid 2^-62
    double y[Model<M>::D], acc[Model<M>::D];
    double X[Model<M>::NX > 0 ? Model<M>::NX : 1]; // local stage-input variables
};

template <int M, int STAGE>
__device__ __forceinline__ void lattice_node_load(const LatticePlan &p, int64_t n, LatNodeIn<M> &in)
{
    constexpr int D = Model<M>::D, NX = Model<M>::NX, XOFF = D - NX;
    const int64_t nodes = p.nodes;
#pragma unroll
    for (int v = 0; v < D; ++v) {
        in.y[v] = p.y[v * nodes + n];
        in.acc[v] = STAGE >= 2 ? p.acc[v * nodes + n] : 0.0;
    }
    if (STAGE > 0) {
        const longlong2 v = reinterpret_cast<const longlong2 *>(p.f)[n];
        in.f62[0] = v.x;
        in.f62[1] = v.y;
#pragma unroll
        for (int g = 0; g < NX; ++g) in.X[g] = STAGE == 1 ? in.y[XOFF + g] : p.xs[g * nodes + n];
    }
}

// The RK4 update of a node from its slope k (stages 1-4), the next stage
// input's local variables and (sin, cos); STAGE 0 (prologue) only the (sin,
// cos) of y.  Acc: the type of the thread's order-parameter sums (int64 where a
// thread handles few enough nodes that |sum| <= nodes 2^F stays below 2^63).
template <int M, int STAGE, typename Acc>
__device__ __forceinline__ void lattice_node_update(const LatticePlan &p, int64_t n, const double (&k)[Model<M>::D],
                                                    const LatNodeIn<M> &in, const StepSize &h, bool &ok, Acc &ps,
                                                    Acc &pc, int64_t *sc_out = nullptr)
{
    constexpr int D = Model<M>::D, NX = Model<M>::NX, XOFF = D - NX;
    const int64_t nodes = p.nodes;
    double xn[D];
    if (STAGE == 0) {
#pragma unroll
        for (int v = 0; v < D; ++v) xn[v] = in.y[v];
    } else {
#pragma unroll
        for (int v = 0; v < D; ++v) {
            if (STAGE == 1) {
                p.acc[v * nodes + n] = k[v];
                xn[v] = in.y[v] + h.half * k[v];
            } else if (STAGE == 2) {
                p.acc[v * nodes + n] = in.acc[v] + 2.0 * k[v];
                xn[v] = in.y[v] + h.half * k[v];
            } else if (STAGE == 3) {
                p.acc[v * nodes + n] = in.acc[v] + 2.0 * k[v];
                xn[v] = in.y[v] + h.dt * k[v];
            } else {
                xn[v] = in.y[v] + h.sixth * (in.acc[v] + k[v]);
                p.y[v * nodes + n] = xn[v];
            }
        }
        if (NX > 0 && STAGE <= 3) {
#pragma unroll
            for (int g = 0; g < NX; ++g) p.xs[g * nodes + n] = xn[XOFF + g];
        }
    }
    int64_t s62, c62;
    fixed_sincos(xn[0], p.mp.tab, s62, c62, ok);
    reinterpret_cast<longlong2 *>(p.f)[n] = make_longlong2(s62, c62);
    if (STAGE == 0 || STAGE == 4) {
        ps += q62_to(s62, p.F);
        pc += q62_to(c62, p.F);
    }
    if (sc_out) {
        sc_out[0] = s62;
        sc_out[1] = c62;
    }
}

// The whole node stage: right-hand side from the window sums and the node's own
// stage input, then lattice_node_update.
template <int M, int STAGE, typename Acc>
__device__ __forceinline__ void lattice_node_finish(const LatticePlan &p, int64_t n, int64_t W0, int64_t W1,
                                                    const LatNodeIn<M> &in, const StepSize &h, bool &ok, Acc &ps,
                                                    Acc &pc)
{
    double k[Model<M>::D] = {};
    if (STAGE > 0) Model<M>::rhs_lattice(p.mp, in.f62, W0, W1, in.X, k);
    lattice_node_update<M, STAGE, Acc>(p, n, k, in, h, ok, ps, pc);
}

// TURN (the cube): the window sums are unrotated, and the node's own phase is
// turned by +alpha for the cross product instead (own_phase_turned).
template <int M, int STAGE, bool TURN = false>
__device__ __forceinline__ void lattice_node(const LatticePlan &p, int64_t n, int64_t W0, int64_t W1, const StepSize &h,
                                             bool &ok, i128 &ps, i128 &pc)
{
    LatNodeIn<M> in;
    lattice_node_load<M, STAGE>(p, n, in);
    if (TURN && STAGE > 0) {
        int64_t t62[2];
        own_phase_turned(p.mp, in.f62, t62);
        in.f62[0] = t62[0];
        in.f62[1] = t62[1];
    }
    lattice_node_finish<M, STAGE, i128>(p, n, W0, W1, in, h, ok, ps, pc);
}

// Batched cube z pass: one thread per segment of an (i, j) column, sliding
// window along k, fused with the node update.
template <int M, int STAGE>
__device__ __forceinline__ void cube_z_col(const LatticePlan &p, const StepSize &h, int64_t bx, int64_t j,
                                           int64_t seg, unsigned bid, unsigned nblk)
{
    const int64_t N1 = p.N1, P = p.P, nodes = p.nodes, plane = N1 * N1;
    const int64_t i = bx * kColThreads + threadIdx.x;
    const int64_t len = col_seg_len(N1), kb = seg * len;
    const int64_t ke = kb + len < N1 ? kb + len : N1;
    i128 ps = 0, pc = 0;
    bool ok = true;
    if (i < N1) {
        const int64_t col = j * N1 + i; // + k * plane
        const int64_t *__restrict__ a0 = p.sxy + col;
        const int64_t *__restrict__ a1 = p.sxy + nodes + col;
        int64_t s0 = 0, s1 = 0;
        if (STAGE > 0 && kb < N1) {
            for (int64_t d = -P; d <= P; ++d) {
                int64_t k = kb + d;
                k += k < 0 ? N1 : 0;
                k -= k >= N1 ? N1 : 0;
                s0 += __ldg(a0 + k * plane);
                s1 += __ldg(a1 + k * plane);
            }
        }
        for (int64_t k = kb; k < ke; ++k) {
            lattice_node<M, STAGE, true>(p, col + k * plane, s0, s1, h, ok, ps, pc);
            if (STAGE > 0) {
                int64_t kin = k + P + 1, kout = k - P;
                if (kin >= N1) kin -= N1;
                if (kout < 0) kout += N1;
                s0 += __ldg(a0 + kin * plane) - __ldg(a0 + kout * plane);
                s1 += __ldg(a1 + kin * plane) - __ldg(a1 + kout * plane);
            }
        }
    }
    if (!ok) raise_error(p.err, ERR_RANGE);
    if (STAGE == 0 || STAGE == 4) lattice_record_order(p, ps, pc, bid, nblk, p.done_ctr);
}

// ---------------------------------------------------------------------------
// Tiled y and z passes of a single cube (the batched cubes keep the sliding
// windows above and below; both give the same exact sums).  CTA (ib, m) loads
// the 2 x N1 x BI block of one plane (y pass: plane k = m, i-block ib, all j) or
// one row of columns (z pass: row j = m, i-block ib, all k) into shared memory,
// so that every element crosses HBM once (a sliding window re-reads the element
// leaving the window, 2P+1 rows or planes after it entered, long gone from L2
// on large cubes).  The block is scanned in place into the exact inclusive
// prefix along the window axis (wrapping int64 arithmetic, as the x pass), and
// every window sum is Pe(a+P+1) - Pe(a-P) on its periodic extension.
constexpr int kTileThreads = 256;

// Asynchronous 8-byte copy global -> shared (zero fill when !live); the copies
// of a thread complete at cp_async_wait_all.
__device__ __forceinline__ void cp_async8(uint64_t *dst, const uint64_t *src, bool live)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(live ? 8 : 0)
                 : "memory");
}

// Asynchronous 16-byte copy global -> shared (both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async16(uint64_t *dst, const uint64_t *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__host__ __device__ inline size_t cube_tile_smem(int64_t N1)
{
    return (size_t)2 * (size_t)(N1 + 1) * (size_t)cube_tile_bi(N1) * sizeof(int64_t);
}

// Turn every column (c, ii) of a loaded tile into its inclusive prefix along a
// (wrapping uint64): NT / (2 BI) segments per column, segment sums, their
// exclusive scan, rewrite.  Called by every thread of the CTA after the tile's
// rows 1..N1 and its zero row 0 are in place and visible; ends with a barrier.
template <int NT>
__device__ __forceinline__ void cube_tile_scan(int N1, int lg, uint64_t *tile)
{
    const int tid = threadIdx.x, BI = 1 << lg;
    const unsigned cstride = (unsigned)(N1 + 1) << lg; // tile words per component
    __shared__ uint64_t s_seg[NT];
    const int ncol = 2 * BI, nseg = NT / ncol;
    const int col = tid & (ncol - 1), sg = tid >> (lg + 1);
    uint64_t *colp = tile + (col >> lg) * cstride + (col & (BI - 1));
    const int seg = (N1 + nseg - 1) / nseg;
    const int a0 = 1 + sg * seg, a1 = min(N1 + 1, a0 + seg);
    uint64_t t = 0;
    for (int a = a0; a < a1; ++a) t += colp[(unsigned)a << lg];
    s_seg[sg * ncol + col] = t;
    __syncthreads();
    uint64_t run = 0;
    for (int q = 0; q < sg; ++q) run += s_seg[q * ncol + col];
    for (int a = a0; a < a1; ++a) {
        run += colp[(unsigned)a << lg];
        colp[(unsigned)a << lg] = run;
    }
    __syncthreads();
}

// Load src[c nodes + base + a stride + ii] for c < 2, a < N1, ii < BI = 2^lg (0
// for ii >= bi, past the cube's edge) into tile[(c (N1 + 1) + a + 1) BI + ii]
// (asynchronous 8-byte copies, so that the whole tile is in flight at once),
// zero row 0 of both components, then scan (cube_tile_scan).  Offsets inside
// the cube are 32-bit (N1 <= 1024, so a * stride < 2^30).  Called by every
// thread of the CTA; ends with a barrier.
template <int NT>
__device__ __forceinline__ void cube_tile_load_scan(const int64_t *__restrict__ src, int64_t nodes, int64_t base,
                                                    unsigned stride, int N1, int lg, int bi, uint64_t *tile)
{
    const int tid = threadIdx.x, BI = 1 << lg, rstep = NT >> lg;
    const int ii = tid & (BI - 1), r0 = tid >> lg;
    const bool live = ii < bi;
    const unsigned cstride = (unsigned)(N1 + 1) << lg;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        // past the cube's edge: a zero fill from an in-bounds address
        const uint64_t *__restrict__ s = reinterpret_cast<const uint64_t *>(src) + c * nodes + base + (live ? ii : 0);
        uint64_t *t = tile + c * cstride + BI + ii;
        for (int a = r0; a < N1; a += rstep) cp_async8(t + ((unsigned)a << lg), s + (unsigned)a * stride, live);
    }
    if (tid < 2 * BI) tile[(tid >> lg) * cstride + (tid & (BI - 1))] = 0ull;
    cp_async_wait_all();
    __syncthreads();
    cube_tile_scan<NT>(N1, lg, tile);
}

// The same from a contiguous block per component (the i-block-major layout of
// the xy-window sums, blk[c] + a BI + ii, zeros already stored past the edge):
// asynchronous 16-byte copies.
template <int NT>
__device__ __forceinline__ void cube_tile_load_scan_contig(const int64_t *blk0, const int64_t *blk1, int N1, int lg,
                                                           uint64_t *tile)
{
    const int tid = threadIdx.x, BI = 1 << lg;
    const unsigned cstride = (unsigned)(N1 + 1) << lg;
    const int words = N1 << lg; // even: BI >= 4
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const uint64_t *__restrict__ s = reinterpret_cast<const uint64_t *>(c ? blk1 : blk0);
        uint64_t *t = tile + c * cstride + BI;
        for (int e = 2 * tid; e < words; e += 2 * NT) cp_async16(t + e, s + e);
    }
    if (tid < 2 * BI) tile[(tid >> lg) * cstride + (tid & (BI - 1))] = 0ull;
    cp_async_wait_all();
    __syncthreads();
    cube_tile_scan<NT>(N1, lg, tile);
}

// Window sum at a (0 <= a < N1) of a scanned column colp (its words BI = 2^lg
// apart, total = colp[N1 BI]): Pe(a + P + 1) - Pe(a - P) on the periodic
// extension Pe(x) = pre(x mod N1) + floor(x / N1) total.  As 2P + 1 <= N1, at
// most one end wraps, and either wrap adds the total once.
__device__ __forceinline__ int64_t cube_tile_window(const uint64_t *colp, int N1, int P, int lg, int a, uint64_t total)
{
    int b = a + P + 1, lo = a - P;
    const bool wb = b > N1, wl = lo < 0;
    b -= wb ? N1 : 0;
    lo += wl ? N1 : 0;
    return (int64_t)(colp[(unsigned)b << lg] - colp[(unsigned)lo << lg] + ((wb || wl) ? total : 0ull));
}

// Tiled cube y pass: CTA (ib, k); writes the window sums in the i-block-major
// layout the z-window pass reads as one contiguous block.
__global__ void __launch_bounds__(kTileThreads) cube_y_tile_kernel(LatticePlan p)
{
    if (p.skip && *(const volatile int *)p.skip) return;
    extern __shared__ int64_t tile_mem[];
    uint64_t *tile = reinterpret_cast<uint64_t *>(tile_mem);
    const int N1 = (int)p.N1, P = (int)p.P, lg = cube_tile_lg(N1), BI = 1 << lg;
    const int i0 = (int)blockIdx.x << lg, k = blockIdx.y;
    const int bi = min(BI, N1 - i0);
    const int64_t tiles = (N1 + BI - 1) >> lg;
    const int64_t *blk = p.sx + ((int64_t)k * tiles + blockIdx.x) * N1 * BI; // plane-wise i-block-major
    cube_tile_load_scan_contig<kTileThreads>(blk, blk + cube_sxy_cstride(N1), N1, lg, tile);
    const int ii = threadIdx.x & (BI - 1), r0 = threadIdx.x >> lg, rstep = kTileThreads >> lg;
    const unsigned cstride = (unsigned)(N1 + 1) << lg;
    const uint64_t *col0 = tile + ii, *col1 = tile + cstride + ii;
    const uint64_t t0 = col0[(unsigned)N1 << lg], t1 = col1[(unsigned)N1 << lg];
    // i-block-major output: element (ii, j = a, k) at ((ib N1 + a) N1 + k) BI + ii,
    // zeros past the cube's edge
    int64_t *__restrict__ d0 = p.sxy + (((int64_t)blockIdx.x * N1) * N1 + k) * BI + ii;
    int64_t *__restrict__ d1 = d0 + cube_sxy_cstride(N1);
    const unsigned dstep = (unsigned)N1 << lg;
#pragma unroll 4 // 464^3: 0.493 ms, against 0.515 (unroll 2) and 0.516-0.517 (6, 8)
    for (int a = r0; a < N1; a += rstep) {
        const bool live = ii < bi;
        d0[(unsigned)a * dstep] = live ? cube_tile_window(col0, N1, P, lg, a, t0) : 0;
        d1[(unsigned)a * dstep] = live ? cube_tile_window(col1, N1, P, lg, a, t1) : 0;
    }
}

// Tiled cube z pass, split in two kernels per stage:
//   window pass  CTA (ib, j) scans the xy-window sums of its columns along k and
//                writes every node's coupling term (lattice_coupling_term, the
//                cross product of its own (sin, cos) with its window sums) to
//                cpl; thread (ii, r0) takes the planes k = r0, r0 + kZThreads /
//                BI, ..., the own (sin, cos) of the next two in flight;
//   node pass    one warp per row of consecutive nodes (cube_nodex_kernel): the
//                slope from cpl, the RK4 update, the next (sin, cos), the next
//                stage's x-window sums of the row, and in stage 4 the order
//                parameter's partials.  STAGE 0 is the prologue: the (sin, cos)
//                of y, its x sums and its order parameter.
// The window pass keeps the tile's 64-byte row segments (the z columns are
// N1^2 elements apart), the node pass reads and writes whole warps of
// consecutive nodes.  Three window CTAs per SM at the tile sizes of N1 <= 594.
// At 464^3 (interleaved (sin, cos) pairs): two planes per unrolled iteration
// with three planes of prefetch 0.826 ms, two planes of prefetch 0.831 ms, one
// plane per iteration 0.860 ms; 512 threads (at most 42 registers) 0.884 ms.
constexpr int kZThreads = 384, kZAhead = 3, kZBlocks = 3; // kZAhead: planes of own (sin, cos) in flight

__global__ void __launch_bounds__(kZThreads, kZBlocks) cube_zw_tile_kernel(LatticePlan p)
{
    if (p.skip && *(const volatile int *)p.skip) return;
    extern __shared__ int64_t tile_mem[];
    uint64_t *tile = reinterpret_cast<uint64_t *>(tile_mem);
    const int N1 = (int)p.N1, P = (int)p.P, lg = cube_tile_lg(N1), BI = 1 << lg;
    const int i0 = (int)blockIdx.x << lg, j = blockIdx.y;
    const int bi = min(BI, N1 - i0);
    const unsigned plane = (unsigned)N1 * (unsigned)N1;
    const int64_t base = (int64_t)j * N1 + i0;
    const int64_t *blk = p.sxy + (((int64_t)blockIdx.x * N1 + j) * N1) * BI; // i-block-major
    cube_tile_load_scan_contig<kZThreads>(blk, blk + cube_sxy_cstride(N1), N1, lg, tile);
    const int ii = threadIdx.x & (BI - 1), r0 = threadIdx.x >> lg, rstep = kZThreads >> lg;
    if (ii >= bi || r0 >= N1) return; // past every barrier
    const unsigned cstride = (unsigned)(N1 + 1) << lg;
    const uint64_t *col0 = tile + ii, *col1 = tile + cstride + ii;
    const uint64_t t0 = col0[(unsigned)N1 << lg], t1 = col1[(unsigned)N1 << lg];
    const longlong2 *__restrict__ fp = reinterpret_cast<const longlong2 *>(p.f) + base + ii; // (sin, cos) pairs
    double *__restrict__ cpl = p.cpl + base + ii;
    int64_t f[kZAhead + 1][2]; // own (sin, cos) of the planes a, a + rstep, ...
#pragma unroll
    for (int d = 0; d < kZAhead; ++d) {
        const int ad = r0 + d * rstep;
        const longlong2 v = ad < N1 ? fp[(unsigned)ad * plane] : make_longlong2(0, 0);
        f[d][0] = v.x;
        f[d][1] = v.y;
    }
#pragma unroll 2 // two planes' independent chains interleaved
    for (int a = r0; a < N1; a += rstep) {
        const int an = a + kZAhead * rstep;
        const longlong2 v = an < N1 ? fp[(unsigned)an * plane] : make_longlong2(0, 0);
        f[kZAhead][0] = v.x;
        f[kZAhead][1] = v.y;
        int64_t t62[2];
        own_phase_turned(p.mp, f[0], t62);
        cpl[(unsigned)a * plane] = lattice_coupling_term(p.mp, t62, cube_tile_window(col0, N1, P, lg, a, t0),
                                                         cube_tile_window(col1, N1, P, lg, a, t1));
#pragma unroll
        for (int d = 0; d < kZAhead; ++d) {
            f[d][0] = f[d + 1][0];
            f[d][1] = f[d + 1][1];
        }
    }
}

template <int M, int STAGE>
__device__ __forceinline__ void cube_node_load(const LatticePlan &p, int64_t n, LatNodeIn<M> &in, double &c)
{
    constexpr int D = Model<M>::D, NX = Model<M>::NX, XOFF = D - NX;
    const int64_t nodes = p.nodes;
#pragma unroll
    for (int v = 0; v < D; ++v) {
        in.y[v] = __ldcg(p.y + v * nodes + n); // streamed once: L2 only, L1 left to the sin/cos table
        in.acc[v] = STAGE >= 2 ? __ldcg(p.acc + v * nodes + n) : 0.0;
    }
#pragma unroll
    for (int g = 0; g < NX; ++g) in.X[g] = STAGE <= 1 ? in.y[XOFF + g] : p.xs[g * nodes + n];
    c = STAGE > 0 ? __ldcg(p.cpl + n) : 0.0;
}

// Node pass fused with the next stage's x pass: one warp per row (k, j).  Every
// lane updates its nodes i = lane, lane + 32, ..., and their new (sin, cos)
// rounded onto 2^-F fill the row's prefix rows in shared memory; the row's
// x-window sums then go out in the plane-wise i-block-major layout the y pass
// reads.  In stage 4 (and the prologue, STAGE 0: the (sin, cos) of y, no
// update) the row's sums give the order parameter.
// The loads go through registers, U nodes of a lane ahead: six for Kuramoto
// (compiled for six CTAs per SM, at most 80 registers), four for the model
// with inertia.  Measured on the 464^3 cube, stages 2-4: U = 6 1.18 ms, U = 7 (94
// registers) 1.25 ms, U = 8 1.21 ms, U = 5 (70 registers) 1.34 ms, U = 4
// 1.33 ms; staging the row's y and coupling terms through shared memory by
// cp.async instead took 1.39 ms.  The loads bypass L1 (1% faster).
template <int M, int STAGE>
__device__ __forceinline__ void cube_nodex_row(const LatticePlan &p, const StepSize &h, int64_t row, int64_t *pre0,
                                               int64_t *pre1, bool &ok, int64_t &ps, int64_t &pc)
{
    constexpr int D = Model<M>::D, U = D == 1 ? 6 : 4;
    const int lane = threadIdx.x & 31, n1 = (int)p.N1;
    // the row's own pointers, so that every node address is a 32-bit offset
    const int64_t base = row * p.N1;
    LatticePlan q = p;
    q.y += base;
    q.acc += base;
    q.f += 2 * base; // (sin, cos) pairs
    q.cpl += base;
    if (Model<M>::NX > 0) q.xs += base;
    for (int mb = lane; mb < n1; mb += 32 * U) {
        LatNodeIn<M> in[U];
        double c[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = mb + 32 * u;
            if (i < n1) cube_node_load<M, STAGE>(q, (unsigned)i, in[u], c[u]);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = mb + 32 * u;
            if (i < n1) {
                double k[D] = {};
                if (STAGE > 0) Model<M>::rhs_from_coupling(q.mp, c[u], in[u].X, k);
                int64_t sc[2];
                int64_t unused_s = 0, unused_c = 0;
                lattice_node_update<M, STAGE, int64_t>(q, (unsigned)i, k, in[u], h, ok, unused_s, unused_c, sc);
                const int64_t qs = q62_to(sc[0], p.F), qc = q62_to(sc[1], p.F);
                pre0[i + 1] = qs;
                pre1[i + 1] = qc;
                if (STAGE == 0 || STAGE == 4) {
                    ps += qs;
                    pc += qc;
                }
            }
        }
    }
    lattice_x_scan_out<0, true>(p, row, pre0, pre1);
}

template <int M, int STAGE>
__global__ void __launch_bounds__(32 * kNodexWarpsMax, kNodexBlocks<M>) cube_nodex_kernel(LatticePlan p, const StepSize h)
{
    if (p.skip && *(const volatile int *)p.skip) return;
    extern __shared__ int64_t smem[];
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int64_t stride = p.N1 + 1, rows = p.nodes / p.N1;
    int64_t *pre0 = smem + (int64_t)warp * 2 * stride;
    int64_t *pre1 = pre0 + stride;
    const int64_t row = (int64_t)blockIdx.x * nwarps + warp;
    // a lane's order sums: at most ceil(N1 / 32) <= 32 terms of |Q| <= 2^F <= 2^56
    // (F = 61 - ceil(log2 K+) and K+ >= 27), so int64 holds them
    int64_t ps = 0, pc = 0;
    bool ok = true;
    if (row < rows) cube_nodex_row<M, STAGE>(p, h, row, pre0, pre1, ok, ps, pc); // uniform over the warp
    if (!ok) raise_error(p.err, ERR_RANGE);
    if (STAGE == 0 || STAGE == 4) { // the order parameter's partials (lattice_order_kernel adds them up)
        i128 ts = ps, tc = pc;
        cta_sum_pair(ts, tc);
        if (threadIdx.x == 0) {
            st_i128(p.partial + 2 * blockIdx.x, ts);
            st_i128(p.partial + 2 * blockIdx.x + 1, tc);
        }
    }
}

// Batched cube z pass (stages 1-4): CTA b is CTA b - yz_base[m] of member m.
template <int M, int STAGE>
__global__ void __launch_bounds__(kColThreads)
    cube_batch_z_kernel(const LatticePlan *__restrict__ plans, const int *__restrict__ yz_item,
                        const int64_t *__restrict__ yz_base, const StepSize h)
{
    const int inst = yz_item[blockIdx.x];
    const LatticePlan &p = plans[inst];
    const int64_t lb = (int64_t)blockIdx.x - yz_base[inst];
    int64_t bx, j, seg;
    cube_col_item(p, lb, bx, j, seg);
    const int64_t nbx = (p.N1 + kColThreads - 1) / kColThreads;
    cube_z_col<M, STAGE>(p, h, bx, j, seg, (unsigned)lb, (unsigned)(nbx * p.N1 * col_segments(p.N1)));
}

// ball / disk gather: one node per thread; the window is the union of the chords
// (dy, dz, w) of the plan's table.  WMODE: one load per chord, the x-window sum
// S_w of the chord's row; otherwise two, the difference of the row's extended
// prefix at both ends (wrapping arithmetic; every chord sum and the window sum
// itself are exact either way, so both give the same bits).
template <int M, int STAGE, bool WMODE>
__global__ void __launch_bounds__(kGatherThreads) lattice_gather_kernel(LatticePlan p, const StepSize h)
{
    if (STAGE == 1 && p.skip && *(const volatile int *)p.skip) return; // stage 1 records nothing
    const int64_t N1 = p.N1, nodes = p.nodes;
    const int64_t n = (int64_t)blockIdx.x * kGatherThreads + threadIdx.x;
    i128 ps = 0, pc = 0;
    bool ok = true;
    if (n < nodes) {
        const int i = (int)(n % N1), j = (int)((n / N1) % N1), k = p.dims == 3 ? (int)(n / (N1 * N1)) : 0;
        const int n1 = (int)N1;
        uint64_t w0 = 0, w1 = 0;
        if (STAGE > 0) {
            const longlong2 *__restrict__ E =
                reinterpret_cast<const longlong2 *>(p.sx) + (WMODE ? (int64_t)i : (int64_t)(i + p.P + 1));
            const int nch = p.nchords;
#pragma unroll 4
            for (int c = 0; c < nch; ++c) {
                const int4 ch = __ldg(p.chords + c); // (dy, dz, w, 0)
                int jj = j + ch.x, kk = k + ch.y;
                jj += jj < 0 ? n1 : 0;
                jj -= jj >= n1 ? n1 : 0;
                kk += kk < 0 ? n1 : 0;
                kk -= kk >= n1 ? n1 : 0;
                if (WMODE) {
                    const longlong2 v = __ldg(E + (int64_t)ch.z * nodes + (int64_t)(kk * n1 + jj) * N1);
                    w0 += (uint64_t)v.x;
                    w1 += (uint64_t)v.y;
                } else {
                    const longlong2 *r = E + (int64_t)(kk * n1 + jj) * p.rs;
                    const longlong2 b = __ldg(r + ch.z), a = __ldg(r - ch.z - 1);
                    w0 += (uint64_t)b.x - (uint64_t)a.x;
                    w1 += (uint64_t)b.y - (uint64_t)a.y;
                }
            }
        }
        lattice_node<M, STAGE>(p, n, (int64_t)w0, (int64_t)w1, h, ok, ps, pc);
    }
    if (!ok) raise_error(p.err, ERR_RANGE);
    if (STAGE == 0 || STAGE == 4) lattice_record_order(p, ps, pc, blockIdx.x, gridDim.x, p.done_ctr);
}

// ---------------------------------------------------------------------------
static dim3 tile_grid(int64_t N1)
{
    const int BI = cube_tile_bi(N1);
    return dim3((unsigned)((N1 + BI - 1) / BI), (unsigned)N1, 1);
}

static unsigned gather_grid(const LatticePlan &p)
{
    return (unsigned)((p.nodes + kGatherThreads - 1) / kGatherThreads);
}

int64_t lattice_sx_elems(int topo, int64_t N1, int64_t P, bool wmode)
{
    if (topo == 1) return lattice_sxy_elems(N1); // both layouts of the x pass's output
    const int64_t rows = topo == 3 ? N1 : N1 * N1;
    return wmode ? 2 * (P + 1) * rows * N1 : 2 * rows * (N1 + 2 * P + 1);
}

int64_t lattice_sxy_elems(int64_t N1)
{
    const int64_t a = N1 * N1 * N1, b = cube_sxy_cstride(N1);
    return 2 * (a > b ? a : b);
}

int64_t lattice_partial_blocks(int topo, int64_t N1)
{
    const int64_t a = lattice_order_blocks(topo, N1);
    if (topo != 1) return a;
    // the fused node pass (one row per warp) and the order kernel's second level
    const int64_t b = (N1 * N1 + nodex_warps(N1) - 1) / nodex_warps(N1) + kOrderCtas;
    return a > b ? a : b;
}

int64_t lattice_order_blocks(int topo, int64_t N1)
{
    if (topo == 1) return ((N1 + kColThreads - 1) / kColThreads) * N1 * col_segments(N1);
    const int64_t nodes = topo == 3 ? N1 * N1 : N1 * N1 * N1;
    return (nodes + kGatherThreads - 1) / kGatherThreads;
}

cudaError_t lattice_configure()
{
    cudaError_t e = cudaFuncSetAttribute(lattice_x_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kRowSmemMax);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(lattice_x_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kRowSmemMax);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(lattice_x_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kRowSmemMax);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(cube_batch_x_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kRowSmemMax);
    // the largest tile of any edge: the top edge of each tile width
    const int tmax = (int)std::max(std::max(cube_tile_smem(297), cube_tile_smem(594)), cube_tile_smem(1024));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(cube_y_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, tmax);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(cube_zw_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, tmax);
#define SIM_NODEX_ATTR(M, S)                                                                                           \
    if (e == cudaSuccess)                                                                                              \
        e = cudaFuncSetAttribute(cube_nodex_kernel<M, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRowSmemMax);
    SIM_NODEX_ATTR(0, 0) SIM_NODEX_ATTR(0, 1) SIM_NODEX_ATTR(0, 2) SIM_NODEX_ATTR(0, 3) SIM_NODEX_ATTR(0, 4)
    SIM_NODEX_ATTR(3, 0) SIM_NODEX_ATTR(3, 1) SIM_NODEX_ATTR(3, 2) SIM_NODEX_ATTR(3, 3) SIM_NODEX_ATTR(3, 4)
#undef SIM_NODEX_ATTR
    return e;
}

int lattice_row_warps(int64_t N1) { return row_warps(N1); }

// Batched cube members of one model: one x, one y and one z launch over all of
// them per pass (each member with its own plan, prefix rows and order-parameter
// counter).  Between steps a cube's x-window sums hold the sums of y (the
// prologue, the fused node pass of a single cube's stage 4 and the batch's last
// x pass keep it so), so a step begins with the y pass and a member can be
// stepped alone or in a batch in any order; the results are the same bits.
static cudaError_t cube_batch_x(const CubeBatchGroup &g, cudaStream_t s)
{
    const size_t smem = (size_t)g.w * 2 * (size_t)(g.n1_max + 1) * sizeof(int64_t);
    cube_batch_x_kernel<<<(unsigned)g.n_x, 32 * g.w, smem, s>>>(g.plans, g.x_item, g.x_base);
    return cudaGetLastError();
}

template <int M>
static cudaError_t cube_batch_yz(int stage, const CubeBatchGroup &g, double dt, cudaStream_t s)
{
    cube_batch_y_kernel<<<(unsigned)g.n_yz, kColThreads, 0, s>>>(g.plans, g.yz_item, g.yz_base);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const StepSize h = step_size(dt);
    const dim3 grid((unsigned)g.n_yz);
    switch (stage) {
    case 1: cube_batch_z_kernel<M, 1><<<grid, kColThreads, 0, s>>>(g.plans, g.yz_item, g.yz_base, h); break;
    case 2: cube_batch_z_kernel<M, 2><<<grid, kColThreads, 0, s>>>(g.plans, g.yz_item, g.yz_base, h); break;
    case 3: cube_batch_z_kernel<M, 3><<<grid, kColThreads, 0, s>>>(g.plans, g.yz_item, g.yz_base, h); break;
    default: cube_batch_z_kernel<M, 4><<<grid, kColThreads, 0, s>>>(g.plans, g.yz_item, g.yz_base, h); break;
    }
    return cudaGetLastError();
}

cudaError_t cube_batch_step(const CubeBatchGroup &g, double dt, cudaStream_t s)
{
    if (g.n_x == 0) return cudaSuccess;
    for (int stage = 1; stage <= 4; ++stage) {
        cudaError_t e = stage > 1 ? cube_batch_x(g, s) : cudaSuccess;
        if (e == cudaSuccess) e = g.model == 3 ? cube_batch_yz<3>(stage, g, dt, s) : cube_batch_yz<0>(stage, g, dt, s);
        if (e != cudaSuccess) return e;
    }
    return cube_batch_x(g, s); // the x sums of y_{n+1}
}

// CTAs of a lattice x pass: one row per warp.
static unsigned x_grid(const LatticePlan &p)
{
    const int w = row_warps(p.N1);
    const int64_t rows = p.nodes / p.N1;
    return (unsigned)((rows + w - 1) / w);
}

static size_t x_smem(const LatticePlan &p)
{
    return (size_t)row_warps(p.N1) * 2 * (size_t)(p.N1 + 1) * sizeof(int64_t);
}

static cudaError_t launch_x(const LatticePlan &p, cudaStream_t s)
{
    const int w = row_warps(p.N1);
    if (p.topo == 1) lattice_x_kernel<0><<<x_grid(p), 32 * w, x_smem(p), s>>>(p);
    else if (p.wmode) lattice_x_kernel<2><<<x_grid(p), 32 * w, x_smem(p), s>>>(p);
    else lattice_x_kernel<1><<<x_grid(p), 32 * w, x_smem(p), s>>>(p);
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) kernel_mark(s, 0);
    return e;
}

// Stage STAGE of a single cube after its x pass: y pass, z-window pass, and the
// node pass fused with the next x pass (STAGE 0: the fused pass alone, the
// prologue).
template <int M, int STAGE>
static cudaError_t launch_cube_stage(const LatticePlan &p, double dt, cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    if (STAGE > 0) {
        cube_y_tile_kernel<<<tile_grid(p.N1), kTileThreads, cube_tile_smem(p.N1), s>>>(p);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        kernel_mark(s, 1);
        cube_zw_tile_kernel<<<tile_grid(p.N1), kZThreads, cube_tile_smem(p.N1), s>>>(p);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        kernel_mark(s, 3);
    }
    const int w = nodex_warps(p.N1);
    const int64_t rows = p.nodes / p.N1;
    const unsigned nblk = (unsigned)((rows + w - 1) / w);
    cube_nodex_kernel<M, STAGE><<<nblk, 32 * w, (size_t)w * 2 * (size_t)(p.N1 + 1) * sizeof(int64_t), s>>>(
        p, step_size(dt));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    kernel_mark(s, 2);
    if (STAGE == 0 || STAGE == 4) {
        lattice_order_kernel<<<kOrderCtas, kOrderThreads, 0, s>>>(p, nblk);
        if ((e = cudaGetLastError()) == cudaSuccess) kernel_mark(s, 0);
    }
    return e;
}

// Stage STAGE of a ball or disk: x pass and gather (STAGE 0: the gather alone,
// the prologue).
template <int M, int STAGE>
static cudaError_t launch_gather_stage(const LatticePlan &p, double dt, cudaStream_t s)
{
    cudaError_t e = STAGE > 0 ? launch_x(p, s) : cudaSuccess;
    if (e != cudaSuccess) return e;
    if (p.wmode && STAGE > 0)
        lattice_gather_kernel<M, STAGE, true><<<gather_grid(p), kGatherThreads, 0, s>>>(p, step_size(dt));
    else lattice_gather_kernel<M, STAGE, false><<<gather_grid(p), kGatherThreads, 0, s>>>(p, step_size(dt));
    if ((e = cudaGetLastError()) == cudaSuccess && STAGE > 0) kernel_mark(s, 2);
    return e;
}

template <int M>
static cudaError_t launch_stage(int stage, const LatticePlan &p, double dt, cudaStream_t s)
{
    if (p.topo == 1) {
        switch (stage) {
        case 0: return launch_cube_stage<M, 0>(p, dt, s);
        case 1: return launch_cube_stage<M, 1>(p, dt, s);
        case 2: return launch_cube_stage<M, 2>(p, dt, s);
        case 3: return launch_cube_stage<M, 3>(p, dt, s);
        default: return launch_cube_stage<M, 4>(p, dt, s);
        }
    }
    switch (stage) {
    case 0: return launch_gather_stage<M, 0>(p, dt, s);
    case 1: return launch_gather_stage<M, 1>(p, dt, s);
    case 2: return launch_gather_stage<M, 2>(p, dt, s);
    case 3: return launch_gather_stage<M, 3>(p, dt, s);
    default: return launch_gather_stage<M, 4>(p, dt, s);
    }
}

static cudaError_t launch_any(int stage, const LatticePlan &p, double dt, cudaStream_t s)
{
    return p.model == 3 ? launch_stage<3>(stage, p, dt, s) : launch_stage<0>(stage, p, dt, s);
}

// The (sin, cos) of y and its order parameter (the cube: also its x sums).
cudaError_t lattice_prologue(const LatticePlan &p, cudaStream_t s)
{
    return launch_any(0, p, 0.0, s);
}

// k = f(y) into acc (stage 1 with dt = 0, from the stored (sin, cos) of y).
cudaError_t lattice_rhs(const LatticePlan &p, cudaStream_t s)
{
    if (p.topo == 1) {
        const cudaError_t e = launch_x(p, s); // y may be a stage input that has no x sums yet
        if (e != cudaSuccess) return e;
    }
    return launch_any(1, p, 0.0, s);
}

cudaError_t lattice_step(const LatticePlan &p, double dt, cudaStream_t s)
{
    for (int stage = 1; stage <= 4; ++stage) {
        const cudaError_t e = launch_any(stage, p, dt, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

} // namespace simk
