// General link matrices (Section III.C) stepped with RK4 through the compressed
// form of Algorithm 2.
//
// COMPRESS (on the host, sim_api.cu) keeps a common vector V (the most frequent
// shifted row; the paper takes row 0) and, for
// every row i, a reference C_i to the difference entry D = XOR(ROL(row_i, i), V);
// EXTRACT gives row i = ROR(XOR(V, D_{C_i}), i).  So the coupling sum of node i is
//   W(i) = sum_{p in V} Q(x_{i+p}) + sum_{p in D_{C_i}} s_p Q(x_{i+p})   (indices mod N)
// with s_p = -1 where p is in V (the XOR clears that bit) and +1 elsewhere.  Here
// V is stored as runs of consecutive offsets [a, a + len), and the sum over a run
// is the difference of two entries of the exact prefix of Q in node order,
//   P(i + a + len) - P(i + a),
// the same exact fixed-point prefix the ring stage kernels build (P over the
// periodic extension).  A node therefore costs O(number of runs + size of its
// difference entry) reads instead of one per link: a ring is two runs and the
// empty entry, a periodic lattice one run per row of its window plus the
// wrapped links near the boundary.  As in the ring kernel, the exact prefix at
// the pieces the CTA's run ends fall in is computed once per CTA, so a run costs
// a node one load per end and component.  The degree of the node (its link
// count, which normalises the coupling) comes with its entry.
#include "ring_parts.cuh"

namespace simk {

// Exact prefix P(pos) = sum_{m < pos} Q_m of component c on the periodic
// extension, pos in [0, 2N).
__device__ __forceinline__ i128 graph_prefix_at(const RingPlan &P, const RingStageIO &a, int c, int64_t pos)
{
    const int64_t N = P.N;
    const i128 *grpofs = a.grpofs_in + c * (P.ngroups + 1);
    i128 base = 0;
    if (pos >= N) {
        pos -= N;
        base = ldg_i128(grpofs + P.ngroups);
    }
    if (pos == 0) return base;
    const int64_t s = (pos - 1) >> kSubLog2;
    return base + ldg_i128(grpofs + (s >> kGroupLog2)) + ldg_i128(a.ingrp_in + c * P.nsub + s) +
           (i128)__ldg(a.lam_in + c * N + pos - 1);
}

// Per-CTA bases of the run ends: for run r, end 2r is i + a (the run's first
// offset) and end 2r+1 is i + a + len; over the CTA's consecutive nodes each end
// covers at most three pieces (split at sub-tile starts and at N), whose exact
// prefix at the piece start is computed once, so a node needs one in-sub-tile
// prefix load per end.  Runs past kGraphSmemRuns use graph_prefix_at.
constexpr int kGraphSmemRuns = 128;
template <int NQ> struct GraphBases {
    i128 base[2 * kGraphSmemRuns][3][NQ];
    int64_t start[2 * kGraphSmemRuns][3], qn[2 * kGraphSmemRuns][3];
};

template <int NQ>
__device__ __forceinline__ void graph_load_bases(const GraphPlan &G, const RingStageIO &a, int64_t sub, int nb,
                                                 GraphBases<NQ> &B)
{
    const RingPlan &P = G.r;
    const int64_t N = P.N, nsub = P.nsub, ngroups = P.ngroups;
    const int64_t nvalid = N - sub * kSubTile < kSubTile ? N - sub * kSubTile : kSubTile;
    for (int e = threadIdx.x; e < 2 * nb; e += blockDim.x) {
        const int2 run = __ldg(G.runs + (e >> 1));
        const int64_t p0 = sub * kSubTile + run.x + ((e & 1) ? run.y : 0);
        const int64_t p1 = p0 + nvalid - 1; // in [0, 2N)
        int64_t p = p0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (p > p1) {
                B.start[e][k] = INT64_MAX;
                B.qn[e][k] = 0;
                continue;
            }
            const int64_t qn = p >= N ? N : 0, pp = p - qn;
            const int64_t st = pp >> kSubLog2;
            int64_t end = ((st + 1) << kSubLog2) - 1;
            if (end > N - 1) end = N - 1;
#pragma unroll
            for (int c = 0; c < NQ; ++c) {
                const i128 *grpofs = a.grpofs_in + c * (ngroups + 1);
                const i128 tot = ldg_i128(grpofs + ngroups);
                // st == nsub only for pp == N (never: pp < N here)
                B.base[e][k][c] = ldg_i128(grpofs + (st >> kGroupLog2)) + ldg_i128(a.ingrp_in + c * nsub + st) +
                                  (qn ? tot : (i128)0);
            }
            B.start[e][k] = p;
            B.qn[e][k] = qn;
            p = end + qn + 1;
        }
    }
    __syncthreads();
}

template <int NQ> struct GraphGather {
    struct Pre {
        int64_t l[NQ], lp[NQ];
    };
    const GraphPlan &G;
    const RingStageIO &a;
    GraphBases<NQ> &B;
    int nb;      // runs with per-CTA bases
    int64_t sub; // the CTA's sub-tile
    __device__ __forceinline__ void load(int tid, int64_t i, Pre &pre) const
    {
        const int64_t N = G.r.N;
#pragma unroll
        for (int c = 0; c < NQ; ++c) {
            const int64_t *lam = a.lam_in + c * N;
            pre.l[c] = __ldg(lam + i);
            pre.lp[c] = tid ? __ldg(lam + i - 1) : 0;
        }
    }
    __device__ __forceinline__ void sync() const { graph_load_bases<NQ>(G, a, sub, nb, B); }
    __device__ __forceinline__ void finish(int tid, int64_t i, const Pre &pre, int64_t (&qo)[NQ], double (&fo)[NQ],
                                           i128 (&W)[NQ], int64_t &wsize, double &cs) const
    {
        const RingPlan &P = G.r;
        const int64_t N = P.N;
#pragma unroll
        for (int c = 0; c < NQ; ++c) {
            qo[c] = pre.l[c] - pre.lp[c];
            fo[c] = fixed_to_double(qo[c], P.F);
            W[c] = 0;
        }
        // the common vector: runs of consecutive offsets, through the CTA's bases
        for (int r = 0; r < nb; ++r) {
            const int2 run = __ldg(G.runs + r);
            const int64_t lo = i + run.x, hi = lo + run.y;
            const int el = 2 * r, eh = 2 * r + 1;
            const int kl = (lo >= B.start[el][1]) + (lo >= B.start[el][2]);
            const int kh = (hi >= B.start[eh][1]) + (hi >= B.start[eh][2]);
            const int64_t pl = lo - B.qn[el][kl], ph = hi - B.qn[eh][kh];
#pragma unroll
            for (int c = 0; c < NQ; ++c) {
                const int64_t *lam = a.lam_in + c * N;
                const int64_t ll = (pl & (kSubTile - 1)) ? __ldg(lam + pl - 1) : 0;
                const int64_t lh = (ph & (kSubTile - 1)) ? __ldg(lam + ph - 1) : 0;
                W[c] += (B.base[eh][kh][c] - B.base[el][kl][c]) + (i128)(lh - ll);
            }
        }
        for (int r = nb; r < G.nruns; ++r) {
            const int2 run = __ldg(G.runs + r); // (a, len), a + len <= N
            const int64_t lo = i + run.x, hi = lo + run.y;
#pragma unroll
            for (int c = 0; c < NQ; ++c) W[c] += graph_prefix_at(P, a, c, hi) - graph_prefix_at(P, a, c, lo);
        }
        // the node's difference entry: signed single links
        const int e = __ldg(G.ent + i);
        const int64_t t0 = __ldg(G.dptr + e), t1 = __ldg(G.dptr + e + 1);
        for (int64_t t = t0; t < t1; ++t) {
            const int2 d = __ldg(G.dpos + t); // (offset, sign)
            int64_t j = i + d.x;
            j -= j >= N ? N : 0;
#pragma unroll
            for (int c = 0; c < NQ; ++c) {
                const int64_t *lam = a.lam_in + c * N;
                const int64_t q = (j & (kSubTile - 1)) ? __ldg(lam + j) - __ldg(lam + j - 1) : __ldg(lam + j);
                W[c] += d.y > 0 ? (i128)q : -(i128)q;
            }
        }
        wsize = __ldg(G.ek + e);
        cs = __ldg(G.ecs + e);
    }
};

// the run loop and 128-bit window sums need more registers than the ring kernel
template <int M> struct GraphMinBlocks { static constexpr int value = 3; };
template <> struct GraphMinBlocks<2> { static constexpr int value = 2; };

template <int M, int STAGE>
__global__ void __launch_bounds__(kRingThreads, GraphMinBlocks<M>::value)
    graph_stage_kernel(const GraphPlan g, const StepSize h)
{
    if (g.r.skip && *(const volatile int *)g.r.skip) return; // uniform over the launch
    constexpr int NQ = Model<M>::NQ;
    __shared__ GraphBases<NQ> s_bases;
    const RingStageIO a = stage_io<M, STAGE>(g.r);
    const int nb = g.nruns < kGraphSmemRuns ? g.nruns : kGraphSmemRuns;
    stage_body<M, STAGE>(g.r, a, h, blockIdx.x, GraphGather<NQ>{g, a, s_bases, nb, (int64_t)blockIdx.x});
}

template <int M>
static cudaError_t launch_stage(int stage, const GraphPlan &g, double dt, cudaStream_t s)
{
    const dim3 grid((unsigned)g.r.nsub), block(kRingThreads);
    switch (stage) {
    case 1: graph_stage_kernel<M, 1><<<grid, block, 0, s>>>(g, step_size(dt)); break;
    case 2: graph_stage_kernel<M, 2><<<grid, block, 0, s>>>(g, step_size(dt)); break;
    case 3: graph_stage_kernel<M, 3><<<grid, block, 0, s>>>(g, step_size(dt)); break;
    default: graph_stage_kernel<M, 4><<<grid, block, 0, s>>>(g, step_size(dt)); break;
    }
    return cudaGetLastError();
}

static cudaError_t launch_any(int stage, const GraphPlan &g, double dt, cudaStream_t s)
{
    switch (g.r.model) {
    case 0: return launch_stage<0>(stage, g, dt, s);
    case 1: return launch_stage<1>(stage, g, dt, s);
    case 2: return launch_stage<2>(stage, g, dt, s);
    default: return launch_stage<3>(stage, g, dt, s);
    }
}

cudaError_t graph_rhs(const GraphPlan &g, cudaStream_t s)
{
    return launch_any(1, g, 0.0, s);
}

cudaError_t graph_step(const GraphPlan &g, double dt, cudaStream_t s)
{
    for (int stage = 1; stage <= 4; ++stage) {
        const cudaError_t e = launch_any(stage, g, dt, s);
        if (e != cudaSuccess) return e;
        kernel_mark(s, 0);
    }
    return cudaSuccess;
}

} // namespace simk
