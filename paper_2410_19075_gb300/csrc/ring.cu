// Ring topology: one fused kernel per RK4 stage.
//
// Stage s (s = 1..4) of node i, in one pass over the ring (Section IV 1D
// networks; the per-node right-hand side of Algorithm 1):
//   a3  window sums   W(i) = P(i+R+1) - P(i-R), P(p) = sum_{j<p} Q(f_j) over the
//                     periodic extension, read from the exact prefix arrays the
//                     previous kernel wrote (two shifted reads per quantity);
//   a4  right-hand side k_s(i) from W(i) and the node's own stage input;
//   a5  RK4 accumulate acc += b_s k_s (stage 4: y <- y + dt/6 (acc + k_4));
//   a1  next stage input x_{s+1} = y + c_{s+1} dt k_s;
//   a2  coupled quantity f(x_{s+1}), its exact prefix inside each 256-node
//       sub-tile (one CTA), and, without any CTA waiting for another, the exact
//       prefix at every sub-tile start: the last CTA to finish in each group of
//       64 sub-tiles scans that group, and the last group scans the groups; or,
//       for rings of at most 64 groups (one-pass prefix, ring_parts.cuh), the
//       sub-tile totals and group accumulators the next kernel sums itself;
//   a6  (stage 4) the Kuramoto order parameter of y_{n+1} from the global totals.
// The prologue kernel does a1/a2/a6 for the initial state.  The Kuramoto and
// FHN rings run ring_stage_kernel2 (two adjacent nodes per thread) unless the
// autotuner chose ring_stage_kernel (one node per thread), which HH always
// runs.  The building blocks are in ring_parts.cuh.
#include "ring_parts.cuh"

namespace simk {

// Ring window in three phases.  load(): the node's own prefix entries and the
// in-sub-tile prefix at both window ends, b = i+R+1 and a = i-R on the periodic
// extension (a piece never straddles 0 or N, so the copy of the ring each end
// falls in is known without the bases).  sync(): the bases threads 0 and 1
// computed become visible.  finish(): W = base(b) - base(a) + the loaded parts,
// exactly as ring_window computes it.
template <int NQ> struct RingGather {
    struct Pre {
        int64_t l[NQ], lp[NQ], lb[NQ], la[NQ];
    };
    const RingPlan &P;
    const int64_t *lam_in;
    const RingBases<NQ> &B;
    __device__ __forceinline__ void load(int tid, int64_t i, Pre &pre) const
    {
        const int64_t N = P.N;
        const int64_t b = i + P.R + 1, am = i - P.R;
        const int64_t bp = b >= N ? b - N : b, ap = am < 0 ? am + N : am;
#pragma unroll
        for (int c = 0; c < NQ; ++c) {
            const int64_t *lam = lam_in + c * N;
            pre.l[c] = __ldg(lam + i);
            pre.lp[c] = tid ? __ldg(lam + i - 1) : 0;
            pre.lb[c] = (bp & (kSubTile - 1)) ? __ldg(lam + bp - 1) : 0;
            pre.la[c] = (ap & (kSubTile - 1)) ? __ldg(lam + ap - 1) : 0;
        }
    }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
    __device__ __forceinline__ void finish(int tid, int64_t i, const Pre &pre, int64_t (&qo)[NQ], double (&fo)[NQ],
                                           i128 (&W)[NQ], int64_t &wsize, double &cs) const
    {
        const int64_t b = i + P.R + 1, am = i - P.R;
        const int kb = (b >= B.start[0][1]) + (b >= B.start[0][2]);
        const int ka = (am >= B.start[1][1]) + (am >= B.start[1][2]);
#pragma unroll
        for (int c = 0; c < NQ; ++c) {
            qo[c] = pre.l[c] - pre.lp[c];
            fo[c] = fixed_to_double(qo[c], P.F);
            W[c] = (B.base[0][kb][c] - B.base[1][ka][c]) + (i128)(pre.lb[c] - pre.la[c]);
        }
        wsize = -1; // the network's window size
        cs = 1.0;
    }
};

// One 256-node sub-tile `sub` of ring P, one node per thread (the whole CTA).
// FLAT_OK: the plain kernel, which may run the one-pass prefix (batched members
// always keep the two-level scan).
template <int M, int STAGE, bool FLAT_OK>
__device__ __forceinline__ void ring_stage_body(const RingPlan &P, const RingStageIO &a, const StepSize &h,
                                                int64_t sub)
{
    constexpr int NQ = Model<M>::NQ;
    __shared__ RingBases<NQ> s_bases;
    if (STAGE > 0) {
        if (FLAT_OK && P.flat) ring_flat_bases<NQ>(P, a.fsub_in, a.facc_in, sub, s_bases);
        else ring_compute_bases<NQ>(P, a.ingrp_in, a.grpofs_in, sub, s_bases);
    }
    stage_body<M, STAGE, RingGather<NQ>, FLAT_OK>(P, a, h, sub, RingGather<NQ>{P, a.lam_in, s_bases});
}

// Two adjacent nodes per thread, 128 threads per 256-node sub-tile: two
// independent right-hand sides per thread and one warp scan per node pair.  The
// same integers and FP64 expressions as ring_stage_body, so the same bits.
constexpr int kRing2Threads = kSubTile / 2;
#ifndef SIM_RING2_MIN_BLOCKS
#define SIM_RING2_MIN_BLOCKS 8
#endif

template <int M, int STAGE>
__device__ __forceinline__ void ring_stage_body2(const RingPlan &P, const RingStageIO &a, const StepSize &h,
                                                 int64_t sub)
{
    using Mo = Model<M>;
    constexpr int D = Mo::D, NQ = Mo::NQ, NX = Mo::NX;
    constexpr int XOFF = D - NX;
    __shared__ RingBases<NQ> s_bases;
    const int tid = threadIdx.x;
    const int64_t N = P.N;
    const int64_t i0 = sub * kSubTile + 2 * tid;
    const bool flat = P.flat != 0;
    if (STAGE > 0) {
        if (flat) ring_flat_bases<NQ>(P, a.fsub_in, a.facc_in, sub, s_bases);
        else ring_compute_bases<NQ>(P, a.ingrp_in, a.grpofs_in, sub, s_bases);
    }

    int64_t l[NQ][2], lp[NQ], lb[NQ][2], la[NQ][2];
    double yv[2][D], av[2][D], X[2][NX > 0 ? NX : 1], Iext[2] = {0.0, 0.0};
    if (STAGE > 0) {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int64_t i = i0 + u;
            if (i < N) {
                const int64_t b = i + P.R + 1, am = i - P.R;
                const int64_t bp = b >= N ? b - N : b, ap = am < 0 ? am + N : am;
#pragma unroll
                for (int c = 0; c < NQ; ++c) {
                    const int64_t *lam = a.lam_in + c * N;
                    l[c][u] = __ldg(lam + i);
                    if (u == 0) lp[c] = tid ? __ldg(lam + i - 1) : 0;
                    lb[c][u] = (bp & (kSubTile - 1)) ? __ldg(lam + bp - 1) : 0;
                    la[c][u] = (ap & (kSubTile - 1)) ? __ldg(lam + ap - 1) : 0;
                }
#pragma unroll
                for (int v = 0; v < D; ++v) {
                    yv[u][v] = P.y[v * N + i];
                    av[u][v] = STAGE >= 2 ? P.acc[v * N + i] : 0.0;
                }
#pragma unroll
                for (int g = 0; g < NX; ++g) X[u][g] = a.x_in[g * N + i];
                if (M == 2 && P.node_param) Iext[u] = P.node_param[i];
            }
        }
        __syncthreads();
    }

    int64_t qv[NQ][2];
    bool ok = true;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int64_t i = i0 + u;
#pragma unroll
        for (int c = 0; c < NQ; ++c) qv[c][u] = 0;
        if (i >= N) continue;
        double xn[D];
        if (STAGE == 0) {
#pragma unroll
            for (int v = 0; v < D; ++v) xn[v] = P.y[v * N + i];
        } else {
            const int64_t b = i + P.R + 1, am = i - P.R;
            const int kb = (b >= s_bases.start[0][1]) + (b >= s_bases.start[0][2]);
            const int ka = (am >= s_bases.start[1][1]) + (am >= s_bases.start[1][2]);
            int64_t qo[NQ];
            double fo[NQ];
            i128 W[NQ];
#pragma unroll
            for (int c = 0; c < NQ; ++c) {
                qo[c] = l[c][u] - (u == 0 ? lp[c] : l[c][0]);
                fo[c] = fixed_to_double(qo[c], P.F);
                W[c] = (s_bases.base[0][kb][c] - s_bases.base[1][ka][c]) + (i128)(lb[c][u] - la[c][u]);
            }
            double k[D];
            Mo::rhs(P.mp, P.F, fo, qo, W, X[u], Iext[u], k);
#pragma unroll
            for (int v = 0; v < D; ++v) {
                if (STAGE == 1) {
                    P.acc[v * N + i] = k[v];
                    xn[v] = yv[u][v] + h.half * k[v];
                } else if (STAGE == 2) {
                    P.acc[v * N + i] = av[u][v] + 2.0 * k[v];
                    xn[v] = yv[u][v] + h.half * k[v];
                } else if (STAGE == 3) {
                    P.acc[v * N + i] = av[u][v] + 2.0 * k[v];
                    xn[v] = yv[u][v] + h.dt * k[v];
                } else {
                    const double yn = yv[u][v] + h.sixth * (av[u][v] + k[v]);
                    P.y[v * N + i] = yn;
                    xn[v] = yn;
                }
            }
            if (NX > 0 && STAGE >= 1 && STAGE <= 3) {
#pragma unroll
                for (int g = 0; g < NX; ++g) a.x_out[g * N + i] = xn[XOFF + g];
            }
        }
        int64_t qn[NQ];
        Mo::coupled_q(P.mp, xn, P.F, P.lim, ok, qn);
#pragma unroll
        for (int c = 0; c < NQ; ++c) qv[c][u] = qn[c];
    }
    if (!ok) raise_error(P.err, ERR_RANGE);
    // the prologue writes both prefix forms (a later kernel of either kind may read it)
    ring_prefix_tail_n<NQ, 2, (M == 0 || M == 3) && (STAGE == 0 || STAGE == 4), STAGE == 4>(
        P, a.lam_out, a.ingrp_out, a.grpofs_out, sub, i0, qv, flat, STAGE == 0 || !flat, a.fsub_out, a.facc_out,
        a.facc_zero);
}

template <int M, int STAGE>
__global__ void __launch_bounds__(kRing2Threads, SIM_RING2_MIN_BLOCKS)
    ring_stage_kernel2(const RingPlan p, const StepSize h)
{
    if (p.skip && *(const volatile int *)p.skip) return; // uniform over the launch
    ring_stage_body2<M, STAGE>(p, stage_io<M, STAGE>(p), h, blockIdx.x);
}

// Plain path: one ring, one sub-tile per CTA.
template <int M, int STAGE>
__global__ void __launch_bounds__(kRingThreads, MinBlocks<M>::value) ring_stage_kernel(const RingPlan p, const StepSize h)
{
    if (p.skip && *(const volatile int *)p.skip) return; // uniform over the launch
    ring_stage_body<M, STAGE, true>(p, stage_io<M, STAGE>(p), h, blockIdx.x);
}

// Batched path: CTA b works on sub-tile b - item_base[inst] of ring inst =
// inst_of_item[b]; every ring keeps its own exact prefix hierarchy.  A ring whose
// step budget (steps_left) is used up is skipped whole, so its arrival counters
// stay consistent.
template <int M, int STAGE>
__global__ void __launch_bounds__(kRingThreads, MinBlocks<M>::value)
    ring_batch_stage_kernel(const RingPlan *__restrict__ plans, const int *__restrict__ inst_of_item,
                            const int64_t *__restrict__ item_base, const StepSize h)
{
    const int inst = inst_of_item[blockIdx.x];
    const RingPlan &p = plans[inst];
    if (p.steps_left && *(volatile long long *)p.steps_left <= 0) return;
    ring_stage_body<M, STAGE, false>(p, stage_io<M, STAGE>(p), h, (int64_t)blockIdx.x - item_base[inst]);
}

// The same with two adjacent nodes per thread (ring_stage_body2).
template <int M, int STAGE>
__global__ void __launch_bounds__(kRing2Threads, SIM_RING2_MIN_BLOCKS)
    ring_batch_stage_kernel2(const RingPlan *__restrict__ plans, const int *__restrict__ inst_of_item,
                             const int64_t *__restrict__ item_base, const StepSize h)
{
    const int inst = inst_of_item[blockIdx.x];
    const RingPlan &p = plans[inst];
    if (p.steps_left && *(volatile long long *)p.steps_left <= 0) return;
    ring_stage_body2<M, STAGE>(p, stage_io<M, STAGE>(p), h, (int64_t)blockIdx.x - item_base[inst]);
}

// The kernel variant is the plan's (p.npt, from sim_create or the autotuner):
// two nodes per thread (128 threads per sub-tile) or one (256).
template <int M>
static cudaError_t launch_stage(int stage, const RingPlan &p, double dt, cudaStream_t s)
{
    const dim3 grid((unsigned)p.nsub), block(kRingThreads);
    if constexpr (M != 2) {
        if (p.npt == 2) {
            const dim3 block2(kRing2Threads);
            switch (stage) {
            case 0: ring_stage_kernel2<M, 0><<<grid, block2, 0, s>>>(p, step_size(dt)); break;
            case 1: ring_stage_kernel2<M, 1><<<grid, block2, 0, s>>>(p, step_size(dt)); break;
            case 2: ring_stage_kernel2<M, 2><<<grid, block2, 0, s>>>(p, step_size(dt)); break;
            case 3: ring_stage_kernel2<M, 3><<<grid, block2, 0, s>>>(p, step_size(dt)); break;
            default: ring_stage_kernel2<M, 4><<<grid, block2, 0, s>>>(p, step_size(dt)); break;
            }
            return cudaGetLastError();
        }
    }
    switch (stage) {
    case 0: ring_stage_kernel<M, 0><<<grid, block, 0, s>>>(p, step_size(dt)); break;
    case 1: ring_stage_kernel<M, 1><<<grid, block, 0, s>>>(p, step_size(dt)); break;
    case 2: ring_stage_kernel<M, 2><<<grid, block, 0, s>>>(p, step_size(dt)); break;
    case 3: ring_stage_kernel<M, 3><<<grid, block, 0, s>>>(p, step_size(dt)); break;
    default: ring_stage_kernel<M, 4><<<grid, block, 0, s>>>(p, step_size(dt)); break;
    }
    return cudaGetLastError();
}

static cudaError_t launch_any(int stage, const RingPlan &p, double dt, cudaStream_t s)
{
    switch (p.model) {
    case 0: return launch_stage<0>(stage, p, dt, s);
    case 1: return launch_stage<1>(stage, p, dt, s);
    case 2: return launch_stage<2>(stage, p, dt, s);
    default: return launch_stage<3>(stage, p, dt, s);
    }
}

template <int M>
static cudaError_t launch_batch_stage(int stage, const RingBatchGroup &g, double dt, cudaStream_t s)
{
    const dim3 grid((unsigned)g.n_items), block(kRingThreads);
    const StepSize h = step_size(dt);
    if constexpr (M != 2) {
        if (g.npt == 2) {
            const dim3 block2(kRing2Threads);
            switch (stage) {
            case 1: ring_batch_stage_kernel2<M, 1><<<grid, block2, 0, s>>>(g.plans, g.inst_of_item, g.item_base, h); break;
            case 2: ring_batch_stage_kernel2<M, 2><<<grid, block2, 0, s>>>(g.plans, g.inst_of_item, g.item_base, h); break;
            case 3: ring_batch_stage_kernel2<M, 3><<<grid, block2, 0, s>>>(g.plans, g.inst_of_item, g.item_base, h); break;
            default: ring_batch_stage_kernel2<M, 4><<<grid, block2, 0, s>>>(g.plans, g.inst_of_item, g.item_base, h); break;
            }
            return cudaGetLastError();
        }
    }
    switch (stage) {
    case 1: ring_batch_stage_kernel<M, 1><<<grid, block, 0, s>>>(g.plans, g.inst_of_item, g.item_base, h); break;
    case 2: ring_batch_stage_kernel<M, 2><<<grid, block, 0, s>>>(g.plans, g.inst_of_item, g.item_base, h); break;
    case 3: ring_batch_stage_kernel<M, 3><<<grid, block, 0, s>>>(g.plans, g.inst_of_item, g.item_base, h); break;
    default: ring_batch_stage_kernel<M, 4><<<grid, block, 0, s>>>(g.plans, g.inst_of_item, g.item_base, h); break;
    }
    return cudaGetLastError();
}

cudaError_t ring_batch_step(const RingBatchGroup &g, double dt, cudaStream_t s)
{
    if (g.n_items == 0) return cudaSuccess;
    for (int stage = 1; stage <= 4; ++stage) {
        cudaError_t e;
        switch (g.model) {
        case 0: e = launch_batch_stage<0>(stage, g, dt, s); break;
        case 1: e = launch_batch_stage<1>(stage, g, dt, s); break;
        case 2: e = launch_batch_stage<2>(stage, g, dt, s); break;
        default: e = launch_batch_stage<3>(stage, g, dt, s); break;
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static size_t flat_slot_bytes(const RingPlan &p)
{
    return sizeof(unsigned) * 4 * (size_t)(p.model == 2 ? Model<2>::NQ : Model<0>::NQ) * (size_t)p.ngroups;
}

cudaError_t ring_prologue(const RingPlan &p, cudaStream_t s)
{
    if (p.flat) { // the four accumulator slots are contiguous; slot 0 must start from zero
        const cudaError_t e = cudaMemsetAsync(p.facc[0], 0, 4 * flat_slot_bytes(p), s);
        if (e != cudaSuccess) return e;
    }
    return launch_any(0, p, 0.0, s);
}

cudaError_t ring_rhs(const RingPlan &p, cudaStream_t s)
{
    cudaError_t e = launch_any(1, p, 0.0, s);
    // a stage 1 on its own leaves slot 1 filled; the next RK4 step adds into it
    if (e == cudaSuccess && p.flat) e = cudaMemsetAsync(p.facc[1], 0, flat_slot_bytes(p), s);
    return e;
}

cudaError_t ring_step(const RingPlan &p, double dt, cudaStream_t s)
{
    for (int stage = 1; stage <= 4; ++stage) {
        const cudaError_t e = launch_any(stage, p, dt, s);
        if (e != cudaSuccess) return e;
        kernel_mark(s, 0);
    }
    return cudaSuccess;
}

} // namespace simk
