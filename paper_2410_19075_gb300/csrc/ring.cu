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
//       64 sub-tiles scans that group, and the last group scans the groups;
//   a6  (stage 4) the Kuramoto order parameter of y_{n+1} from the global totals.
// The prologue kernel does a1/a2/a6 for the initial state.
#include "ring_parts.cuh"

namespace simk {

// Buffers one stage reads and writes (chosen by the stage's parity).
struct RingStageIO {
    const int64_t *lam_in;
    const i128 *ingrp_in, *grpofs_in;
    int64_t *lam_out;
    i128 *ingrp_out, *grpofs_out;
    const double *x_in; // local stage-input variables of this stage (HH gates)
    double *x_out;      // local stage-input variables of the next stage
};

// Stage 0 (prologue) writes buffer 0; stage s reads buffer (s+1)&1 and writes
// s&1, so stage 4 leaves f(y_{n+1}) in buffer 0 for the next step.
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
    a.x_in = nullptr;
    a.x_out = nullptr;
    if (NX > 0) {
        a.x_in = STAGE == 1 ? p.y + (int64_t)(D - NX) * p.N : STAGE == 3 ? p.xg[1] : STAGE ? p.xg[0] : nullptr;
        a.x_out = STAGE == 1 || STAGE == 3 ? p.xg[0] : STAGE == 2 ? p.xg[1] : nullptr;
    }
    return a;
}

// One 256-node sub-tile `sub` of ring P, one node per thread (the whole CTA).
template <int M, int STAGE>
__device__ __forceinline__ void ring_stage_body(const RingPlan &P, const RingStageIO &a, double dt, int64_t sub)
{
    using Mo = Model<M>;
    constexpr int D = Mo::D, NQ = Mo::NQ, NX = Mo::NX;
    constexpr int XOFF = D - NX; // first local (non-coupled) state variable
    __shared__ RingBases<NQ> s_bases;

    const int tid = threadIdx.x;
    const int64_t N = P.N;
    const int64_t i = sub * kSubTile + tid;
    if (STAGE > 0) ring_load_bases<NQ>(P, a.ingrp_in, a.grpofs_in, sub, s_bases);

    int64_t qv[NQ];
    bool ok = true;
#pragma unroll
    for (int c = 0; c < NQ; ++c) qv[c] = 0;
    if (i < N) {
        double xn[D];
        if (STAGE == 0) {
#pragma unroll
            for (int v = 0; v < D; ++v) xn[v] = P.y[v * N + i];
        } else {
            int64_t qo[NQ];
            double fo[NQ];
            i128 W[NQ];
            ring_window<NQ>(P, a.lam_in, s_bases, tid, i, qo, fo, W);
            double X[NX > 0 ? NX : 1];
#pragma unroll
            for (int g = 0; g < NX; ++g) X[g] = a.x_in[g * N + i];
            const double Iext = (M == 2 && P.node_param) ? P.node_param[i] : 0.0;
            double k[D];
            Mo::rhs(P.mp, P.F, fo, qo, W, X, Iext, k);
#pragma unroll
            for (int v = 0; v < D; ++v) {
                const double yv = P.y[v * N + i];
                if (STAGE == 1) {
                    P.acc[v * N + i] = k[v];
                    xn[v] = yv + (0.5 * dt) * k[v];
                } else if (STAGE == 2) {
                    P.acc[v * N + i] = P.acc[v * N + i] + 2.0 * k[v];
                    xn[v] = yv + (0.5 * dt) * k[v];
                } else if (STAGE == 3) {
                    P.acc[v * N + i] = P.acc[v * N + i] + 2.0 * k[v];
                    xn[v] = yv + dt * k[v];
                } else {
                    const double yn = yv + (dt / 6.0) * (P.acc[v * N + i] + k[v]);
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
        double f[NQ];
        Mo::coupled(P.mp, xn, f);
#pragma unroll
        for (int c = 0; c < NQ; ++c) qv[c] = to_fixed(f[c], P.F, P.lim, ok);
    }
    if (!ok) raise_error(P.err, ERR_RANGE);
    ring_prefix_tail<NQ, (M == 0 || M == 3) && (STAGE == 0 || STAGE == 4), STAGE == 4>(P, a.lam_out, a.ingrp_out,
                                                                                     a.grpofs_out, sub, i, qv);
}

// Plain path: one ring, one sub-tile per CTA.
template <int M, int STAGE>
__global__ void __launch_bounds__(kRingThreads, MinBlocks<M>::value) ring_stage_kernel(const RingPlan p, double dt)
{
    ring_stage_body<M, STAGE>(p, stage_io<M, STAGE>(p), dt, blockIdx.x);
}

// Batched path: CTA b works on sub-tile b - item_base[inst] of ring inst =
// inst_of_item[b]; every ring keeps its own exact prefix hierarchy.  A ring whose
// step budget (steps_left) is used up is skipped whole, so its arrival counters
// stay consistent.
template <int M, int STAGE>
__global__ void __launch_bounds__(kRingThreads, MinBlocks<M>::value)
    ring_batch_stage_kernel(const RingPlan *__restrict__ plans, const int *__restrict__ inst_of_item,
                            const int64_t *__restrict__ item_base, double dt)
{
    const int inst = inst_of_item[blockIdx.x];
    const RingPlan &p = plans[inst];
    if (p.steps_left && *(volatile long long *)p.steps_left <= 0) return;
    ring_stage_body<M, STAGE>(p, stage_io<M, STAGE>(p), dt, (int64_t)blockIdx.x - item_base[inst]);
}

template <int M>
static cudaError_t launch_stage(int stage, const RingPlan &p, double dt, cudaStream_t s)
{
    const dim3 grid((unsigned)p.nsub), block(kRingThreads);
    switch (stage) {
    case 0: ring_stage_kernel<M, 0><<<grid, block, 0, s>>>(p, dt); break;
    case 1: ring_stage_kernel<M, 1><<<grid, block, 0, s>>>(p, dt); break;
    case 2: ring_stage_kernel<M, 2><<<grid, block, 0, s>>>(p, dt); break;
    case 3: ring_stage_kernel<M, 3><<<grid, block, 0, s>>>(p, dt); break;
    default: ring_stage_kernel<M, 4><<<grid, block, 0, s>>>(p, dt); break;
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
    switch (stage) {
    case 1: ring_batch_stage_kernel<M, 1><<<grid, block, 0, s>>>(g.plans, g.inst_of_item, g.item_base, dt); break;
    case 2: ring_batch_stage_kernel<M, 2><<<grid, block, 0, s>>>(g.plans, g.inst_of_item, g.item_base, dt); break;
    case 3: ring_batch_stage_kernel<M, 3><<<grid, block, 0, s>>>(g.plans, g.inst_of_item, g.item_base, dt); break;
    default: ring_batch_stage_kernel<M, 4><<<grid, block, 0, s>>>(g.plans, g.inst_of_item, g.item_base, dt); break;
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

cudaError_t ring_prologue(const RingPlan &p, cudaStream_t s)
{
    return launch_any(0, p, 0.0, s);
}

cudaError_t ring_rhs(const RingPlan &p, cudaStream_t s)
{
    return launch_any(1, p, 0.0, s);
}

cudaError_t ring_step(const RingPlan &p, double dt, cudaStream_t s)
{
    for (int stage = 1; stage <= 4; ++stage) {
        const cudaError_t e = launch_any(stage, p, dt, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

} // namespace simk
