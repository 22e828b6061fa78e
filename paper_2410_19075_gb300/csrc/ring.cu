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
//       sub-tile, and the prefix at sub-tile starts through a single-pass
//       decoupled look-back across CTAs;
//   a6  (stage 4) the Kuramoto order parameter of y_{n+1} from the global totals.
// The prologue kernel does a1/a2/a6 for the initial state.
#include "internal.h"

namespace simk {

struct RingStageArgs {
    RingPlan p;
    double dt;
    const int64_t *lam_in;
    const i128 *ofs_in;
    int64_t *lam_out;
    i128 *ofs_out;
    const double *x_in; // local stage-input variables of this stage (HH gates)
    double *x_out;      // local stage-input variables of the next stage
};

__device__ __forceinline__ i128 ldg_i128(const i128 *p)
{
    const longlong2 v = __ldg(reinterpret_cast<const longlong2 *>(p));
    return (i128)(u128)(unsigned long long)v.x | ((i128)v.y << 64);
}

// P(p) = sum_{j<p} Q(f_j) over the periodic extension of the ring, p in [-N, 2N).
__device__ __forceinline__ i128 prefix_at(const int64_t *lam, const i128 *ofs, int64_t N, int64_t p, i128 tot)
{
    i128 add = 0;
    if (p < 0) {
        p += N;
        add = -tot;
    } else if (p >= N) {
        p -= N;
        add = tot;
    }
    i128 v = ldg_i128(ofs + (p >> kSubLog2)) + add;
    if (p & (kSubTile - 1)) v += (i128)__ldg(lam + p - 1);
    return v;
}

template <int M, int STAGE>
__global__ void __launch_bounds__(kRingThreads) ring_stage_kernel(const RingStageArgs a)
{
    using Mo = Model<M>;
    constexpr int D = Mo::D, NQ = Mo::NQ, NX = Mo::NX, V = kRingNodesPerThread;
    constexpr int XOFF = D - NX; // first local (non-coupled) state variable
    const RingPlan &P = a.p;
    __shared__ unsigned long long s_ticket;
    __shared__ int64_t s_wtot[kRingThreads / 32][NQ];
    __shared__ i128 s_excl[NQ];

    if (threadIdx.x == 0) s_ticket = atomicAdd(P.ticket, 1ull);
    __syncthreads();
    const unsigned long long ticket = s_ticket;
    const long long tile = (long long)(ticket % (unsigned long long)P.nctas);
    const unsigned long long epoch = ticket / (unsigned long long)P.nctas + 1ull;
    const int64_t N = P.N;
    const int64_t base = (int64_t)tile * kRingTile + (int64_t)threadIdx.x * V;

    double xn[V][D];
    if (STAGE == 0) {
#pragma unroll
        for (int q = 0; q < V; ++q)
#pragma unroll
            for (int v = 0; v < D; ++v) xn[q][v] = (base + q < N) ? P.y[v * N + base + q] : 0.0;
    } else {
        i128 tot[NQ];
#pragma unroll
        for (int c = 0; c < NQ; ++c) tot[c] = ldg_i128(a.ofs_in + c * (P.nsub + 1) + P.nsub);
#pragma unroll
        for (int q = 0; q < V; ++q) {
            const int64_t i = base + q;
            if (i >= N) {
#pragma unroll
                for (int v = 0; v < D; ++v) xn[q][v] = 0.0;
                continue;
            }
            int64_t qo[NQ];
            double fo[NQ];
            i128 W[NQ];
#pragma unroll
            for (int c = 0; c < NQ; ++c) {
                const int64_t *lam = a.lam_in + c * N;
                const i128 *ofs = a.ofs_in + c * (P.nsub + 1);
                const int64_t l = __ldg(lam + i);
                qo[c] = (i & (kSubTile - 1)) ? l - __ldg(lam + i - 1) : l;
                fo[c] = fixed_to_double(qo[c], P.F);
                W[c] = prefix_at(lam, ofs, N, i + P.R + 1, tot[c]) - prefix_at(lam, ofs, N, i - P.R, tot[c]);
            }
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
                    xn[q][v] = yv + (0.5 * a.dt) * k[v];
                } else if (STAGE == 2) {
                    P.acc[v * N + i] = P.acc[v * N + i] + 2.0 * k[v];
                    xn[q][v] = yv + (0.5 * a.dt) * k[v];
                } else if (STAGE == 3) {
                    P.acc[v * N + i] = P.acc[v * N + i] + 2.0 * k[v];
                    xn[q][v] = yv + a.dt * k[v];
                } else {
                    const double yn = yv + (a.dt / 6.0) * (P.acc[v * N + i] + k[v]);
                    P.y[v * N + i] = yn;
                    xn[q][v] = yn;
                }
            }
            if (NX > 0 && STAGE >= 1 && STAGE <= 3) {
#pragma unroll
                for (int g = 0; g < NX; ++g) a.x_out[g * N + i] = xn[q][XOFF + g];
            }
        }
    }

    // a2: coupled quantity of the next stage input on the fixed-point grid.
    int64_t qv[V][NQ];
    bool ok = true;
#pragma unroll
    for (int q = 0; q < V; ++q) {
        double f[NQ];
        Mo::coupled(xn[q], f);
#pragma unroll
        for (int c = 0; c < NQ; ++c) qv[q][c] = (base + q < N) ? to_fixed(f[c], P.F, P.lim, ok) : 0;
    }
    if (!ok) raise_error(P.err, ERR_RANGE);

    // Exact inclusive prefix inside each 256-node sub-tile (= 2 warps).
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t tsum[NQ], incl[NQ];
#pragma unroll
    for (int c = 0; c < NQ; ++c) {
        int64_t run = 0;
#pragma unroll
        for (int q = 0; q < V; ++q) {
            run += qv[q][c];
            qv[q][c] = run;
        }
        tsum[c] = run;
        incl[c] = warp_incl_scan(run);
        if (lane == 31) s_wtot[warp][c] = incl[c];
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NQ; ++c) {
        const int64_t off = incl[c] - tsum[c] + ((warp & 1) ? s_wtot[warp - 1][c] : 0);
#pragma unroll
        for (int q = 0; q < V; ++q)
            if (base + q < N) a.lam_out[c * N + base + q] = off + qv[q][c];
    }

    // Exclusive prefix of this CTA's tile across the ring.
    if (threadIdx.x == 0) {
        i128 agg[NQ], excl[NQ];
#pragma unroll
        for (int c = 0; c < NQ; ++c) {
            agg[c] = 0;
            for (int w = 0; w < kRingThreads / 32; ++w) agg[c] += (i128)s_wtot[w][c];
        }
        lookback<NQ>(P.slots, tile, epoch, agg, excl, P.err);
#pragma unroll
        for (int c = 0; c < NQ; ++c) s_excl[c] = excl[c];
        if (tile == P.nctas - 1) {
            // Global totals: the last prefix entry, and the order parameter.
#pragma unroll
            for (int c = 0; c < NQ; ++c) a.ofs_out[c * (P.nsub + 1) + P.nsub] = excl[c] + agg[c];
            if (M == 0 && (STAGE == 0 || STAGE == 4)) {
                const double S = fixed_to_double(excl[0] + agg[0], P.F);
                const double C = fixed_to_double(excl[NQ - 1] + agg[NQ - 1], P.F);
                const unsigned long long n = *P.obs_ctr;
                P.obs[n % (unsigned long long)P.obs_cap] = sqrt(S * S + C * C) / (double)N;
                *P.obs_ctr = n + 1;
            }
        }
    }
    __syncthreads();
    constexpr int kSubPerCta = kRingTile / kSubTile;
    if (threadIdx.x < kSubPerCta) {
        const int s = threadIdx.x;
        const int64_t sub = (int64_t)tile * kSubPerCta + s;
        if (sub < P.nsub) {
#pragma unroll
            for (int c = 0; c < NQ; ++c) {
                i128 v = s_excl[c];
                for (int t = 0; t < s; ++t) v += (i128)s_wtot[2 * t][c] + (i128)s_wtot[2 * t + 1][c];
                a.ofs_out[c * (P.nsub + 1) + sub] = v;
            }
        }
    }
}

template <int M>
static cudaError_t launch_stage(int stage, const RingPlan &p, double dt, cudaStream_t s)
{
    constexpr int D = Model<M>::D, NX = Model<M>::NX;
    RingStageArgs a;
    a.p = p;
    a.dt = dt;
    const int in = (stage + 1) & 1, out = stage & 1; // stage 0 writes buffer 0
    a.lam_in = stage ? p.lam[in] : nullptr;
    a.ofs_in = stage ? p.ofs[in] : nullptr;
    a.lam_out = p.lam[stage == 0 ? 0 : out];
    a.ofs_out = p.ofs[stage == 0 ? 0 : out];
    a.x_in = nullptr;
    a.x_out = nullptr;
    if (NX > 0) {
        const double *src[5] = {nullptr, p.y + (int64_t)(D - NX) * p.N, p.xg[0], p.xg[1], p.xg[0]};
        double *dst[5] = {nullptr, p.xg[0], p.xg[1], p.xg[0], nullptr};
        a.x_in = src[stage];
        a.x_out = dst[stage];
    }
    const dim3 grid((unsigned)p.nctas), block(kRingThreads);
    switch (stage) {
    case 0: ring_stage_kernel<M, 0><<<grid, block, 0, s>>>(a); break;
    case 1: ring_stage_kernel<M, 1><<<grid, block, 0, s>>>(a); break;
    case 2: ring_stage_kernel<M, 2><<<grid, block, 0, s>>>(a); break;
    case 3: ring_stage_kernel<M, 3><<<grid, block, 0, s>>>(a); break;
    default: ring_stage_kernel<M, 4><<<grid, block, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

static cudaError_t launch_any(int stage, const RingPlan &p, double dt, cudaStream_t s)
{
    switch (p.model) {
    case 0: return launch_stage<0>(stage, p, dt, s);
    case 1: return launch_stage<1>(stage, p, dt, s);
    default: return launch_stage<2>(stage, p, dt, s);
    }
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
