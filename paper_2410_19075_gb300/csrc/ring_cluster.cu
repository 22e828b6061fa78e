// Small rings resident in one thread-block cluster for a whole sim_step call.
//
// For N <= kClusterMaxNodes the stage kernels of the streaming path are
// launch-latency bound (a few CTAs per stage, four launches per RK4 step).  Here
// one cluster of up to 16 CTAs (16 SMs) runs all stages of all steps of a call:
//   * every CTA owns a contiguous slice of nodes; their y, acc and HH gates stay
//     in registers for the whole call;
//   * after each stage every CTA writes the fixed-point coupled quantities of
//     its nodes into the shared memory of every CTA of the cluster (distributed
//     shared memory), into the buffer of the next stage (double-buffered), and
//     one cluster barrier per stage publishes them;
//   * every CTA then builds the exact prefix of the whole ring in its own shared
//     memory (int64 inside 256-node blocks, int128 block offsets) and gathers its
//     nodes' window sums from it.
// The arithmetic (grid, exact sums, right-hand sides, RK4) is the streaming
// path's, so the results are bit-for-bit the same.  At the end the cluster
// writes y, the order parameters of every step, and the streaming path's
// prefix buffers of f(y) (so that later calls may take either path).
#include <cooperative_groups.h>

#include "internal.h"

namespace cg = cooperative_groups;

namespace simk {

constexpr int kClusterThreads = 256;
constexpr int kClusterMaxNodesPerThread = 2;

// Byte offset of the int128 block offsets: after two Q buffers and the in-block
// prefix (int64 each), rounded up to 16 bytes (int128 accesses need it).
template <int NQ>
__host__ __device__ constexpr size_t cluster_bofs_offset(int64_t N)
{
    return ((size_t)(3 * NQ) * (size_t)N * sizeof(int64_t) + 15) / 16 * 16;
}

template <int NQ>
__host__ __device__ constexpr size_t cluster_smem_bytes(int64_t N)
{
    return cluster_bofs_offset<NQ>(N) + (size_t)NQ * ((N + 255) / 256 + 1) * sizeof(i128);
}

template <int M>
__global__ void __launch_bounds__(kClusterThreads, 1)
    ring_cluster_kernel(const RingPlan P, double dt, int64_t n_steps)
{
    using Mo = Model<M>;
    constexpr int D = Mo::D, NQ = Mo::NQ, NX = Mo::NX, XOFF = D - NX, MPT = kClusterMaxNodesPerThread;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank(), CL = (int)cluster.num_blocks();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t N = P.N, R = P.R, nb = (N + 255) / 256;
    const int64_t per = (N + CL - 1) / CL, i0 = rank * per, i1 = i0 + per < N ? i0 + per : N;

    extern __shared__ __align__(16) unsigned char smem[];
    int64_t *qbuf0 = reinterpret_cast<int64_t *>(smem);
    int64_t *qbuf1 = qbuf0 + NQ * N;
    int64_t *lam = qbuf1 + NQ * N;
    i128 *bofs = reinterpret_cast<i128 *>(smem + cluster_bofs_offset<NQ>(N)); // NQ * (nb + 1)

    // own nodes: i = i0 + tid + k * blockDim
    double y[MPT][D], acc[MPT][D], xs[MPT][NX > 0 ? NX : 1], iext[MPT];
    int64_t qn[MPT][NQ];
    bool ok = true;
#pragma unroll
    for (int k = 0; k < MPT; ++k) {
        const int64_t i = i0 + tid + (int64_t)k * kClusterThreads;
        iext[k] = 0.0;
#pragma unroll
        for (int v = 0; v < D; ++v) {
            y[k][v] = i < i1 ? P.y[v * N + i] : 0.0;
            acc[k][v] = 0.0;
        }
#pragma unroll
        for (int g = 0; g < NX; ++g) xs[k][g] = y[k][XOFF + g];
        if (M == 2 && P.node_param && i < i1) iext[k] = P.node_param[i];
    }

    // Q of f(x) for own nodes, written into `dst` of every CTA of the cluster
    auto broadcast = [&](int64_t *dst) {
#pragma unroll
        for (int k = 0; k < MPT; ++k) {
            const int64_t i = i0 + tid + (int64_t)k * kClusterThreads;
            if (i >= i1) continue;
            for (int r = 0; r < CL; ++r) {
                int64_t *remote = cluster.map_shared_rank(dst, r);
#pragma unroll
                for (int c = 0; c < NQ; ++c) remote[c * N + i] = qn[k][c];
            }
        }
    };

    // Exact prefix of a Q buffer: lam (inclusive inside 256-node blocks) and
    // bofs (exclusive at block starts, bofs[nb] = total).  Each warp scans whole
    // blocks (8 values per lane); warp 0 then scans the block totals.
    auto build_prefix = [&](const int64_t *q) {
        for (int64_t blk = warp; blk < (int64_t)NQ * nb; blk += kClusterThreads / 32) {
            const int c = (int)(blk / nb);
            const int64_t b = blk - (int64_t)c * nb;
            const int64_t j0 = b * 256 + lane * 8;
            int64_t v[8], run = 0;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                v[e] = j0 + e < N ? q[c * N + j0 + e] : 0;
                run += v[e];
                v[e] = run;
            }
            const int64_t incl = warp_incl_scan(run);
            const int64_t off = incl - run;
#pragma unroll
            for (int e = 0; e < 8; ++e)
                if (j0 + e < N) lam[c * N + j0 + e] = off + v[e];
            if (lane == 31) bofs[c * (nb + 1) + b] = (i128)incl; // block total, scanned below
        }
        __syncthreads();
        if (warp == 0) {
#pragma unroll
            for (int c = 0; c < NQ; ++c) {
                // nb <= 32 blocks (N <= 8192): one per lane
                const i128 t = lane < nb ? bofs[c * (nb + 1) + lane] : (i128)0;
                i128 x = t;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const i128 u = shfl_up_i128(x, o);
                    if (lane >= o) x += u;
                }
                __syncwarp();
                if (lane < nb) bofs[c * (nb + 1) + lane] = x - t;
                if (lane == 31) bofs[c * (nb + 1) + nb] = x;
            }
        }
        __syncthreads();
    };
    auto prefix_at = [&](int c, int64_t p) -> i128 { // p in [-N, 2N)
        i128 add = 0;
        const i128 tot = bofs[c * (nb + 1) + nb];
        if (p < 0) {
            p += N;
            add = -tot;
        } else if (p >= N) {
            p -= N;
            add = tot;
        }
        i128 v = bofs[c * (nb + 1) + (p >> 8)] + add;
        if (p & 255) v += (i128)lam[c * N + p - 1];
        return v;
    };
    auto record_order = [&]() {
        if ((M == 0 || M == 3) && rank == 0 && tid == 0) {
            const double S = fixed_to_double(bofs[nb], P.F);
            const double C = fixed_to_double(bofs[(NQ - 1) * (nb + 1) + nb], P.F);
            const unsigned long long n = *P.obs_ctr;
            P.obs[n % (unsigned long long)P.obs_cap] = sqrt(S * S + C * C) / (double)N;
            *P.obs_ctr = n + 1;
        }
    };

    // prologue: f(y) into buffer 0 (the observable of y was recorded when the
    // state was set)
#pragma unroll
    for (int k = 0; k < MPT; ++k) {
        Mo::coupled_q(P.mp, y[k], P.F, P.lim, ok, qn[k]);
    }
    broadcast(qbuf0);
    cluster.sync();

    int cur = 0; // buffer holding f of the current stage input
    for (int64_t step = 0; step < n_steps; ++step) {
#pragma unroll 1
        for (int stage = 1; stage <= 4; ++stage) {
            const int64_t *q = cur ? qbuf1 : qbuf0;
            build_prefix(q);
            if (stage == 1 && step > 0) record_order(); // order parameter of y after the previous step
#pragma unroll
            for (int k = 0; k < MPT; ++k) {
                const int64_t i = i0 + tid + (int64_t)k * kClusterThreads;
                if (i >= i1) continue;
                int64_t qo[NQ];
                double fo[NQ];
                i128 W[NQ];
#pragma unroll
                for (int c = 0; c < NQ; ++c) {
                    qo[c] = q[c * N + i];
                    fo[c] = fixed_to_double(qo[c], P.F);
                    W[c] = prefix_at(c, i + R + 1) - prefix_at(c, i - R);
                }
                double kk[D], xn[D];
                Mo::rhs(P.mp, P.F, fo, qo, W, xs[k], iext[k], kk);
#pragma unroll
                for (int v = 0; v < D; ++v) {
                    if (stage == 1) {
                        acc[k][v] = kk[v];
                        xn[v] = y[k][v] + (0.5 * dt) * kk[v];
                    } else if (stage == 2) {
                        acc[k][v] = acc[k][v] + 2.0 * kk[v];
                        xn[v] = y[k][v] + (0.5 * dt) * kk[v];
                    } else if (stage == 3) {
                        acc[k][v] = acc[k][v] + 2.0 * kk[v];
                        xn[v] = y[k][v] + dt * kk[v];
                    } else {
                        y[k][v] = y[k][v] + (dt / 6.0) * (acc[k][v] + kk[v]);
                        xn[v] = y[k][v];
                    }
                }
#pragma unroll
                for (int g = 0; g < NX; ++g) xs[k][g] = xn[XOFF + g];
                Mo::coupled_q(P.mp, xn, P.F, P.lim, ok, qn[k]);
            }
            cur ^= 1;
            broadcast(cur ? qbuf1 : qbuf0);
            cluster.sync();
        }
    }
    if (!ok) raise_error(P.err, ERR_RANGE);

    // results: y, the last order parameter, and the streaming path's prefix
    // buffers of f(y) (buffer 0)
    build_prefix(cur ? qbuf1 : qbuf0);
    if (n_steps > 0) record_order();
#pragma unroll
    for (int k = 0; k < MPT; ++k) {
        const int64_t i = i0 + tid + (int64_t)k * kClusterThreads;
        if (i >= i1) continue;
#pragma unroll
        for (int v = 0; v < D; ++v) P.y[v * N + i] = y[k][v];
#pragma unroll
        for (int c = 0; c < NQ; ++c) P.lam[0][c * N + i] = lam[c * N + i];
    }
    if (rank == 0) {
        // one prefix group (nsub <= 64): in-group offsets are the block offsets
        for (int64_t t = tid; t < (int64_t)NQ * nb; t += kClusterThreads) {
            const int c = (int)(t / nb);
            const int64_t b = t - (int64_t)c * nb;
            P.ingrp[0][c * P.nsub + b] = bofs[c * (nb + 1) + b];
        }
        if (tid < NQ) {
            P.grpofs[0][tid * (P.ngroups + 1)] = 0;
            P.grpofs[0][tid * (P.ngroups + 1) + 1] = bofs[tid * (nb + 1) + nb];
        }
    }
    cluster.sync(); // no CTA exits while others may still write its shared memory
}

static int g_max_cluster = 8; // 16 when the device can co-schedule it (set by configure)

int cluster_size_for(int64_t N)
{
    if (N > kClusterMaxNodes) return 0;
    int cl = (int)((N + 127) / 128);
    if (cl < 2) cl = 2;
    if (cl > g_max_cluster) cl = g_max_cluster;
    return (N + cl - 1) / cl <= (int64_t)kClusterThreads * kClusterMaxNodesPerThread ? cl : 0;
}

template <int M>
static cudaError_t configure_one(int64_t max_nodes)
{
    constexpr int NQ = Model<M>::NQ;
    cudaError_t e = cudaFuncSetAttribute(ring_cluster_kernel<M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)cluster_smem_bytes<NQ>(max_nodes));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(ring_cluster_kernel<M>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

cudaError_t ring_cluster_configure()
{
    cudaError_t e = configure_one<0>(kClusterMaxNodes);
    if (e == cudaSuccess) e = configure_one<1>(kClusterMaxNodes);
    if (e == cudaSuccess) e = configure_one<2>(kClusterMaxNodes);
    if (e == cudaSuccess) e = configure_one<3>(kClusterMaxNodes);
    if (e != cudaSuccess) return e;
    // largest cluster the device can co-schedule with the largest shared-memory use
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3(kClusterThreads);
    cfg.dynamicSmemBytes = cluster_smem_bytes<2>(kClusterMaxNodes);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 16;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, ring_cluster_kernel<0>, &cfg) == cudaSuccess && n >= 1) g_max_cluster = 16;
    else g_max_cluster = 8;
    cudaGetLastError();
    return cudaSuccess;
}

template <int M>
static cudaError_t launch_cluster(const RingPlan &p, double dt, int64_t n_steps, int cl, cudaStream_t s)
{
    constexpr int NQ = Model<M>::NQ;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cl);
    cfg.blockDim = dim3(kClusterThreads);
    cfg.dynamicSmemBytes = cluster_smem_bytes<NQ>(p.N);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, ring_cluster_kernel<M>, p, dt, n_steps);
}

cudaError_t ring_cluster_steps(const RingPlan &p, double dt, int64_t n_steps, cudaStream_t s)
{
    const int cl = cluster_size_for(p.N);
    if (cl == 0) return cudaErrorInvalidValue;
    cudaError_t e;
    switch (p.model) {
    case 0: e = launch_cluster<0>(p, dt, n_steps, cl, s); break;
    case 1: e = launch_cluster<1>(p, dt, n_steps, cl, s); break;
    case 2: e = launch_cluster<2>(p, dt, n_steps, cl, s); break;
    default: e = launch_cluster<3>(p, dt, n_steps, cl, s); break;
    }
    if (e == cudaSuccess) kernel_mark(s, 0);
    return e;
}

} // namespace simk
