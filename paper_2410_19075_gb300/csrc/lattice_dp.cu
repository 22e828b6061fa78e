// Adaptive Dormand-Prince 5(4) on the lattices (cube, ball, disk; Kuramoto with
// and without inertia; the solver of the paper's performance tests on the 3D
// network with inertia, Sections III.A and V) and on link matrices (every model).
//
// Each stage s of an attempt of size h is
//   input   x_s = y + h sum_{j<s} a_sj k_j into the stage-input buffer, and the
//           (sin, cos) of its phase (x_7 is also kept as the candidate y_{n+1});
//   slope   k_s = f(x_s): the network's own right-hand side (lattice: x pass and
//           gather; link matrix: exact prefix and the graph kernel) on a plan
//           whose state is the stage-input buffer and whose output is k_s;
// then the error kernel forms e = h sum_j (b_j - bhat_j) k_j, the per-CTA sums of
// (e / sc)^2 and of the (sin, cos) of the Hermite-interpolated phases at the
// output times, and the last CTA reduces them in a fixed order and decides (the
// same controller as on rings, dp_control.cuh); the accept kernel then moves
// y_{n+1} and k_7 into y and k_1.  Every kernel of a finished run returns at once.
#include "dp_control.cuh"

namespace simk {

constexpr int kLdpThreads = 256;

__device__ __forceinline__ bool ldp_done(const ElemDpPlan &d) { return *(const volatile int *)&d.ctl->done; }

template <int M, int S>
__global__ void __launch_bounds__(kLdpThreads) lat_dp_input_kernel(const ElemDpPlan d)
{
    constexpr int D = Model<M>::D;
    if (ldp_done(d)) return;
    const int64_t nodes = d.nodes;
    const int64_t n = (int64_t)blockIdx.x * kLdpThreads + threadIdx.x;
    if (n >= nodes) return;
    const double h = d.ctl->h_att;
    double phase = 0.0;
#pragma unroll
    for (int v = 0; v < D; ++v) {
        const int64_t q = v * nodes + n;
        double x;
        if (S == 1) {
            x = d.y[q];
        } else {
            double acc = c_dp_a[S - 1][0] * d.k[1][q];
#pragma unroll
            for (int j = 1; j < S - 1; ++j) acc += c_dp_a[S - 1][j] * d.k[j + 1][q];
            x = d.y[q] + h * acc;
        }
        d.xbuf[q] = x;
        if (S == 7) d.y5[q] = x;
        if (v == 0) phase = x;
    }
    if (d.f) { // lattices: the x pass reads the (sin, cos) of the phase on the grid 2^-62
        int64_t s62, c62;
        bool ok = true;
        fixed_sincos(phase, d.tab, s62, c62, ok);
        reinterpret_cast<longlong2 *>(d.f)[n] = make_longlong2(s62, c62); // (sin, cos) pairs
        if (!ok) raise_error(d.err, ERR_RANGE);
    }
}

template <int M>
__global__ void __launch_bounds__(kLdpThreads) lat_dp_error_kernel(const ElemDpPlan d)
{
    constexpr int D = Model<M>::D;
    constexpr int NW = kLdpThreads / 32;
    __shared__ double s_err[NW];
    __shared__ i128 s_w[NW][2];
    __shared__ i128 s_out[kDpMaxOut][2];
    __shared__ int s_last;
    if (ldp_done(d)) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t nodes = d.nodes;
    const int64_t n = (int64_t)blockIdx.x * kLdpThreads + tid;
    const DpCtl *ctl = d.ctl;
    const double h = ctl->h_att, atol = ctl->atol, rtol = ctl->rtol;
    double err = 0.0;
    if (n < nodes) {
#pragma unroll
        for (int v = 0; v < D; ++v) {
            const int64_t q = v * nodes + n;
            double e = c_dp_e[0] * d.k[1][q];
#pragma unroll
            for (int j = 2; j <= 7; ++j) e += c_dp_e[j - 1] * d.k[j][q];
            e *= h;
            const double sc = atol + rtol * fmax(fabs(d.y[q]), fabs(d.y5[q]));
            const double r = e / sc;
            err += r * r;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) err += __shfl_xor_sync(0xffffffffu, err, o);
    if (lane == 0) s_err[warp] = err;

    // dense output: the order parameter of the Hermite-interpolated phases
    const double t = ctl->t, t0 = ctl->t0, odt = ctl->out_dt;
    const long long next_out = ctl->next_out, n_out = ctl->n_out;
    const int last = ctl->last;
    int n_here = 0;
    if ((M == 0 || M == 3) && odt > 0.0) {
        while (n_here < kDpMaxOut && next_out + n_here <= n_out) {
            const double to = t0 + (double)(next_out + n_here) * odt;
            if (!last && to > t + h) break;
            ++n_here;
        }
    }
    bool ok = true;
    for (int o = 0; o < n_here; ++o) {
        i128 ss = 0, cc = 0;
        if (n < nodes) {
            const double to = t0 + (double)(next_out + o) * odt;
            double th = (to - t) / h;
            th = th > 1.0 ? 1.0 : th;
            const double a0 = d.y[n], a1 = d.y5[n], f0 = d.k[1][n], f1 = d.k[7][n];
            const double ph = (1.0 - th) * a0 + th * a1 +
                              th * (th - 1.0) * ((1.0 - 2.0 * th) * (a1 - a0) + (th - 1.0) * h * f0 + th * h * f1);
            int64_t s62, c62;
            fixed_sincos(ph, d.tab, s62, c62, ok);
            ss = q62_to(s62, d.F);
            cc = q62_to(c62, d.F);
        }
        ss = warp_sum_i128(ss);
        cc = warp_sum_i128(cc);
        if (lane == 0) {
            s_w[warp][0] = ss;
            s_w[warp][1] = cc;
        }
        __syncthreads();
        if (tid == 0) {
            i128 a = 0, b = 0;
            for (int w = 0; w < NW; ++w) {
                a += s_w[w][0];
                b += s_w[w][1];
            }
            st_i128(d.out_part + ((int64_t)blockIdx.x * kDpMaxOut + o) * 2, a);
            st_i128(d.out_part + ((int64_t)blockIdx.x * kDpMaxOut + o) * 2 + 1, b);
        }
        __syncthreads();
    }
    if (!ok) raise_error(d.err, ERR_RANGE);
    __syncthreads();
    if (tid == 0) {
        double a = 0.0;
        for (int w = 0; w < NW; ++w) a += s_err[w];
        d.err_part[blockIdx.x] = a;
        __threadfence();
        s_last = last_arrival(d.dp_ctr, (unsigned long long)d.nblk);
    }
    __syncthreads();
    if (!s_last) return;

    // the last CTA: fixed assignment of the per-CTA sums to threads, then decide
    double es = 0.0;
    for (int64_t b = tid; b < d.nblk; b += kLdpThreads) es += __ldcg(d.err_part + b);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) es += __shfl_xor_sync(0xffffffffu, es, o);
    __syncthreads();
    if (lane == 0) s_err[warp] = es;
    for (int o = 0; o < n_here; ++o) {
        i128 a = 0, b = 0;
        for (int64_t sb = tid; sb < d.nblk; sb += kLdpThreads) {
            a += ld_cg_i128(d.out_part + (sb * kDpMaxOut + o) * 2);
            b += ld_cg_i128(d.out_part + (sb * kDpMaxOut + o) * 2 + 1);
        }
        a = warp_sum_i128(a);
        b = warp_sum_i128(b);
        if (lane == 0) {
            s_w[warp][0] = a;
            s_w[warp][1] = b;
        }
        __syncthreads();
        if (tid == 0) {
            i128 ta = 0, tb = 0;
            for (int w = 0; w < NW; ++w) {
                ta += s_w[w][0];
                tb += s_w[w][1];
            }
            s_out[o][0] = ta;
            s_out[o][1] = tb;
        }
        __syncthreads();
    }
    __syncthreads();
    if (tid == 0) {
        double tot = 0.0;
        for (int w = 0; w < NW; ++w) tot += s_err[w];
        dp_decide_ctl(d.ctl, d.remaining, tot, (int64_t)D * nodes, n_here, s_out,
                      DpRecord{d.obs, d.obs_cap, d.obs_ctr, d.F, nodes});
    }
}

// An accepted attempt: y <- y_{n+1}, k_1 <- k_7 (idempotent, so repeating it after
// the run ended changes nothing).
template <int M>
__global__ void __launch_bounds__(kLdpThreads) lat_dp_accept_kernel(const ElemDpPlan d)
{
    constexpr int D = Model<M>::D;
    if (!*(const volatile int *)&d.ctl->acc_flag) return;
    const int64_t n = (int64_t)blockIdx.x * kLdpThreads + threadIdx.x;
    if (n >= d.nodes) return;
#pragma unroll
    for (int v = 0; v < D; ++v) {
        const int64_t q = v * d.nodes + n;
        d.y[q] = d.y5[q];
        d.k[1][q] = d.k[7][q];
    }
}

// Stage S: the stage input, then the network's right-hand side into k_S.
template <int M, int S, class Rhs>
static cudaError_t stage(const ElemDpPlan &e, const Rhs &rhs, cudaStream_t s)
{
    lat_dp_input_kernel<M, S><<<(unsigned)e.nblk, kLdpThreads, 0, s>>>(e);
    const cudaError_t err = cudaGetLastError();
    return err != cudaSuccess ? err : rhs(e.k[S], s);
}

template <int M, class Rhs>
static cudaError_t attempt(const ElemDpPlan &e, const Rhs &rhs, cudaStream_t s)
{
    cudaError_t err = stage<M, 2>(e, rhs, s);
    if (err == cudaSuccess) err = stage<M, 3>(e, rhs, s);
    if (err == cudaSuccess) err = stage<M, 4>(e, rhs, s);
    if (err == cudaSuccess) err = stage<M, 5>(e, rhs, s);
    if (err == cudaSuccess) err = stage<M, 6>(e, rhs, s);
    if (err == cudaSuccess) err = stage<M, 7>(e, rhs, s);
    if (err != cudaSuccess) return err;
    lat_dp_error_kernel<M><<<(unsigned)e.nblk, kLdpThreads, 0, s>>>(e);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    lat_dp_accept_kernel<M><<<(unsigned)e.nblk, kLdpThreads, 0, s>>>(e);
    return cudaGetLastError();
}

// the right-hand sides: k <- f(stage-input buffer)
struct LatticeRhs {
    const LatticePlan &p;
    cudaError_t operator()(double *k, cudaStream_t s) const
    {
        LatticePlan q = p;
        q.acc = k;
        return lattice_rhs(q, s);
    }
};
struct GraphRhs {
    const GraphPlan &g;
    cudaError_t operator()(double *k, cudaStream_t s) const
    {
        GraphPlan q = g;
        q.r.acc = k;
        cudaError_t err = ring_prologue(q.r, s); // exact prefix of the stage input's coupled quantity
        return err != cudaSuccess ? err : graph_rhs(q, s);
    }
};

template <class Rhs>
static cudaError_t start_any(const ElemDpPlan &e, const Rhs &rhs, cudaStream_t s)
{
    switch (e.model) {
    case 0: return stage<0, 1>(e, rhs, s);
    case 1: return stage<1, 1>(e, rhs, s);
    case 2: return stage<2, 1>(e, rhs, s);
    default: return stage<3, 1>(e, rhs, s);
    }
}

template <class Rhs>
static cudaError_t attempt_any(const ElemDpPlan &e, const Rhs &rhs, cudaStream_t s)
{
    switch (e.model) {
    case 0: return attempt<0>(e, rhs, s);
    case 1: return attempt<1>(e, rhs, s);
    case 2: return attempt<2>(e, rhs, s);
    default: return attempt<3>(e, rhs, s);
    }
}

cudaError_t lat_dp_start(const LatDpPlan &d, cudaStream_t s) { return start_any(d.e, LatticeRhs{d.rhs}, s); }
cudaError_t lat_dp_attempt(const LatDpPlan &d, cudaStream_t s) { return attempt_any(d.e, LatticeRhs{d.rhs}, s); }
cudaError_t graph_dp_start(const GraphDpPlan &d, cudaStream_t s) { return start_any(d.e, GraphRhs{d.rhs}, s); }
cudaError_t graph_dp_attempt(const GraphDpPlan &d, cudaStream_t s)
{
    return attempt_any(d.e, GraphRhs{d.rhs}, s);
}

} // namespace simk
