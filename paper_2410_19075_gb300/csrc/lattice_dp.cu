// Adaptive Dormand-Prince 5(4) on the lattices (cube, ball, disk; Kuramoto with
// and without inertia), the solver of the paper's performance tests on the 3D
// network with inertia (Sections III.A and V).
//
// Each stage s of an attempt of size h is
//   input   x_s = y + h sum_{j<s} a_sj k_j into the stage-input buffer, and the
//           (sin, cos) of its phase (x_7 is also kept as the candidate y_{n+1});
//   slope   k_s = f(x_s): the lattice right-hand side (x pass, gather) on a plan
//           whose state is the stage-input buffer and whose output is k_s;
// then the error kernel forms e = h sum_j (b_j - bhat_j) k_j, the per-CTA sums of
// (e / sc)^2 and of the (sin, cos) of the Hermite-interpolated phases at the
// output times, and the last CTA reduces them in a fixed order and decides (the
// same controller as on rings, dp_control.cuh); the accept kernel then moves
// y_{n+1} and k_7 into y and k_1.  Every kernel of a finished run returns at once.
#include "dp_control.cuh"

namespace simk {

constexpr int kLdpThreads = 256;

__device__ __forceinline__ bool ldp_done(const LatDpPlan &d) { return *(const volatile int *)&d.ctl->done; }

template <int M, int S>
__global__ void __launch_bounds__(kLdpThreads) lat_dp_input_kernel(const LatDpPlan d)
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
    double sn, cn;
    fast_sincos(phase, d.rhs.mp.tab, sn, cn);
    d.rhs.f[n] = sn;
    d.rhs.f[nodes + n] = cn;
}

template <int M>
__global__ void __launch_bounds__(kLdpThreads) lat_dp_error_kernel(const LatDpPlan d)
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
    if (odt > 0.0) {
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
            double sn, cn;
            fast_sincos(ph, d.rhs.mp.tab, sn, cn);
            ss = to_fixed(sn, d.rhs.F, 1, ok);
            cc = to_fixed(cn, d.rhs.F, 1, ok);
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
    if (!ok) raise_error(d.rhs.err, ERR_RANGE);
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
                      DpRecord{d.rhs.obs, d.rhs.obs_cap, d.rhs.obs_ctr, d.rhs.F, nodes});
    }
}

// An accepted attempt: y <- y_{n+1}, k_1 <- k_7 (idempotent, so repeating it after
// the run ended changes nothing).
template <int M>
__global__ void __launch_bounds__(kLdpThreads) lat_dp_accept_kernel(const LatDpPlan d)
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

template <int M, int S>
static cudaError_t stage(const LatDpPlan &d, cudaStream_t s)
{
    lat_dp_input_kernel<M, S><<<(unsigned)d.nblk, kLdpThreads, 0, s>>>(d);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    LatticePlan p = d.rhs;
    p.acc = d.k[S];
    return lattice_rhs(p, s);
}

template <int M>
static cudaError_t attempt(const LatDpPlan &d, cudaStream_t s)
{
    cudaError_t e = stage<M, 2>(d, s);
    if (e == cudaSuccess) e = stage<M, 3>(d, s);
    if (e == cudaSuccess) e = stage<M, 4>(d, s);
    if (e == cudaSuccess) e = stage<M, 5>(d, s);
    if (e == cudaSuccess) e = stage<M, 6>(d, s);
    if (e == cudaSuccess) e = stage<M, 7>(d, s);
    if (e != cudaSuccess) return e;
    lat_dp_error_kernel<M><<<(unsigned)d.nblk, kLdpThreads, 0, s>>>(d);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    lat_dp_accept_kernel<M><<<(unsigned)d.nblk, kLdpThreads, 0, s>>>(d);
    return cudaGetLastError();
}

cudaError_t lat_dp_start(const LatDpPlan &d, cudaStream_t s)
{
    return d.model == 3 ? stage<3, 1>(d, s) : stage<0, 1>(d, s);
}

cudaError_t lat_dp_attempt(const LatDpPlan &d, cudaStream_t s)
{
    return d.model == 3 ? attempt<3>(d, s) : attempt<0>(d, s);
}

} // namespace simk
