// Adaptive Dormand-Prince 5(4) on rings, one step control per instance (the
// paper's default solver, Section III.A; dense output of the order parameter at
// every output time, Section V).
//
// One attempted step of size h is seven kernels per group of rings of one model,
// every CTA one 256-node sub-tile of one instance (the batched layout of the
// RK4 kernels, and the same exact window sums):
//   ds 0    input of stage 2, x2 = y + h a21 k1 (k1 = f(y_n) is kept from the
//           last stage of the previous accepted step: first same as last), and
//           the exact prefix of its coupled quantity;
//   ds 2..6 k_s = f(x_s) from the window sums, then x_{s+1} = y + h sum_j a_{s+1,j} k_j
//           and its prefix (x7 is the candidate y_{n+1});
//   ds 7    k7 = f(y_{n+1}), the error e = h sum_j (b_j - bhat_j) k_j, per-sub-tile
//           sums of (e / sc)^2 with sc = atol + rtol max(|y_n|, |y_{n+1}|), and the
//           fixed-point sums of sin and cos of the Hermite-interpolated phases at
//           the output times inside (t, t + h].  The last CTA of the instance
//           reduces them in a fixed order, accepts (err <= 1) or rejects, sets
//           the next step size and records the dense order parameters.  An
//           attempt whose stage inputs left the fixed-point range of the window
//           sums is rejected with the smallest step factor (as a non-finite
//           error is), not reported as a failure.
// ds 8 starts a run: the prefix of f(y_n) and R(t0); ds 1 then computes
// k1 = f(y_n) from it and continues as ds 0.  ds 9 ends a run: the state moves
// back to the first buffer if needed and the prefix of f(y) is rebuilt for the
// RK4 kernels (without recording R).
// An instance that is done skips every kernel whole (its arrival counters stay
// consistent); accepting swaps the roles of the two state buffers and of the
// two first-stage buffers instead of copying.
#include "dp_control.cuh"
#include "ring_parts.cuh"

namespace simk {

template <int M> struct DpMinBlocks { static constexpr int value = 4; };
template <> struct DpMinBlocks<2> { static constexpr int value = 2; };

__device__ __forceinline__ double warp_sum_f64(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ long long warp_sum_i64(long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int M, int DS>
__global__ void __launch_bounds__(kRingThreads, DpMinBlocks<M>::value)
    dp_stage_kernel(const DpPlan *__restrict__ plans, const int *__restrict__ inst_of_item,
                    const int64_t *__restrict__ item_base)
{
    using Mo = Model<M>;
    constexpr int D = Mo::D, NQ = Mo::NQ, NX = Mo::NX, XOFF = D - NX;
    constexpr bool KURAMOTO = M == 0 || M == 3;
    constexpr bool EDGE = DS >= 8;                // run start (8) or end (9)
    constexpr int pin = (DS + 1) & 1;             // prefix buffer read (ds 1..7)
    constexpr int pout = EDGE ? 0 : (DS <= 1 ? 1 : (DS & 1)); // prefix buffer written
    constexpr int NW = kRingThreads / 32;
    __shared__ RingBases<NQ> s_bases;

    const int inst = inst_of_item[blockIdx.x];
    const DpPlan &Q = plans[inst];
    const RingPlan &P = Q.r;
    const DpCtl *ctl = Q.ctl;
    if (!EDGE && *(const volatile int *)&ctl->done) return;
    const int64_t sub = (int64_t)blockIdx.x - item_base[inst];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t N = P.N;
    const int64_t i = sub * kSubTile + tid;
    const int cur = ctl->cur;
    const double h = ctl->h_att;
    const double *__restrict__ y = Q.ybuf[cur];
    double *__restrict__ y5 = Q.ybuf[cur ^ 1];
    const double *k1 = Q.k[cur];
    if (DS >= 1 && DS <= 7) ring_load_bases<NQ>(P, P.ingrp[pin], P.grpofs[pin], sub, s_bases);

    int64_t qv[NQ];
    bool ok = true;
#pragma unroll
    for (int c = 0; c < NQ; ++c) qv[c] = 0;
    double err_acc = 0.0;
    double k[D];
    if (EDGE && i < N) {
        double xn[D];
#pragma unroll
        for (int v = 0; v < D; ++v) {
            const int64_t q = v * N + i;
            xn[v] = y[q];
            if (DS == 9 && cur == 1) Q.ybuf[0][q] = xn[v];
        }
        Mo::coupled_q(P.mp, xn, P.F, P.lim, ok, qv);
    }
    if (EDGE) {
        if (!ok) raise_error(P.err, ERR_RANGE);
        ring_prefix_tail<NQ, DS == 8 && KURAMOTO, false>(P, P.lam[0], P.ingrp[0], P.grpofs[0], sub, i, qv);
        return;
    }
    if (i < N) {
        if (DS >= 1) {
            int64_t qo[NQ];
            double fo[NQ];
            i128 W[NQ];
            ring_window<NQ>(P, P.lam[pin], s_bases, tid, i, qo, fo, W);
            double X[NX > 0 ? NX : 1];
#pragma unroll
            for (int g = 0; g < NX; ++g) X[g] = DS == 1 ? y[(XOFF + g) * N + i] : P.xg[pin][g * N + i];
            const double Iext = (M == 2 && P.node_param) ? P.node_param[i] : 0.0;
            Mo::rhs(P.mp, P.F, fo, qo, W, X, Iext, k);
        }
        if (DS <= 6) {
            double xn[D];
#pragma unroll
            for (int v = 0; v < D; ++v) {
                const int64_t q = v * N + i;
                double acc;
                if (DS == 0) {
                    acc = c_dp_a[1][0] * k1[q];
                } else if (DS == 1) {
                    Q.k[cur][q] = k[v];
                    acc = c_dp_a[1][0] * k[v];
                } else {
                    Q.k[DS][q] = k[v];
                    acc = c_dp_a[DS][0] * k1[q];
#pragma unroll
                    for (int j = 1; j < DS - 1; ++j) acc += c_dp_a[DS][j] * Q.k[j + 1][q];
                    acc += c_dp_a[DS][DS - 1] * k[v];
                }
                xn[v] = y[q] + h * acc;
                if (DS == 6) y5[q] = xn[v];
            }
            if (NX > 0) {
#pragma unroll
                for (int g = 0; g < NX; ++g) P.xg[pout][g * N + i] = xn[XOFF + g];
            }
            Mo::coupled_q(P.mp, xn, P.F, P.lim, ok, qv);
        } else {
            const double atol = ctl->atol, rtol = ctl->rtol;
#pragma unroll
            for (int v = 0; v < D; ++v) {
                const int64_t q = v * N + i;
                Q.k[cur ^ 1][q] = k[v];
                double e = c_dp_e[0] * k1[q];
#pragma unroll
                for (int j = 2; j <= 5; ++j) e += c_dp_e[j] * Q.k[j + 1][q];
                e += c_dp_e[6] * k[v];
                e *= h;
                const double sc = atol + rtol * fmax(fabs(y[q]), fabs(y5[q]));
                const double r = e / sc;
                err_acc += r * r;
            }
        }
    }

    if (DS <= 6) {
        if (!ok) *(volatile int *)&Q.ctl->bad = 1; // the decision rejects this attempt
        ring_prefix_tail<NQ, false, false>(P, P.lam[pout], P.ingrp[pout], P.grpofs[pout], sub, i, qv);
        return;
    }

    // ds 7: per-sub-tile error sum and dense-output sums, then the decision.
    __shared__ double s_err[NW];
    __shared__ long long s_o[NW][2];
    __shared__ i128 s_w[NW][2];
    __shared__ int s_last;
    err_acc = warp_sum_f64(err_acc);
    if (lane == 0) s_err[warp] = err_acc;

    const double t = ctl->t, t0 = ctl->t0, odt = ctl->out_dt;
    const long long next_out = ctl->next_out, n_out = ctl->n_out;
    const int last = ctl->last;
    int n_here = 0;
    if (KURAMOTO && odt > 0.0) {
        while (n_here < kDpMaxOut && next_out + n_here <= n_out) {
            const double to = t0 + (double)(next_out + n_here) * odt;
            if (!last && to > t + h) break;
            ++n_here;
        }
    }
    for (int o = 0; o < n_here; ++o) {
        long long ss = 0, cc = 0;
        if (i < N) {
            const double to = t0 + (double)(next_out + o) * odt;
            double th = (to - t) / h;
            th = th > 1.0 ? 1.0 : th;
            const double a0 = y[i], a1 = y5[i], f0 = k1[i], f1 = k[0];
            const double ph = (1.0 - th) * a0 + th * a1 +
                              th * (th - 1.0) * ((1.0 - 2.0 * th) * (a1 - a0) + (th - 1.0) * h * f0 + th * h * f1);
            int64_t s62, c62;
            fixed_sincos(ph, P.mp.tab, s62, c62, ok);
            ss = q62_to(s62, P.F);
            cc = q62_to(c62, P.F);
        }
        ss = warp_sum_i64(ss);
        cc = warp_sum_i64(cc);
        if (lane == 0) {
            s_o[warp][0] = ss;
            s_o[warp][1] = cc;
        }
        __syncthreads();
        if (tid == 0) {
            long long a = 0, b = 0;
            for (int w = 0; w < NW; ++w) {
                a += s_o[w][0];
                b += s_o[w][1];
            }
            Q.out_part[(sub * kDpMaxOut + o) * 2] = a;
            Q.out_part[(sub * kDpMaxOut + o) * 2 + 1] = b;
        }
        __syncthreads();
    }
    if (!ok) *(volatile int *)&Q.ctl->bad = 1;
    __syncthreads();
    if (tid == 0) {
        double a = 0.0;
        for (int w = 0; w < NW; ++w) a += s_err[w];
        Q.err_part[sub] = a;
        __threadfence();
        s_last = last_arrival(Q.dp_ctr, (unsigned long long)P.nsub);
    }
    __syncthreads();
    if (!s_last) return;

    // The instance's last CTA: reduce the per-sub-tile sums with a fixed
    // assignment of sub-tiles to threads (deterministic), then decide.
    const int64_t nsub = P.nsub;
    double es = 0.0;
    for (int64_t b = tid; b < nsub; b += kRingThreads) es += __ldcg(Q.err_part + b);
    es = warp_sum_f64(es);
    __syncthreads();
    if (lane == 0) s_err[warp] = es;
    __shared__ i128 s_out[kDpMaxOut][2];
    for (int o = 0; o < n_here; ++o) {
        i128 a = 0, b = 0;
        for (int64_t sb = tid; sb < nsub; sb += kRingThreads) {
            a += (i128)__ldcg(Q.out_part + (sb * kDpMaxOut + o) * 2);
            b += (i128)__ldcg(Q.out_part + (sb * kDpMaxOut + o) * 2 + 1);
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
        const int D = P.model == 2 ? 4 : (P.model == 0 ? 1 : 2);
        dp_decide_ctl(Q.ctl, Q.remaining, tot, (int64_t)D * P.N, n_here, s_out,
                      DpRecord{P.obs, P.obs_cap, P.obs_ctr, P.F, P.N});
    }
}

template <int M>
static cudaError_t launch_m(int ds, const DpGroup &g, cudaStream_t s)
{
    const dim3 grid((unsigned)g.n_items), block(kRingThreads);
    switch (ds) {
    case 0: dp_stage_kernel<M, 0><<<grid, block, 0, s>>>(g.plans, g.inst_of_item, g.item_base); break;
    case 1: dp_stage_kernel<M, 1><<<grid, block, 0, s>>>(g.plans, g.inst_of_item, g.item_base); break;
    case 2: dp_stage_kernel<M, 2><<<grid, block, 0, s>>>(g.plans, g.inst_of_item, g.item_base); break;
    case 3: dp_stage_kernel<M, 3><<<grid, block, 0, s>>>(g.plans, g.inst_of_item, g.item_base); break;
    case 4: dp_stage_kernel<M, 4><<<grid, block, 0, s>>>(g.plans, g.inst_of_item, g.item_base); break;
    case 5: dp_stage_kernel<M, 5><<<grid, block, 0, s>>>(g.plans, g.inst_of_item, g.item_base); break;
    case 6: dp_stage_kernel<M, 6><<<grid, block, 0, s>>>(g.plans, g.inst_of_item, g.item_base); break;
    case 7: dp_stage_kernel<M, 7><<<grid, block, 0, s>>>(g.plans, g.inst_of_item, g.item_base); break;
    case 8: dp_stage_kernel<M, 8><<<grid, block, 0, s>>>(g.plans, g.inst_of_item, g.item_base); break;
    default: dp_stage_kernel<M, 9><<<grid, block, 0, s>>>(g.plans, g.inst_of_item, g.item_base); break;
    }
    return cudaGetLastError();
}

cudaError_t dp_launch(int ds, const DpGroup &g, cudaStream_t s)
{
    if (g.n_items == 0) return cudaSuccess;
    switch (g.model) {
    case 0: return launch_m<0>(ds, g, s);
    case 1: return launch_m<1>(ds, g, s);
    case 2: return launch_m<2>(ds, g, s);
    default: return launch_m<3>(ds, g, s);
    }
}

} // namespace simk
