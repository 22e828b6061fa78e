// Periodic cubic lattice, Kuramoto nodes (Section IV, 3D networks; node index
// k*N1^2 + j*N1 + i).  The (2P+1)^3 box sum is separable, so every RK4 stage is
// three passes over the lattice:
//   x pass  SX(i,j,k)  = sum_{|dx|<=P} Q(f(i+dx,j,k))      (row prefix in shared memory)
//   y pass  SXY(i,j,k) = sum_{|dy|<=P} SX(i,j+dy,k)        (sliding window along j)
//   z pass  W(i,j,k)   = sum_{|dz|<=P} SXY(i,j,k+dz)       (sliding window along k)
//           fused with the right-hand side, the RK4 update, the next stage input
//           and its (sin, cos), and at stage 4 the order parameter.
// f = (sin, cos) of the stage input; Q rounds onto the grid 2^-F with F chosen so
// that a full box sum fits in int64 (every sum is then exact and order-free).
#include "internal.h"

namespace simk {

constexpr int kCubeRowWarps = 8;      // x pass: one warp per row, 8 rows per CTA
constexpr int kCubeMaxN1 = 1024;      // x-pass shared-memory row buffer
constexpr int kCubeColThreads = 128;  // y and z passes: threads per CTA along i

// x pass: one warp per (j, k) row.  pre(p) = sum_{m<p} Q(f(m)) for p in [0, N1]
// is built in shared memory (row stride N1 + 1 per component, sized at launch);
// SX(i) = Pe(i+P+1) - Pe(i-P) on the periodic extension
// Pe(p) = pre(p mod N1) + floor(p / N1) * pre(N1).  Rows are read and written
// with coalesced accesses; the scan runs on the shared-memory copy.
__global__ void __launch_bounds__(32 * kCubeRowWarps) cube_x_kernel(CubePlan p)
{
    extern __shared__ int64_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t N1 = p.N1, P = p.P, nodes = N1 * N1 * N1, stride = N1 + 1;
    int64_t *pre0 = smem + (int64_t)warp * 2 * stride;
    int64_t *pre1 = pre0 + stride;
    const int per = (int)((N1 + 31) / 32); // contiguous chunk per lane in the scan
    bool ok = true;
    for (int64_t row = (int64_t)blockIdx.x * kCubeRowWarps + warp; row < N1 * N1;
         row += (int64_t)gridDim.x * kCubeRowWarps) {
        const double *__restrict__ fs = p.f + row * N1;
        const double *__restrict__ fc = p.f + nodes + row * N1;
        // coalesced loads, 8 per lane in flight before they are used
        for (int64_t mb = lane; mb < N1; mb += 32 * 8) {
            double vs[8], vc[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int64_t m = mb + 32 * u;
                vs[u] = m < N1 ? __ldg(fs + m) : 0.0;
                vc[u] = m < N1 ? __ldg(fc + m) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int64_t m = mb + 32 * u;
                if (m < N1) {
                    pre0[m + 1] = to_fixed(vs[u], p.F, 1, ok);
                    pre1[m + 1] = to_fixed(vc[u], p.F, 1, ok);
                }
            }
        }
        __syncwarp();
        const int m0 = lane * per;
        int64_t r0 = 0, r1 = 0;
        for (int t = 0; t < per; ++t) {
            const int m = m0 + t;
            if (m < N1) {
                r0 += pre0[m + 1];
                r1 += pre1[m + 1];
                pre0[m + 1] = r0;
                pre1[m + 1] = r1;
            }
        }
        const int64_t e0 = warp_incl_scan(r0) - r0, e1 = warp_incl_scan(r1) - r1;
        for (int t = 0; t < per; ++t) {
            const int m = m0 + t;
            if (m < N1) {
                pre0[m + 1] += e0;
                pre1[m + 1] += e1;
            }
        }
        if (lane == 0) {
            pre0[0] = 0;
            pre1[0] = 0;
        }
        __syncwarp();
        const int64_t t0 = pre0[N1], t1 = pre1[N1];
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
        __syncwarp();
    }
    if (!ok) raise_error(p.err, ERR_RANGE);
}

// y pass: one thread per (i, k) column, sliding window along j (exact int64).
// The loop runs in blocks of 8 rows whose 16 window loads per component are
// issued together, so each thread keeps several loads in flight.
__global__ void __launch_bounds__(kCubeColThreads) cube_y_kernel(CubePlan p)
{
    constexpr int U = 8;
    const int64_t N1 = p.N1, P = p.P, nodes = N1 * N1 * N1;
    const int64_t i = (int64_t)blockIdx.x * kCubeColThreads + threadIdx.x;
    const int64_t k = blockIdx.y;
    if (i >= N1) return;
    const int64_t col = k * N1 * N1 + i; // + j * N1
    const int64_t *__restrict__ a0 = p.sx + col;
    const int64_t *__restrict__ a1 = p.sx + nodes + col;
    int64_t *__restrict__ o0 = p.sxy + col;
    int64_t *__restrict__ o1 = p.sxy + nodes + col;
    int64_t s0 = 0, s1 = 0;
    for (int64_t d = -P; d <= P; ++d) {
        const int64_t j = d < 0 ? d + N1 : d;
        s0 += __ldg(a0 + j * N1);
        s1 += __ldg(a1 + j * N1);
    }
    for (int64_t j0 = 0; j0 < N1; j0 += U) {
        int64_t in0[U], out0[U], in1[U], out1[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t j = j0 + u;
            int64_t jin = j + P + 1, jout = j - P;
            if (jin >= N1) jin -= N1;
            if (jout < 0) jout += N1;
            const bool live = j < N1;
            in0[u] = live ? __ldg(a0 + jin * N1) : 0;
            out0[u] = live ? __ldg(a0 + jout * N1) : 0;
            in1[u] = live ? __ldg(a1 + jin * N1) : 0;
            out1[u] = live ? __ldg(a1 + jout * N1) : 0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t j = j0 + u;
            if (j < N1) {
                o0[j * N1] = s0;
                o1[j * N1] = s1;
            }
            s0 += in0[u] - out0[u];
            s1 += in1[u] - out1[u];
        }
    }
}

// Block-wide deterministic reduction of the order-parameter partials; the last
// CTA to finish (ticket order) sums all partials in index order and records R.
__device__ void cube_record_order(const CubePlan &p, int64_t ps, int64_t pc)
{
    __shared__ int64_t s_s[kCubeColThreads], s_c[kCubeColThreads];
    __shared__ bool s_last;
    s_s[threadIdx.x] = ps;
    s_c[threadIdx.x] = pc;
    __syncthreads();
    const unsigned nblk = gridDim.x * gridDim.y;
    const unsigned bid = blockIdx.y * gridDim.x + blockIdx.x;
    if (threadIdx.x == 0) {
        i128 ts = 0, tc = 0;
        for (int t = 0; t < kCubeColThreads; ++t) {
            ts += s_s[t];
            tc += s_c[t];
        }
        p.partial[2 * bid] = ts;
        p.partial[2 * bid + 1] = tc;
        __threadfence();
        const unsigned long long done = atomicAdd(p.done_ctr, 1ull);
        s_last = ((done + 1ull) % nblk) == 0ull;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        i128 ts = 0, tc = 0;
        for (unsigned b = 0; b < nblk; ++b) {
            ts += ld_cg_i128(p.partial + 2 * b);
            tc += ld_cg_i128(p.partial + 2 * b + 1);
        }
        const double S = fixed_to_double(ts, p.F), C = fixed_to_double(tc, p.F);
        const unsigned long long n = *p.obs_ctr;
        p.obs[n % (unsigned long long)p.obs_cap] = sqrt(S * S + C * C) / (double)(p.N1 * p.N1 * p.N1);
        *p.obs_ctr = n + 1;
    }
}

// z pass (STAGE 1..4): one thread per (i, j) column, sliding window along k,
// fused with a4 (RHS), a5 (RK4), a1 (next stage input) and its (sin, cos).
// STAGE 0 is the prologue: f = (sin, cos) of y and the order parameter.
template <int STAGE>
__global__ void __launch_bounds__(kCubeColThreads) cube_z_kernel(CubePlan p, double dt)
{
    const int64_t N1 = p.N1, P = p.P, nodes = N1 * N1 * N1, plane = N1 * N1;
    const int64_t i = (int64_t)blockIdx.x * kCubeColThreads + threadIdx.x;
    const int64_t j = blockIdx.y;
    int64_t ps = 0, pc = 0; // order-parameter partials (stage 0 and 4)
    bool ok = true;
    if (i < N1) {
        const int64_t col = j * N1 + i; // + k * plane
        const int64_t *a0 = p.sxy + col, *a1 = p.sxy + nodes + col;
        int64_t s0 = 0, s1 = 0;
        if (STAGE > 0) {
            for (int64_t d = -P; d <= P; ++d) {
                const int64_t k = d < 0 ? d + N1 : d;
                s0 += a0[k * plane];
                s1 += a1[k * plane];
            }
        }
        for (int64_t k = 0; k < N1; ++k) {
            const int64_t n = col + k * plane;
            double x;
            if (STAGE == 0) {
                x = p.y[n];
            } else {
                const double fo[2] = {p.f[n], p.f[nodes + n]};
                const int64_t qo[2] = {to_fixed(fo[0], p.F, 1, ok), to_fixed(fo[1], p.F, 1, ok)};
                const i128 W[2] = {(i128)s0, (i128)s1};
                double kk[1];
                Model<0>::rhs(p.mp, p.F, fo, qo, W, nullptr, 0.0, kk);
                const double yv = p.y[n];
                if (STAGE == 1) {
                    p.acc[n] = kk[0];
                    x = yv + (0.5 * dt) * kk[0];
                } else if (STAGE == 2) {
                    p.acc[n] = p.acc[n] + 2.0 * kk[0];
                    x = yv + (0.5 * dt) * kk[0];
                } else if (STAGE == 3) {
                    p.acc[n] = p.acc[n] + 2.0 * kk[0];
                    x = yv + dt * kk[0];
                } else {
                    x = yv + (dt / 6.0) * (p.acc[n] + kk[0]);
                    p.y[n] = x;
                }
                int64_t kin = k + P + 1, kout = k - P;
                if (kin >= N1) kin -= N1;
                if (kout < 0) kout += N1;
                s0 += a0[kin * plane] - a0[kout * plane];
                s1 += a1[kin * plane] - a1[kout * plane];
            }
            double sn, cn;
            fast_sincos(x, p.mp.tab, sn, cn);
            p.f[n] = sn;
            p.f[nodes + n] = cn;
            if (STAGE == 0 || STAGE == 4) {
                ps += to_fixed(sn, p.F, 1, ok);
                pc += to_fixed(cn, p.F, 1, ok);
            }
        }
    }
    if (!ok) raise_error(p.err, ERR_RANGE);
    if (STAGE == 0 || STAGE == 4) cube_record_order(p, ps, pc);
}

static dim3 col_grid(int64_t N1)
{
    return dim3((unsigned)((N1 + kCubeColThreads - 1) / kCubeColThreads), (unsigned)N1);
}

constexpr size_t kCubeXSmem = (size_t)kCubeRowWarps * 2 * (kCubeMaxN1 + 1) * sizeof(int64_t); // largest N1

cudaError_t cube_configure()
{
    return cudaFuncSetAttribute(cube_x_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCubeXSmem);
}

static cudaError_t launch_x(const CubePlan &p, cudaStream_t s)
{
    const size_t smem = (size_t)kCubeRowWarps * 2 * (size_t)(p.N1 + 1) * sizeof(int64_t);
    const int64_t rows = p.N1 * p.N1;
    const int64_t want = (rows + kCubeRowWarps - 1) / kCubeRowWarps;
    const unsigned grid = (unsigned)(want < 152 * 16 ? want : 152 * 16);
    cube_x_kernel<<<grid, 32 * kCubeRowWarps, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t cube_prologue(const CubePlan &p, cudaStream_t s)
{
    cube_z_kernel<0><<<col_grid(p.N1), kCubeColThreads, 0, s>>>(p, 0.0);
    return cudaGetLastError();
}

cudaError_t cube_rhs(const CubePlan &p, cudaStream_t s)
{
    cudaError_t e = launch_x(p, s);
    if (e != cudaSuccess) return e;
    cube_y_kernel<<<col_grid(p.N1), kCubeColThreads, 0, s>>>(p);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    cube_z_kernel<1><<<col_grid(p.N1), kCubeColThreads, 0, s>>>(p, 0.0);
    return cudaGetLastError();
}

cudaError_t cube_step(const CubePlan &p, double dt, cudaStream_t s)
{
    for (int stage = 1; stage <= 4; ++stage) {
        cudaError_t e = launch_x(p, s);
        if (e != cudaSuccess) return e;
        cube_y_kernel<<<col_grid(p.N1), kCubeColThreads, 0, s>>>(p);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        switch (stage) {
        case 1: cube_z_kernel<1><<<col_grid(p.N1), kCubeColThreads, 0, s>>>(p, dt); break;
        case 2: cube_z_kernel<2><<<col_grid(p.N1), kCubeColThreads, 0, s>>>(p, dt); break;
        case 3: cube_z_kernel<3><<<col_grid(p.N1), kCubeColThreads, 0, s>>>(p, dt); break;
        default: cube_z_kernel<4><<<col_grid(p.N1), kCubeColThreads, 0, s>>>(p, dt); break;
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

} // namespace simk
