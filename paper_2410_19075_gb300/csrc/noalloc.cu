// sim_ring_step_noalloc: RK4 steps of a ring network without any device
// allocation, for callers that cannot allocate device memory.
//
// Some host programs cannot call cudaMalloc once they are running: a plugin
// inside a larger application that owns every byte of device memory through its
// own arena, a long-running service whose device footprint must be fixed at
// start-up, or a control loop that cannot afford the device-wide
// synchronisation an allocation may cause.  They pass their own device buffer
// for the state; every other buffer the fused stage kernels need lives in the
// static device array below, which each GPU that loads this library keeps until
// the process exits.
//
// The array is sized for rings of at most kNoAllocMaxNodes nodes.  The first
// call on a device looks the array's address up and fills its fast-math tables;
// both are kept for the life of the process, so a cudaDeviceReset() between
// calls (which gives the device a fresh, zeroed copy of the array at a possibly
// different address) is not supported.  Every call
// shares it and it keeps the last call's contents: the call clears the parts
// that must start at zero (arrival counters, error word) itself.  Two calls whose
// work overlaps on the GPU (different streams, or different host threads) race
// on the array and give wrong results; callers must serialise them.
#include <cmath>
#include <cstring>
#include <mutex>

#include "internal.h"
#include "sim.h"

using namespace simk;

namespace {

constexpr int64_t kNoAllocMaxNodes = 65536;
constexpr size_t kNoAllocScratchBytes = size_t(8) << 20; // 8 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
struct DeviceSetup {
    bool done;
    unsigned char *scratch; // device address of g_noalloc_scratch on this device
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mu;
double g_host_tables[kMathTableWords]; // filled once, static (no allocation)
bool g_host_tables_ready = false;

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

// The fast-math tables sit at the start of the scratch array (written once per
// device); the ring buffers follow (sizes as in sim_create).
constexpr size_t kTablesBytes = sizeof(double) * kMathTableWords;
struct NoAllocLayout {
    size_t acc, xg0, xg1, lam0, lam1, ingrp0, ingrp1, grpofs0, grpofs1, subtot, grptot, grpctr, ctrs, obs, total;
};

NoAllocLayout noalloc_layout(int d, int nq, int nx, int64_t N)
{
    const int64_t nsub = (N + kSubTile - 1) / kSubTile, ngroups = (nsub + kGroup - 1) / kGroup;
    NoAllocLayout L{};
    size_t o = up256(kTablesBytes);
    auto take = [&](size_t bytes) { const size_t at = o; o = up256(o + bytes); return at; };
    L.acc = take(sizeof(double) * d * N);
    L.xg0 = take(sizeof(double) * nx * N);
    L.xg1 = take(sizeof(double) * nx * N);
    L.lam0 = take(sizeof(int64_t) * nq * N);
    L.lam1 = take(sizeof(int64_t) * nq * N);
    L.ingrp0 = take(sizeof(i128) * nq * nsub);
    L.ingrp1 = take(sizeof(i128) * nq * nsub);
    L.grpofs0 = take(sizeof(i128) * nq * (ngroups + 1));
    L.grpofs1 = take(sizeof(i128) * nq * (ngroups + 1));
    L.subtot = take(sizeof(int64_t) * nq * nsub);
    L.grptot = take(sizeof(i128) * nq * ngroups);
    L.grpctr = take(sizeof(unsigned long long) * ngroups);
    L.ctrs = take(64);
    L.obs = take(sizeof(double));
    L.total = o;
    return L;
}

// Once per device, with that device current: the device address of the scratch
// array (cudaGetSymbolAddress), and the fast-math tables copied into its start.
int setup_device(unsigned char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return report_cuda_error(e, "sim_ring_step_noalloc: cudaGetDevice");
    }
    if (dev < 0 || dev >= kMaxDevices)
        return report_error(SIM_EDEVICE, "sim_ring_step_noalloc: device index beyond the set-up table (64)");
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_setup[dev].done) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return report_cuda_error(e, "sim_ring_step_noalloc: cudaGetSymbolAddress of the static array");
        }
        if (!g_host_tables_ready) {
            fill_math_tables(g_host_tables);
            g_host_tables_ready = true;
        }
        e = cudaMemcpy(p, g_host_tables, kTablesBytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return report_cuda_error(e, "sim_ring_step_noalloc: copy of the fast-math tables");
        }
        g_setup[dev].scratch = static_cast<unsigned char *>(p);
        g_setup[dev].done = true;
    }
    *out = g_setup[dev].scratch;
    return SIM_OK;
}

} // namespace

extern "C" int sim_ring_step_noalloc(int model, int64_t N, int64_t radius, const double *params, int n_params,
                                     unsigned flags, double *dev_state, const double *dev_node_param,
                                     int64_t n_steps, double dt, void *stream)
{
    const int d = model == SIM_KS ? 1 : model == SIM_FHN ? 2 : model == SIM_HH ? 4 : 0;
    const int np = model == SIM_KS ? 3 : model == SIM_FHN ? 4 : model == SIM_HH ? 8 : -1;
    if (d == 0) return report_error(SIM_EINVAL, "sim_ring_step_noalloc: model must be SIM_KS, SIM_FHN or SIM_HH");
    if (!params || n_params != np) return report_error(SIM_EINVAL, "sim_ring_step_noalloc: wrong parameter count");
    if (!dev_state) return report_error(SIM_EINVAL, "sim_ring_step_noalloc: dev_state is NULL");
    if (radius < 1 || N < 2 * radius + 1)
        return report_error(SIM_EINVAL, "sim_ring_step_noalloc: need radius >= 1 and 2 * radius + 1 <= N");
    if (N > kNoAllocMaxNodes)
        return report_error(SIM_EINVAL, "sim_ring_step_noalloc: N exceeds the static scratch array (65536 nodes)");
    if (flags & ~SIM_FLAG_INCLUDE_SELF) return report_error(SIM_EINVAL, "sim_ring_step_noalloc: unknown flags");
    if (n_steps < 0 || !(dt > 0.0) || !std::isfinite(dt))
        return report_error(SIM_EINVAL, "sim_ring_step_noalloc: need n_steps >= 0 and a finite dt > 0");
    for (int i = 0; i < n_params; ++i)
        if (!std::isfinite(params[i])) return report_error(SIM_EINVAL, "sim_ring_step_noalloc: non-finite parameter");
    if ((model == SIM_FHN || model == SIM_HH) && params[0] == 0.0)
        return report_error(SIM_EINVAL, "sim_ring_step_noalloc: eps (FHN) or Cm (HH) must be non-zero");

    const int nq = model == SIM_HH ? 1 : 2, nx = model == SIM_HH ? 3 : 0;
    const NoAllocLayout L = noalloc_layout(d, nq, nx, N);
    if (L.total > kNoAllocScratchBytes)
        return report_error(SIM_EINVAL, "sim_ring_step_noalloc: the ring's buffers exceed the static scratch array");

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // The call reads the error word back and synchronises the stream, neither of
    // which a capturing stream allows: refuse before touching the stream, so that
    // the caller's capture stays intact.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t ce = cudaStreamIsCapturing(s, &cap);
    if (ce != cudaSuccess) return report_cuda_error(ce, "sim_ring_step_noalloc: cudaStreamIsCapturing");
    if (cap != cudaStreamCaptureStatusNone)
        return report_error(SIM_EINVAL, "sim_ring_step_noalloc: the stream is capturing; this call synchronises and cannot be captured");

    unsigned char *b = nullptr;
    int st = setup_device(&b);
    if (st != SIM_OK) return st;

    // Derived constants, as sim_create computes them.
    ModelParams mp{};
    const bool self = (flags & SIM_FLAG_INCLUDE_SELF) != 0;
    mp.include_self = self ? 1 : 0;
    mp.wsize = 2 * radius + 1;
    model_constants(model, params, (double)(self ? mp.wsize : mp.wsize - 1), mp);
    mp.tab = math_tables_at(b);

    RingPlan p{};
    p.model = model;
    p.npt = model == SIM_HH ? 1 : 2;
    p.N = N;
    p.R = radius;
    p.nsub = (N + kSubTile - 1) / kSubTile;
    p.ngroups = (p.nsub + kGroup - 1) / kGroup;
    p.F = model == SIM_KS ? Model<0>::F : model == SIM_FHN ? Model<1>::F : Model<2>::F;
    p.lim = 54 - p.F;
    p.mp = mp;
    if (model == SIM_KS) ring_coupling_constants(p.mp, model, p.F);
    p.y = dev_state;
    p.acc = reinterpret_cast<double *>(b + L.acc);
    p.xg[0] = reinterpret_cast<double *>(b + L.xg0);
    p.xg[1] = reinterpret_cast<double *>(b + L.xg1);
    p.node_param = model == SIM_HH ? dev_node_param : nullptr;
    p.lam[0] = reinterpret_cast<int64_t *>(b + L.lam0);
    p.lam[1] = reinterpret_cast<int64_t *>(b + L.lam1);
    p.ingrp[0] = reinterpret_cast<i128 *>(b + L.ingrp0);
    p.ingrp[1] = reinterpret_cast<i128 *>(b + L.ingrp1);
    p.grpofs[0] = reinterpret_cast<i128 *>(b + L.grpofs0);
    p.grpofs[1] = reinterpret_cast<i128 *>(b + L.grpofs1);
    p.subtot = reinterpret_cast<int64_t *>(b + L.subtot);
    p.grptot = reinterpret_cast<i128 *>(b + L.grptot);
    p.grp_ctr = reinterpret_cast<unsigned long long *>(b + L.grpctr);
    unsigned long long *ctrs = reinterpret_cast<unsigned long long *>(b + L.ctrs);
    p.err = reinterpret_cast<unsigned *>(ctrs + 0);
    p.obs_ctr = ctrs + 1;
    p.top_ctr = ctrs + 2;
    p.obs = reinterpret_cast<double *>(b + L.obs);
    p.obs_cap = 1;

    // The array keeps the previous call's contents: zero the arrival counters,
    // the error word and the observable counter (every other buffer is written
    // before it is read).
    cudaError_t e = cudaMemsetAsync(b + L.grpctr, 0, sizeof(unsigned long long) * p.ngroups, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b + L.ctrs, 0, 64, s);
    if (e == cudaSuccess) e = ring_prologue(p, s);
    for (int64_t t = 0; t < n_steps && e == cudaSuccess; ++t) e = ring_step(p, dt, s);
    unsigned err_word = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err_word, p.err, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return report_cuda_error(e, "sim_ring_step_noalloc");
    }
    if (err_word & ERR_RANGE)
        return report_error(SIM_ENONFINITE,
                            "sim_ring_step_noalloc: the state became non-finite or left the fixed-point range");
    if (err_word & ERR_TIMEOUT)
        return report_error(SIM_ETIMEOUT, "sim_ring_step_noalloc: a device-side wait exceeded its bound");
    return SIM_OK;
}
