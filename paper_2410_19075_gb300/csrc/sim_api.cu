// C ABI of libsim: handles, argument validation, device buffers, the
// CUDA-graph-captured step loop and error reporting (declared in include/sim.h).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <iterator>
#include <map>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "internal.h"
#include "sim.h"

using namespace simk;

thread_local KernelMarks *simk::g_kernel_marks = nullptr;

namespace {

thread_local std::string g_last_error = "no error";

int fail(int status, const std::string &msg)
{
    g_last_error = msg;
    return status;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(SIM_EDEVICE, std::string(what) + ": " + cudaGetErrorString(e));
}

} // namespace

// The thread's last-error message for the other translation units (internal.h).
int simk::report_error(int status, const char *msg)
{
    return fail(status, msg);
}

int simk::report_cuda_error(cudaError_t e, const char *what)
{
    return cuda_fail(e, what);
}

namespace {

constexpr int64_t kObsCap = 65536;
constexpr int kGraphChunk = 16; // RK4 steps per captured graph

size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

int model_dim(int m) { return m == SIM_KS ? 1 : m == SIM_FHN ? 2 : m == SIM_HH ? 4 : m == SIM_KSI ? 2 : 0; }
int model_nq(int m) { return m == SIM_HH ? 1 : 2; }
int model_nx(int m) { return m == SIM_HH ? 3 : m == SIM_KSI ? 1 : 0; }
int model_nparams(int m) { return m == SIM_KS ? 3 : m == SIM_FHN ? 4 : m == SIM_HH ? 8 : m == SIM_KSI ? 4 : -1; }
int ring_F(int m)
{
    return m == SIM_KS ? Model<0>::F : m == SIM_FHN ? Model<1>::F : m == SIM_HH ? Model<2>::F : Model<3>::F;
}
bool is_lattice(int topo) { return topo == SIM_CUBE3D || topo == SIM_BALL3D || topo == SIM_DISK2D; }
int64_t nodes_of(int topo, int64_t N)
{
    return topo == SIM_RING ? N : topo == SIM_DISK2D ? N * N : N * N * N;
}

// Chords (dy, dz, w) of a ball (dims 3) or disk (dims 2) window of radius P:
// for every (dy, dz) with dy^2 + dz^2 <= P^2, the row segment |dx| <= w with
// w = floor(sqrt(P^2 - dy^2 - dz^2)).  Also returns the window size.
std::vector<int4> chords_of(int topo, int64_t P, int64_t *count)
{
    std::vector<int4> out;
    int64_t c = 0;
    const int64_t zr = topo == SIM_BALL3D ? P : 0;
    for (int64_t dz = -zr; dz <= zr; ++dz)
        for (int64_t dy = -P; dy <= P; ++dy) {
            const int64_t r2 = P * P - dy * dy - dz * dz;
            if (r2 < 0) continue;
            int64_t w = (int64_t)std::sqrt((double)r2);
            while ((w + 1) * (w + 1) <= r2) ++w;
            while (w * w > r2) --w;
            out.push_back(make_int4((int)dy, (int)dz, (int)w, 0));
            c += 2 * w + 1;
        }
    *count = c;
    return out;
}

int64_t window_of(int topo, int64_t R)
{
    if (topo == SIM_RING) return 2 * R + 1;
    if (topo == SIM_CUBE3D) return (2 * R + 1) * (2 * R + 1) * (2 * R + 1);
    int64_t c = 0;
    chords_of(topo, R, &c);
    return c;
}

int ceil_log2(uint64_t x)
{
    int r = 0;
    while ((1ull << r) < x) ++r;
    return r;
}

// Rings whose RK4 stage kernels may use the one-pass prefix: few enough groups
// for the 32-bit chunk sums (any model, either kernel variant).
bool ring_flat_eligible(int model, int64_t ngroups)
{
    (void)model;
    return ngroups <= kFlatMaxGroups;
}

// Autotuner cache (process-wide): the kernel variant that measured fastest for
// a plain ring (kind 0: model, N, R) or for a batch (kind 1: the ring members'
// sub-tile count and member count).  sim_create and sim_batch_create apply a
// matching entry; sim_autotune and sim_batch_autotune add entries;
// sim_tune_save / sim_tune_load keep them in a text file.
struct TuneKey {
    int kind, model;
    int64_t a, b;
    bool operator<(const TuneKey &o) const
    {
        return kind != o.kind ? kind < o.kind : model != o.model ? model < o.model : a != o.a ? a < o.a : b < o.b;
    }
};
struct TuneVal {
    int npt, flat;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune;

bool tune_lookup(const TuneKey &k, TuneVal *v)
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(k);
    if (it == g_tune.end()) return false;
    *v = it->second;
    return true;
}

void tune_store(const TuneKey &k, const TuneVal &v)
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[k] = v;
}

// Byte layout of a network's device block.  Each entry is an offset.
struct Layout {
    size_t total = 0;
    size_t y, acc, xg0, xg1, npar, lam0, lam1, ingrp0, ingrp1, grpofs0, grpofs1, subtot, grptot, grpctr;
    size_t fsub0, fsub1, facc; // one-pass prefix (rings of at most kFlatMaxGroups groups)
    size_t f, xs, sx, sxy, cpl, partial, chords, ctrs, obs, tabs;
};

// Ball and disk: one x-window array per chord half-width (one load per chord
// instead of two) for radii of 5 and more, when the arrays fit the budget.
// Measured on the 100^3 ball: 8% faster at P = 6 and 19% on 200^3 at P = 8;
// at P <= 4 the extra x-pass writes cost as much as the loads they save.
constexpr int64_t kWindowMinRadius = 5;
bool lattice_wmode(int topo, int64_t N, int64_t R, unsigned flags)
{
    if (topo != SIM_BALL3D && topo != SIM_DISK2D) return false;
    if ((flags & SIM_FLAG_LOW_MEMORY) || R < kWindowMinRadius) return false;
    return (R + 1) * 16 * nodes_of(topo, N) <= kLatticeWindowBudget;
}

Layout layout_of(int model, int topo, int64_t N, int64_t R, unsigned flags = 0)
{
    Layout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align_up(o + bytes);
        return at;
    };
    const int d = model_dim(model);
    if (topo == SIM_RING) {
        const int nq = model_nq(model), nx = model_nx(model);
        const int64_t nsub = (N + kSubTile - 1) / kSubTile, ngroups = (nsub + kGroup - 1) / kGroup;
        L.y = take(sizeof(double) * d * N);
        L.acc = take(sizeof(double) * d * N);
        L.xg0 = take(sizeof(double) * nx * N);
        L.xg1 = take(sizeof(double) * nx * N);
        L.npar = take(model == SIM_HH ? sizeof(double) * N : 0);
        L.lam0 = take(sizeof(int64_t) * nq * N);
        L.lam1 = take(sizeof(int64_t) * nq * N);
        L.ingrp0 = take(sizeof(i128) * nq * nsub);
        L.ingrp1 = take(sizeof(i128) * nq * nsub);
        L.grpofs0 = take(sizeof(i128) * nq * (ngroups + 1));
        L.grpofs1 = take(sizeof(i128) * nq * (ngroups + 1));
        L.subtot = take(sizeof(int64_t) * nq * nsub);
        L.grptot = take(sizeof(i128) * nq * ngroups);
        L.grpctr = take(sizeof(unsigned long long) * ngroups);
        const bool flat = ring_flat_eligible(model, ngroups);
        L.fsub0 = take(flat ? sizeof(int64_t) * nq * nsub : 0);
        L.fsub1 = take(flat ? sizeof(int64_t) * nq * nsub : 0);
        L.facc = take(flat ? sizeof(unsigned) * 4 * 4 * nq * ngroups : 0);
    } else {
        const int64_t n = nodes_of(topo, N);
        const int64_t nblk = lattice_partial_blocks(topo, N);
        L.y = take(sizeof(double) * d * n);
        L.acc = take(sizeof(double) * d * n);
        L.f = take(sizeof(int64_t) * 2 * n);
        L.xs = take(sizeof(double) * model_nx(model) * n);
        L.sx = take(sizeof(int64_t) * lattice_sx_elems(topo, N, R, lattice_wmode(topo, N, R, flags)));
        L.sxy = take(topo == SIM_CUBE3D ? sizeof(int64_t) * lattice_sxy_elems(N) : 0);
        L.cpl = take(topo == SIM_CUBE3D ? sizeof(double) * n : 0);
        L.partial = take(sizeof(i128) * 2 * nblk);
        L.chords = take(topo == SIM_CUBE3D ? 0 : sizeof(int4) * (2 * R + 1) * (2 * R + 1));
    }
    L.ctrs = take(64);
    L.obs = take(sizeof(double) * kObsCap);
    L.tabs = take(sizeof(double) * kMathTableWords);
    L.total = o;
    return L;
}

const char *validate(int model, int topo, int64_t N, int64_t R, const double *params, int n_params)
{
    if (model_dim(model) == 0) return "unknown model";
    if (topo == SIM_GRAPH) return "link-matrix networks are created with sim_create_graph";
    if (topo != SIM_RING && !is_lattice(topo)) return "unknown topology";
    if (is_lattice(topo) && model != SIM_KS && model != SIM_KSI)
        return "the lattices support the Kuramoto models (with or without inertia) only";
    if (R < 1) return "radius must be >= 1";
    if (N < 2 * R + 1) return "window does not fit: need 2*radius+1 <= N";
    if (topo == SIM_RING && N > (int64_t(1) << 34)) return "ring too large";
    if ((topo == SIM_CUBE3D || topo == SIM_BALL3D) && N > 1024) return "3D lattice edge N1 must be <= 1024";
    if (topo == SIM_DISK2D && N > 8192) return "disk lattice edge N1 must be <= 8192";
    if (n_params != model_nparams(model)) return "wrong number of parameters for this model";
    if (!params) return "params is NULL";
    for (int i = 0; i < n_params; ++i)
        if (!std::isfinite(params[i])) return "non-finite parameter";
    if (model == SIM_FHN && params[0] == 0.0) return "FHN eps must be non-zero";
    if (model == SIM_HH && params[0] == 0.0) return "HH Cm must be non-zero";
    if (model == SIM_KSI && params[0] == 0.0) return "the mass m must be non-zero";
    return nullptr;
}

} // namespace

struct sim_handle {
    int model = 0, topo = 0, d = 0;
    int64_t N = 0, R = 0, nodes = 0;
    unsigned flags = 0;
    cudaStream_t stream = nullptr;       // where work is issued
    cudaStream_t cap_stream = nullptr;   // private stream used only for graph capture
    void *block = nullptr;
    size_t bytes = 0;
    Layout L;
    RingPlan ring{};
    LatticePlan lat{};
    std::vector<int4> chords; // host copy (the upload reads it asynchronously)
    unsigned *err = nullptr;
    unsigned long long *obs_ctr = nullptr;
    double *obs = nullptr;
    bool owns_block = true;               // false: caller's workspace (sim_create_in)
    unsigned h_err = 0;                   // host copies of device words
    unsigned long long h_ctr = 0;
    int64_t steps_done = 0;
    int64_t obs_read = 0;
    std::map<std::pair<double, int>, cudaGraphExec_t> graphs;
    void *dp_block = nullptr;             // Dormand-Prince buffers (allocated on first use)
    DpPlan dp{};
    void *edp_block = nullptr;            // lattice / link-matrix Dormand-Prince buffers (first use)
    ElemDpPlan edp{};
    void *graph_block = nullptr;          // compressed link matrix (general topology)
    GraphPlan graph{};
    int64_t graph_entries = 0;            // difference-table entries
    size_t graph_bytes = 0;               // device bytes of the compressed matrix
    // Which prefix forms of f(y) in buffer 0 are current (rings): bit 0 the
    // two-level scan (Dormand-Prince, cluster and link-matrix kernels read it),
    // bit 1 the one-pass form (RK4 stage kernels of a flat ring).
    int pfx = 3;
};

namespace {

// rings and general link matrices share the node-order buffers and prologue
bool ring_like(sim_t h) { return h->topo == SIM_RING || h->topo == SIM_GRAPH; }

int check_device_error(sim_t h)
{
    cudaError_t e = cudaMemcpyAsync(&h->h_err, h->err, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "device work failed");
    const unsigned w = h->h_err;
    if (w & ERR_TIMEOUT) return fail(SIM_ETIMEOUT, "a device-side wait exceeded its bound; results are invalid");
    if (w & ERR_RANGE) return fail(SIM_ENONFINITE, "the state became non-finite or left the fixed-point range");
    return SIM_OK;
}

bool use_cluster(sim_t h)
{
    return h->topo == SIM_RING && !(h->flags & SIM_FLAG_STREAMING) && cluster_size_for(h->N) > 0;
}

cudaError_t launch_steps(sim_t h, int64_t n, double dt, cudaStream_t s)
{
    if (use_cluster(h)) return n > 0 ? ring_cluster_steps(h->ring, dt, n, s) : cudaSuccess;
    for (int64_t t = 0; t < n; ++t) {
        const cudaError_t e = h->topo == SIM_RING    ? ring_step(h->ring, dt, s)
                              : h->topo == SIM_GRAPH ? graph_step(h->graph, dt, s)
                                                     : lattice_step(h->lat, dt, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int get_graph(sim_t h, double dt, int chunk, cudaGraphExec_t *out)
{
    auto it = h->graphs.find({dt, chunk});
    if (it != h->graphs.end()) {
        *out = it->second;
        return SIM_OK;
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaSuccess;
    if (!h->cap_stream && (e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(e, "capture stream");
    e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    const cudaError_t le = launch_steps(h, chunk, dt, h->cap_stream);
    e = cudaStreamEndCapture(h->cap_stream, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(le, "kernel launch during capture");
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    h->graphs[{dt, chunk}] = ex;
    *out = ex;
    return SIM_OK;
}

// Make the one-pass prefix of buffer 0 current again (after kernels that write
// only the two-level form), without recording an order parameter.
cudaError_t ring_refresh(sim_t h, cudaStream_t s)
{
    RingPlan quiet = h->ring;
    quiet.obs = nullptr;
    const cudaError_t e = ring_prologue(quiet, s);
    if (e == cudaSuccess) h->pfx = 3;
    return e;
}

bool ring_flat(sim_t h) { return h->topo == SIM_RING && h->ring.flat; }

int prologue(sim_t h)
{
    cudaError_t e = cudaMemsetAsync(h->obs_ctr, 0, sizeof(unsigned long long), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->err, 0, sizeof(unsigned), h->stream);
    if (e == cudaSuccess)
        e = ring_like(h) ? ring_prologue(h->ring, h->stream) : lattice_prologue(h->lat, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "prologue");
    h->steps_done = 0;
    h->obs_read = 0;
    h->pfx = 3;
    return SIM_OK;
}

} // namespace

// Derived model constants for K links per node (FP64 on the host).
void simk::model_constants(int model, const double *params, double K, ModelParams &mp)
{
    if (model == SIM_KS || model == SIM_KSI) {
        const double alpha = model == SIM_KS ? params[2] : params[3];
        if (model == SIM_KS) {
            mp.c[0] = params[0];
            mp.c[1] = params[1] / K;
        } else {
            mp.c[0] = params[2] / (params[0] * K); // mu / (m K)
            mp.c[1] = params[1] / params[0];       // eps / m
        }
        mp.c[2] = std::sin(alpha);
        mp.c[3] = std::cos(alpha);
        mp.q[0] = (int64_t)std::llround(std::ldexp(mp.c[3], 62)); // exact: |cos| <= 1, 53-bit significand
        mp.q[1] = (int64_t)std::llround(std::ldexp(mp.c[2], 62));
        // alpha = aq pi/2 + alpha0 with alpha0 in [0, pi/2): the angle addition of
        // the ring and link-matrix right-hand side (ring_coupling)
        {
            const long double half_pi = 1.570796326794896619231321691639751442L;
            const long double a = (long double)alpha, q = floorl(a / half_pi), a0 = a - q * half_pi;
            const long double two63 = 9223372036854775808.0L;
            mp.a0[0] = (uint64_t)roundl(fminl(fmaxl(cosl(a0), 0.0L), 1.0L) * two63);
            mp.a0[1] = (uint64_t)roundl(fminl(fmaxl(sinl(a0), 0.0L), 1.0L) * two63);
            const long long qi = (long long)q % 4;
            mp.aq = (int)(qi < 0 ? qi + 4 : qi);
        }
        // lattices: the constant of the right-hand side with the node's own term
        // (-sin alpha in the rotated window sum) taken out
        if (model == SIM_KS) mp.c[4] = mp.include_self ? mp.c[0] : mp.c[0] + mp.c[1] * mp.c[2];
        else mp.c[4] = mp.include_self ? 0.0 : mp.c[0] * mp.c[2];
    } else if (model == SIM_FHN) {
        const double ph = params[3], inv_eps = 1.0 / params[0], sK = params[2] / K;
        mp.c[0] = inv_eps;
        mp.c[1] = params[1];
        mp.c[2] = sK * std::cos(ph) * inv_eps;  // (sigma/K) B00 / eps
        mp.c[3] = sK * std::sin(ph) * inv_eps;  // (sigma/K) B01 / eps
        mp.c[4] = -sK * std::sin(ph);           // (sigma/K) B10
        mp.c[5] = sK * std::cos(ph);            // (sigma/K) B11
    } else {
        mp.c[0] = 1.0 / params[0];
        for (int i = 1; i < 7; ++i) mp.c[i] = params[i];
        mp.c[7] = params[7] / K;
    }
}

// A Kuramoto ring's shift of its exact window sums into int64 and the scale of
// the cross product T on the grid 2^-(F - ksh - 3) (see ring_coupling).
void simk::ring_coupling_constants(ModelParams &mp, int model, int F)
{
    const int lg = ceil_log2((uint64_t)mp.wsize);
    mp.ksh = lg + F - 61 > 0 ? lg + F - 61 : 0;
    mp.c[5] = std::ldexp(model == SIM_KS ? mp.c[1] : mp.c[0], mp.ksh + 3 - F);
}

// A lattice's rotation by -alpha (the ball's and disk's x pass rotate every
// node's (sin, cos); the cube turns the node's own phase by +alpha with the
// model's a0, aq instead) and the scale of the right-hand side's cross product
// (see lattice_coupling).
void simk::lattice_rotation(LatticePlan &p, double alpha)
{
    const long double half_pi = 1.570796326794896619231321691639751442L;
    const long double a = (long double)alpha;
    long double q = floorl(a / half_pi);
    const long double a0 = a - q * half_pi; // in [0, pi/2) up to rounding
    const long double c0 = cosl(a0), s0 = sinl(a0);
    const long double two63 = 9223372036854775808.0L;
    p.rot_c = (uint64_t)roundl(fminl(fmaxl(c0, 0.0L), 1.0L) * two63); // <= 2^63
    p.rot_s = (uint64_t)roundl(fminl(fmaxl(s0, 0.0L), 1.0L) * two63);
    long long qi = (long long)q % 4;
    p.rot_q = (int)(qi < 0 ? qi + 4 : qi);
    // the cross product T lands on the grid 2^-(F-2): fold that scale into the coefficient
    p.mp.c[5] = std::ldexp(p.model == SIM_KS ? p.mp.c[1] : p.mp.c[0], -(p.F - 2));
}

extern "C" {

size_t sim_workspace_bytes(int model, int topology, int64_t N, int64_t radius)
{
    double dummy[8] = {1, 1, 1, 1, 1, 1, 1, 1};
    if (validate(model, topology, N, radius, dummy, model_nparams(model))) return 0;
    return layout_of(model, topology, N, radius).total;
}

static const double *host_tables()
{
    static double tab[kMathTableWords];
    static std::once_flag once;
    std::call_once(once, [] { fill_math_tables(tab); });
    return tab;
}

static int create_impl(sim_t *out, int model, int topology, int64_t N, int64_t radius, const double *params,
                       int n_params, unsigned flags, void *workspace, size_t workspace_bytes, void *stream)
{
    if (!out) return fail(SIM_EINVAL, "out is NULL");
    *out = nullptr;
    if (const char *msg = validate(model, topology, N, radius, params, n_params)) return fail(SIM_EINVAL, msg);
    if (flags & ~(SIM_FLAG_INCLUDE_SELF | SIM_FLAG_STREAMING | SIM_FLAG_LOW_MEMORY))
        return fail(SIM_EINVAL, "unknown flags");

    sim_t h = new sim_handle();
    h->model = model;
    h->topo = topology;
    h->d = model_dim(model);
    h->N = N;
    h->R = radius;
    h->nodes = nodes_of(topology, N);
    h->flags = flags;
    h->stream = static_cast<cudaStream_t>(stream);
    h->L = layout_of(model, topology, N, radius, flags);
    h->bytes = h->L.total;

    cudaError_t e = cudaSuccess;
    if (workspace) {
        if (workspace_bytes < h->bytes || (reinterpret_cast<uintptr_t>(workspace) & 255u)) {
            delete h;
            return fail(SIM_EINVAL, "workspace smaller than sim_workspace_bytes() or not 256-byte aligned");
        }
        h->block = workspace;
        h->owns_block = false;
    } else {
        e = cudaMalloc(&h->block, h->bytes);
        if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();
            h->block = nullptr;
            sim_destroy(h);
            return fail(SIM_ENOMEM, "device allocation of " + std::to_string(h->bytes) + " bytes failed");
        }
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(h->block, 0, h->bytes, h->stream);
    if (e != cudaSuccess) {
        sim_destroy(h);
        return cuda_fail(e, "sim_create");
    }
    char *b = static_cast<char *>(h->block);
    const Layout &L = h->L;
    unsigned long long *ctrs = reinterpret_cast<unsigned long long *>(b + L.ctrs);
    h->err = reinterpret_cast<unsigned *>(ctrs + 0);
    h->obs_ctr = ctrs + 1;
    unsigned long long *ticket = ctrs + 2;
    h->obs = reinterpret_cast<double *>(b + L.obs);

    // Tables of the fast elementary functions (from a static host copy, so the
    // copy needs no synchronisation).
    e = cudaMemcpyAsync(b + L.tabs, host_tables(), sizeof(double) * kMathTableWords, cudaMemcpyHostToDevice,
                        h->stream);
    if (e != cudaSuccess) {
        sim_destroy(h);
        return cuda_fail(e, "table upload");
    }
    // Derived model constants (FP64 on the host).
    ModelParams mp{};
    mp.tab = math_tables_at(b + L.tabs);
    const bool self = (flags & SIM_FLAG_INCLUDE_SELF) != 0;
    mp.include_self = self ? 1 : 0;
    mp.wsize = window_of(topology, radius);
    model_constants(model, params, (double)(self ? mp.wsize : mp.wsize - 1), mp);

    if (topology == SIM_RING) {
        RingPlan &p = h->ring;
        p.model = model;
        p.N = N;
        p.R = radius;
        p.nsub = (N + kSubTile - 1) / kSubTile;
        p.ngroups = (p.nsub + kGroup - 1) / kGroup;
        p.F = ring_F(model);
        p.lim = 54 - p.F;
        p.mp = mp;
        if (model == SIM_KS || model == SIM_KSI) ring_coupling_constants(p.mp, model, p.F);
        p.y = reinterpret_cast<double *>(b + L.y);
        p.acc = reinterpret_cast<double *>(b + L.acc);
        p.xg[0] = reinterpret_cast<double *>(b + L.xg0);
        p.xg[1] = reinterpret_cast<double *>(b + L.xg1);
        p.node_param = model == SIM_HH ? reinterpret_cast<double *>(b + L.npar) : nullptr;
        p.lam[0] = reinterpret_cast<int64_t *>(b + L.lam0);
        p.lam[1] = reinterpret_cast<int64_t *>(b + L.lam1);
        p.ingrp[0] = reinterpret_cast<i128 *>(b + L.ingrp0);
        p.ingrp[1] = reinterpret_cast<i128 *>(b + L.ingrp1);
        p.grpofs[0] = reinterpret_cast<i128 *>(b + L.grpofs0);
        p.grpofs[1] = reinterpret_cast<i128 *>(b + L.grpofs1);
        p.subtot = reinterpret_cast<int64_t *>(b + L.subtot);
        p.grptot = reinterpret_cast<i128 *>(b + L.grptot);
        p.grp_ctr = reinterpret_cast<unsigned long long *>(b + L.grpctr);
        p.top_ctr = ticket;
        p.err = h->err;
        p.obs = h->obs;
        p.obs_cap = kObsCap;
        p.obs_ctr = h->obs_ctr;
        p.flat = ring_flat_eligible(model, p.ngroups) ? 1 : 0;
        p.npt = model == SIM_HH ? 1 : 2;
        TuneVal tv;
        if (tune_lookup(TuneKey{0, model, N, radius}, &tv)) {
            p.npt = model == SIM_HH || tv.npt == 1 ? 1 : 2;
            p.flat = p.flat && tv.flat ? 1 : 0;
        }
        if (p.flat) {
            const size_t slot = 4 * (size_t)model_nq(model) * p.ngroups;
            p.fsub[0] = reinterpret_cast<int64_t *>(b + L.fsub0);
            p.fsub[1] = reinterpret_cast<int64_t *>(b + L.fsub1);
            for (int k = 0; k < 4; ++k) p.facc[k] = reinterpret_cast<unsigned *>(b + L.facc) + k * slot;
            p.flat_ctr = ctrs + 3;
        }
        if (N <= kClusterMaxNodes && !(flags & SIM_FLAG_STREAMING)) {
            static std::once_flag cl_once;
            static cudaError_t cl_err = cudaSuccess;
            std::call_once(cl_once, [] { cl_err = ring_cluster_configure(); });
            if (cl_err != cudaSuccess) h->flags |= SIM_FLAG_STREAMING; // fall back to the streaming kernels
        }
    } else {
        LatticePlan &p = h->lat;
        p.model = model;
        p.topo = topology;
        p.dims = topology == SIM_DISK2D ? 2 : 3;
        p.N1 = N;
        p.P = radius;
        p.nodes = h->nodes;
        p.F = 61 - ceil_log2((uint64_t)mp.wsize);
        p.mp = mp;
        lattice_rotation(p, model == SIM_KS ? params[2] : params[3]);
        p.y = reinterpret_cast<double *>(b + L.y);
        p.acc = reinterpret_cast<double *>(b + L.acc);
        p.f = reinterpret_cast<int64_t *>(b + L.f);
        p.xs = reinterpret_cast<double *>(b + L.xs);
        p.sx = reinterpret_cast<int64_t *>(b + L.sx);
        p.rs = N + 2 * radius + 1;
        p.wmode = lattice_wmode(topology, N, radius, flags) ? 1 : 0;
        p.sxy = reinterpret_cast<int64_t *>(b + L.sxy);
        p.cpl = reinterpret_cast<double *>(b + L.cpl);
        p.partial = reinterpret_cast<i128 *>(b + L.partial);
        p.done_ctr = ticket;
        p.tile_ctr = ctrs + 4;
        p.err = h->err;
        p.obs = h->obs;
        p.obs_cap = kObsCap;
        p.obs_ctr = h->obs_ctr;
        p.chords = nullptr;
        p.nchords = 0;
        if (topology != SIM_CUBE3D) {
            int64_t cnt = 0;
            const std::vector<int4> ch = chords_of(topology, radius, &cnt);
            h->chords = ch;
            p.chords = reinterpret_cast<const int4 *>(b + L.chords);
            p.nchords = (int)ch.size();
            e = cudaMemcpyAsync(b + L.chords, h->chords.data(), sizeof(int4) * ch.size(), cudaMemcpyHostToDevice,
                                h->stream);
        }
        static std::once_flag lat_once;
        static cudaError_t lat_err = cudaSuccess;
        std::call_once(lat_once, [] { lat_err = lattice_configure(); });
        if (e == cudaSuccess) e = lat_err;
        if (e != cudaSuccess) {
            sim_destroy(h);
            return cuda_fail(e, "lattice set-up");
        }
    }
    const int st = prologue(h);
    if (st != SIM_OK) {
        sim_destroy(h);
        return st;
    }
    *out = h;
    return SIM_OK;
}

// Algorithm 2 (Section III.C) on the host.  ROL by i maps link j of row i to
// offset (j - i) mod N; XOR is the symmetric difference of sorted offset sets.
// Every row i is stored as the entry of the difference table holding
// XOR(ROL(row_i, i), V), found through a hash of its offsets, and V is kept as
// runs of consecutive offsets.  The paper takes V = row 0; here V is the most
// frequent shifted row (row 0 among equals), so that the rows of a periodic
// lattice, whose node 0 is a corner with wrapped links, map to the empty entry
// except near the boundary.  EXTRACT is unchanged: row_i = ROR(XOR(V, D), i).
// Each entry keeps its offsets with the sign they carry in the coupling sum and
// the link count of its rows.
struct CompressedLinks {
    std::vector<int2> runs;
    std::vector<int> ent;
    std::vector<int64_t> dptr{0};
    std::vector<int2> dpos;
    std::vector<int64_t> ek;
    std::vector<double> ecs;
};

static std::string offsets_key(const std::vector<int64_t> &v)
{
    return std::string(reinterpret_cast<const char *>(v.data()), v.size() * sizeof(int64_t));
}

// Shifted row i (sorted); nullptr or the reason it is invalid.
static const char *shifted_row(int64_t N, const int64_t *row_ptr, const int64_t *col, int64_t i,
                               std::vector<int64_t> &sh)
{
    sh.clear();
    for (int64_t t = row_ptr[i]; t < row_ptr[i + 1]; ++t) {
        const int64_t j = col[t];
        if (j < 0 || j >= N) return "a link index is outside [0, N)";
        sh.push_back(j >= i ? j - i : j - i + N);
    }
    std::sort(sh.begin(), sh.end());
    if (std::adjacent_find(sh.begin(), sh.end()) != sh.end()) return "a row lists the same link twice";
    return nullptr;
}

static const char *compress_links(int64_t N, const int64_t *row_ptr, const int64_t *col, CompressedLinks &T)
{
    if (row_ptr[0] != 0) return "row_ptr[0] must be 0";
    for (int64_t i = 0; i < N; ++i)
        if (row_ptr[i + 1] < row_ptr[i]) return "row_ptr must not decrease";
    if (row_ptr[N] > 0 && !col) return "col is NULL";
    // pass 1: the most frequent shifted row becomes V
    std::vector<int64_t> sh, d, V;
    {
        std::unordered_map<std::string, std::pair<int64_t, int64_t>> count; // key -> (count, first row)
        int64_t best = -1, best_row = 0;
        for (int64_t i = 0; i < N; ++i) {
            if (const char *why = shifted_row(N, row_ptr, col, i, sh)) return why;
            auto &c = count[offsets_key(sh)];
            if (c.first++ == 0) c.second = i;
            if (c.first > best || (c.first == best && c.second < best_row)) {
                best = c.first;
                best_row = c.second;
            }
        }
        shifted_row(N, row_ptr, col, best_row, V);
    }
    for (size_t t = 0; t < V.size();) { // runs of consecutive offsets
        size_t u = t + 1;
        while (u < V.size() && V[u] == V[u - 1] + 1) ++u;
        T.runs.push_back(make_int2((int)V[t], (int)(u - t)));
        t = u;
    }
    // pass 2: the difference table
    T.ent.resize(N);
    std::unordered_map<std::string, int> index;
    for (int64_t i = 0; i < N; ++i) {
        shifted_row(N, row_ptr, col, i, sh);
        d.clear();
        std::set_symmetric_difference(sh.begin(), sh.end(), V.begin(), V.end(), std::back_inserter(d));
        std::string key = offsets_key(d);
        auto it = index.find(key);
        if (it != index.end()) {
            T.ent[i] = it->second;
            continue;
        }
        const int e = (int)index.size();
        index.emplace(std::move(key), e);
        T.ent[i] = e;
        int64_t K = (int64_t)V.size();
        for (int64_t p : d) {
            const int sign = std::binary_search(V.begin(), V.end(), p) ? -1 : 1;
            T.dpos.push_back(make_int2((int)p, sign));
            K += sign;
        }
        T.dptr.push_back((int64_t)T.dpos.size());
        T.ek.push_back(K);
        T.ecs.push_back(K > 0 ? 1.0 / (double)K : 0.0);
    }
    return nullptr;
}

int sim_create(sim_t *out, int model, int topology, int64_t N, int64_t radius, const double *params,
               int n_params, unsigned flags, void *stream)
{
    return create_impl(out, model, topology, N, radius, params, n_params, flags, nullptr, 0, stream);
}

int sim_create_in(sim_t *out, int model, int topology, int64_t N, int64_t radius, const double *params,
                  int n_params, unsigned flags, void *dev_workspace, size_t workspace_bytes, void *stream)
{
    if (!dev_workspace) return fail(SIM_EINVAL, "workspace is NULL");
    return create_impl(out, model, topology, N, radius, params, n_params, flags, dev_workspace, workspace_bytes,
                       stream);
}

int sim_create_graph(sim_t *out, int model, int64_t N, const int64_t *row_ptr, const int64_t *col,
                     const double *params, int n_params, void *stream)
{
    if (!out) return fail(SIM_EINVAL, "out is NULL");
    *out = nullptr;
    if (N < 3 || N > INT32_MAX) return fail(SIM_EINVAL, "a link matrix needs 3 <= N < 2^31 nodes");
    if (!row_ptr) return fail(SIM_EINVAL, "row_ptr is NULL");
    CompressedLinks T;
    if (const char *why = compress_links(N, row_ptr, col, T)) return fail(SIM_EINVAL, why);
    // The node-order buffers of a ring of N nodes (radius 1 only sizes its window
    // bases, which a link matrix does not use), streaming kernels.
    sim_t h = nullptr;
    int st = create_impl(&h, model, SIM_RING, N, 1, params, n_params, SIM_FLAG_STREAMING, nullptr, 0, stream);
    if (st != SIM_OK) return st;
    h->topo = SIM_GRAPH;
    h->R = 0;
    // constants for K = 1: every node's coupling is scaled by 1 / K_i on the device
    model_constants(model, params, 1.0, h->ring.mp);
    h->ring.mp.include_self = 1; // the link sums are exact; a self link is just one of the links
    h->ring.mp.wsize = 1;
    // device tables
    const size_t o_runs = 0, o_ent = align_up(sizeof(int2) * (T.runs.size() + 1));
    const size_t o_dptr = o_ent + align_up(sizeof(int) * T.ent.size());
    const size_t o_dpos = o_dptr + align_up(sizeof(int64_t) * T.dptr.size());
    const size_t o_ek = o_dpos + align_up(sizeof(int2) * (T.dpos.size() + 1));
    const size_t o_ecs = o_ek + align_up(sizeof(int64_t) * T.ek.size());
    const size_t total = o_ecs + align_up(sizeof(double) * T.ecs.size());
    cudaError_t e = cudaMalloc(&h->graph_block, total);
    if (e != cudaSuccess) {
        h->graph_block = nullptr;
        sim_destroy(h);
        return fail(SIM_ENOMEM, "device allocation of the compressed link matrix failed");
    }
    char *b = static_cast<char *>(h->graph_block);
    auto up = [&](size_t off, const void *src, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(b + off, src, bytes, cudaMemcpyHostToDevice, h->stream);
    };
    up(o_runs, T.runs.data(), sizeof(int2) * T.runs.size());
    up(o_ent, T.ent.data(), sizeof(int) * T.ent.size());
    up(o_dptr, T.dptr.data(), sizeof(int64_t) * T.dptr.size());
    up(o_dpos, T.dpos.data(), sizeof(int2) * T.dpos.size());
    up(o_ek, T.ek.data(), sizeof(int64_t) * T.ek.size());
    up(o_ecs, T.ecs.data(), sizeof(double) * T.ecs.size());
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream); // the host tables go out of scope
    if (e != cudaSuccess) {
        sim_destroy(h);
        return cuda_fail(e, "link matrix upload");
    }
    GraphPlan &g = h->graph;
    h->ring.flat = 0; // the link-matrix kernels read the two-level prefix
    g.r = h->ring;
    g.runs = reinterpret_cast<const int2 *>(b + o_runs);
    g.nruns = (int)T.runs.size();
    g.ent = reinterpret_cast<const int *>(b + o_ent);
    g.dptr = reinterpret_cast<const int64_t *>(b + o_dptr);
    g.dpos = reinterpret_cast<const int2 *>(b + o_dpos);
    g.ek = reinterpret_cast<const int64_t *>(b + o_ek);
    g.ecs = reinterpret_cast<const double *>(b + o_ecs);
    h->graph_entries = (int64_t)T.ek.size();
    h->graph_bytes = total;
    *out = h;
    return SIM_OK;
}

int sim_graph_info(sim_t h, int64_t *n_entries, int64_t *n_runs, size_t *device_bytes)
{
    if (!h || h->topo != SIM_GRAPH) return fail(SIM_EINVAL, "not a link-matrix network");
    if (n_entries) *n_entries = h->graph_entries;
    if (n_runs) *n_runs = h->graph.nruns;
    if (device_bytes) *device_bytes = h->graph_bytes;
    return SIM_OK;
}

int64_t sim_nodes(sim_t h) { return h ? h->nodes : 0; }
int sim_dim(sim_t h) { return h ? h->d : 0; }

static int set_state_impl(sim_t h, const double *src, int64_t n_values, cudaMemcpyKind kind)
{
    if (!h || !src) return fail(SIM_EINVAL, "NULL handle or buffer");
    if (n_values != (int64_t)h->d * h->nodes) return fail(SIM_EINVAL, "n_values must equal dim * nodes");
    double *y = ring_like(h) ? h->ring.y : h->lat.y;
    cudaError_t e = cudaMemcpyAsync(y, src, sizeof(double) * n_values, kind, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "state copy");
    return prologue(h);
}

int sim_set_state(sim_t h, const double *host_soa, int64_t n_values)
{
    return set_state_impl(h, host_soa, n_values, cudaMemcpyHostToDevice);
}

int sim_set_state_device(sim_t h, const double *dev_soa, int64_t n_values)
{
    return set_state_impl(h, dev_soa, n_values, cudaMemcpyDeviceToDevice);
}

int sim_set_node_param(sim_t h, int which, const double *host, int64_t n)
{
    if (!h || !host) return fail(SIM_EINVAL, "NULL handle or buffer");
    if (h->model != SIM_HH || which != 0) return fail(SIM_EINVAL, "only the HH external current (which = 0) is a node parameter");
    if (n != h->nodes) return fail(SIM_EINVAL, "n must equal the number of nodes");
    cudaError_t e = cudaMemcpyAsync(const_cast<double *>(h->ring.node_param), host, sizeof(double) * n,
                                    cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "node parameter copy");
    return SIM_OK;
}

int sim_step(sim_t h, int64_t n_steps, double dt)
{
    if (!h) return fail(SIM_EINVAL, "NULL handle");
    if (n_steps < 0) return fail(SIM_EINVAL, "n_steps must be >= 0");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(SIM_EINVAL, "dt must be finite and > 0");
    if (n_steps > 0 && ring_flat(h)) {
        if (use_cluster(h)) {
            h->pfx = 1; // the cluster kernel leaves the two-level form
        } else {
            if (!(h->pfx & 2)) {
                const cudaError_t e = ring_refresh(h, h->stream);
                if (e != cudaSuccess) return cuda_fail(e, "prefix refresh");
            }
            h->pfx = 2;
        }
    }
    int64_t left = n_steps;
    while (left > 0) {
        const int chunk = left >= kGraphChunk ? kGraphChunk : 1;
        cudaGraphExec_t ex;
        const int st = get_graph(h, dt, chunk, &ex);
        if (st != SIM_OK) return st;
        const cudaError_t e = cudaGraphLaunch(ex, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
        left -= chunk;
        h->steps_done += chunk;
    }
    return SIM_OK;
}

int sim_step_timed(sim_t h, int64_t n_steps, double dt, double *ms_by_kind, int64_t *launches_by_kind)
{
    if (!h) return fail(SIM_EINVAL, "NULL handle");
    if (n_steps < 1 || n_steps > 4096) return fail(SIM_EINVAL, "n_steps must be in [1, 4096]");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(SIM_EINVAL, "dt must be finite and > 0");
    if (!ms_by_kind || !launches_by_kind) return fail(SIM_EINVAL, "NULL output");
    if (ring_flat(h)) {
        if (use_cluster(h)) {
            h->pfx = 1;
        } else {
            if (!(h->pfx & 2)) {
                const cudaError_t e = ring_refresh(h, h->stream);
                if (e != cudaSuccess) return cuda_fail(e, "prefix refresh");
            }
            h->pfx = 2;
        }
    }
    const int per_step = use_cluster(h) ? 1 : h->topo == SIM_CUBE3D ? 13 : is_lattice(h->topo) ? 8 : 4;
    const int cap = (int)(use_cluster(h) ? 1 : per_step * n_steps);
    std::vector<cudaEvent_t> ev(cap + 1, nullptr);
    std::vector<unsigned char> kind(cap, 0);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i <= cap && e == cudaSuccess; ++i) e = cudaEventCreate(&ev[i]);
    KernelMarks marks{ev.data() + 1, kind.data(), cap, 0};
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], h->stream);
    if (e == cudaSuccess) {
        g_kernel_marks = &marks;
        e = launch_steps(h, n_steps, dt, h->stream);
        g_kernel_marks = nullptr;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    for (int k = 0; k < 4; ++k) {
        ms_by_kind[k] = 0.0;
        launches_by_kind[k] = 0;
    }
    for (int i = 0; i < marks.n && e == cudaSuccess; ++i) {
        float ms = 0.0f;
        e = cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
        ms_by_kind[kind[i] & 3] += ms;
        launches_by_kind[kind[i] & 3] += 1;
    }
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    if (e != cudaSuccess) return cuda_fail(e, "sim_step_timed");
    h->steps_done += n_steps;
    return check_device_error(h);
}

static int get_state_impl(sim_t h, double *dst, int64_t n_values, cudaMemcpyKind kind)
{
    if (!h || !dst) return fail(SIM_EINVAL, "NULL handle or buffer");
    if (n_values != (int64_t)h->d * h->nodes) return fail(SIM_EINVAL, "n_values must equal dim * nodes");
    const double *y = ring_like(h) ? h->ring.y : h->lat.y;
    const cudaError_t e = cudaMemcpyAsync(dst, y, sizeof(double) * n_values, kind, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "state copy");
    return SIM_OK;
}

int sim_get_state(sim_t h, double *host_soa, int64_t n_values)
{
    const int st = get_state_impl(h, host_soa, n_values, cudaMemcpyDeviceToHost);
    if (st != SIM_OK) return st;
    return check_device_error(h);
}

int sim_get_state_device(sim_t h, double *dev_soa, int64_t n_values)
{
    return get_state_impl(h, dev_soa, n_values, cudaMemcpyDeviceToDevice);
}

int sim_rhs(sim_t h, double *host_k, int64_t n_values)
{
    if (!h || !host_k) return fail(SIM_EINVAL, "NULL handle or buffer");
    if (n_values != (int64_t)h->d * h->nodes) return fail(SIM_EINVAL, "n_values must equal dim * nodes");
    if (ring_flat(h) && !(h->pfx & 2)) {
        const cudaError_t e = ring_refresh(h, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "prefix refresh");
    }
    cudaError_t e = h->topo == SIM_RING    ? ring_rhs(h->ring, h->stream)
                    : h->topo == SIM_GRAPH ? graph_rhs(h->graph, h->stream)
                                           : lattice_rhs(h->lat, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "rhs launch");
    const double *acc = ring_like(h) ? h->ring.acc : h->lat.acc;
    e = cudaMemcpyAsync(host_k, acc, sizeof(double) * n_values, cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "rhs copy");
    return check_device_error(h);
}

int sim_observables(sim_t h, double *host_R, int64_t max_values, int64_t *n_written)
{
    if (!h || !n_written || (max_values > 0 && !host_R)) return fail(SIM_EINVAL, "NULL argument");
    *n_written = 0;
    if (h->model != SIM_KS && h->model != SIM_KSI) return check_device_error(h);
    cudaError_t e = cudaMemcpyAsync(&h->h_ctr, h->obs_ctr, sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "observable counter copy");
    const int64_t have = (int64_t)h->h_ctr;
    if (have - h->obs_read > kObsCap) h->obs_read = have - kObsCap;
    int64_t n = have - h->obs_read;
    if (n > max_values) n = max_values;
    int64_t done = 0;
    while (done < n) {
        const int64_t start = (h->obs_read + done) % kObsCap;
        int64_t len = n - done;
        if (start + len > kObsCap) len = kObsCap - start;
        e = cudaMemcpyAsync(host_R + done, h->obs + start, sizeof(double) * len, cudaMemcpyDeviceToHost, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "observable copy");
        done += len;
    }
    h->obs_read += n;
    *n_written = n;
    return check_device_error(h);
}

int sim_sync(sim_t h)
{
    if (!h) return fail(SIM_EINVAL, "NULL handle");
    return check_device_error(h);
}

int64_t sim_steps_done(sim_t h) { return h ? h->steps_done : 0; }

const char *sim_last_error(void) { return g_last_error.c_str(); }

// ---------------------------------------------------------------------------
// Batches: many networks advanced together, ring members of one model in one
// launch per RK4 stage.

} // extern "C"

struct sim_batch_handle {
    cudaStream_t stream = nullptr, cap_stream = nullptr;
    std::vector<sim_t> members;
    std::vector<int> ring_slot;      // member -> index of its plan in the group tables (or -1)
    std::vector<RingBatchGroup> groups;
    std::vector<CubeBatchGroup> cube_groups; // cube members, by model
    std::vector<sim_t> lattices;     // members stepped by their own kernels (ball, disk, link matrices)
    void *block = nullptr;           // device tables
    long long *budgets = nullptr;    // device: steps left per ring member (budgeted mode)
    std::vector<long long> host_budget; // host shadow, -1 = unlimited
    unsigned **err_ptrs = nullptr;   // device: every member's error word
    unsigned *err_out = nullptr;     // device: OR of the members' error words
    unsigned h_err = 0;              // host copy of err_out
    bool budgeted = false;
    std::map<std::pair<double, int>, cudaGraphExec_t> graphs;
    std::map<std::pair<double, int>, int> uses; // launches per (dt, chunk) before capturing a graph
    // independent branches (one per model group, lattices spread over a few) run
    // concurrently on side streams, forked from and joined to the main stream
    std::vector<cudaStream_t> side;
    cudaEvent_t ev_fork = nullptr;
    std::vector<cudaEvent_t> ev_join;
};

namespace {

__global__ void batch_error_kernel(unsigned *const *errs, int n, unsigned *out)
{
    __shared__ unsigned acc;
    if (threadIdx.x == 0) acc = 0;
    __syncthreads();
    unsigned v = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v |= *errs[i];
    atomicOr(&acc, v);
    __syncthreads();
    if (threadIdx.x == 0) *out = acc;
}

constexpr int kLatticeBranches = 4;

int n_branches(sim_batch_t b)
{
    const int nc = (int)b->lattices.size();
    return (int)(b->groups.size() + b->cube_groups.size()) + (nc < kLatticeBranches ? nc : kLatticeBranches);
}

// n steps of branch k (a ring group, a cube group, or every kLatticeBranches-th
// other lattice) on stream s.
cudaError_t branch_steps(sim_batch_t b, int k, int64_t n, double dt, cudaStream_t s)
{
    const int ng = (int)b->groups.size(), ncg = (int)b->cube_groups.size();
    for (int64_t t = 0; t < n; ++t) {
        if (k < ng) {
            const cudaError_t e = ring_batch_step(b->groups[k], dt, s);
            if (e != cudaSuccess) return e;
        } else if (k < ng + ncg) {
            const cudaError_t e = cube_batch_step(b->cube_groups[k - ng], dt, s);
            if (e != cudaSuccess) return e;
        } else {
            for (size_t c = (size_t)(k - ng - ncg); c < b->lattices.size(); c += kLatticeBranches) {
                const sim_t m = b->lattices[c];
                const cudaError_t e = m->topo == SIM_GRAPH ? graph_step(m->graph, dt, s) : lattice_step(m->lat, dt, s);
                if (e != cudaSuccess) return e;
            }
        }
    }
    return cudaSuccess;
}

cudaError_t batch_launch_steps(sim_batch_t b, int64_t n, double dt, cudaStream_t s)
{
    const int nb = n_branches(b);
    if (nb <= 1) return nb ? branch_steps(b, 0, n, dt, s) : cudaSuccess;
    cudaError_t e = cudaSuccess;
    if (b->side.empty()) {
        b->side.resize(nb, nullptr);
        b->ev_join.resize(nb, nullptr);
        e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
        for (int k = 0; k < nb && e == cudaSuccess; ++k) {
            e = cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return e;
    }
    e = cudaEventRecord(b->ev_fork, s);
    for (int k = 0; k < nb && e == cudaSuccess; ++k) {
        e = cudaStreamWaitEvent(b->side[k], b->ev_fork, 0);
        if (e == cudaSuccess) e = branch_steps(b, k, n, dt, b->side[k]);
        if (e == cudaSuccess) e = cudaEventRecord(b->ev_join[k], b->side[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->ev_join[k], 0);
    }
    return e;
}

// Autotuner key of a batch: its ring members' sub-tile count and member count.
TuneKey batch_tune_key(sim_batch_t b, size_t n_items)
{
    int64_t rings = 0;
    for (int s : b->ring_slot) rings += s >= 0;
    return TuneKey{1, -1, (int64_t)n_items, rings};
}

void clear_batch_graphs(sim_batch_t b)
{
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
    b->uses.clear();
}

int batch_graph(sim_batch_t b, double dt, int chunk, cudaGraphExec_t *out)
{
    auto it = b->graphs.find({dt, chunk});
    if (it != b->graphs.end()) {
        *out = it->second;
        return SIM_OK;
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaSuccess;
    if (!b->cap_stream && (e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(e, "capture stream");
    e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    const cudaError_t le = batch_launch_steps(b, chunk, dt, b->cap_stream);
    e = cudaStreamEndCapture(b->cap_stream, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(le, "kernel launch during capture");
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    b->graphs[{dt, chunk}] = ex;
    *out = ex;
    return SIM_OK;
}

} // namespace

extern "C" {

int sim_batch_create(sim_batch_t *out, const sim_t *members, int n_members, void *stream)
{
    if (!out) return fail(SIM_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_members < 1 || !members) return fail(SIM_EINVAL, "a batch needs at least one member");
    for (int i = 0; i < n_members; ++i) {
        if (!members[i]) return fail(SIM_EINVAL, "NULL member");
        for (int j = 0; j < i; ++j)
            if (members[j] == members[i]) return fail(SIM_EINVAL, "a network appears twice in the batch");
    }
    sim_batch_t b = new sim_batch_handle();
    b->stream = static_cast<cudaStream_t>(stream);
    b->members.assign(members, members + n_members);
    b->ring_slot.assign(n_members, -1);
    b->host_budget.assign(n_members, -1);

    // Group ring members by model; host copies of the device tables.
    std::vector<std::vector<int>> by_model(4), cubes(2); // cubes: Kuramoto, with inertia
    for (int i = 0; i < n_members; ++i) {
        if (members[i]->topo == SIM_RING) by_model[members[i]->model].push_back(i);
        else if (members[i]->topo == SIM_CUBE3D) cubes[members[i]->model == SIM_KSI ? 1 : 0].push_back(i);
        else b->lattices.push_back(members[i]);
    }
    // cube members: one x, y and z launch per stage for each model (tables below)
    std::vector<LatticePlan> cplans;
    std::vector<int> cx_item, cyz_item;
    std::vector<int64_t> cx_base, cyz_base;
    struct CubeSpan { int model, plan0, n, w; int64_t n1_max, x0, nx, yz0, nyz; };
    std::vector<CubeSpan> cspans;
    for (int c = 0; c < 2; ++c) {
        if (cubes[c].empty()) continue;
        CubeSpan cs{c ? 3 : 0, (int)cplans.size(), (int)cubes[c].size(), 0, 0, (int64_t)cx_item.size(), 0,
                    (int64_t)cyz_item.size(), 0};
        for (int i : cubes[c]) cs.n1_max = std::max(cs.n1_max, members[i]->lat.N1);
        cs.w = lattice_row_warps(cs.n1_max);
        for (int k = 0; k < cs.n; ++k) {
            const LatticePlan &lp = members[cubes[c][k]]->lat;
            cplans.push_back(lp);
            cx_base.push_back(cs.nx);
            cyz_base.push_back(cs.nyz);
            const int64_t nx = (lp.N1 * lp.N1 + cs.w - 1) / cs.w, nyz = lattice_order_blocks(SIM_CUBE3D, lp.N1);
            cx_item.insert(cx_item.end(), (size_t)nx, k);
            cyz_item.insert(cyz_item.end(), (size_t)nyz, k);
            cs.nx += nx;
            cs.nyz += nyz;
        }
        cspans.push_back(cs);
    }
    std::vector<RingPlan> plans;
    std::vector<int> inst_of_item;
    std::vector<int64_t> item_base;
    struct GroupSpan { int model, plan0, n; int64_t item0, n_items; };
    std::vector<GroupSpan> spans;
    for (int m = 0; m < 4; ++m) {
        if (by_model[m].empty()) continue;
        GroupSpan gs{m, (int)plans.size(), (int)by_model[m].size(), (int64_t)inst_of_item.size(), 0};
        for (int k = 0; k < (int)by_model[m].size(); ++k) {
            const sim_t h = members[by_model[m][k]];
            b->ring_slot[by_model[m][k]] = (int)plans.size();
            item_base.push_back(gs.n_items);
            for (int64_t t = 0; t < h->ring.nsub; ++t) inst_of_item.push_back(k);
            gs.n_items += h->ring.nsub;
            plans.push_back(h->ring);
            // batched members keep the two-level scan: another member's work
            // hides each end-of-launch scan (the one-pass form measured no
            // faster on the 4096-ring sweep)
            plans.back().flat = 0;
        }
        spans.push_back(gs);
    }
    if (inst_of_item.size() > (size_t)0x7fffffff) {
        delete b;
        return fail(SIM_EINVAL, "batch too large");
    }
    const size_t nplan = plans.size(), nitem = inst_of_item.size();
    size_t o = 0;
    auto take = [&](size_t bytes) { const size_t at = o; o = align_up(o + bytes); return at; };
    const size_t o_plans = take(sizeof(RingPlan) * nplan), o_items = take(sizeof(int) * nitem);
    const size_t o_base = take(sizeof(int64_t) * nplan), o_budget = take(sizeof(long long) * nplan);
    const size_t o_errs = take(sizeof(unsigned *) * n_members), o_eout = take(64);
    const size_t o_cplans = take(sizeof(LatticePlan) * cplans.size());
    const size_t o_cxi = take(sizeof(int) * cx_item.size()), o_cyi = take(sizeof(int) * cyz_item.size());
    const size_t o_cxb = take(sizeof(int64_t) * cx_base.size()), o_cyb = take(sizeof(int64_t) * cyz_base.size());
    // stream-ordered allocation: no device-wide synchronisation when batches are
    // formed and dropped often (the serving loop re-forms them as jobs come and go)
    cudaError_t e = cudaMallocAsync(&b->block, o, b->stream);
    if (e != cudaSuccess) {
        b->block = nullptr;
        sim_batch_destroy(b);
        return e == cudaErrorMemoryAllocation ? fail(SIM_ENOMEM, "batch tables") : cuda_fail(e, "sim_batch_create");
    }
    char *blk = static_cast<char *>(b->block);
    b->budgets = reinterpret_cast<long long *>(blk + o_budget);
    b->err_ptrs = reinterpret_cast<unsigned **>(blk + o_errs);
    b->err_out = reinterpret_cast<unsigned *>(blk + o_eout);
    // plans carry a step-budget pointer; unlimited budgets start at INT64_MAX
    for (size_t k = 0; k < nplan; ++k) plans[k].steps_left = b->budgets + k;
    std::vector<long long> budgets(nplan, (long long)0x7fffffffffffffffLL);
    std::vector<unsigned *> errs(n_members);
    for (int i = 0; i < n_members; ++i) errs[i] = members[i]->err;
    if (nplan) e = cudaMemcpyAsync(blk + o_plans, plans.data(), sizeof(RingPlan) * nplan, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && nitem)
        e = cudaMemcpyAsync(blk + o_items, inst_of_item.data(), sizeof(int) * nitem, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && nplan)
        e = cudaMemcpyAsync(blk + o_base, item_base.data(), sizeof(int64_t) * nplan, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && nplan)
        e = cudaMemcpyAsync(b->budgets, budgets.data(), sizeof(long long) * nplan, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->err_ptrs, errs.data(), sizeof(unsigned *) * n_members, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && !cplans.empty()) {
        e = cudaMemcpyAsync(blk + o_cplans, cplans.data(), sizeof(LatticePlan) * cplans.size(), cudaMemcpyHostToDevice,
                            b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(blk + o_cxi, cx_item.data(), sizeof(int) * cx_item.size(), cudaMemcpyHostToDevice,
                                b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(blk + o_cyi, cyz_item.data(), sizeof(int) * cyz_item.size(), cudaMemcpyHostToDevice,
                                b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(blk + o_cxb, cx_base.data(), sizeof(int64_t) * cx_base.size(), cudaMemcpyHostToDevice,
                                b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(blk + o_cyb, cyz_base.data(), sizeof(int64_t) * cyz_base.size(),
                                cudaMemcpyHostToDevice, b->stream);
    }

    if (e != cudaSuccess) {
        sim_batch_destroy(b);
        return cuda_fail(e, "batch table upload");
    }
    for (const GroupSpan &gs : spans) {
        RingBatchGroup g;
        g.model = gs.model;
        g.n_inst = gs.n;
        g.n_items = gs.n_items;
        g.plans = reinterpret_cast<const RingPlan *>(blk + o_plans) + gs.plan0;
        g.inst_of_item = reinterpret_cast<const int *>(blk + o_items) + gs.item0;
        g.item_base = reinterpret_cast<const int64_t *>(blk + o_base) + gs.plan0;
        g.npt = gs.model == SIM_HH ? 1 : 2;
        TuneVal tv;
        if (gs.model != SIM_HH && tune_lookup(batch_tune_key(b, nitem), &tv)) g.npt = tv.npt == 1 ? 1 : 2;
        b->groups.push_back(g);
    }
    for (const CubeSpan &cs : cspans) {
        CubeBatchGroup g;
        g.model = cs.model;
        g.n_inst = cs.n;
        g.w = cs.w;
        g.n1_max = cs.n1_max;
        g.n_x = cs.nx;
        g.n_yz = cs.nyz;
        g.plans = reinterpret_cast<const LatticePlan *>(blk + o_cplans) + cs.plan0;
        g.x_item = reinterpret_cast<const int *>(blk + o_cxi) + cs.x0;
        g.yz_item = reinterpret_cast<const int *>(blk + o_cyi) + cs.yz0;
        g.x_base = reinterpret_cast<const int64_t *>(blk + o_cxb) + cs.plan0;
        g.yz_base = reinterpret_cast<const int64_t *>(blk + o_cyb) + cs.plan0;
        b->cube_groups.push_back(g);
    }
    *out = b;
    return SIM_OK;
}

int sim_batch_set_budgets(sim_batch_t b, const int64_t *steps)
{
    if (!b || !steps) return fail(SIM_EINVAL, "NULL argument");
    const int n = (int)b->members.size();
    for (int i = 0; i < n; ++i) {
        if (steps[i] < -1) return fail(SIM_EINVAL, "budgets must be >= 0, or -1 for unlimited");
        if (b->members[i]->topo != SIM_RING && steps[i] != -1)
            return fail(SIM_EINVAL, "step budgets apply to ring members only (lattices take -1)");
    }
    std::vector<long long> dev;
    for (int i = 0; i < n; ++i) {
        b->host_budget[i] = steps[i];
        if (b->ring_slot[i] >= 0) {
            if ((int)dev.size() <= b->ring_slot[i]) dev.resize(b->ring_slot[i] + 1);
            dev[b->ring_slot[i]] = steps[i] < 0 ? (long long)0x7fffffffffffffffLL : steps[i];
        }
    }
    if (!dev.empty()) {
        // from pageable memory: the call returns once the values are staged
        const cudaError_t e = cudaMemcpyAsync(b->budgets, dev.data(), sizeof(long long) * dev.size(),
                                              cudaMemcpyHostToDevice, b->stream);
        if (e != cudaSuccess) return cuda_fail(e, "budget upload");
    }
    return SIM_OK;
}

int sim_batch_step(sim_batch_t b, int64_t n_steps, double dt)
{
    if (!b) return fail(SIM_EINVAL, "NULL batch");
    if (n_steps < 0) return fail(SIM_EINVAL, "n_steps must be >= 0");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(SIM_EINVAL, "dt must be finite and > 0");
    if (n_steps > 0)
        for (sim_t h : b->members) {
            if (!ring_flat(h)) continue;
            if (!(h->pfx & 1)) { // the batched kernels read the two-level prefix
                const cudaError_t e = ring_refresh(h, b->stream);
                if (e != cudaSuccess) return cuda_fail(e, "prefix refresh");
            }
            h->pfx = 1;
        }
    int64_t left = n_steps;
    while (left > 0) {
        const int chunk = left >= kGraphChunk ? kGraphChunk : 1;
        // A graph pays off only when reused: the first launches of a (dt, chunk)
        // go out directly (a serving loop re-forms batches often).
        int &uses = b->uses[{dt, chunk}];
        if (uses < 2 && !b->graphs.count({dt, chunk})) {
            ++uses;
            const cudaError_t e = batch_launch_steps(b, chunk, dt, b->stream);
            if (e != cudaSuccess) return cuda_fail(e, "batched launch");
        } else {
            cudaGraphExec_t ex;
            const int st = batch_graph(b, dt, chunk, &ex);
            if (st != SIM_OK) return st;
            const cudaError_t e = cudaGraphLaunch(ex, b->stream);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
        }
        left -= chunk;
    }
    for (size_t i = 0; i < b->members.size(); ++i) {
        long long &bud = b->host_budget[i];
        int64_t done = n_steps;
        if (bud >= 0) {
            done = n_steps < bud ? n_steps : bud;
            bud -= done;
        }
        b->members[i]->steps_done += done;
    }
    return SIM_OK;
}

int sim_batch_sync(sim_batch_t b)
{
    if (!b) return fail(SIM_EINVAL, "NULL batch");
    batch_error_kernel<<<1, 256, 0, b->stream>>>(b->err_ptrs, (int)b->members.size(), b->err_out);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&b->h_err, b->err_out, sizeof(unsigned), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch work failed");
    const unsigned w = b->h_err;
    if (w & ERR_TIMEOUT) return fail(SIM_ETIMEOUT, "a device-side wait exceeded its bound; results are invalid");
    if (w & ERR_RANGE) return fail(SIM_ENONFINITE, "a member's state became non-finite or left the fixed-point range");
    return SIM_OK;
}

void sim_batch_destroy(sim_batch_t b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream); // the batch's graphs may still be running
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    if (b->block) cudaFreeAsync(b->block, b->stream);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (cudaStream_t x : b->side)
        if (x) cudaStreamDestroy(x);
    for (cudaEvent_t x : b->ev_join)
        if (x) cudaEventDestroy(x);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    delete b;
}

void sim_destroy(sim_t h)
{
    if (!h) return;
    if (h->block) cudaStreamSynchronize(h->stream);
    for (auto &kv : h->graphs) cudaGraphExecDestroy(kv.second);
    if (h->dp_block) cudaFree(h->dp_block);
    if (h->graph_block) cudaFree(h->graph_block);
    if (h->edp_block) cudaFree(h->edp_block);
    if (h->block && h->owns_block) cudaFree(h->block);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    delete h;
}

} // extern "C"

// ---------------------------------------------------------------------------
// Adaptive Dormand-Prince 5(4) on rings (kernels in dp5.cu).
static_assert(kDpStatusSteps == SIM_ESTEPS && kDpStatusSmall == SIM_ESMALL, "status codes");

namespace {

constexpr int kDpGraphAttempts = 16; // attempted steps per captured graph
constexpr int kDpMaxOutPerStep = 8;  // the step is capped at this many output intervals

int64_t dp_n_out(double t0, double t_end, double out_dt)
{
    if (!(out_dt > 0.0)) return 0;
    return (int64_t)std::floor((t_end - t0) / out_dt * (1.0 + 1e-12));
}

const char *dp_check(sim_t h, const sim_dp5_opts &o)
{
    const double v[] = {o.t0, o.t_end, o.rtol, o.atol, o.h0, o.h_max, o.out_dt};
    for (double x : v)
        if (!std::isfinite(x)) return "non-finite option";
    if (!(o.t_end > o.t0)) return "t_end must be after t0";
    if (!(o.h0 > 0.0)) return "h0 must be positive";
    if (o.rtol < 0.0 || o.atol < 0.0 || !(o.rtol > 0.0 || o.atol > 0.0)) return "tolerances must be >= 0, not both 0";
    if (o.h_max < 0.0 || o.out_dt < 0.0) return "h_max and out_dt must be >= 0";
    if (o.max_attempts < 1) return "max_attempts must be >= 1";
    return nullptr;
}

int dp_ensure(sim_t h)
{
    if (h->dp_block) return SIM_OK;
    const int64_t n = (int64_t)h->d * h->N, nsub = h->ring.nsub;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += align_up(bytes);
        return o;
    };
    const size_t oy1 = take(sizeof(double) * n);
    size_t ok[7] = {};
    for (int s = 0; s < 7; ++s)
        if (s != 2) ok[s] = take(sizeof(double) * n);
    const size_t oerr = take(sizeof(double) * nsub);
    const size_t oout = take(sizeof(long long) * nsub * kDpMaxOut * 2);
    const size_t octr = take(sizeof(unsigned long long));
    cudaError_t e = cudaMalloc(&h->dp_block, off);
    if (e != cudaSuccess) {
        h->dp_block = nullptr;
        return fail(SIM_ENOMEM, "device allocation of the Dormand-Prince buffers failed");
    }
    char *b = static_cast<char *>(h->dp_block);
    e = cudaMemsetAsync(b + octr, 0, sizeof(unsigned long long), h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "Dormand-Prince set-up");
    DpPlan &Q = h->dp;
    Q.ybuf[0] = h->ring.y;
    Q.ybuf[1] = reinterpret_cast<double *>(b + oy1);
    for (int s = 0; s < 7; ++s) Q.k[s] = s == 2 ? h->ring.acc : reinterpret_cast<double *>(b + ok[s]);
    Q.err_part = reinterpret_cast<double *>(b + oerr);
    Q.out_part = reinterpret_cast<long long *>(b + oout);
    Q.dp_ctr = reinterpret_cast<unsigned long long *>(b + octr);
    Q.ctl = nullptr;       // set per run (the run's control table)
    Q.remaining = nullptr; // set per run
    return SIM_OK;
}

// Buffers of a lattice or link-matrix run: the candidate state, the stage
// input, the seven slopes (k_2 in the network's own accumulator), per-CTA sums.
int edp_ensure(sim_t h)
{
    if (h->edp_block) return SIM_OK;
    const int64_t n = (int64_t)h->d * h->nodes, nblk = (h->nodes + 255) / 256;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += align_up(bytes);
        return o;
    };
    const size_t oy5 = take(sizeof(double) * n), ox = take(sizeof(double) * n);
    size_t ok[8] = {};
    for (int j = 1; j <= 7; ++j)
        if (j != 2) ok[j] = take(sizeof(double) * n);
    const size_t oerr = take(sizeof(double) * nblk);
    const size_t oout = take(sizeof(i128) * nblk * kDpMaxOut * 2);
    const size_t octr = take(sizeof(unsigned long long));
    cudaError_t e = cudaMalloc(&h->edp_block, off);
    if (e != cudaSuccess) {
        h->edp_block = nullptr;
        return fail(SIM_ENOMEM, "device allocation of the Dormand-Prince buffers failed");
    }
    char *b = static_cast<char *>(h->edp_block);
    e = cudaMemsetAsync(b + octr, 0, sizeof(unsigned long long), h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "Dormand-Prince set-up");
    const bool lat = h->topo != SIM_GRAPH;
    ElemDpPlan &Q = h->edp;
    Q.model = h->model;
    Q.nodes = h->nodes;
    Q.nblk = nblk;
    Q.y = lat ? h->lat.y : h->ring.y;
    Q.y5 = reinterpret_cast<double *>(b + oy5);
    Q.xbuf = reinterpret_cast<double *>(b + ox);
    Q.k[0] = nullptr;
    for (int j = 1; j <= 7; ++j)
        Q.k[j] = j == 2 ? (lat ? h->lat.acc : h->ring.acc) : reinterpret_cast<double *>(b + ok[j]);
    Q.err_part = reinterpret_cast<double *>(b + oerr);
    Q.out_part = reinterpret_cast<i128 *>(b + oout);
    Q.dp_ctr = reinterpret_cast<unsigned long long *>(b + octr);
    Q.f = lat ? h->lat.f : nullptr;
    Q.tab = lat ? h->lat.mp.tab : h->ring.mp.tab;
    Q.F = lat ? h->lat.F : h->ring.F;
    Q.obs = h->obs;
    Q.obs_cap = kObsCap;
    Q.obs_ctr = h->obs_ctr;
    Q.err = h->err;
    return SIM_OK;
}

// Integrate every member from its opts.t0 to opts.t_end on stream s.  Returns a
// machinery or device status; per-member outcomes are in stats.
int dp_run(const std::vector<sim_t> &mem, const sim_dp5_opts *opts, sim_dp5_stats *stats, cudaStream_t s)
{
    const int n = (int)mem.size();
    for (int i = 0; i < n; ++i)
        if (const char *why = dp_check(mem[i], opts[i])) return fail(SIM_EINVAL, why);
    for (int i = 0; i < n; ++i) {
        if (mem[i]->topo != SIM_RING) {
            const int st = edp_ensure(mem[i]);
            if (st != SIM_OK) return st;
            continue;
        }
        const int st = dp_ensure(mem[i]);
        if (st != SIM_OK) return st;
        mem[i]->dp.r = mem[i]->ring; // picks up a node parameter set since the last run
        mem[i]->dp.r.steps_left = nullptr;
    }
    // Step control of every member, and the first attempt.
    std::vector<DpCtl> ctl(n);
    int remaining = 0;
    for (int i = 0; i < n; ++i) {
        const sim_dp5_opts &o = opts[i];
        DpCtl c{};
        c.t = o.t0;
        c.t_end = o.t_end;
        c.t0 = o.t0;
        c.out_dt = o.out_dt;
        c.rtol = o.rtol;
        c.atol = o.atol;
        c.hcap = o.h_max > 0.0 ? o.h_max : INFINITY;
        if (o.out_dt > 0.0 && kDpMaxOutPerStep * o.out_dt < c.hcap) c.hcap = kDpMaxOutPerStep * o.out_dt;
        c.h = o.h0 < c.hcap ? o.h0 : c.hcap;
        c.max_att = o.max_attempts;
        c.n_out = dp_n_out(o.t0, o.t_end, o.out_dt);
        c.next_out = 1;
        c.last = o.t_end - c.t <= c.h;
        c.h_att = c.last ? o.t_end - c.t : c.h;
        if (!(c.h_att > 1e-14 * (std::fabs(c.t) + c.h_att))) {
            c.done = 1;
            c.status = SIM_ESMALL;
        }
        remaining += c.done ? 0 : 1;
        ctl[i] = c;
    }
    // Device tables of the run: plans, work items per model group, control
    // words, the members' error words and the counter of unfinished members.
    std::vector<std::vector<int>> by_model(4);
    std::vector<int> lat_members;
    for (int i = 0; i < n; ++i) {
        if (mem[i]->topo == SIM_RING) by_model[mem[i]->model].push_back(i);
        else lat_members.push_back(i);
    }
    std::vector<DpPlan> plans;
    std::vector<int> inst_of_item, plan_member;
    std::vector<int64_t> item_base;
    struct Span { int model, first_plan, n_inst; int64_t first_item, n_items; };
    std::vector<Span> spans;
    for (int m = 0; m < 4; ++m) {
        if (by_model[m].empty()) continue;
        Span sp{m, (int)plans.size(), (int)by_model[m].size(), (int64_t)inst_of_item.size(), 0};
        for (int k = 0; k < sp.n_inst; ++k) {
            const sim_t h = mem[by_model[m][k]];
            plans.push_back(h->dp);
            plan_member.push_back(by_model[m][k]);
            item_base.push_back(sp.n_items);
            for (int64_t t = 0; t < h->ring.nsub; ++t) inst_of_item.push_back(k);
            sp.n_items += h->ring.nsub;
        }
        spans.push_back(sp);
    }
    std::vector<unsigned *> errs(n);
    for (int i = 0; i < n; ++i) errs[i] = mem[i]->err;
    const size_t o_plans = 0, o_items = align_up(sizeof(DpPlan) * plans.size());
    const size_t o_base = o_items + align_up(sizeof(int) * inst_of_item.size());
    const size_t o_ctl = o_base + align_up(sizeof(int64_t) * item_base.size());
    const size_t o_errs = o_ctl + align_up(sizeof(DpCtl) * n);
    const size_t o_rem = o_errs + align_up(sizeof(unsigned *) * n);
    const size_t o_eout = o_rem + align_up(sizeof(int));
    const size_t total = o_eout + align_up(sizeof(unsigned));
    void *tab = nullptr;
    cudaError_t e = cudaMalloc(&tab, total);
    if (e != cudaSuccess) return fail(SIM_ENOMEM, "device allocation of the run tables failed");
    char *tb = static_cast<char *>(tab);
    int *d_rem = reinterpret_cast<int *>(tb + o_rem);
    DpCtl *d_ctl = reinterpret_cast<DpCtl *>(tb + o_ctl);
    unsigned *d_eout = reinterpret_cast<unsigned *>(tb + o_eout);
    for (size_t q = 0; q < plans.size(); ++q) {
        plans[q].remaining = d_rem;
        plans[q].ctl = d_ctl + plan_member[q];
    }
    // lattices and link matrices: elementwise stage kernels around the network's
    // own right-hand side, evaluated from the stage-input buffer
    std::vector<LatDpPlan> lplans;
    std::vector<GraphDpPlan> gplans;
    std::vector<int> lat_idx, graph_idx;
    for (int i : lat_members) {
        ElemDpPlan e = mem[i]->edp;
        e.ctl = d_ctl + i;
        e.remaining = d_rem;
        if (mem[i]->topo == SIM_GRAPH) {
            GraphDpPlan q{e, mem[i]->graph};
            q.rhs.r.y = e.xbuf;
            q.rhs.r.obs = nullptr;
            q.rhs.r.skip = &(d_ctl + i)->done;
            q.rhs.r.err = reinterpret_cast<unsigned *>(&(d_ctl + i)->bad); // out of range: reject
            gplans.push_back(q);
            graph_idx.push_back(i);
        } else {
            LatDpPlan q{e, mem[i]->lat};
            q.rhs.y = e.xbuf;
            q.rhs.skip = &(d_ctl + i)->done;
            lplans.push_back(q);
            lat_idx.push_back(i);
        }
    }
    std::vector<DpGroup> groups;
    for (const Span &sp : spans)
        groups.push_back(DpGroup{sp.model, sp.n_inst, sp.n_items,
                                 reinterpret_cast<const DpPlan *>(tb + o_plans) + sp.first_plan,
                                 reinterpret_cast<const int *>(tb + o_items) + sp.first_item,
                                 reinterpret_cast<const int64_t *>(tb + o_base) + sp.first_plan});
    cudaGraphExec_t ex = nullptr;
    cudaStream_t cap = nullptr;
    int status = SIM_OK;
    auto finish = [&](int st) {
        for (sim_t h : mem)
            if (h->topo == SIM_RING) h->pfx = 1; // the run leaves the two-level prefix of f(y)
        if (ex) cudaGraphExecDestroy(ex);
        cudaStreamSynchronize(s);
        if (cap) cudaStreamDestroy(cap);
        cudaFree(tab);
        return st;
    };
    e = cudaMemcpyAsync(tb + o_plans, plans.data(), sizeof(DpPlan) * plans.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(tb + o_items, inst_of_item.data(), sizeof(int) * inst_of_item.size(),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(tb + o_base, item_base.data(), sizeof(int64_t) * item_base.size(),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_ctl, ctl.data(), sizeof(DpCtl) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(tb + o_errs, errs.data(), sizeof(unsigned *) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_rem, &remaining, sizeof(int), cudaMemcpyHostToDevice, s);
    // prefix of f(y_n) and R(t0) of every member, then the first right-hand side
    for (int ds : {8, 1})
        for (const DpGroup &g : groups)
            if (e == cudaSuccess) e = dp_launch(ds, g, s);
    for (size_t q = 0; q < lplans.size() && e == cudaSuccess; ++q) {
        e = lattice_prologue(mem[lat_idx[q]]->lat, s);
        if (e == cudaSuccess) e = lat_dp_start(lplans[q], s);
    }
    for (size_t q = 0; q < gplans.size() && e == cudaSuccess; ++q) {
        e = ring_prologue(mem[graph_idx[q]]->ring, s); // R(t0)
        if (e == cudaSuccess) e = graph_dp_start(gplans[q], s);
    }
    if (e != cudaSuccess) return finish(cuda_fail(e, "Dormand-Prince start"));
    // Attempts in captured graphs until every member is done.
    if (remaining > 0) {
        e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return finish(cuda_fail(e, "Dormand-Prince capture"));
        cudaError_t le = cudaSuccess;
        for (int a = 0; a < kDpGraphAttempts && le == cudaSuccess; ++a) {
            for (int ds : {2, 3, 4, 5, 6, 7, 0})
                for (const DpGroup &g : groups)
                    if (le == cudaSuccess) le = dp_launch(ds, g, cap);
            for (const LatDpPlan &q : lplans)
                if (le == cudaSuccess) le = lat_dp_attempt(q, cap);
            for (const GraphDpPlan &q : gplans)
                if (le == cudaSuccess) le = graph_dp_attempt(q, cap);
        }
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(cap, &graph);
        if (le != cudaSuccess || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return finish(cuda_fail(le != cudaSuccess ? le : e, "Dormand-Prince capture"));
        }
        e = cudaGraphInstantiate(&ex, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return finish(cuda_fail(e, "cudaGraphInstantiate"));
        long long max_att = 0;
        for (int i = 0; i < n; ++i) max_att = opts[i].max_attempts > max_att ? opts[i].max_attempts : max_att;
        const long long max_replays = max_att / kDpGraphAttempts + 2;
        int h_rem = remaining;
        for (long long r = 0; r < max_replays && h_rem > 0; ++r) {
            e = cudaGraphLaunch(ex, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(&h_rem, d_rem, sizeof(int), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return finish(cuda_fail(e, "Dormand-Prince attempts"));
        }
        if (h_rem > 0) status = fail(SIM_EDEVICE, "Dormand-Prince run did not finish within its attempt budget");
    }
    // State back in the handles' buffers with the prefix of f(y) for the RK4
    // path, the control words and the OR of the members' error words.
    for (const DpGroup &g : groups)
        if (e == cudaSuccess) e = dp_launch(9, g, s);
    for (int i : lat_idx) { // (sin, cos) of y and a cube's x sums of y for the RK4 kernels, without recording R
        LatticePlan quiet = mem[i]->lat;
        quiet.obs = nullptr;
        if (e == cudaSuccess) e = lattice_prologue(quiet, s);
    }
    for (int i : graph_idx) { // the prefix of f(y) for the RK4 kernels, without recording R
        RingPlan quiet = mem[i]->ring;
        quiet.obs = nullptr;
        if (e == cudaSuccess) e = ring_prologue(quiet, s);
    }
    if (e == cudaSuccess) {
        batch_error_kernel<<<1, 256, 0, s>>>(reinterpret_cast<unsigned *const *>(tb + o_errs), n, d_eout);
        e = cudaGetLastError();
    }
    unsigned h_eout = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctl.data(), d_ctl, sizeof(DpCtl) * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_eout, d_eout, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return finish(cuda_fail(e, "Dormand-Prince results"));
    for (int i = 0; i < n && stats; ++i) {
        stats[i].accepted = ctl[i].n_acc;
        stats[i].rejected = ctl[i].n_rej;
        stats[i].t = ctl[i].t;
        stats[i].h_next = ctl[i].h;
        stats[i].status = ctl[i].status;
    }
    status = finish(status);
    if (status == SIM_OK && (h_eout & ERR_TIMEOUT))
        status = fail(SIM_ETIMEOUT, "a device-side wait exceeded its bound; results are invalid");
    if (status == SIM_OK && (h_eout & ERR_RANGE))
        status = fail(SIM_ENONFINITE, "the state became non-finite or left the fixed-point range");
    return status;
}

} // namespace

extern "C" {

int sim_dp5(sim_t h, const sim_dp5_opts *opts, sim_dp5_stats *stats)
{
    if (!h || !opts) return fail(SIM_EINVAL, "NULL argument");
    sim_dp5_stats st{};
    const int r = dp_run({h}, opts, &st, h->stream);
    if (stats) *stats = st;
    if (r != SIM_OK) return r;
    if (st.status == SIM_ESTEPS) return fail(SIM_ESTEPS, "the attempt budget ran out before t_end");
    if (st.status == SIM_ESMALL) return fail(SIM_ESMALL, "the step size fell below the resolution of t");
    return SIM_OK;
}

int sim_batch_dp5(sim_batch_t b, const sim_dp5_opts *opts, sim_dp5_stats *stats)
{
    if (!b || !opts) return fail(SIM_EINVAL, "NULL argument");
    return dp_run(b->members, opts, stats, b->stream);
}

} // extern "C"


// ----------------------------------------------------------------------------- autotuner
namespace {

void clear_graphs(sim_t h)
{
    for (auto &kv : h->graphs) cudaGraphExecDestroy(kv.second);
    h->graphs.clear();
}

// Recompute the prefix buffers of f(y) of any member without recording R.
cudaError_t quiet_prologue(sim_t h, cudaStream_t s)
{
    if (h->topo == SIM_RING) return ring_refresh(h, s);
    if (ring_like(h)) {
        RingPlan quiet = h->ring;
        quiet.obs = nullptr;
        return ring_prologue(quiet, s);
    }
    LatticePlan quiet = h->lat;
    quiet.obs = nullptr;
    return lattice_prologue(quiet, s);
}

double *state_of(sim_t h) { return ring_like(h) ? h->ring.y : h->lat.y; }

// Device time of `launches` launches of a captured graph after one warm-up launch.
cudaError_t time_graph(cudaGraphExec_t ex, int64_t launches, cudaStream_t s, float *ms)
{
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e == cudaSuccess) e = cudaGraphLaunch(ex, s);
    if (e == cudaSuccess) e = cudaEventRecord(a, s);
    for (int64_t k = 0; k < launches && e == cudaSuccess; ++k) e = cudaGraphLaunch(ex, s);
    if (e == cudaSuccess) e = cudaEventRecord(b, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    return e;
}

} // namespace

extern "C" {

int sim_autotune(sim_t h, double dt, int64_t trial_steps, int *npt_out, int *flat_out)
{
    if (!h) return fail(SIM_EINVAL, "NULL handle");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(SIM_EINVAL, "dt must be finite and > 0");
    if (trial_steps < 1) return fail(SIM_EINVAL, "trial_steps must be >= 1");
    auto report = [&] {
        if (npt_out) *npt_out = h->topo == SIM_RING ? h->ring.npt : 0;
        if (flat_out) *flat_out = h->topo == SIM_RING ? h->ring.flat : 0;
        return SIM_OK;
    };
    // only the stage kernels of rings have variants (HH: one node per thread)
    if (h->topo != SIM_RING || use_cluster(h)) return report();
    const bool flat_ok = ring_flat_eligible(h->model, h->ring.ngroups);
    std::vector<TuneVal> cand;
    for (int npt : {2, 1}) {
        if (npt == 2 && h->model == SIM_HH) continue;
        if (flat_ok) cand.push_back({npt, 1});
        cand.push_back({npt, 0});
    }
    if (cand.size() < 2) return report();
    const size_t ybytes = sizeof(double) * h->d * h->nodes;
    void *save = nullptr;
    cudaError_t e = cudaMallocAsync(&save, ybytes, h->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SIM_ENOMEM, "autotune: no room for a copy of the state");
    }
    e = cudaMemcpyAsync(save, h->ring.y, ybytes, cudaMemcpyDeviceToDevice, h->stream);
    const int chunk = trial_steps >= kGraphChunk ? kGraphChunk : 1;
    const int64_t launches = (trial_steps + chunk - 1) / chunk;
    float best = 0.0f;
    TuneVal pick = cand[0];
    int st = SIM_OK;
    for (size_t c = 0; c < cand.size() && e == cudaSuccess && st == SIM_OK; ++c) {
        h->ring.npt = cand[c].npt;
        h->ring.flat = cand[c].flat;
        clear_graphs(h);
        e = cudaMemcpyAsync(h->ring.y, save, ybytes, cudaMemcpyDeviceToDevice, h->stream);
        if (e == cudaSuccess) e = ring_refresh(h, h->stream);
        cudaGraphExec_t ex = nullptr;
        if (e == cudaSuccess) st = get_graph(h, dt, chunk, &ex);
        float ms = 0.0f;
        if (e == cudaSuccess && st == SIM_OK) e = time_graph(ex, launches, h->stream, &ms);
        if (e == cudaSuccess && st == SIM_OK && (c == 0 || ms < best)) {
            best = ms;
            pick = cand[c];
        }
    }
    h->ring.npt = pick.npt;
    h->ring.flat = pick.flat;
    clear_graphs(h);
    // the state as it was; prefix buffers, counters and R(t0) as after sim_set_state
    const cudaError_t e2 = cudaMemcpyAsync(h->ring.y, save, ybytes, cudaMemcpyDeviceToDevice, h->stream);
    cudaFreeAsync(save, h->stream);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return cuda_fail(e, "autotune");
    if (st != SIM_OK) return st;
    const int r = prologue(h);
    if (r != SIM_OK) return r;
    tune_store(TuneKey{0, h->model, h->N, h->R}, pick);
    return report();
}

int sim_tune_info(sim_t h, int *npt, int *flat)
{
    if (!h || !npt || !flat) return fail(SIM_EINVAL, "NULL argument");
    *npt = h->topo == SIM_RING ? h->ring.npt : 0;
    *flat = h->topo == SIM_RING ? h->ring.flat : 0;
    return SIM_OK;
}

int sim_batch_autotune(sim_batch_t b, double dt, int64_t trial_steps, int *npt_out)
{
    if (!b) return fail(SIM_EINVAL, "NULL batch");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(SIM_EINVAL, "dt must be finite and > 0");
    if (trial_steps < 1) return fail(SIM_EINVAL, "trial_steps must be >= 1");
    bool variants = false;
    size_t n_items = 0;
    for (const RingBatchGroup &g : b->groups) {
        variants = variants || g.model != SIM_HH;
        n_items += (size_t)g.n_items;
    }
    auto report = [&] {
        int v = 1;
        for (const RingBatchGroup &g : b->groups)
            if (g.model != SIM_HH) v = g.npt;
        if (npt_out) *npt_out = v;
        return SIM_OK;
    };
    if (!variants) return report();
    cudaStream_t s = b->stream;
    const int n = (int)b->members.size();
    // everything the trial steps change: states, error words, order-parameter
    // counters and step budgets
    std::vector<size_t> at(n + 1, 0);
    for (int i = 0; i < n; ++i)
        at[i + 1] = at[i] + align_up(sizeof(double) * b->members[i]->d * b->members[i]->nodes);
    size_t nplan = 0;
    for (const RingBatchGroup &g : b->groups) nplan += (size_t)g.n_inst;
    const size_t o_err = at[n], o_ctr = align_up(o_err + sizeof(unsigned) * n);
    const size_t o_bud = align_up(o_ctr + sizeof(unsigned long long) * n);
    const size_t total = o_bud + sizeof(long long) * nplan;
    char *save = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&save), total, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SIM_ENOMEM, "autotune: no room for a copy of the members' states");
    }
    auto copy_all = [&](bool to_save) {
        cudaError_t r = cudaSuccess;
        for (int i = 0; i < n && r == cudaSuccess; ++i) {
            sim_t h = b->members[i];
            const size_t yb = sizeof(double) * h->d * h->nodes;
            double *y = state_of(h);
            r = to_save ? cudaMemcpyAsync(save + at[i], y, yb, cudaMemcpyDeviceToDevice, s)
                        : cudaMemcpyAsync(y, save + at[i], yb, cudaMemcpyDeviceToDevice, s);
            if (r == cudaSuccess)
                r = to_save ? cudaMemcpyAsync(save + o_err + sizeof(unsigned) * i, h->err, sizeof(unsigned),
                                              cudaMemcpyDeviceToDevice, s)
                            : cudaMemcpyAsync(h->err, save + o_err + sizeof(unsigned) * i, sizeof(unsigned),
                                              cudaMemcpyDeviceToDevice, s);
            if (r == cudaSuccess)
                r = to_save ? cudaMemcpyAsync(save + o_ctr + 8 * i, h->obs_ctr, 8, cudaMemcpyDeviceToDevice, s)
                            : cudaMemcpyAsync(h->obs_ctr, save + o_ctr + 8 * i, 8, cudaMemcpyDeviceToDevice, s);
        }
        if (r == cudaSuccess && nplan)
            r = to_save ? cudaMemcpyAsync(save + o_bud, b->budgets, sizeof(long long) * nplan, cudaMemcpyDeviceToDevice, s)
                        : cudaMemcpyAsync(b->budgets, save + o_bud, sizeof(long long) * nplan, cudaMemcpyDeviceToDevice, s);
        for (int i = 0; i < n && r == cudaSuccess; ++i)
            if (!to_save) r = quiet_prologue(b->members[i], s);
        return r;
    };
    e = copy_all(true);
    float best = 0.0f;
    int pick = 2;
    const int cands[2] = {2, 1};
    for (int c = 0; c < 2 && e == cudaSuccess; ++c) {
        for (RingBatchGroup &g : b->groups)
            if (g.model != SIM_HH) g.npt = cands[c];
        clear_batch_graphs(b);
        e = copy_all(false);
        cudaEvent_t ea = nullptr, eb = nullptr;
        if (e == cudaSuccess) e = cudaEventCreate(&ea);
        if (e == cudaSuccess) e = cudaEventCreate(&eb);
        if (e == cudaSuccess) e = batch_launch_steps(b, 1, dt, s); // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(ea, s);
        if (e == cudaSuccess) e = batch_launch_steps(b, trial_steps, dt, s);
        if (e == cudaSuccess) e = cudaEventRecord(eb, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(eb);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ea, eb);
        if (ea) cudaEventDestroy(ea);
        if (eb) cudaEventDestroy(eb);
        if (e == cudaSuccess && (c == 0 || ms < best)) {
            best = ms;
            pick = cands[c];
        }
    }
    for (RingBatchGroup &g : b->groups)
        if (g.model != SIM_HH) g.npt = pick;
    clear_batch_graphs(b);
    const cudaError_t e2 = copy_all(false);
    cudaFreeAsync(save, s);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "batch autotune");
    tune_store(batch_tune_key(b, n_items), TuneVal{pick, 0});
    return report();
}

int sim_tune_save(const char *path)
{
    if (!path) return fail(SIM_EINVAL, "NULL path");
    FILE *f = std::fopen(path, "w");
    if (!f) return fail(SIM_EINVAL, std::string("cannot write ") + path);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    std::fprintf(f, "# kind model a b npt flat\n");
    for (const auto &kv : g_tune)
        std::fprintf(f, "%d %d %lld %lld %d %d\n", kv.first.kind, kv.first.model, (long long)kv.first.a,
                     (long long)kv.first.b, kv.second.npt, kv.second.flat);
    const bool ok = std::fclose(f) == 0;
    return ok ? SIM_OK : fail(SIM_EINVAL, std::string("cannot write ") + path);
}

int sim_tune_load(const char *path)
{
    if (!path) return fail(SIM_EINVAL, "NULL path");
    FILE *f = std::fopen(path, "r");
    if (!f) return fail(SIM_EINVAL, std::string("cannot read ") + path);
    char line[256];
    int st = SIM_OK;
    std::map<TuneKey, TuneVal> read;
    while (std::fgets(line, sizeof line, f)) {
        if (line[0] == '#' || line[0] == '\n') continue;
        int kind, model, npt, flat;
        long long a, bb;
        if (std::sscanf(line, "%d %d %lld %lld %d %d", &kind, &model, &a, &bb, &npt, &flat) != 6 ||
            (kind != 0 && kind != 1) || (npt != 1 && npt != 2) || (flat != 0 && flat != 1)) {
            st = fail(SIM_EINVAL, std::string("malformed line in ") + path);
            break;
        }
        read[TuneKey{kind, model, a, bb}] = TuneVal{npt, flat};
    }
    std::fclose(f);
    if (st != SIM_OK) return st;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (const auto &kv : read) g_tune[kv.first] = kv.second;
    return SIM_OK;
}

int sim_tune_clear(void)
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune.clear();
    return SIM_OK;
}

} // extern "C"
