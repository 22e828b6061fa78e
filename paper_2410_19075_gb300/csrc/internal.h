// Internal declarations shared by the translation units of libsim (not part of
// the public C ABI in include/sim.h).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"
#include "models.cuh"

namespace simk {

constexpr int kRingThreads = 256;       // threads per CTA, one node each
constexpr int kSubTile = 256;           // nodes per CTA = exact-prefix sub-tile
constexpr int kSubLog2 = 8;
constexpr int kGroup = 64;              // sub-tiles per prefix group
constexpr int kGroupLog2 = 6;

// RK4 step size and the multiples the stage updates use, computed once on the
// host (IEEE division: the same bits as on the device), so that no thread
// divides.
struct StepSize {
    double dt, half, sixth; // dt, dt / 2, dt / 6
};
inline StepSize step_size(double dt) { return StepSize{dt, 0.5 * dt, dt / 6.0}; }

// Device buffers and sizes of one ring network (plain path).
struct RingPlan {
    int model;
    int64_t N, R;
    int64_t nsub;    // ceil(N / kSubTile) = CTAs per stage launch
    int64_t ngroups; // ceil(nsub / kGroup)
    int F, lim;    // fixed-point grid 2^-F, range |f| < 2^lim
    ModelParams mp;
    double *y;          // D * N, the state y_n
    double *acc;        // D * N, RK4 accumulator k1 + 2 k2 + 2 k3
    double *xg[2];      // NX * N each, local stage-input variables (HH gates)
    const double *node_param; // N (HH I_ext) or nullptr
    int64_t *lam[2];    // NQ * N each: inclusive prefix of Q(f) inside each sub-tile
    i128 *ingrp[2];     // NQ * nsub each: exclusive prefix of each sub-tile inside its group
    i128 *grpofs[2];    // NQ * (ngroups + 1) each: exclusive prefix at group starts, then the total
    int64_t *subtot;    // NQ * nsub: sub-tile totals (scratch of the launch)
    i128 *grptot;       // NQ * ngroups: group totals (scratch of the launch)
    unsigned long long *grp_ctr; // ngroups arrival counters
    unsigned long long *top_ctr; // arrival counter of the groups
    unsigned *err;
    double *obs;        // order-parameter ring buffer
    int64_t obs_cap;
    unsigned long long *obs_ctr;
    long long *steps_left; // batched runs with a step budget: steps still to do (else nullptr)
    const int *skip;       // if set and nonzero, the plain and link-matrix stage kernels return at
                           // once (a finished Dormand-Prince run); nullptr for every other use
    // One-pass prefix of the RK4 stage kernels (flat = 1; rings of at most
    // kFlatMaxGroups groups): each CTA stores its sub-tile total t and adds it
    // into its group's accumulator as four chunks (bits 0-17, 18-35, 36-53
    // unsigned, and t >> 54 signed) in 32-bit words, exact because no sum of
    // chunks over at most 8192 sub-tiles reaches 2^31; the next kernel's CTAs
    // sum those themselves, so no CTA waits for the last one of its launch.
    int flat;             // plain stage kernels only (batched members keep the two-level scan)
    int npt;              // nodes per thread of the stage kernels: 2 (128 threads per sub-tile;
                          // not HH) or 1 (256); set by sim_create and the autotuner
    int64_t *fsub[2];     // NQ * nsub each: sub-tile totals (same parity as lam)
    unsigned *facc[4];    // NQ * ngroups * 4 each: group accumulators of stage slot s & 3
    unsigned long long *flat_ctr; // arrival counter of the one-pass kernels that record or count steps
};

constexpr int kFlatMaxGroups = 128; // lanes sum four groups each; 8192 sub-tiles keep chunk sums below 2^31

// Ring members of one model in a batch: device tables of the batched launch.
struct RingBatchGroup {
    int model;
    int n_inst;
    int64_t n_items;        // sum of the members' sub-tile counts = CTAs per launch
    const RingPlan *plans;  // n_inst plans (device)
    const int *inst_of_item; // n_items (device)
    const int64_t *item_base; // n_inst: first item of each member (device)
    int npt;                  // nodes per thread of the batched stage kernels (1, or 2 if not HH)
};

// Batched ring stage kernels: one RK4 step of every member of the group.
cudaError_t ring_batch_step(const RingBatchGroup &g, double dt, cudaStream_t s);

// General link matrix in the compressed form of Algorithm 2 (graph.cu): the ring
// buffers (exact prefix in node order, states, observables) plus the tables.
struct GraphPlan {
    RingPlan r;            // r.R is unused; r.mp carries K = 1 and include_self = 1
    const int2 *runs;      // the common vector V as runs (first offset, length), first + length <= N
    int nruns;
    const int *ent;        // N: difference-table entry of every node
    const int64_t *dptr;   // entries + 1: start of every entry in dpos
    const int2 *dpos;      // (offset p, sign): -1 where p is in V (the bit is cleared), +1 elsewhere
    const int64_t *ek;     // per entry: the link count K = |V| + sum of its signs
    const double *ecs;     // per entry: 1 / K (0 for a node without links)
};
cudaError_t graph_rhs(const GraphPlan &g, cudaStream_t s);             // acc <- f(y), stage 1 with dt = 0
cudaError_t graph_step(const GraphPlan &g, double dt, cudaStream_t s); // one RK4 step

// Adaptive Dormand-Prince 5(4) on rings (dp5.cu), per instance in a batch.
constexpr int kDpMaxOut = 16; // dense outputs handled inside one step (the step is capped at 8 of them)
constexpr int kDpStatusSteps = -7, kDpStatusSmall = -8; // = SIM_ESTEPS, SIM_ESMALL

// Step control of one instance (device memory; written by the host before a
// run and by the deciding CTA of every attempt).
struct DpCtl {
    double t, t_end, t0, out_dt;
    double h;      // proposed step
    double h_att;  // step of the current attempt (h, or t_end - t for the last one)
    double hcap;   // largest step: h_max and 8 out_dt
    double rtol, atol;
    long long n_acc, n_rej, max_att, n_out, next_out;
    int last;      // the current attempt ends at t_end
    int last_rej;  // the previous attempt was rejected
    int cur;       // which of the two state / first-stage buffers holds y_n, k_1
    int done;      // 1: finished (t_end reached or status set)
    int status;    // 0, or the sim_status that ended the run
    int bad;       // a stage input of the current attempt left the fixed-point range
    int acc_flag;  // the last decided attempt was accepted
};

struct DpPlan {
    RingPlan r;              // prefix buffers, local-variable buffers, observables; r.y = ybuf[0]
    double *ybuf[2];         // D * N each: y_n and the candidate y_{n+1}
    double *k[7];            // D * N each: k[0], k[1] first-same-as-last pair, k[2..6] stages 2..6
    DpCtl *ctl;
    double *err_part;        // nsub: per-sub-tile sums of (e / sc)^2
    long long *out_part;     // nsub * kDpMaxOut * 2: per-sub-tile fixed-point sums of the dense sin, cos
    unsigned long long *dp_ctr; // arrival counter of the decision
    int *remaining;          // instances of the run not done yet (shared by the run)
};

struct DpGroup {
    int model;
    int n_inst;
    int64_t n_items;
    const DpPlan *plans;
    const int *inst_of_item;
    const int64_t *item_base;
};

// Kernel ds for every instance of the group: 8 = run start (prefix of f(y_n),
// R(t0)); 1 = first right-hand side of a run and the input of stage 2;
// 2..6 = stages 2..6; 7 = stage 7, the error norm, dense output and the
// decision; 0 = the input of stage 2 of the next attempt; 9 = run end (state
// back in the first buffer, prefix of f(y) for the RK4 kernels).
cudaError_t dp_launch(int ds, const DpGroup &g, cudaStream_t s);

// Ring: f(y) -> lam[0], ofs[0] and the order parameter of y (Kuramoto).
cudaError_t ring_prologue(const RingPlan &p, cudaStream_t s);
// Small rings (N <= kClusterMaxNodes): all stages of n_steps RK4 steps in one
// thread-block-cluster launch (ring_cluster.cu).  Same results as ring_step.
constexpr int64_t kClusterMaxNodes = 4096;
cudaError_t ring_cluster_configure(); // per device, before the first cluster launch
int cluster_size_for(int64_t N);      // CTAs of the cluster for a ring of N nodes (0: not eligible)
cudaError_t ring_cluster_steps(const RingPlan &p, double dt, int64_t n_steps, cudaStream_t s);

// Ring: stage 1 only with dt = 0, so acc receives f(y) and y is untouched.
cudaError_t ring_rhs(const RingPlan &p, cudaStream_t s);
// Ring: one RK4 step, 4 fused stage kernels.
cudaError_t ring_step(const RingPlan &p, double dt, cudaStream_t s);

// Device buffers of one periodic lattice (cube, ball or disk; Kuramoto models 0
// and 3).  topo: 1 cube, 2 ball, 3 disk.
struct LatticePlan {
    int model, topo, dims;
    int64_t N1, P, nodes;
    int F;            // fixed-point grid of the window sums
    // ball, disk: the x pass rotates every node's (sin, cos) by -alpha =
    // -(rot_q pi/2 + alpha0), alpha0 in [0, pi/2): rot_c, rot_s = cos alpha0,
    // sin alpha0 on the grid 2^-63 (lattice_rotated_q)
    uint64_t rot_c, rot_s;
    int rot_q;
    ModelParams mp;
    double *y, *acc;  // D * nodes
    int64_t *f;       // nodes (sin, cos) pairs (f[2n], f[2n+1]) of the current stage-input phase on the grid 2^-62
    double *xs;       // NX * nodes: local stage-input variables (psi of model 3)
    int64_t *sx;      // cube: 2 * nodes window sums along x (SoA); ball, disk: per row,
                      // rs (sin, cos) pairs of the periodically extended inclusive
                      // prefix E(x), x in [-P-1, N1+P-1], stored at x + P + 1
    int64_t rs;       // ball, disk: row stride of sx in (sin, cos) pairs, N1 + 2P + 1
    int wmode;        // ball, disk: sx holds, for w = 0..P, nodes (sin, cos) pairs of the
                      // x-window sums S_w (one load per chord) instead of the row prefixes
    int64_t *sxy;     // cube box sums over x and y: 2 components, i-block-major (tiled passes)
                      // or node order (the batched sliding passes)
    double *cpl;      // cube: nodes coupling terms of the current stage (window pass -> node pass)
    i128 *partial;    // per-CTA partial sums of the order parameter
    unsigned long long *done_ctr; // arrival counter of the sliding-window node passes (and the prologue)
    unsigned long long *tile_ctr; // arrival counter of the cube node pass (another CTA count per launch)
    unsigned *err;
    double *obs;
    int64_t obs_cap;
    unsigned long long *obs_ctr;
    const int4 *chords; // ball/disk: (dy, dz, w, 0) chords of the window
    int nchords;
    const int *skip;    // if set and nonzero, the x, y and gather passes of stage 1 return at once
                        // (a finished Dormand-Prince run); nullptr for every other use
};

// Adaptive Dormand-Prince 5(4) on lattices and link matrices (lattice_dp.cu):
// elementwise stage-input, error/decision and accept kernels around the
// network's own right-hand side, evaluated from a stage-input buffer.
struct ElemDpPlan {
    int model;
    int64_t nodes, nblk; // nodes; CTAs of the elementwise kernels (256 nodes each)
    double *y, *y5, *xbuf;
    double *k[8];        // k[1..7]: the stage slopes (k[1] = f(y_n) kept from the last accepted step)
    DpCtl *ctl;
    int *remaining;
    double *err_part;    // nblk
    i128 *out_part;      // nblk * kDpMaxOut * 2
    unsigned long long *dp_ctr;
    int64_t *f;          // lattices: (sin, cos) pairs of the stage input's phase on the grid 2^-62 (else nullptr)
    MathTables tab;
    int F;               // fixed-point grid of the dense order-parameter sums
    double *obs;
    int64_t obs_cap;
    unsigned long long *obs_ctr;
    unsigned *err;
};
struct LatDpPlan {
    ElemDpPlan e;
    LatticePlan rhs;     // the network's plan with y = xbuf and skip = &ctl->done; acc set per stage
};
struct GraphDpPlan {
    ElemDpPlan e;
    GraphPlan rhs;       // the network's plan with r.y = xbuf, r.obs = nullptr, r.skip = &ctl->done
};
cudaError_t lat_dp_start(const LatDpPlan &d, cudaStream_t s);     // k1 = f(y_n)
cudaError_t lat_dp_attempt(const LatDpPlan &d, cudaStream_t s);   // one attempted step
cudaError_t graph_dp_start(const GraphDpPlan &d, cudaStream_t s);
cudaError_t graph_dp_attempt(const GraphDpPlan &d, cudaStream_t s);

cudaError_t lattice_configure(); // once per process, before the first launch
int64_t lattice_order_blocks(int topo, int64_t N1); // CTAs of the order-parameter passes (sliding-window grid)
int64_t lattice_sxy_elems(int64_t N1); // cube: xy-window sums (both layouts of the y pass's output)
int64_t lattice_partial_blocks(int topo, int64_t N1); // order-parameter partials to allocate (every grid)
int64_t lattice_sx_elems(int topo, int64_t N1, int64_t P, bool wmode); // int64 elements of sx
constexpr int64_t kLatticeWindowBudget = int64_t(8) << 30; // bytes of the per-w window arrays
cudaError_t lattice_prologue(const LatticePlan &p, cudaStream_t s);
cudaError_t lattice_step(const LatticePlan &p, double dt, cudaStream_t s);
cudaError_t lattice_rhs(const LatticePlan &p, cudaStream_t s); // acc <- f(y)

// Cube members of one model in a batch: device tables of the batched x, y and z
// launches (lattice.cu).  x: CTA b does rows of member x_item[b] (w warps, one
// row each, counted from x_base[member]); y and z: CTA b is the member's CTA
// b - yz_base[member] of its single-network column grid.
struct CubeBatchGroup {
    int model;
    int n_inst;
    int w;                    // warps per x CTA (for the largest edge)
    int64_t n1_max;           // largest edge (sizes the x pass's shared rows)
    int64_t n_x, n_yz;        // CTAs of the x and of the y / z launches
    const LatticePlan *plans; // n_inst (device)
    const int *x_item, *yz_item;
    const int64_t *x_base, *yz_base; // n_inst each
};
cudaError_t cube_batch_step(const CubeBatchGroup &g, double dt, cudaStream_t s); // one RK4 step of every member
int lattice_row_warps(int64_t N1); // warps per CTA of the x pass for edge N1
void lattice_rotation(LatticePlan &p, double alpha); // rot_* and mp.c[5] of a lattice (sim_api.cu)
void ring_coupling_constants(ModelParams &mp, int model, int F); // ksh and c[5] of a Kuramoto ring (sim_api.cu)

// Per-kernel timing of sim_step_timed: while set on the launching host thread,
// every stage-kernel launch of ring_step, graph_step, lattice_step and
// ring_cluster_steps records an event of its kind right after itself (kinds:
// 0 fused ring / link-matrix stage kernel, lattice x pass or the cube's
// order-parameter total, 1 cube y pass, 2 lattice node pass (cube node pass
// fused with the next x pass, ball / disk gather), 3 cube z-window pass).  Never set during a stream capture.
struct KernelMarks {
    cudaEvent_t *ev;
    unsigned char *kind;
    int cap, n;
};
extern thread_local KernelMarks *g_kernel_marks;
inline void kernel_mark(cudaStream_t s, int kind)
{
    KernelMarks *m = g_kernel_marks;
    if (m && m->n < m->cap && cudaEventRecord(m->ev[m->n], s) == cudaSuccess) m->kind[m->n++] = (unsigned char)kind;
}

// Derived model constants of ModelParams (c, q) for K links per node, computed
// on the host in FP64 (sim_api.cu).
void model_constants(int model, const double *params, double K, ModelParams &mp);

// Set the calling thread's sim_last_error() message and return status
// (report_cuda_error: SIM_EDEVICE with "what: <CUDA error string>").
int report_error(int status, const char *msg);
int report_cuda_error(cudaError_t e, const char *what);

// Host-side values of the fast-math tables (long double, rounded to double, and
// the fixed-point sin/cos table rounded onto 2^-62): kMathTableWords 64-bit
// words in the layout of math_tables_at().
void fill_math_tables(double *block);

} // namespace simk
