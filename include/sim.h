/*
 * sim.h -- C ABI of the GB300 network-dynamics stepper.
 *
 * One explicit RK4 time step of a large network of nonlocally coupled
 * oscillators (Sudakov & Maistrenko, "Parallelization of Network Dynamics
 * Computations in Heterogeneous Distributed Environment", arXiv:2410.19075):
 * every RK4 stage gathers each node's coupling sum over its nonlocal
 * neighbourhood, evaluates the node's right-hand side and updates the stage
 * state.  Everything runs on one GPU; there is no CPU fallback.
 *
 * Conventions shared by every entry point
 *   - Return value: a sim_status (0 = SIM_OK, negative = error).  Nothing aborts
 *     the process.  sim_last_error() gives a message for the calling thread.
 *   - Handles are not thread-safe: use one handle per host thread.
 *   - Host buffers are owned by the caller and only read or written during the
 *     call.  The handle owns every device buffer it allocates and frees it in
 *     sim_destroy().
 *   - State layout: variable-major (SoA), FP64, little-endian.  Variable v of
 *     node i is at [v * nodes + i].  Ring: node i in [0, N).  Cube and ball:
 *     node k*N1^2 + j*N1 + i; disk: node j*N1 + i (Section IV, 3D networks).
 *   - Work is issued asynchronously on the handle's CUDA stream (the stream
 *     given at creation; NULL means the legacy default stream).  Device errors
 *     from earlier asynchronous work surface at the next call that synchronises.
 */
#ifndef SIM_H
#define SIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sim_handle *sim_t;

/* Node models.
 * SIM_KS  Kuramoto-Sakaguchi, Eq. (3) with m = 0, eps = 1 (Algorithm 1):
 *         dphi_i/dt = omega - (mu/K) sum_{j in W(i)} sin(phi_i - phi_j + alpha).
 *         1 variable (phi).  params = {omega, mu, alpha}.
 * SIM_FHN FitzHugh-Nagumo, Eq. (2) with tau = 0, D = 0, I_app = 0 and a
 *         rotational coupling matrix B = [[cos p, sin p], [-sin p, cos p]]:
 *         eps du_i/dt = u_i - u_i^3/3 - v_i + (sigma/K) sum_j [B00 (u_j-u_i) + B01 (v_j-v_i)]
 *             dv_i/dt = u_i + a         + (sigma/K) sum_j [B10 (u_j-u_i) + B11 (v_j-v_i)]
 *         2 variables (u, v).  params = {eps, a, sigma, p}.
 * SIM_HH  Hodgkin-Huxley, Eq. (1) specialised to the classic neuron (V, m, h, n)
 *         with textbook rates (rest near -65 mV) and diffusive coupling of V to
 *         the mean of its window: Cm dV/dt = I_ext,i - I_Na - I_K - I_L
 *         + g (mean_{j in W(i)} V_j - V_i).  4 variables.
 *         params = {Cm, gNa, gK, gL, ENa, EK, EL, g}; I_ext per node via
 *         sim_set_node_param (default 0).
 * SIM_KSI Kuramoto with inertia, Eq. (3) with m != 0 (Section IV.C, 3D chimeras):
 *         m phi_i'' + eps phi_i' = (mu/K) sum_{j in W(i)} sin(phi_j - phi_i - alpha),
 *         integrated as phi' = psi, psi' = ((mu/K) sum_j ... - eps psi) / m.
 *         2 variables (phi, psi), stored phi block then psi block.
 *         params = {m, eps, mu, alpha}; m must be non-zero.
 * K is the number of links of a node: 2R on the ring, (2P+1)^3 - 1 on the cube,
 * the lattice-point count of the ball or disk of radius P minus one (one more
 * of each with SIM_FLAG_INCLUDE_SELF). */
typedef enum { SIM_KS = 0, SIM_FHN = 1, SIM_HH = 2, SIM_KSI = 3 } sim_model;

/* Topologies (Section IV).
 * SIM_RING    node i couples to i-R..i+R (mod N), R = radius, 2R+1 <= N.
 * SIM_CUBE3D  periodic N1^3 lattice (N = N1, N1 <= 1024), node couples to the
 *             (2P+1)^3 box around it, P = radius, 2P+1 <= N1.
 * SIM_BALL3D  periodic N1^3 lattice (N1 <= 1024), node couples to every node at
 *             offset (dx, dy, dz) with dx^2 + dy^2 + dz^2 <= P^2 (the nonlocal
 *             3D coupling of Section IV.C), 2P+1 <= N1.
 * SIM_DISK2D  periodic N1^2 lattice (N1 <= 8192), dx^2 + dy^2 <= P^2, 2P+1 <= N1.
 * Lattice nodes are numbered k N1^2 + j N1 + i (x = i fastest).  The lattices
 * take the Kuramoto models (SIM_KS, SIM_KSI) only. */
typedef enum { SIM_RING = 0, SIM_CUBE3D = 1, SIM_BALL3D = 2, SIM_DISK2D = 3, SIM_GRAPH = 4 } sim_topology;
/* SIM_GRAPH   a general link matrix (Section III.C), created with
 *             sim_create_graph, not sim_create. */

typedef enum {
    SIM_OK = 0,
    SIM_EINVAL = -1,      /* invalid argument; nothing was changed */
    SIM_ENOMEM = -2,      /* device allocation failed (or over an admission budget) */
    SIM_EDEVICE = -3,     /* a CUDA call failed; the message says which */
    SIM_ETIMEOUT = -4,    /* a bounded device-side wait gave up; results are invalid */
    SIM_ENONFINITE = -5,  /* the state left the representable range (NaN, Inf or overflow) */
    SIM_EBUSY = -6,       /* the handle is in use (e.g. captured) */
    SIM_ESTEPS = -7,      /* Dormand-Prince: the attempt budget ran out before t_end */
    SIM_ESMALL = -8       /* Dormand-Prince: the step size fell below the resolution of t */
} sim_status;

/* Creation flags. */
#define SIM_FLAG_INCLUDE_SELF 1u /* count the node itself as one of its links */
#define SIM_FLAG_STREAMING 2u    /* rings of <= 4096 nodes: use the multi-launch streaming kernels
                                    instead of the thread-block-cluster kernel (same results) */
#define SIM_FLAG_LOW_MEMORY 4u   /* ball and disk lattices: keep one periodically extended row
                                    prefix (about 16 B per node) instead of one x-window array
                                    per chord half-width ((P+1) * 16 B per node, the default for
                                    P >= 5 when it stays within 8 GiB), at two loads per chord
                                    instead of one; the results are the same bits */

/* Bytes of device memory sim_create() allocates for this network with flags 0
 * (an upper bound for any flags; for admission control).  Returns 0 for invalid
 * arguments. */
size_t sim_workspace_bytes(int model, int topology, int64_t N, int64_t radius);

/* Create a network.  params: n_params doubles in the model's order (above).
 * flags: SIM_FLAG_* above (0 for the defaults).
 * stream: a cudaStream_t (may be torch's current stream) or NULL.
 * The initial state is all zeros until sim_set_state().
 * Errors: SIM_EINVAL (unknown model/topology, 2*radius+1 > N, radius < 1,
 * non-finite params, wrong n_params), SIM_ENOMEM, SIM_EDEVICE. */
int sim_create(sim_t *out, int model, int topology, int64_t N, int64_t radius,
               const double *params, int n_params, unsigned flags, void *stream);

/* Same as sim_create, but the network lives in caller-provided device memory
 * (dev_workspace: at least sim_workspace_bytes() bytes, 256-byte aligned, for
 * example a slice of a PyTorch tensor or of a caller's arena).  The handle does
 * not free it; sim_destroy() synchronises the stream so the memory can be
 * reused afterwards.  Errors: as sim_create, plus SIM_EINVAL for a NULL,
 * misaligned or too small workspace. */
int sim_create_in(sim_t *out, int model, int topology, int64_t N, int64_t radius, const double *params,
                  int n_params, unsigned flags, void *dev_workspace, size_t workspace_bytes, void *stream);

/* A network on a general link matrix (Section III.C: L_ij = 1 when node j
 * influences node i), every model.  Host arrays, read during the call only:
 * row_ptr[N + 1] (row_ptr[0] = 0, non-decreasing) and col[row_ptr[N]]; the links
 * of node i are col[row_ptr[i] .. row_ptr[i+1]), each in [0, N), no duplicates
 * within a row (a self link is allowed and counts as a link).  The coupling of
 * node i is normalised by its own link count K_i (the mean over its links, as
 * Algorithm 1 does with links_amount); a node without links has no coupling
 * term.  The matrix is compressed with Algorithm 2 (common vector V = row 0,
 * difference table of XOR(ROL(row_i, i), V), one entry index per node) and the
 * device evaluates each node's sum as runs of V read from an exact prefix of
 * the coupled quantity plus its entry's signed links: O(runs of V + entry size)
 * reads per node instead of one per link.  3 <= N < 2^31.  The network then
 * steps with sim_step (RK4) or sim_dp5 and supports every call taking a sim_t
 * except step budgets and the server.  Errors: SIM_EINVAL (invalid matrix, model
 * or parameters; the message says which), SIM_ENOMEM, SIM_EDEVICE. */
int sim_create_graph(sim_t *out, int model, int64_t N, const int64_t *row_ptr, const int64_t *col,
                     const double *params, int n_params, void *stream);

/* Size of the compressed link matrix of a SIM_GRAPH network: difference-table
 * entries, runs of the common vector, device bytes of the tables.  Any output
 * may be NULL.  SIM_EINVAL for other networks. */
int sim_graph_info(sim_t h, int64_t *n_entries, int64_t *n_runs, size_t *device_bytes);

/* Number of nodes (N, N1^3 or N1^2) and of state variables per node. */
int64_t sim_nodes(sim_t h);
int sim_dim(sim_t h);

/* Copy a full state (d * nodes doubles, SoA) from host memory.  Resets the
 * observable record: the order parameter of this state is recorded as t = 0.
 * Returns after the copy has been issued; the host buffer may be reused when
 * the call returns.  Errors: SIM_EINVAL if n_values != d * nodes. */
int sim_set_state(sim_t h, const double *host_soa, int64_t n_values);

/* Same, from device memory (dev_soa must stay valid until the stream reaches
 * the copy). */
int sim_set_state_device(sim_t h, const double *dev_soa, int64_t n_values);

/* Per-node parameter: which = 0 is the HH external current I_ext,i
 * (n = nodes doubles, host memory).  SIM_EINVAL for other models. */
int sim_set_node_param(sim_t h, int which, const double *host, int64_t n);

/* Advance the network by n_steps classic RK4 steps of size dt (asynchronous on
 * the handle's stream; launched as a captured CUDA graph).  dt > 0.
 * Errors from the device (SIM_ETIMEOUT, SIM_ENONFINITE) surface at the next
 * synchronising call. */
int sim_step(sim_t h, int64_t n_steps, double dt);

/* As sim_step, for measurement: the n_steps RK4 steps (1 <= n_steps <= 4096)
 * are launched kernel by kernel, not as CUDA graphs, with a CUDA event recorded
 * on the handle's stream after every launch, and the call synchronises.
 * ms_by_kind[k] receives the summed time between consecutive events that ended
 * with a kernel of kind k, launches_by_kind[k] their number (4 entries each):
 * kind 0 = the fused stage kernel of a ring or link matrix (one per stage; the
 * whole call for the cluster-resident small-ring kernel), the x pass of a ball
 * or disk, or the cube's order-parameter total (once per step), 1 = the y pass
 * of the cube, 2 = the node pass of a lattice (the cube's elementwise RK4 pass
 * fused with the next stage's x pass, the chord gather of the ball and disk),
 * 3 = the z-window pass of the cube.  The
 * state advances exactly as with sim_step (the same bits).  Returns the device
 * error status like sim_sync.  Errors: SIM_EINVAL (NULL handle or output,
 * n_steps out of range, invalid dt), SIM_EDEVICE. */
int sim_step_timed(sim_t h, int64_t n_steps, double dt, double *ms_by_kind, int64_t *launches_by_kind);

/* Copy the state to host memory (synchronises the stream).  Returns the device
 * error status accumulated since creation, if any. */
int sim_get_state(sim_t h, double *host_soa, int64_t n_values);

/* Copy the state to device memory (asynchronous). */
int sim_get_state_device(sim_t h, double *dev_soa, int64_t n_values);

/* Evaluate the right-hand side f(y) of every node at the current state, through
 * the same fused stage kernel sim_step() uses for RK4 stage 1, and copy it to
 * host memory (d * nodes doubles, SoA; synchronises).  The state is not changed.
 * Useful for sampled checks of large networks and for Jacobian studies. */
int sim_rhs(sim_t h, double *host_k, int64_t n_values);

/* Kuramoto order parameter |mean_j exp(i phi_j)| at t = 0 and after every step
 * since the last call (synchronises).  Writes at most max_values values to
 * host_R and their count to *n_written.  Values not yet read are kept for the
 * most recent 65536 steps; older ones are dropped.  Recorded for SIM_KS and
 * SIM_KSI (phases = variable 0); other models write 0 values. */
int sim_observables(sim_t h, double *host_R, int64_t max_values, int64_t *n_written);

/* Wait for all work issued on the handle's stream and report device errors. */
int sim_sync(sim_t h);

/* Steps completed (issued) since the last sim_set_state. */
int64_t sim_steps_done(sim_t h);

/* ---------------------------------------------------------------------------
 * Adaptive Dormand-Prince 5(4) (Section III.A: the paper's default solver is a
 * Dormand-Prince method with step-size control; Section V: the solution is
 * interpolated for dense output and synchronisation is analysed at every
 * output).  Every topology: rings and link matrices (every model), the cube,
 * ball and disk lattices (the Kuramoto models).
 *
 * Method: the RK5(4)7M pair of Dormand and Prince (1980), first same as last
 * (six right-hand sides per attempted step).  Error of an attempt of size h:
 * e = h sum_j (b_j - bhat_j) k_j, err = sqrt(mean over all d * N values of
 * (e / sc)^2) with sc = atol + rtol max(|y_n|, |y_n+1|).  Accepted when err <= 1
 * (a non-finite err is a rejection).  Next step h * clamp(0.9 err^(-1/5), 0.2, 10),
 * not growing right after a rejection, and at most h_max and 8 * out_dt.  The
 * attempt that reaches t_end is cut to end there exactly.  Every decision is
 * taken on the device; the host only waits for the run to end.
 * Dense output (SIM_KS, SIM_KSI): the order parameter of the cubic Hermite
 * interpolant of the phases (from y_n, y_n+1 and their slopes) at
 * t0 + k out_dt, k = 1 .. floor((t_end - t0) / out_dt (1 + 1e-12)); together with
 * R(t0) these values are appended to the record sim_observables() returns.
 * The state is integrated in place: after the call the handle holds y(t), t as
 * reported in the stats.  The first call on a handle allocates its
 * Dormand-Prince buffers (7 d N doubles and per-sub-tile sums). */
typedef struct {
    double t0, t_end;   /* integrate from t0 to t_end > t0 */
    double rtol, atol;  /* >= 0, not both 0 */
    double h0;          /* first trial step, > 0 */
    double h_max;       /* largest step; 0 = no limit */
    double out_dt;      /* dense-output interval; 0 = none */
    int64_t max_attempts; /* accepted + rejected attempts allowed, >= 1 */
} sim_dp5_opts;

typedef struct {
    int64_t accepted, rejected;
    double t;       /* time reached: t_end unless status != 0 */
    double h_next;  /* the next proposed step size (before any cut at t_end) */
    int status;     /* SIM_OK, SIM_ESTEPS or SIM_ESMALL */
} sim_dp5_stats;

/* One network.  Returns SIM_OK, the run's SIM_ESTEPS / SIM_ESMALL (the state is
 * then that of the last accepted step, stats->t), SIM_EINVAL (invalid options),
 * SIM_ENOMEM, or a device error.  stats may be NULL.  Synchronises the handle's
 * stream.  A ring run uses fused Dormand-Prince stage kernels; a lattice or
 * link-matrix run evaluates each stage with the network's own right-hand-side
 * kernels from a stage-input buffer. */
int sim_dp5(sim_t h, const sim_dp5_opts *opts, sim_dp5_stats *stats);

/* ---------------------------------------------------------------------------
 * Batches: many independent networks advanced together (the paper's "large
 * number of small unconnected subnets within a single run", Section III.C, and
 * its parameter and multistability studies, Section IV).  Ring members of the
 * same model are stepped by one launch per RK4 stage whose CTAs are
 * (member, 256-node sub-tile) work items; lattice members by their own kernels.
 * Every member keeps its own state, prefix buffers and observables, so results
 * are bit-for-bit those of sim_step on each member alone.
 */
typedef struct sim_batch_handle *sim_batch_t;

/* Group existing networks into a batch.  Members are networks made with
 * sim_create (or sim_create_in / sim_create_graph), each with its own model,
 * topology, size, parameters and state, so that a batch can mix everything a
 * single network can be and members keep working on their own between batches;
 * the batch does not own the members;
 * they must outlive it and must not be stepped on their own streams while the
 * batch's work is in flight.  stream: where the batch issues work (NULL =
 * legacy default).  Errors: SIM_EINVAL (no members, NULL or duplicate member),
 * SIM_ENOMEM, SIM_EDEVICE. */
int sim_batch_create(sim_batch_t *out, const sim_t *members, int n_members, void *stream);

/* Per-member step budgets (n_members values): a ring member with budget b stops
 * after b more RK4 steps of the following sim_batch_step calls (its state then
 * stays as it is); -1 = unlimited (the default).  Cube members take -1 only.
 * Synchronises the batch stream. */
int sim_batch_set_budgets(sim_batch_t b, const int64_t *steps);

/* Advance every member by n_steps RK4 steps of size dt (asynchronous; CUDA
 * graphs of 16 steps).  sim_steps_done() of each member is updated.
 * How a batch is launched: per RK4 stage one launch for all ring members of a
 * model, whose CTAs are (member, 256-node sub-tile) work items listed in a
 * device table built at sim_batch_create (CTA b reads its item directly); the
 * stage boundary is the launch boundary, and the step loop is captured in CUDA
 * graphs.  This takes the place of one persistent launch pulling (member, tile)
 * items from a device work queue, which would need every stage of every member
 * to wait, inside the launch, for the CTAs of its previous stage; here no CTA
 * ever waits for another.  The 256-node sub-tile is fixed (it is the unit of
 * the exact prefix); what sim_batch_autotune chooses is the number of nodes per
 * thread (1 or 2). */
int sim_batch_step(sim_batch_t b, int64_t n_steps, double dt);

/* Dormand-Prince runs of every member, each with its own
 * options opts[i], tolerances, step sizes and decisions; every attempt of every
 * unfinished member is one set of launches per model group.  stats[i] gets each
 * member's outcome (status SIM_OK, SIM_ESTEPS or SIM_ESMALL).  Returns SIM_OK
 * unless the arguments, an allocation or the device failed.  Results are those
 * of sim_dp5 on each member alone. */
int sim_batch_dp5(sim_batch_t b, const sim_dp5_opts *opts, sim_dp5_stats *stats);

/* Wait for the batch's work and report the first device error of any member. */
int sim_batch_sync(sim_batch_t b);

/* Free the batch's own tables (synchronises first); members are untouched. */
void sim_batch_destroy(sim_batch_t b);

/* ---------------------------------------------------------------------------
 * Autotuner.  The ring stage kernels come in variants that give the same bits:
 * two adjacent nodes per thread (128 threads per 256-node sub-tile) or one
 * (256 threads), and, on rings of at most 128 prefix groups (N <= 2^21), the
 * one-pass or the two-level prefix of the coupled quantity.  Which is fastest
 * depends on the model, the ring and the batch, so it is measured.
 *
 * sim_autotune times trial_steps RK4 steps of dt with every variant of a ring
 * network, on its current state, and keeps the fastest: *npt_out = nodes per
 * thread (1 or 2; HH always 1), *flat_out = 1 for the one-pass prefix (either
 * may be NULL).
 * Afterwards the state is the one before the call, and the order-parameter
 * record, step count and error word are as after sim_set_state (R(t0) is
 * recorded again).  Networks without variants (lattices, link matrices, rings
 * small enough for the cluster kernel) report their fixed choice and run
 * nothing.  Needs a device copy of the state; SIM_ENOMEM if it does not fit.
 * The choice is also stored in a process-wide cache under (model, N, radius):
 * later sim_create calls with the same key start with it. */
int sim_autotune(sim_t h, double dt, int64_t trial_steps, int *npt_out, int *flat_out);

/* The variant a ring network runs (npt 1 or 2, flat 0 or 1; 0 and 0 for
 * lattices and link matrices).  SIM_EINVAL for a NULL argument. */
int sim_tune_info(sim_t h, int *npt, int *flat);

/* The same for a batch: times trial_steps batched RK4 steps with one and with
 * two nodes per thread for every ring group (HH groups run one), keeps the
 * faster in *npt_out, and restores every member's state, error word,
 * order-parameter count and the batch's step budgets.  Cached under the batch's
 * ring sub-tile and member counts for later sim_batch_create calls. */
int sim_batch_autotune(sim_batch_t b, double dt, int64_t trial_steps, int *npt_out);

/* Write the cache as text (one "kind model a b npt flat" line per entry; kind 0
 * = plain ring (model, N, radius), kind 1 = batch (-1, ring sub-tiles, ring
 * members)), merge a file written that way into it, or empty it.  Host only;
 * the caller owns path.  SIM_EINVAL if the file cannot be written or read, or
 * if a line is malformed (then nothing of the file is merged).  An entry only
 * selects among variants that give the same results, so a stale file can cost
 * speed, never correctness. */
int sim_tune_save(const char *path);
int sim_tune_load(const char *path);
int sim_tune_clear(void);

/* ---------------------------------------------------------------------------
 * Serving: a request loop with continuous batching.  Jobs (one network each)
 * are submitted at any time; a worker thread admits them in arrival order while
 * the resident jobs' device memory (sim_workspace_bytes each) stays within
 * hbm_budget_bytes and fewer than max_slots are resident, keeps their state on
 * the device, advances all resident jobs together (sim_batch_* in chunks of
 * chunk_steps RK4 steps, each job stopped exactly at its horizon by a step
 * budget) and retires finished jobs (final state and Kuramoto order
 * parameters copied to host memory, device memory released).  A job's result is
 * bit-for-bit the same alone and in any mix.  max_slots = 1 runs one job at a
 * time on the plain path (sim_step): the baseline.
 */
typedef struct srv_handle *srv_t;

/* Start a server (and its worker thread) on the current device.  stream: where
 * its work is issued (NULL = legacy default). */
int srv_create(srv_t *out, size_t hbm_budget_bytes, int max_slots, int64_t chunk_steps, void *stream);

/* Queue one job (arguments as sim_create / sim_set_state / sim_set_node_param;
 * host buffers are copied before the call returns).  n_steps RK4 steps of dt.
 * Writes the job id.  SIM_ENOMEM if the job alone exceeds the HBM budget. */
int srv_submit(srv_t s, int model, int topology, int64_t N, int64_t radius, const double *params, int n_params,
               const double *host_init_state, const double *host_node_param, int64_t n_steps, double dt,
               int64_t *job_id);

/* *done = 1 once the job has finished.  Then copies its final state
 * (n_values = d * nodes doubles, or host_state_out = NULL), up to max_order
 * order-parameter values (t = 0 and every step; Kuramoto only) with their count
 * in *n_order, and times_out[0..2] = submit, admission and completion times
 * (seconds, steady clock; may be NULL), releases the job and returns its
 * status.  While not done it returns SIM_OK with *done = 0.  SIM_EINVAL for an
 * unknown (or already collected) id. */
int srv_poll(srv_t s, int64_t job_id, int *done, double *host_state_out, int64_t n_values, double *host_order_out,
             int64_t max_order, int64_t *n_order, double *times_out);

/* Block until every submitted job has finished. */
int srv_wait_idle(srv_t s);

/* out6 = {completed jobs, jobs not yet finished, queued (not admitted) jobs,
 * node-steps done, batches formed, device bytes in use}. */
int srv_stats(srv_t s, int64_t *out6);

/* Device-memory accounting of the admission loop: out3 = {bytes of the budget
 * in use now, the largest number of bytes in use at any moment since
 * srv_create (never above hbm_budget_bytes), jobs whose admission had to wait
 * for device memory (the head of the queue did not fit the budget, or no free
 * block of the arena was large enough, while a slot was free)}. */
int srv_memory(srv_t s, int64_t *out3);

/* out5 = the worker thread's cumulative time (seconds) in admission (network
 * creation and state upload), batch formation, stepping (launches of each chunk
 * and the wait for it), retirement (result download, release) and waiting for
 * work.  Read while running or after srv_wait_idle. */
int srv_timings(srv_t s, double *out5);

/* Stop the worker (unfinished jobs are dropped) and free everything. */
void srv_destroy(srv_t s);

/* RK4 steps of a ring network with no device allocation at all.
 *
 * The paper has no counterpart; this entry point is for callers that cannot
 * allocate device memory while they run (for example a plugin inside an
 * application that owns all device memory through its own fixed arena, or a
 * service whose device footprint must not change after start-up).  The caller
 * passes the state as a device buffer (dev_state: d * N doubles, SoA, updated in
 * place) and, for SIM_HH, dev_node_param (N doubles of I_ext, or NULL for 0).
 * Every other buffer lives in one static device array of this library (8 MiB,
 * held by each GPU that loads the library until the process exits), so the
 * ring must have N <= 65536 nodes; larger N returns SIM_EINVAL.  Arguments and
 * model parameters are as for sim_create with topology SIM_RING.
 * The work is issued on `stream` (a cudaStream_t, NULL = legacy default) and the
 * call synchronises that stream before it returns, so that it can report
 * SIM_ENONFINITE; it therefore cannot be captured into a CUDA graph, and a call
 * on a capturing stream returns SIM_EINVAL without touching the stream.  It
 * calls no cudaMalloc, cudaFree or other allocator.
 * The first call on each device does a one-time set-up with that device
 * current (it looks up the static array's device address and copies the
 * fast-math tables into it); make that first call before any stream capture.
 * The set-up is kept for the life of the process: calls after a
 * cudaDeviceReset() of that device are not supported.
 * All calls share the static array, which keeps the last call's contents (each
 * call clears the counters and the error word it needs at zero): calls whose
 * work overlaps on the GPU (other streams or host threads) race with each
 * other and must be serialised by the caller.
 * Errors: SIM_EINVAL (the same argument checks as sim_create, N > 65536, or a
 * capturing stream), SIM_ENONFINITE, SIM_ETIMEOUT, SIM_EDEVICE;
 * sim_last_error() gives the reason. */
int sim_ring_step_noalloc(int model, int64_t N, int64_t radius, const double *params, int n_params,
                          unsigned flags, double *dev_state, const double *dev_node_param, int64_t n_steps,
                          double dt, void *stream);

/* Evaluate the library's device elementary functions on n arguments (host
 * buffers; synchronous), for accuracy checks: fn 0 = sin, 1 = cos, 2 = exp,
 * 3 = reciprocal 1/x, 4 = x / (1 - exp(-x)).  These are the table-driven FP64
 * routines the node right-hand sides use (Kuramoto phases, Hodgkin-Huxley
 * rates of Eq. (1)).  Allocates and frees its own device buffers. */
int sim_math_eval(int fn, const double *host_x, double *host_out, int64_t n);

/* Measured peak rate of one arithmetic pipe of the current device, for roofline
 * denominators (not part of the method; a utility of the benchmark): kind 0 =
 * FP64 fused multiply-adds per second (count 2 flops each), 1 = 64-bit integer
 * multiply-highs (mul.hi.u64) per second, 2 = 32-bit integer multiply-adds per
 * second, 3 = int64 -> double conversions (cvt.rn.f64.s64) per second, 4 =
 * signed 64-bit multiply-highs (mul.hi.s64) per second.  Every thread of a grid of 8 CTAs per SM runs 8 independent dependent
 * chains of the operation; one warm-up launch, then one launch timed with CUDA
 * events (tens of milliseconds).  Allocates and frees 64 bytes of device memory
 * and a stream; synchronous.  Errors: SIM_EINVAL (unknown kind or NULL output),
 * SIM_EDEVICE. */
int sim_probe_peak(int kind, double *ops_per_s);

/* Message of the last non-OK status returned on this thread (never NULL).  It
 * takes no handle: a failed sim_create has no handle to ask, and the message is
 * per host thread, as handles are used from one thread each. */
const char *sim_last_error(void);

/* Free all device memory of the handle (synchronises first).  NULL is a no-op. */
void sim_destroy(sim_t h);

#ifdef __cplusplus
}
#endif
#endif /* SIM_H */
