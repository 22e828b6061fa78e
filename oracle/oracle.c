/*
 * Oracle for the explicit RK4 time step of nonlocally coupled oscillator networks.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, obviously correct CPU
 * implementation in IEEE FP64.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header, table or
 * constant with the CUDA path, and the CUDA path never calls it.
 *
 * What it computes (brute force, straight from the equations):
 *   - Coupling sums are evaluated pair by pair over every neighbour in the
 *     window, in increasing offset order (or decreasing, with ORC_REVERSE, to
 *     measure the floating-point floor of a chaotic run).
 *   - Kuramoto-Sakaguchi, Eq. (3) with m = 0, eps = 1 and Algorithm 1 (mean of
 *     sin(phi_j - phi_i - alpha) over the links of node i); written in the
 *     equivalent form  dphi_i/dt = omega - (mu/K) sum_j sin(phi_i - phi_j + alpha).
 *   - FitzHugh-Nagumo, Eq. (2) with tau = 0, D = 0, I_app = 0, and a rotational
 *     2x2 coupling matrix B(phi) = [[cos, sin], [-sin, cos]] acting on (u, v).
 *   - Hodgkin-Huxley, Eq. (1) specialised to the classic four-variable neuron
 *     (V, m, h, n) with diffusive coupling of V to the mean of its window.
 *     The rate functions are the textbook ones (rest near -65 mV); the paper does
 *     not print them.
 *   - Topologies: a ring where node i couples to the R nodes on each side
 *     (Section IV, 1D networks), and a periodic cubic lattice of N1^3 nodes,
 *     node index k*N1^2 + j*N1 + i (Section IV, 3D networks), coupled to the
 *     (2P+1)^3 box around it.  Self is excluded unless ORC_INCLUDE_SELF.
 *   - Classic fixed-step fourth-order Runge-Kutta.
 *   - Kuramoto-Sakaguchi with inertia, Eq. (3) with m != 0, as phi' = psi,
 *     psi' = ((mu/K) sum_j sin(phi_j - phi_i - alpha) - eps psi) / m.
 *   - Kuramoto order parameter |sum_j exp(i phi_j)| / n.
 *   - A general link matrix given by rows (Section III.C), every model, each node
 *     normalised by its own link count; and the differential compression of
 *     the link matrix, Algorithm 2 (COMPRESS and EXTRACT).
 *   - Adaptive Dormand-Prince 5(4) (the paper's default solver, Section III.A):
 *     the published RK5(4)7M tableau, the mixed error norm and step-size
 *     controller of the textbook, and cubic Hermite dense output (the paper
 *     interpolates its dense output and analyses synchronisation at every
 *     output, Section V).
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fopenmp -shared -fPIC (see build.py).
 * Parallelism: OpenMP over nodes only; every node's sum is computed by one thread
 * in a fixed order, so results do not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORC_KS = 0, ORC_FHN = 1, ORC_HH = 2, ORC_KSI = 3 };
enum { ORC_RING = 0, ORC_CUBE = 1, ORC_BALL = 2, ORC_DISK = 3, ORC_GRAPH = 4 };

/* A general link matrix (Section III.C: L_ij = 1 when oscillator j influences
 * oscillator i), given by rows: the links of node i are col[row_ptr[i] ..
 * row_ptr[i+1]).  Set with orc_set_graph before using topology ORC_GRAPH (N is
 * then the number of nodes and R is ignored).  The oracle keeps a pointer to the
 * caller's arrays; they must stay valid while it is used. */
static int64_t g_graph_n = 0;
static const int64_t *g_graph_ptr = NULL, *g_graph_col = NULL;

int orc_set_graph(int64_t n, const int64_t *row_ptr, const int64_t *col)
{
    if (n < 1 || !row_ptr || (row_ptr[n] > 0 && !col)) return -1;
    for (int64_t i = 0; i < n; ++i)
        if (row_ptr[i + 1] < row_ptr[i]) return -1;
    for (int64_t t = 0; t < row_ptr[n]; ++t)
        if (col[t] < 0 || col[t] >= n) return -1;
    g_graph_n = n;
    g_graph_ptr = row_ptr;
    g_graph_col = col;
    return 0;
}
enum { ORC_REVERSE = 1, ORC_INCLUDE_SELF = 2 };
enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ENOMEM = -2, ORC_ESTEPS = -3, ORC_ESMALL = -4 };

/* Number of state variables per node. */
int orc_dim(int model)
{
    switch (model) {
    case ORC_KS: return 1;
    case ORC_FHN: return 2;
    case ORC_HH: return 4;
    case ORC_KSI: return 2;
    default: return 0;
    }
}

/* Number of nodes: N for the ring, N1^3 for the cube and the ball, N1^2 for the
 * disk (N is the edge N1). */
int64_t orc_nodes(int topo, int64_t N)
{
    if (topo == ORC_CUBE || topo == ORC_BALL) return N * N * N;
    if (topo == ORC_DISK) return N * N;
    return N; /* ring, graph */
}

static int n_params_of(int model)
{
    switch (model) {
    case ORC_KS: return 3;  /* omega, mu, alpha */
    case ORC_FHN: return 4; /* eps, a, sigma, phi */
    case ORC_HH: return 8;  /* Cm, gNa, gK, gL, ENa, EK, EL, g */
    case ORC_KSI: return 4; /* m, eps, mu, alpha */
    default: return -1;
    }
}

int orc_validate(int model, int topo, int64_t N, int64_t R, int n_params)
{
    if (orc_dim(model) == 0) return ORC_EINVAL;
    if (topo < ORC_RING || topo > ORC_GRAPH) return ORC_EINVAL;
    if (n_params != n_params_of(model)) return ORC_EINVAL;
    if (topo == ORC_GRAPH) return (g_graph_ptr && N == g_graph_n) ? ORC_OK : ORC_EINVAL;
    if (R < 1 || N < 2 * R + 1) return ORC_EINVAL;
    if (topo != ORC_RING && model != ORC_KS && model != ORC_KSI) return ORC_EINVAL;
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Neighbour enumeration.  The window of node `node` is listed into `nb` in
 * increasing offset order (ring: d = -R..R; lattices: dz, then dy, then dx,
 * each -P..P), skipping the node itself unless include_self.  The cube keeps
 * every offset of the (2P+1)^3 box; the ball keeps dx^2 + dy^2 + dz^2 <= P^2
 * (Section IV, 3D networks: the sphere of radius P, index k N1^2 + j N1 + i);
 * the disk keeps dx^2 + dy^2 <= P^2 (Section IV, 2D networks, index j N1 + i).
 * Returns the count. */
static int64_t wrap(int64_t a, int64_t n)
{
    int64_t r = a % n;
    return r < 0 ? r + n : r;
}

static int64_t list_window(int topo, int64_t N, int64_t R, int64_t node, int include_self, int64_t *nb)
{
    int64_t c = 0;
    if (topo == ORC_GRAPH) { /* the row of the link matrix, as given (self only if listed) */
        (void)include_self;
        for (int64_t t = g_graph_ptr[node]; t < g_graph_ptr[node + 1]; ++t) nb[c++] = g_graph_col[t];
    } else if (topo == ORC_RING) {
        for (int64_t d = -R; d <= R; ++d) {
            if (d == 0 && !include_self) continue;
            nb[c++] = wrap(node + d, N);
        }
    } else if (topo == ORC_DISK) {
        int64_t i = node % N, j = node / N;
        for (int64_t dy = -R; dy <= R; ++dy)
            for (int64_t dx = -R; dx <= R; ++dx) {
                if (dx * dx + dy * dy > R * R) continue;
                if (dx == 0 && dy == 0 && !include_self) continue;
                nb[c++] = wrap(j + dy, N) * N + wrap(i + dx, N);
            }
    } else {
        int64_t i = node % N, j = (node / N) % N, k = node / (N * N);
        for (int64_t dz = -R; dz <= R; ++dz)
            for (int64_t dy = -R; dy <= R; ++dy)
                for (int64_t dx = -R; dx <= R; ++dx) {
                    if (topo == ORC_BALL && dx * dx + dy * dy + dz * dz > R * R) continue;
                    if (dx == 0 && dy == 0 && dz == 0 && !include_self) continue;
                    nb[c++] = wrap(k + dz, N) * N * N + wrap(j + dy, N) * N + wrap(i + dx, N);
                }
    }
    return c;
}

/* An upper bound of the window size (the enclosing box). */
static int64_t window_size(int topo, int64_t R, int include_self)
{
    if (topo == ORC_GRAPH) {
        int64_t m = 1;
        for (int64_t i = 0; i < g_graph_n; ++i)
            if (g_graph_ptr[i + 1] - g_graph_ptr[i] > m) m = g_graph_ptr[i + 1] - g_graph_ptr[i];
        return m;
    }
    int64_t w = 2 * R + 1;
    int64_t full = topo == ORC_RING ? w : (topo == ORC_DISK ? w * w : w * w * w);
    return include_self ? full : full - 1;
}

/* Links of a node (the window size): used by tests against the paper's counts. */
int64_t orc_links(int topo, int64_t N, int64_t R, int include_self)
{
    if (R < 1 || N < 2 * R + 1) return -1;
    int64_t *nb = malloc(sizeof(int64_t) * (size_t)window_size(topo, R, 1));
    if (!nb) return -1;
    int64_t c = list_window(topo, N, R, 0, include_self, nb);
    free(nb);
    return c;
}

/* ------------------------------------------------------------------------- */
/* Hodgkin-Huxley rate functions, V in mV, rates in 1/ms (textbook set, rest
 * near -65 mV).  x / (1 - exp(-x)) is written with expm1 and takes its limit 1
 * at x = 0 (the removable singularities at V = -40 and V = -55). */
static double x_over_1mexp(double x)
{
    if (x == 0.0) return 1.0;
    return x / -expm1(-x);
}
double orc_hh_alpha_m(double V) { return x_over_1mexp((V + 40.0) / 10.0); }
double orc_hh_beta_m(double V) { return 4.0 * exp(-(V + 65.0) / 18.0); }
double orc_hh_alpha_h(double V) { return 0.07 * exp(-(V + 65.0) / 20.0); }
double orc_hh_beta_h(double V) { return 1.0 / (1.0 + exp(-(V + 35.0) / 10.0)); }
double orc_hh_alpha_n(double V) { return 0.1 * x_over_1mexp((V + 55.0) / 10.0); }
double orc_hh_beta_n(double V) { return 0.125 * exp(-(V + 65.0) / 80.0); }

/* ------------------------------------------------------------------------- */
/* Right-hand side of one node i.  x is variable-major (SoA): variable v of node
 * j is at x[v * nodes + j].  k receives the d derivatives of node i, k[0..d).
 * node_param: HH external current per node (NULL means 0).  nb is scratch for
 * the neighbour list. */
static void rhs_node(int model, int topo, int64_t N, int64_t R, const double *p,
                     const double *node_param, const double *x, double *k,
                     int64_t nodes, int flags, int64_t i, int64_t *nb)
{
    int include_self = (flags & ORC_INCLUDE_SELF) != 0;
    int64_t cnt = list_window(topo, N, R, i, include_self, nb);
    double K = (double)cnt;
    /* cnt = 0 (a node without links, only on a graph): no coupling term */
    int64_t first = 0, last = cnt, step = 1;
    if (flags & ORC_REVERSE) { first = cnt - 1; last = -1; step = -1; }

    if (model == ORC_KS) {
        double omega = p[0], mu = p[1], alpha = p[2];
        double phi_i = x[i], sum = 0.0;
        for (int64_t t = first; t != last; t += step)
            sum += sin(phi_i - x[nb[t]] + alpha);
        k[0] = cnt > 0 ? omega - (mu / K) * sum : omega;
    } else if (model == ORC_KSI) {
        /* Eq. (3) with inertia: m phi'' + eps phi' = (mu/K) sum_j sin(phi_j - phi_i - alpha),
         * as the first-order system phi' = psi, psi' = ((mu/K) sum_j ... - eps psi) / m. */
        double m = p[0], eps = p[1], mu = p[2], alpha = p[3];
        const double *phi = x, *psi = x + nodes;
        double phi_i = phi[i], sum = 0.0;
        for (int64_t t = first; t != last; t += step)
            sum += sin(phi[nb[t]] - phi_i - alpha);
        k[0] = psi[i];
        k[1] = ((cnt > 0 ? (mu / K) * sum : 0.0) - eps * psi[i]) / m;
    } else if (model == ORC_FHN) {
        double eps = p[0], a = p[1], sigma = p[2], phi = p[3];
        double buu = cos(phi), buv = sin(phi), bvu = -sin(phi), bvv = cos(phi);
        const double *u = x, *v = x + nodes;
        double ui = u[i], vi = v[i], cu = 0.0, cv = 0.0;
        for (int64_t t = first; t != last; t += step) {
            int64_t j = nb[t];
            cu += buu * (u[j] - ui) + buv * (v[j] - vi);
            cv += bvu * (u[j] - ui) + bvv * (v[j] - vi);
        }
        const double sK = cnt > 0 ? sigma / K : 0.0;
        k[0] = (ui - ui * ui * ui / 3.0 - vi + sK * cu) / eps;
        k[1] = ui + a + sK * cv;
    } else { /* ORC_HH */
        double Cm = p[0], gNa = p[1], gK = p[2], gL = p[3];
        double ENa = p[4], EK = p[5], EL = p[6], g = p[7];
        const double *V = x, *m = x + nodes, *h = x + 2 * nodes, *n = x + 3 * nodes;
        double Vi = V[i], mi = m[i], hi = h[i], ni = n[i];
        double sumV = 0.0;
        for (int64_t t = first; t != last; t += step) sumV += V[nb[t]];
        double coupling = cnt > 0 ? g * (sumV / K - Vi) : 0.0;
        double Iext = node_param ? node_param[i] : 0.0;
        double INa = gNa * mi * mi * mi * hi * (Vi - ENa);
        double IK = gK * ni * ni * ni * ni * (Vi - EK);
        double IL = gL * (Vi - EL);
        k[0] = (Iext - INa - IK - IL + coupling) / Cm;
        k[1] = orc_hh_alpha_m(Vi) * (1.0 - mi) - orc_hh_beta_m(Vi) * mi;
        k[2] = orc_hh_alpha_h(Vi) * (1.0 - hi) - orc_hh_beta_h(Vi) * hi;
        k[3] = orc_hh_alpha_n(Vi) * (1.0 - ni) - orc_hh_beta_n(Vi) * ni;
    }
}

static int set_threads(int nthreads)
{
#ifdef _OPENMP
    return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

/* Right-hand side of every node; x and k are SoA (d * nodes doubles). */
int orc_rhs(int model, int topo, int64_t N, int64_t R, const double *params, int n_params,
            const double *node_param, const double *x, double *k, int flags, int nthreads)
{
    int st = orc_validate(model, topo, N, R, n_params);
    if (st != ORC_OK) return st;
    int64_t nodes = orc_nodes(topo, N);
    int64_t wmax = window_size(topo, R, 1);
    int nt = set_threads(nthreads);
    int failed = 0;
#pragma omp parallel num_threads(nt)
    {
        int64_t *nb = (int64_t *)malloc(sizeof(int64_t) * (size_t)wmax);
        if (!nb) {
#pragma omp atomic write
            failed = 1;
        } else {
            int d = orc_dim(model);
#pragma omp for schedule(static)
            for (int64_t i = 0; i < nodes; ++i) {
                double kn[4];
                rhs_node(model, topo, N, R, params, node_param, x, kn, nodes, flags, i, nb);
                for (int v = 0; v < d; ++v) k[v * nodes + i] = kn[v];
            }
            free(nb);
        }
    }
    return failed ? ORC_ENOMEM : ORC_OK;
}

/* Kuramoto order parameter |(1/n) sum_j exp(i phi_j)|. */
double orc_order_parameter(int64_t n, const double *phi)
{
    double c = 0.0, s = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        c += cos(phi[j]);
        s += sin(phi[j]);
    }
    return sqrt(c * c + s * s) / (double)n;
}

/* Classic RK4:
 *   k1 = f(y), k2 = f(y + dt/2 k1), k3 = f(y + dt/2 k2), k4 = f(y + dt k3),
 *   y <- y + dt/6 (k1 + 2 k2 + 2 k3 + k4).
 * y (d * nodes doubles, SoA) is advanced in place by n_steps steps.  If order_out
 * is not NULL (Kuramoto only), it receives the order parameter at t = 0 and after
 * every step: n_steps + 1 values. */
int orc_rk4(int model, int topo, int64_t N, int64_t R, const double *params, int n_params,
            const double *node_param, double *y, int64_t n_steps, double dt,
            double *order_out, int flags, int nthreads)
{
    int st = orc_validate(model, topo, N, R, n_params);
    if (st != ORC_OK) return st;
    if (n_steps < 0 || !(dt > 0.0)) return ORC_EINVAL;
    int64_t nodes = orc_nodes(topo, N);
    int64_t len = nodes * orc_dim(model);
    double *k1 = malloc(sizeof(double) * (size_t)len), *k2 = malloc(sizeof(double) * (size_t)len);
    double *k3 = malloc(sizeof(double) * (size_t)len), *k4 = malloc(sizeof(double) * (size_t)len);
    double *tmp = malloc(sizeof(double) * (size_t)len);
    if (!k1 || !k2 || !k3 || !k4 || !tmp) {
        free(k1); free(k2); free(k3); free(k4); free(tmp);
        return ORC_ENOMEM;
    }
    int nt = set_threads(nthreads);
    int has_order = model == ORC_KS || model == ORC_KSI; /* phases are the first variable */
    if (order_out && has_order) order_out[0] = orc_order_parameter(nodes, y);
    for (int64_t s = 0; s < n_steps && st == ORC_OK; ++s) {
        st = orc_rhs(model, topo, N, R, params, n_params, node_param, y, k1, flags, nt);
        for (int64_t q = 0; q < len; ++q) tmp[q] = y[q] + dt / 2.0 * k1[q];
        if (st == ORC_OK) st = orc_rhs(model, topo, N, R, params, n_params, node_param, tmp, k2, flags, nt);
        for (int64_t q = 0; q < len; ++q) tmp[q] = y[q] + dt / 2.0 * k2[q];
        if (st == ORC_OK) st = orc_rhs(model, topo, N, R, params, n_params, node_param, tmp, k3, flags, nt);
        for (int64_t q = 0; q < len; ++q) tmp[q] = y[q] + dt * k3[q];
        if (st == ORC_OK) st = orc_rhs(model, topo, N, R, params, n_params, node_param, tmp, k4, flags, nt);
        for (int64_t q = 0; q < len; ++q)
            y[q] = y[q] + dt / 6.0 * (k1[q] + 2.0 * k2[q] + 2.0 * k3[q] + k4[q]);
        if (order_out && has_order) order_out[s + 1] = orc_order_parameter(nodes, y);
    }
    free(k1); free(k2); free(k3); free(k4); free(tmp);
    return st;
}

/* Coupling sum of one quantity over the window of each listed node, brute force:
 * out[t] = sum_{j in W(nodes[t])} f[j].  Used to check window sums on tiny inputs. */
int orc_window_sum(int topo, int64_t N, int64_t R, const double *f, int64_t n_query,
                   const int64_t *query, double *out, int flags)
{
    if (R < 1 || N < 2 * R + 1) return ORC_EINVAL;
    int64_t *nb = malloc(sizeof(int64_t) * (size_t)window_size(topo, R, 1));
    if (!nb) return ORC_ENOMEM;
    for (int64_t t = 0; t < n_query; ++t) {
        int64_t cnt = list_window(topo, N, R, query[t], (flags & ORC_INCLUDE_SELF) != 0, nb);
        double s = 0.0;
        for (int64_t q = 0; q < cnt; ++q) s += f[nb[q]];
        out[t] = s;
    }
    free(nb);
    return ORC_OK;
}

/* RHS of the listed nodes only (brute force), for sampled checks on networks too
 * large for a full oracle step: k_out[v * n_query + t] = f_v(x)[query[t]]. */
int orc_rhs_sampled(int model, int topo, int64_t N, int64_t R, const double *params, int n_params,
                    const double *node_param, const double *x, int64_t n_query,
                    const int64_t *query, double *k_out, int flags, int nthreads)
{
    int st = orc_validate(model, topo, N, R, n_params);
    if (st != ORC_OK) return st;
    int64_t nodes = orc_nodes(topo, N);
    int d = orc_dim(model);
    int64_t wmax = window_size(topo, R, 1);
    int nt = set_threads(nthreads);
    int failed = 0;
#pragma omp parallel num_threads(nt)
    {
        int64_t *nb = malloc(sizeof(int64_t) * (size_t)wmax);
        if (!nb) {
#pragma omp atomic write
            failed = 1;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (int64_t t = 0; t < n_query; ++t) {
                double kn[4];
                rhs_node(model, topo, N, R, params, node_param, x, kn, nodes, flags, query[t], nb);
                for (int v = 0; v < d; ++v) k_out[v * n_query + t] = kn[v];
            }
        }
        free(nb);
    }
    return failed ? ORC_ENOMEM : ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Dormand-Prince 5(4) (J. R. Dormand and P. J. Prince, "A family of embedded
 * Runge-Kutta formulae", J. Comput. Appl. Math. 6 (1980) 19-26; the RK5(4)7M
 * pair).  Seven stages, c_7 = 1 and a_7j = b_j, so the last stage is f(y_{n+1})
 * and serves as the first stage of the next step (first same as last). */
static const double DP_C[7] = {0.0, 1.0 / 5.0, 3.0 / 10.0, 4.0 / 5.0, 8.0 / 9.0, 1.0, 1.0};
static const double DP_A[7][6] = {
    {0, 0, 0, 0, 0, 0},
    {1.0 / 5.0, 0, 0, 0, 0, 0},
    {3.0 / 40.0, 9.0 / 40.0, 0, 0, 0, 0},
    {44.0 / 45.0, -56.0 / 15.0, 32.0 / 9.0, 0, 0, 0},
    {19372.0 / 6561.0, -25360.0 / 2187.0, 64448.0 / 6561.0, -212.0 / 729.0, 0, 0},
    {9017.0 / 3168.0, -355.0 / 33.0, 46732.0 / 5247.0, 49.0 / 176.0, -5103.0 / 18656.0, 0},
    {35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0}};
/* fifth-order weights (= the last row of A, b_7 = 0) and the embedded fourth-order ones */
static const double DP_B[7] = {35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0, 0.0};
static const double DP_BHAT[7] = {5179.0 / 57600.0, 0.0, 7571.0 / 16695.0, 393.0 / 640.0, -92097.0 / 339200.0,
                                  187.0 / 2100.0, 1.0 / 40.0};

/* The tableau, for checks of the order conditions: a is 7 x 7 row-major. */
void orc_dp5_tableau(double *a, double *b, double *bhat, double *c)
{
    for (int i = 0; i < 7; ++i) {
        for (int j = 0; j < 7; ++j) a[7 * i + j] = j < 6 ? DP_A[i][j] : 0.0;
        b[i] = DP_B[i];
        bhat[i] = DP_BHAT[i];
        c[i] = DP_C[i];
    }
}

/* Cubic Hermite interpolant on [t, t + h] from y0, y1 and the slopes f0, f1 at
 * both ends, at theta = (s - t) / h (textbook dense output of order 3). */
static double hermite(double y0, double y1, double f0, double f1, double h, double th)
{
    return (1.0 - th) * y0 + th * y1 +
           th * (th - 1.0) * ((1.0 - 2.0 * th) * (y1 - y0) + (th - 1.0) * h * f0 + th * h * f1);
}

/* Step-size controller constants (textbook values): safety factor, smallest and
 * largest factor per step, and the error exponent 1/5 of a 5(4) pair. */
#define DP_SAFE 0.9
#define DP_FACMIN 0.2
#define DP_FACMAX 10.0
/* At most this many dense outputs inside one step: the step is capped at
 * DP_MAX_OUT * out_dt. */
#define DP_MAX_OUT 8

/* Number of dense-output times t0 + k out_dt, k = 1..n, with t0 + k out_dt <= t_end
 * (up to a relative 1e-12 of the span, so that an end point on the grid counts). */
int64_t orc_dp5_n_out(double t0, double t_end, double out_dt)
{
    if (!(out_dt > 0.0)) return 0;
    return (int64_t)floor((t_end - t0) / out_dt * (1.0 + 1e-12));
}

/* Integrate y (d * nodes doubles, SoA) from t0 to t_end with the adaptive
 * Dormand-Prince 5(4) pair.
 *   Error of an attempted step of size h: e = h sum_j (b_j - bhat_j) k_j and
 *     err = sqrt(mean_q (e_q / sc_q)^2),  sc_q = atol + rtol max(|y_q|, |y_new,q|);
 *   the step is accepted when err <= 1 (a non-finite err is a rejection with
 *   factor 0.2).  New step h * clamp(0.9 err^(-1/5), 0.2, 10),
 *   not larger than h after a rejected attempt, and at most h_max (if > 0) and
 *   DP_MAX_OUT * out_dt (if out_dt > 0).  The attempt that reaches t_end is cut
 *   to t_end - t and ends exactly at t_end.
 *   Dense output (Kuramoto models): order_out[0] = R(t0) and order_out[k] = the
 *   order parameter of the Hermite-interpolated phases at t0 + k out_dt,
 *   k = 1..orc_dp5_n_out(t0, t_end, out_dt).
 *   stats (may be NULL): accepted, rejected attempts, final t, the next proposed
 *   step (before any cut at t_end).
 * Returns ORC_ESTEPS if max_attempts attempts did not reach t_end, ORC_ESMALL if
 * the step fell below 1e-14 (|t| + h), leaving y at the last accepted step. */
int orc_dp5(int model, int topo, int64_t N, int64_t R, const double *params, int n_params,
            const double *node_param, double *y, double t0, double t_end, double rtol, double atol,
            double h0, double h_max, double out_dt, int64_t max_attempts, double *order_out,
            int64_t *stats_i, double *stats_d, int flags, int nthreads)
{
    int st = orc_validate(model, topo, N, R, n_params);
    if (st != ORC_OK) return st;
    if (!(t_end > t0) || !(h0 > 0.0) || rtol < 0.0 || atol < 0.0 || !(rtol > 0.0 || atol > 0.0) ||
        h_max < 0.0 || out_dt < 0.0 || max_attempts < 1)
        return ORC_EINVAL;
    const int64_t nodes = orc_nodes(topo, N);
    const int64_t len = nodes * orc_dim(model);
    double *k[7], *tmp = malloc(sizeof(double) * (size_t)len), *ynew = malloc(sizeof(double) * (size_t)len);
    double *phi = malloc(sizeof(double) * (size_t)nodes);
    int bad = !tmp || !ynew || !phi;
    for (int s = 0; s < 7; ++s) {
        k[s] = malloc(sizeof(double) * (size_t)len);
        bad |= !k[s];
    }
    if (bad) {
        for (int s = 0; s < 7; ++s) free(k[s]);
        free(tmp); free(ynew); free(phi);
        return ORC_ENOMEM;
    }
    const int nt = set_threads(nthreads);
    const int has_order = model == ORC_KS || model == ORC_KSI;
    const int64_t n_out = orc_dp5_n_out(t0, t_end, out_dt);
    double hcap = h_max > 0.0 ? h_max : INFINITY;
    if (out_dt > 0.0 && DP_MAX_OUT * out_dt < hcap) hcap = DP_MAX_OUT * out_dt;
    if (order_out && has_order) order_out[0] = orc_order_parameter(nodes, y);

    double t = t0, h = h0 < hcap ? h0 : hcap;
    int64_t n_acc = 0, n_rej = 0, next_out = 1;
    int last_rejected = 0;
    st = orc_rhs(model, topo, N, R, params, n_params, node_param, y, k[0], flags, nt);
    while (st == ORC_OK) {
        if (n_acc + n_rej >= max_attempts) {
            st = ORC_ESTEPS;
            break;
        }
        const int last = t_end - t <= h;
        const double hs = last ? t_end - t : h;
        if (!(hs > 1e-14 * (fabs(t) + hs))) {
            st = ORC_ESMALL;
            break;
        }
        /* stages 2..7: stage input y + hs sum_{j<s} a_sj k_j */
        for (int s = 1; s < 7 && st == ORC_OK; ++s) {
            double *xin = s == 6 ? ynew : tmp;
            for (int64_t q = 0; q < len; ++q) {
                double acc = 0.0;
                for (int j = 0; j < s; ++j) acc += DP_A[s][j] * k[j][q];
                xin[q] = y[q] + hs * acc;
            }
            st = orc_rhs(model, topo, N, R, params, n_params, node_param, xin, k[s], flags, nt);
        }
        if (st != ORC_OK) break;
        /* error norm */
        double sum = 0.0;
        for (int64_t q = 0; q < len; ++q) {
            double e = 0.0;
            for (int j = 0; j < 7; ++j) e += (DP_B[j] - DP_BHAT[j]) * k[j][q];
            e *= hs;
            const double sc = atol + rtol * fmax(fabs(y[q]), fabs(ynew[q]));
            sum += (e / sc) * (e / sc);
        }
        const double err = sqrt(sum / (double)len);
        /* a non-finite error (the attempt overflowed) is a rejection with the
         * smallest factor; a zero error takes the largest */
        double fac = !isfinite(err) ? DP_FACMIN : err > 0.0 ? DP_SAFE * pow(err, -0.2) : DP_FACMAX;
        fac = fac < DP_FACMIN ? DP_FACMIN : (fac > DP_FACMAX ? DP_FACMAX : fac);
        if (err <= 1.0) {
            /* dense output inside (t, t + hs] */
            if (order_out && has_order) {
                while (next_out <= n_out) {
                    const double to = t0 + (double)next_out * out_dt;
                    if (!last && to > t + hs) break;
                    double th = (to - t) / hs;
                    th = th > 1.0 ? 1.0 : th;
                    for (int64_t q = 0; q < nodes; ++q) phi[q] = hermite(y[q], ynew[q], k[0][q], k[6][q], hs, th);
                    order_out[next_out] = orc_order_parameter(nodes, phi);
                    ++next_out;
                }
            }
            memcpy(y, ynew, sizeof(double) * (size_t)len);
            memcpy(k[0], k[6], sizeof(double) * (size_t)len);
            ++n_acc;
            double hn = h * fac;
            if (last_rejected && hn > h) hn = h;
            h = hn < hcap ? hn : hcap;
            last_rejected = 0;
            if (last) {
                t = t_end;
                break;
            }
            t = t + hs;
        } else {
            ++n_rej;
            h = hs * fac;
            last_rejected = 1;
        }
    }
    if (stats_i) {
        stats_i[0] = n_acc;
        stats_i[1] = n_rej;
    }
    if (stats_d) {
        stats_d[0] = t;
        stats_d[1] = h;
    }
    for (int s = 0; s < 7; ++s) free(k[s]);
    free(tmp); free(ynew); free(phi);
    return st;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 2 (Section III.C): differential compression of the link matrix.
 * A row is the sorted set of positions of its set bits.  ROL by i moves bit p to
 * (p - i) mod N; XOR of two rows is the symmetric difference of the sets.
 *   COMPRESS: V = row 0; for each row i, d = XOR(ROL(row_i, i), V); C_i is the
 *   index of d in the difference table D (d is appended if new).
 *   EXTRACT(i) = ROR(XOR(V, D[C_i]), i), ROR by i moving bit p to (p + i) mod N.
 * Outputs (caller-allocated, sizes from a first call with NULL outputs):
 *   v[n_v], the sorted set V; d_ptr[n_d + 1] and d_pos[d_ptr[n_d]], the table D;
 *   c[n] the entry of every row.  Returns n_d, or -1 on invalid input. */
static int cmp_i64(const void *a, const void *b)
{
    const int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return x < y ? -1 : (x > y);
}

/* symmetric difference of two sorted sets; returns its size */
static int64_t sym_diff(const int64_t *a, int64_t na, const int64_t *b, int64_t nb, int64_t *out)
{
    int64_t i = 0, j = 0, c = 0;
    while (i < na || j < nb) {
        if (j >= nb || (i < na && a[i] < b[j])) out[c++] = a[i++];
        else if (i >= na || b[j] < a[i]) out[c++] = b[j++];
        else { ++i; ++j; }
    }
    return c;
}

int64_t orc_compress(int64_t n, const int64_t *row_ptr, const int64_t *col, int64_t *n_v, int64_t *v,
                     int64_t *d_ptr, int64_t *d_pos, int64_t *c)
{
    if (n < 1) return -1;
    int64_t maxrow = 0;
    for (int64_t i = 0; i < n; ++i)
        if (row_ptr[i + 1] - row_ptr[i] > maxrow) maxrow = row_ptr[i + 1] - row_ptr[i];
    const int64_t nv = row_ptr[1] - row_ptr[0];
    int64_t *V = malloc(sizeof(int64_t) * (size_t)(nv + 1));
    int64_t *sh = malloc(sizeof(int64_t) * (size_t)(maxrow + 1));
    int64_t *d = malloc(sizeof(int64_t) * (size_t)(maxrow + nv + 1));
    /* the difference table, grown as needed */
    int64_t cap_e = 16, cap_p = 1024, ne = 0;
    int64_t *eptr = malloc(sizeof(int64_t) * (size_t)(cap_e + 1));
    int64_t *epos = malloc(sizeof(int64_t) * (size_t)cap_p);
    if (!V || !sh || !d || !eptr || !epos) {
        free(V); free(sh); free(d); free(eptr); free(epos);
        return -1;
    }
    for (int64_t t = 0; t < nv; ++t) V[t] = col[row_ptr[0] + t];
    qsort(V, (size_t)nv, sizeof(int64_t), cmp_i64);
    eptr[0] = 0;
    int64_t result = 0;
    for (int64_t i = 0; i < n && result >= 0; ++i) {
        const int64_t len = row_ptr[i + 1] - row_ptr[i];
        for (int64_t t = 0; t < len; ++t) sh[t] = wrap(col[row_ptr[i] + t] - i, n); /* ROL by i */
        qsort(sh, (size_t)len, sizeof(int64_t), cmp_i64);
        const int64_t nd = sym_diff(sh, len, V, nv, d); /* XOR with V */
        int64_t found = -1;
        for (int64_t e = 0; e < ne && found < 0; ++e) /* FIND in the table */
            if (eptr[e + 1] - eptr[e] == nd && memcmp(epos + eptr[e], d, sizeof(int64_t) * (size_t)nd) == 0)
                found = e;
        if (found < 0) {
            if (ne == cap_e) {
                cap_e *= 2;
                int64_t *q = realloc(eptr, sizeof(int64_t) * (size_t)(cap_e + 1));
                if (!q) { result = -1; break; }
                eptr = q;
            }
            while (eptr[ne] + nd > cap_p) {
                cap_p *= 2;
                int64_t *q = realloc(epos, sizeof(int64_t) * (size_t)cap_p);
                if (!q) { result = -1; break; }
                epos = q;
            }
            if (result < 0) break;
            memcpy(epos + eptr[ne], d, sizeof(int64_t) * (size_t)nd);
            eptr[ne + 1] = eptr[ne] + nd;
            found = ne++;
        }
        if (c) c[i] = found;
    }
    if (result >= 0) {
        *n_v = nv;
        if (v) memcpy(v, V, sizeof(int64_t) * (size_t)nv);
        if (d_ptr) memcpy(d_ptr, eptr, sizeof(int64_t) * (size_t)(ne + 1));
        if (d_pos) memcpy(d_pos, epos, sizeof(int64_t) * (size_t)eptr[ne]);
        result = ne;
    }
    free(V); free(sh); free(d); free(eptr); free(epos);
    return result;
}

/* EXTRACT(i): writes the sorted links of row i into row (at most n_v plus the
 * entry's size values) and returns their count. */
int64_t orc_extract(int64_t n, int64_t i, int64_t n_v, const int64_t *v, const int64_t *d_ptr,
                    const int64_t *d_pos, const int64_t *c, int64_t *row)
{
    const int64_t e = c[i];
    const int64_t cnt = sym_diff(v, n_v, d_pos + d_ptr[e], d_ptr[e + 1] - d_ptr[e], row); /* XOR */
    for (int64_t t = 0; t < cnt; ++t) row[t] = wrap(row[t] + i, n); /* ROR by i */
    qsort(row, (size_t)cnt, sizeof(int64_t), cmp_i64);
    return cnt;
}
