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
enum { ORC_RING = 0, ORC_CUBE = 1, ORC_BALL = 2, ORC_DISK = 3 };
enum { ORC_REVERSE = 1, ORC_INCLUDE_SELF = 2 };
enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ENOMEM = -2 };

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
    return N;
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
    if (topo < ORC_RING || topo > ORC_DISK) return ORC_EINVAL;
    if (n_params != n_params_of(model)) return ORC_EINVAL;
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
    if (topo == ORC_RING) {
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
    int64_t first = 0, last = cnt, step = 1;
    if (flags & ORC_REVERSE) { first = cnt - 1; last = -1; step = -1; }

    if (model == ORC_KS) {
        double omega = p[0], mu = p[1], alpha = p[2];
        double phi_i = x[i], sum = 0.0;
        for (int64_t t = first; t != last; t += step)
            sum += sin(phi_i - x[nb[t]] + alpha);
        k[0] = omega - (mu / K) * sum;
    } else if (model == ORC_KSI) {
        /* Eq. (3) with inertia: m phi'' + eps phi' = (mu/K) sum_j sin(phi_j - phi_i - alpha),
         * as the first-order system phi' = psi, psi' = ((mu/K) sum_j ... - eps psi) / m. */
        double m = p[0], eps = p[1], mu = p[2], alpha = p[3];
        const double *phi = x, *psi = x + nodes;
        double phi_i = phi[i], sum = 0.0;
        for (int64_t t = first; t != last; t += step)
            sum += sin(phi[nb[t]] - phi_i - alpha);
        k[0] = psi[i];
        k[1] = ((mu / K) * sum - eps * psi[i]) / m;
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
        k[0] = (ui - ui * ui * ui / 3.0 - vi + (sigma / K) * cu) / eps;
        k[1] = ui + a + (sigma / K) * cv;
    } else { /* ORC_HH */
        double Cm = p[0], gNa = p[1], gK = p[2], gL = p[3];
        double ENa = p[4], EK = p[5], EL = p[6], g = p[7];
        const double *V = x, *m = x + nodes, *h = x + 2 * nodes, *n = x + 3 * nodes;
        double Vi = V[i], mi = m[i], hi = h[i], ni = n[i];
        double sumV = 0.0;
        for (int64_t t = first; t != last; t += step) sumV += V[nb[t]];
        double coupling = g * (sumV / K - Vi);
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
