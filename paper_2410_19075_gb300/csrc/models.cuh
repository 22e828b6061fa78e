// Node right-hand sides evaluated from exact window sums (FP64).
//
// Every model is written as: a coupled quantity f(x) of a node's stage input
// (the "exchange" variables of the paper's memory layout, Section III.B), whose
// window sums W = sum_{j in window incl. self} Q(f_j) arrive as exact
// fixed-point integers, and a local right-hand side.
#pragma once
#include "common.cuh"
#include "fastmath.cuh"

namespace simk {

// coupled_q() rounds a node's coupled quantity f(x) onto the grid 2^-F (sin and
// cos of the phase through the integer-only fixed_sincos for the Kuramoto
// models; u, v or V themselves otherwise), checking |f| < 2^lim (ok = false
// outside it or for a non-finite value).
// Every rhs() takes the node's window sums W; on a general link matrix it also
// takes the node's link count (wsize, the FHN/HH self-term multiplier; -1 = the
// network's) and a coupling scale cs = 1/K_i applied to the converted sums (the
// constants c then carry K = 1).  The ring and lattice paths use the defaults.

// Derived constants, computed once on the host in FP64.
struct ModelParams {
    double c[8];
    int64_t q[2];     // Kuramoto models: cos alpha and sin alpha on the grid 2^-62
    uint64_t a0[2];   // Kuramoto models: alpha = aq pi/2 + alpha0, alpha0 in [0, pi/2):
    int aq;           //   cos alpha0, sin alpha0 on the grid 2^-63 (non-negative), aq in 0..3
    int ksh;          // Kuramoto rings: right shift taking the exact window sums into int64
    MathTables tab;   // device tables of the fast elementary functions
    int64_t wsize;    // window size including the node itself (2R+1 or (2P+1)^3)
    int include_self; // 1: the node is one of its own links
};

template <int M> struct Model;

// Kuramoto coupling on a lattice.  On the ball and disk the window sums arrive
// rotated by -alpha: W' = W'c + i W's = sum over the window (the node itself
// included) of e^{-i alpha} Q(e^{i phi_j}), int64 on the grid 2^-F (their x pass
// rotates every node's quantity).  The cube keeps its sums unrotated and turns
// the node's own phase by +alpha instead (own_phase_turned), which gives the
// same T.  Then
//   T = Im[e^{-i phi_i} W'] = cos(phi_i) W's - sin(phi_i) W'c
//     = sum_j sin(phi_j - phi_i - alpha)   (the node's own term is -sin alpha),
// two 64 x 64 high products of the node's own (sin, cos) on the grid 2^-62 with
// the sums, on the grid 2^-(F-2).  The caller converts T once (correctly
// rounded, the grid's power of two folded into c[5]); the window without the
// node itself is T + sin alpha, the constant folded into c[4] on the host
// (quantisation makes the node's own rotated term differ from -sin alpha by a
// few units of 2^-F).
__device__ __forceinline__ double lattice_coupling(const int64_t (&f62)[2], int64_t W0, int64_t W1)
{
    return __ll2double_rn(mulhi_ss(f62[1], W0) - mulhi_ss(f62[0], W1));
}

// The node's own (sin, cos) on the grid 2^-62 turned by +alpha = aq pi/2 +
// alpha0: e^{i alpha0} (c + i s) by four high products with the non-negative cos
// alpha0, sin alpha0 (grid 2^-63, landing on 2^-61), back onto 2^-62 by one bit
// (|values| <= 1, so they stay below 2^62 + 2), then aq quarter turns.  With
// the turned phase the cross product of lattice_coupling takes the unrotated
// window sums: Im[e^{-i(phi + alpha)} S] = Im[e^{-i phi} e^{-i alpha} S] (the
// cube; the ball and disk rotate their sums instead).
__device__ __forceinline__ void own_phase_turned(const ModelParams &P, const int64_t (&f62)[2], int64_t (&t62)[2])
{
    const int64_t s = f62[0], c = f62[1];
    const int64_t c1 = mulhi_su(c, P.a0[0]) - mulhi_su(s, P.a0[1]);
    const int64_t s1 = mulhi_su(s, P.a0[0]) + mulhi_su(c, P.a0[1]);
    int64_t ca, sa;
    switch (P.aq) { // times i^aq
    case 0: ca = c1; sa = s1; break;
    case 1: ca = -s1; sa = c1; break;
    case 2: ca = -c1; sa = -s1; break;
    default: ca = s1; sa = -c1; break;
    }
    t62[0] = (int64_t)((uint64_t)sa << 1);
    t62[1] = (int64_t)((uint64_t)ca << 1);
}

// Both Kuramoto models' coupling term on a lattice, c[5] T + c[4] (the whole
// slope of the plain model, the coupling part of dpsi/dt with inertia).
__device__ __forceinline__ double lattice_coupling_term(const ModelParams &P, const int64_t (&f62)[2], int64_t W0,
                                                        int64_t W1)
{
    return fma(P.c[5], lattice_coupling(f62, W0, W1), P.c[4]);
}

// Kuramoto coupling on a ring or a link matrix: T = Im[e^{-i(phi+alpha)} S] =
// cos(phi+alpha) S_sin - sin(phi+alpha) S_cos, with S the exact window sum
// (int128 on the grid 2^-F; without the node itself unless it is one of its own
// links) shifted right by sh bits into int64, and (cos, sin)(phi + alpha) from
// the node's own grid values by the angle-addition formula: four high products
// with the non-negative cos alpha0, sin alpha0 (grid 2^-61), then aq quarter
// turns.  Two signed high products give T on the grid 2^-(F - sh - 3).  No FP64
// instruction and no conversion until the caller's single one.
__device__ __forceinline__ int64_t ring_coupling(const ModelParams &P, const int64_t (&qo)[2], int F,
                                                 const i128 (&W)[2], int sh)
{
    const i128 ss = P.include_self ? W[0] : W[0] - (i128)qo[0];
    const i128 sc = P.include_self ? W[1] : W[1] - (i128)qo[1];
    const int64_t S_s = (int64_t)(ss >> sh), S_c = (int64_t)(sc >> sh);
    const int64_t s = qo[0] * (int64_t(1) << (62 - F)), c = qo[1] * (int64_t(1) << (62 - F));
    const int64_t c1 = mulhi_su(c, P.a0[0]) - mulhi_su(s, P.a0[1]); // e^{i alpha0} (c + i s), grid 2^-61
    const int64_t s1 = mulhi_su(s, P.a0[0]) + mulhi_su(c, P.a0[1]);
    int64_t ca, sa;
    switch (P.aq) { // times i^aq
    case 0: ca = c1; sa = s1; break;
    case 1: ca = -s1; sa = c1; break;
    case 2: ca = -c1; sa = -s1; break;
    default: ca = s1; sa = -c1; break;
    }
    return mulhi_ss(ca, S_s) - mulhi_ss(sa, S_c);
}

// The shift and the scale of ring_coupling's T for a window of ws links (the
// node itself included or not): sh = max(0, ceil(log2 ws) + F - 61) keeps
// |S >> sh| < 2^62; the returned scale is coef 2^(sh + 3 - F), with coef the
// coupling constant (times the link-matrix node's 1/K_i).
__device__ __forceinline__ double ring_coupling_scale(int64_t ws, int F, double coef, int &sh)
{
    const int lg = ws > 1 ? 64 - __clzll((long long)(ws - 1)) : 0;
    sh = lg + F - 61 > 0 ? lg + F - 61 : 0;
    // coef 2^(sh + 3 - F) by the exponent field (coef is a normal double, the
    // power of two keeps it one)
    return __longlong_as_double(__double_as_longlong(coef) + ((long long)(sh + 3 - F) << 52));
}

// Kuramoto-Sakaguchi, Eq. (3) with m = 0, eps = 1 (Algorithm 1):
//   dphi_i/dt = omega - (mu/K) sum_{j in W(i)} sin(phi_i - phi_j + alpha)
//             = omega + (mu/K) [cos(phi_i+alpha) S_sin - sin(phi_i+alpha) S_cos],
// S_sin = sum_j sin phi_j, S_cos = sum_j cos phi_j (angle-difference identity,
// so the window only needs sums of sin and cos).
// c = {omega, mu/K, sin alpha, cos alpha}, q = {cos alpha, sin alpha} on the grid
// 2^-62.  Coupled quantity (sin phi, cos phi).
template <> struct Model<0> {
    static constexpr int D = 1, NQ = 2, NX = 0, F = 53;
    __device__ __forceinline__ static void coupled_q(const ModelParams &P, const double (&x)[D], int F, int,
                                                     bool &ok, int64_t (&q)[NQ])
    {
        int64_t s62, c62;
        fixed_sincos(x[0], P.tab, s62, c62, ok);
        q[0] = q62_to(s62, F);
        q[1] = q62_to(c62, F);
    }
    // Rings and link matrices: c[5] = (mu/K) 2^(ksh + 3 - F) (rings; a link
    // matrix's node of wsize links scales mu cs instead).
    __device__ __forceinline__ static void rhs(const ModelParams &P, int F_, const double (&)[NQ],
                                               const int64_t (&qo)[NQ], const i128 (&W)[NQ],
                                               const double *, double, double (&k)[D],
                                               int64_t wsize = -1, double cs = 1.0, const int64_t * = nullptr)
    {
        int sh = P.ksh;
        const double sc = wsize < 0 ? P.c[5] : ring_coupling_scale(wsize, F_, P.c[1] * cs, sh);
        k[0] = fma(sc, __ll2double_rn(ring_coupling(P, qo, F_, W, sh)), P.c[0]);
    }
    // Lattices: c[4] = omega + (mu/K) sin alpha (omega with the node itself as a
    // link), c[5] = (mu/K) 2^-(F-2).
    __device__ __forceinline__ static void rhs_lattice(const ModelParams &P, const int64_t (&f62)[2], int64_t W0,
                                                       int64_t W1, const double *, double (&k)[D])
    {
        k[0] = lattice_coupling_term(P, f62, W0, W1);
    }
    __device__ __forceinline__ static void rhs_from_coupling(const ModelParams &, double c, const double *,
                                                             double (&k)[D])
    {
        k[0] = c;
    }
};

// FitzHugh-Nagumo, Eq. (2) with tau = 0, D = 0, I_app = 0 and the rotational
// coupling matrix B = [[b00, b01], [b10, b11]] = [[cos p, sin p], [-sin p, cos p]]:
//   du/dt = (u - u^3/3 - v + (sigma/K) [b00 Cu + b01 Cv]) / eps
//   dv/dt =  u + a        + (sigma/K) [b10 Cu + b11 Cv]
// with Cu = sum_{j in W(i)} (u_j - u_i) = W_u - wsize * Q(u_i), exact in fixed point.
// c = {1/eps, a, (sigma/K) b00/eps, (sigma/K) b01/eps, (sigma/K) b10, (sigma/K) b11}
// (constants folded on the host so that the RHS costs 9 FP64 instructions).
// Coupled quantity (u, v).
template <> struct Model<1> {
    static constexpr int D = 2, NQ = 2, NX = 0, F = 51;
    __device__ __forceinline__ static void coupled_q(const ModelParams &, const double (&x)[D], int F, int lim,
                                                     bool &ok, int64_t (&q)[NQ])
    {
        q[0] = to_fixed(x[0], F, lim, ok);
        q[1] = to_fixed(x[1], F, lim, ok);
    }
    __device__ __forceinline__ static void rhs(const ModelParams &P, int F_, const double (&fo)[NQ],
                                               const int64_t (&qo)[NQ], const i128 (&W)[NQ],
                                               const double *X, double Iext, double (&k)[D],
                                               int64_t wsize = -1, double cs = 1.0, const int64_t * = nullptr)
    {
        const int64_t ws = wsize < 0 ? P.wsize : wsize;
        const double Cu = cs * fixed_to_double_wide(W[0] - (i128)qo[0] * ws, F_);
        const double Cv = cs * fixed_to_double_wide(W[1] - (i128)qo[1] * ws, F_);
        const double u = fo[0], v = fo[1];
        const double w = fma(u * u, -1.0 / 3.0, 1.0);      // 1 - u^2/3
        const double local = fma(u, w, -v);                // u - u^3/3 - v
        k[0] = fma(P.c[0], local, fma(P.c[2], Cu, P.c[3] * Cv));
        k[1] = fma(P.c[4], Cu, fma(P.c[5], Cv, u + P.c[1]));
    }
};

// Hodgkin-Huxley, Eq. (1) as the classic neuron (V, m, h, n), textbook rates
// (V in mV, rates in 1/ms, rest near -65 mV):
//   Cm dV/dt = I_ext - gNa m^3 h (V-ENa) - gK n^4 (V-EK) - gL (V-EL) + (g/K) CV
//   dx/dt    = alpha_x(V) (1-x) - beta_x(V) x,   x in {m, h, n}
// with CV = sum_{j in W(i)} (V_j - V_i) = W_V - wsize * Q(V_i), exact in fixed point.
// c = {1/Cm, gNa, gK, gL, ENa, EK, EL, g/K}.  Coupled quantity V; the gates are
// local variables.  Rates use the table-driven exp and reciprocal of fastmath.cuh.
template <> struct Model<2> {
    static constexpr int D = 4, NQ = 1, NX = 3, F = 46;
    __device__ __forceinline__ static void coupled_q(const ModelParams &, const double (&x)[D], int F, int lim,
                                                     bool &ok, int64_t (&q)[NQ])
    {
        q[0] = to_fixed(x[0], F, lim, ok);
    }
    __device__ __forceinline__ static void rhs(const ModelParams &P, int F_, const double (&fo)[NQ],
                                               const int64_t (&qo)[NQ], const i128 (&W)[NQ],
                                               const double *X, double Iext, double (&k)[D],
                                               int64_t wsize = -1, double cs = 1.0, const int64_t * = nullptr)
    {
        const int64_t ws = wsize < 0 ? P.wsize : wsize;
        const double CV = cs * fixed_to_double_wide(W[0] - (i128)qo[0] * ws, F_);
        const double V = fo[0], m = X[0], h = X[1], n = X[2];
        const MathTables &T = P.tab;
        const double am = fast_x_over_1mexp(fma(V, 0.1, 4.0), T);                    // (V+40)/10
        const double bm = 4.0 * fast_exp(fma(V, -1.0 / 18.0, -65.0 / 18.0), T);     // -(V+65)/18
        const double ah = 0.07 * fast_exp(fma(V, -0.05, -3.25), T);                 // -(V+65)/20
        const double bh = fast_rcp(1.0 + fast_exp(fma(V, -0.1, -3.5), T));          // -(V+35)/10
        const double an = 0.1 * fast_x_over_1mexp(fma(V, 0.1, 5.5), T);             // (V+55)/10
        const double bn = 0.125 * fast_exp(fma(V, -0.0125, -0.8125), T);            // -(V+65)/80
        const double m3h = m * m * m * h, n4 = (n * n) * (n * n);
        const double I = Iext - P.c[1] * m3h * (V - P.c[4]) - P.c[2] * n4 * (V - P.c[5]) -
                         P.c[3] * (V - P.c[6]) + P.c[7] * CV;
        k[0] = I * P.c[0];
        k[1] = am * (1.0 - m) - bm * m;
        k[2] = ah * (1.0 - h) - bh * h;
        k[3] = an * (1.0 - n) - bn * n;
    }
};

// Kuramoto-Sakaguchi with inertia, Eq. (3) with m != 0, as a first-order system:
//   dphi/dt = psi,   dpsi/dt = ((mu/K) sum_{j in W(i)} sin(phi_j - phi_i - alpha) - eps psi) / m
// with sum_j sin(phi_j - phi_i - alpha) = cos(phi_i+alpha) S_sin - sin(phi_i+alpha) S_cos.
// c = {mu/(m K), eps/m, sin alpha, cos alpha}, q as for Model<0>.  Coupled
// quantity (sin phi, cos phi);
// psi is a local variable.
template <> struct Model<3> {
    static constexpr int D = 2, NQ = 2, NX = 1, F = 53;
    __device__ __forceinline__ static void coupled_q(const ModelParams &P, const double (&x)[D], int F, int,
                                                     bool &ok, int64_t (&q)[NQ])
    {
        int64_t s62, c62;
        fixed_sincos(x[0], P.tab, s62, c62, ok);
        q[0] = q62_to(s62, F);
        q[1] = q62_to(c62, F);
    }
    // Rings and link matrices: c[5] = (mu/(m K)) 2^(ksh + 3 - F).
    __device__ __forceinline__ static void rhs(const ModelParams &P, int F_, const double (&)[NQ],
                                               const int64_t (&qo)[NQ], const i128 (&W)[NQ],
                                               const double *X, double, double (&k)[D],
                                               int64_t wsize = -1, double cs = 1.0, const int64_t * = nullptr)
    {
        int sh = P.ksh;
        const double sc = wsize < 0 ? P.c[5] : ring_coupling_scale(wsize, F_, P.c[0] * cs, sh);
        const double psi = X[0];
        k[0] = psi;
        k[1] = fma(sc, __ll2double_rn(ring_coupling(P, qo, F_, W, sh)), -P.c[1] * psi);
    }
    // Lattices: c[4] = (mu/(m K)) sin alpha (0 with the node itself as a link),
    // c[5] = (mu/(m K)) 2^-(F-2).  The coupling term first, then the damping
    // (the order of the split cube node pass, which takes the coupling term
    // from the window pass).
    __device__ __forceinline__ static void rhs_lattice(const ModelParams &P, const int64_t (&f62)[2], int64_t W0,
                                                       int64_t W1, const double *X, double (&k)[D])
    {
        k[0] = X[0];
        k[1] = fma(-P.c[1], X[0], lattice_coupling_term(P, f62, W0, W1));
    }
    // The slope from the coupling term c of lattice_coupling_term.
    __device__ __forceinline__ static void rhs_from_coupling(const ModelParams &P, double c, const double *X,
                                                             double (&k)[D])
    {
        k[0] = X[0];
        k[1] = fma(-P.c[1], X[0], c);
    }
};

} // namespace simk
