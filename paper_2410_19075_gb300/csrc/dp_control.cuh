// Step-size control of the adaptive Dormand-Prince 5(4) runs (rings in dp5.cu,
// lattices in lattice_dp.cu): the decision one thread takes after an attempt's
// error norm and dense-output sums have been reduced.
#pragma once
#include "internal.h"

namespace simk {

// Dormand and Prince (1980), the RK5(4)7M pair.  Row s (0-based stage) holds the
// weights of k_1..k_s in the input of stage s + 1; row 6 is the fifth-order
// solution.  c_dp_e = b - bhat (b the fifth-order weights, bhat the embedded
// fourth-order ones).
__constant__ double c_dp_a[7][6] = {
    {0, 0, 0, 0, 0, 0},
    {1.0 / 5.0, 0, 0, 0, 0, 0},
    {3.0 / 40.0, 9.0 / 40.0, 0, 0, 0, 0},
    {44.0 / 45.0, -56.0 / 15.0, 32.0 / 9.0, 0, 0, 0},
    {19372.0 / 6561.0, -25360.0 / 2187.0, 64448.0 / 6561.0, -212.0 / 729.0, 0, 0},
    {9017.0 / 3168.0, -355.0 / 33.0, 46732.0 / 5247.0, 49.0 / 176.0, -5103.0 / 18656.0, 0},
    {35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0}};
__constant__ double c_dp_e[7] = {71.0 / 57600.0, 0.0, -71.0 / 16695.0, 71.0 / 1920.0, -17253.0 / 339200.0,
                                 22.0 / 525.0, -1.0 / 40.0};

// Step-size controller: safety factor, smallest and largest factor per step.
constexpr double kDpSafe = 0.9, kDpFacMin = 0.2, kDpFacMax = 10.0;

// Where the decision records the dense order parameters.
struct DpRecord {
    double *obs;              // ring buffer of order parameters (nullptr: none)
    int64_t obs_cap;
    unsigned long long *obs_ctr;
    int F;                    // fixed-point grid of the dense sums
    int64_t nodes;
};

// err = sqrt(esum / n_values) (infinite if the attempt left the fixed-point
// range); accept when err <= 1, set the next step, record the n_here dense order
// parameters of an accepted attempt, and decide whether the run is done.
// Returns 1 if the attempt was accepted.
__device__ __forceinline__ int dp_decide_ctl(DpCtl *ctl, int *remaining, double esum, int64_t n_values, int n_here,
                                             const i128 (*out_tot)[2], const DpRecord &rec)
{
    DpCtl c = *ctl;
    // an attempt whose stage inputs left the fixed-point range is rejected like
    // one whose error is not finite
    const double err = c.bad ? INFINITY : sqrt(esum / (double)n_values);
    c.bad = 0;
    double fac = !isfinite(err) ? kDpFacMin : err > 0.0 ? kDpSafe * pow(err, -0.2) : kDpFacMax;
    fac = fac < kDpFacMin ? kDpFacMin : (fac > kDpFacMax ? kDpFacMax : fac);
    const int accepted = err <= 1.0;
    if (accepted) {
        for (int o = 0; o < n_here && rec.obs; ++o) {
            const double S = fixed_to_double(out_tot[o][0], rec.F), C = fixed_to_double(out_tot[o][1], rec.F);
            const unsigned long long n = *rec.obs_ctr;
            rec.obs[n % (unsigned long long)rec.obs_cap] = sqrt(S * S + C * C) / (double)rec.nodes;
            *rec.obs_ctr = n + 1;
        }
        c.next_out += n_here;
        c.cur ^= 1;
        ++c.n_acc;
        double hn = c.h * fac;
        if (c.last_rej && hn > c.h) hn = c.h;
        c.h = hn < c.hcap ? hn : c.hcap;
        c.last_rej = 0;
        if (c.last) {
            c.t = c.t_end;
            c.done = 1;
        } else {
            c.t = c.t + c.h_att;
        }
    } else {
        ++c.n_rej;
        c.h = c.h_att * fac;
        c.last_rej = 1;
    }
    if (!c.done) {
        if (c.n_acc + c.n_rej >= c.max_att) {
            c.done = 1;
            c.status = kDpStatusSteps;
        } else {
            c.last = c.t_end - c.t <= c.h;
            c.h_att = c.last ? c.t_end - c.t : c.h;
            if (!(c.h_att > 1e-14 * (fabs(c.t) + c.h_att))) {
                c.done = 1;
                c.status = kDpStatusSmall;
            }
        }
    }
    c.acc_flag = accepted;
    *ctl = c;
    if (c.done) atomicSub(remaining, 1);
    return accepted;
}

} // namespace simk
