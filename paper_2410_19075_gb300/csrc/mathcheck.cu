// Tables of the fast elementary functions, and sim_math_eval(): evaluation of
// those device routines on caller-given arguments, so that their accuracy can
// be checked against a reference libm.
#include <cmath>
#include <vector>

#include "internal.h"
#include "sim.h"

namespace simk {

void fill_math_tables(double *block)
{
    const long double pi = 3.141592653589793238462643383279502884L;
    double *sincos = block, *exp2j = block + 2 * kSinTab;
    int64_t *sincos_q = reinterpret_cast<int64_t *>(block + 2 * kSinTab + kExpTab);
    for (int j = 0; j < kSinTab; ++j) {
        const long double a = pi * (long double)j / 512.0L;
        sincos[2 * j] = (double)sinl(a);
        sincos[2 * j + 1] = (double)cosl(a);
        sincos_q[2 * j] = (int64_t)llroundl(sinl(a) * 4611686018427387904.0L); // 2^62
        sincos_q[2 * j + 1] = (int64_t)llroundl(cosl(a) * 4611686018427387904.0L);
    }
    for (int j = 0; j < kExpTab; ++j) exp2j[j] = (double)exp2l((long double)j / 64.0L);
}

__global__ void math_eval_kernel(int fn, const double *x, double *out, int64_t n, MathTables T)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = x[i];
    double r = 0.0, s, c;
    switch (fn) {
    case 0: fast_sincos(v, T, s, c); r = s; break;
    case 1: fast_sincos(v, T, s, c); r = c; break;
    case 2: r = fast_exp(v, T); break;
    case 3: r = fast_rcp(v); break;
    default: r = fast_x_over_1mexp(v, T); break;
    }
    out[i] = r;
}

} // namespace simk

using namespace simk;

extern "C" int sim_math_eval(int fn, const double *host_x, double *host_out, int64_t n)
{
    if (fn < 0 || fn > 4 || n < 0 || (n > 0 && (!host_x || !host_out))) return SIM_EINVAL;
    if (n == 0) return SIM_OK;
    std::vector<double> tab(kMathTableWords);
    fill_math_tables(tab.data());
    double *d = nullptr;
    const size_t bytes = sizeof(double) * (tab.size() + 2 * (size_t)n);
    if (cudaMalloc(&d, bytes) != cudaSuccess) {
        cudaGetLastError();
        return SIM_ENOMEM;
    }
    double *dtab = d, *dx = d + tab.size(), *dout = dx + n;
    cudaError_t e = cudaMemcpy(dtab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dx, host_x, sizeof(double) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        const MathTables T = math_tables_at(dtab);
        math_eval_kernel<<<(unsigned)((n + 255) / 256), 256>>>(fn, dx, dout, n, T);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(host_out, dout, sizeof(double) * n, cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e == cudaSuccess ? SIM_OK : SIM_EDEVICE;
}
