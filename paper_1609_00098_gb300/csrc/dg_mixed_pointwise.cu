// dg_mixed_pointwise.cu -- node-wise kernels of the mixed-precision path: the
// CFL pass: FP32 primitives of U^n, the largest wave speed, and the pressures
// that warm-start the first stage's con2prim.
#include "dg_mixed.cuh"

namespace dg {

namespace {

constexpr int kThreads = 256;

template <int SYS>
__global__ void __launch_bounds__(kThreads) k_cfl_mixed(const double *Un, const float *pin, float *pout,
                                                        unsigned long long *lam, unsigned int *err, long long total,
                                                        int nn, float gamma, double gamma_d, float kappa_sw,
                                                        double d_atm, double tau_atm)
{
    float lmax = 0.0f;
    unsigned errs = 0;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        const long long e = g / nn;
        const int q = (int)(g - e * nn);
        float u[5], P[NPRIM];
#pragma unroll
        for (int v = 0; v < 5; ++v) u[v] = f64_to_f32(Un[(e * 5 + v) * nn + q]);
        if (SYS == 0) {
            ne_primitives32(gamma, u, P);
        } else {
            errs |= sr_prims_mixed(gamma, gamma_d, kappa_sw, d_atm, tau_atm, u, Un + e * 5 * nn + q, nn,
                                   pin ? pin[g] : -1.0f, P);
            pout[g] = P[3];
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float lo, hi;
            speeds_axis32<SYS>(gamma, u, P, a, lo, hi);
            lmax = fmaxf(lmax, fmaxf(fabsf(lo), fabsf(hi)));
        }
    }
    if (errs) atomicOr(err, errs);
    __shared__ float red[kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lmax;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = red[0];
        for (int w = 1; w < kThreads / 32; ++w) m = fmaxf(m, red[w]);
        atomicMax(lam, (unsigned long long)__double_as_longlong(f32_to_f64(m)));
    }
}

unsigned grid_for(long long count)
{
    long long b = (count + kThreads - 1) / kThreads;
    if (b > 152LL * 64) b = 152LL * 64;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_cfl_mixed(const dg_mesh *m, const double *Un, const float *pin, float *pout, float kappa_sw,
                             cudaStream_t s)
{
    const long long total = m->E * m->nn;
    if (m->d.system == 0)
        k_cfl_mixed<0><<<grid_for(total), kThreads, 0, s>>>(Un, pin, pout, m->lam, m->err, total, m->nn,
                                                            (float)m->d.gamma, m->d.gamma, kappa_sw, m->d.d_atm,
                                                            m->d.tau_atm);
    else
        k_cfl_mixed<1><<<grid_for(total), kThreads, 0, s>>>(Un, pin, pout, m->lam, m->err, total, m->nn,
                                                            (float)m->d.gamma, m->d.gamma, kappa_sw, m->d.d_atm,
                                                            m->d.tau_atm);
    return cudaGetLastError();
}

}  // namespace dg
