// dg_mixed_pointwise.cu -- node-wise kernels of the mixed-precision path: the
// CFL pass: FP32 primitives of U^n, the largest wave speed, and the pressures
// that warm-start the first stage's con2prim.
#include <cstring>

#include "dg_mixed.cuh"

namespace dg {

namespace {

constexpr int kThreads = 256;

struct CflArgs {
    const double *Un;
    const float *pin;              // previous pass's pressures (guesses), or nullptr
    float *pout;                   // this pass's pressures, or nullptr
    unsigned long long *lam;
    unsigned int *err;
    long long total;
    int nn;
    float gamma;
    double gamma_d;
    float kappa_sw;
    double d_atm, tau_atm;
    const float *netP;             // learned-guess network, or nullptr
    const __nv_bfloat16 *netW2;
    float net_sc[6];
};

// Shared memory of the learned-guess variant: weights, features, guesses.
struct CflNetSmem {
    NetWeightsSmem W;
    float feat[kThreads][6];
    float guess[kThreads];
};

// CFL pass: FP32 primitives of U^n at every node, the largest wave speed (block
// max, then an integer atomicMax on the bit pattern: exact and order-independent),
// and (warm start) the pressures for the first stage.  GUESS: con2prim starts from
// the learned network's guess, evaluated per 256-node chunk on the tensor cores.
template <int SYS, int GUESS>
__global__ void __launch_bounds__(kThreads) k_cfl_mixed(const CflArgs a)
{
    extern __shared__ __align__(16) unsigned char cfl_smem[];
    CflNetSmem &N = *reinterpret_cast<CflNetSmem *>(cfl_smem);
    if (GUESS) net_stage_weights(N.W, a.netP, a.netW2);
    float lmax = 0.0f;
    unsigned errs = 0;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < a.total;
         base += (long long)gridDim.x * blockDim.x) {
        const long long g = base + threadIdx.x;
        const bool act = g < a.total;
        const long long e = act ? g / a.nn : 0;
        const int q = act ? (int)(g - e * a.nn) : 0;
        float u[5], P[NPRIM];
#pragma unroll
        for (int v = 0; v < 5; ++v) u[v] = act ? f64_to_f32(a.Un[(e * 5 + v) * a.nn + q]) : 1.0f;
        float guess = (a.pin && act) ? a.pin[g] : -1.0f;
        if (GUESS) {
            net_features(u, a.net_sc, N.feat[threadIdx.x]);
            __syncthreads();
            net_guess_rows(N.W, N.feat, N.guess, kThreads, a.gamma, a.net_sc);
            __syncthreads();
            guess = N.guess[threadIdx.x];
        }
        if (!act) continue;
        if (SYS == 0) {
            ne_primitives32(a.gamma, u, P);
        } else {
            errs |= sr_prims_mixed(a.gamma, a.gamma_d, a.kappa_sw, a.d_atm, a.tau_atm, u, a.Un + e * 5 * a.nn + q,
                                   a.nn, guess, P);
            if (a.pout) a.pout[g] = P[3];
        }
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            float lo, hi;
            speeds_axis32<SYS>(a.gamma, u, P, ax, lo, hi);
            lmax = fmaxf(lmax, fmaxf(fabsf(lo), fabsf(hi)));
        }
    }
    if (errs) atomicOr(a.err, errs);
    __shared__ float red[kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lmax;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = red[0];
        for (int w = 1; w < kThreads / 32; ++w) m = fmaxf(m, red[w]);
        atomicMax(a.lam, (unsigned long long)__double_as_longlong(f32_to_f64(m)));
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
    CflArgs a;
    std::memset(&a, 0, sizeof(a));
    a.Un = Un;
    a.pin = pin;
    a.pout = pout;
    a.lam = m->lam;
    a.err = m->err;
    a.total = m->E * m->nn;
    a.nn = m->nn;
    a.gamma = (float)m->d.gamma;
    a.gamma_d = m->d.gamma;
    a.kappa_sw = kappa_sw;
    a.d_atm = m->d.d_atm;
    a.tau_atm = m->d.tau_atm;
    const bool learned = m->d.system == 1 && m->net != nullptr;
    if (learned) {
        const void *w2 = nullptr;
        net_device_view(m->net, &a.netP, &w2, a.net_sc);
        a.netW2 = static_cast<const __nv_bfloat16 *>(w2);
    }
    const unsigned grid = grid_for(a.total);
    if (m->d.system == 0) {
        k_cfl_mixed<0, 0><<<grid, kThreads, 0, s>>>(a);
    } else if (!learned) {
        k_cfl_mixed<1, 0><<<grid, kThreads, 0, s>>>(a);
    } else {
        const size_t smem = sizeof(CflNetSmem);
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(k_cfl_mixed<1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        k_cfl_mixed<1, 1><<<grid, kThreads, smem, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace dg
