// dg_mixed_pointwise.cu -- node-wise kernels of the mixed-precision path: the
// CFL pass: FP32 primitives of U^n, the largest wave speed, and the pressures
// that warm-start the first stage's con2prim.
#include <cstring>

#include "dg_mixed.cuh"

namespace dg {

namespace {

constexpr int kThreads = CFL_CHUNK;

// Shared memory of the learned-guess variant: weights, features, guesses.
struct CflNetSmem {
    NetWeightsSmem W;
    float feat[kThreads][6];
    float guess[kThreads];
};

// CFL pass: FP32 primitives of U^n at every node, the largest wave speed (block
// max, then an integer atomicMax on the bit pattern: exact and order-independent),
// and (warm start) the pressures for the first stage.  GUESS: con2prim starts from
// the learned network's guess, evaluated per chunk on the tensor cores.  Four CTAs
// per SM cap the registers at 64 (the SR variants used 74-80, three CTAs).
template <int SYS, int GUESS>
__global__ void __launch_bounds__(kThreads, 4) k_cfl_mixed(const CflArgs a)
{
    extern __shared__ __align__(16) unsigned char cfl_smem[];
    CflNetSmem &N = *reinterpret_cast<CflNetSmem *>(cfl_smem);
    __shared__ uint64_t bar;  // completion of the network weights' bulk copy
    if (GUESS) {
        if (threadIdx.x == 0) net_bar_init(&bar);
        __syncthreads();
        if (threadIdx.x == 0) net_copy_issue(&N.W, a.netImg, &bar);
    }
    int m = 0;
    long long c = blockIdx.x;
    if (a.slots) {
        m = find_slot(a.chunk0, a.nslots, blockIdx.x);
        c = blockIdx.x - a.chunk0[m];
    }
    const CflSlot &sl = a.slots ? a.slots[m] : a.one;
    const long long g = c * kThreads + threadIdx.x;
    const bool act = g < sl.nodes;
    const long long e = act ? g / a.nn : 0;
    const int q = act ? (int)(g - e * a.nn) : 0;
    float u[5] = {1.0f, 0.0f, 0.0f, 0.0f, 1.0f}, P[NPRIM];
    if (act)
#pragma unroll
        for (int v = 0; v < 5; ++v) u[v] = f64_to_f32(sl.Un[(e * 5 + v) * a.nn + q]);
    float guess = (sl.pin && act) ? sl.pin[g] : -1.0f;
    unsigned errs = 0;
    if (GUESS) {
        net_features(u, a.net_sc, N.feat[threadIdx.x]);
        if (!net_copy_wait(&bar, NET_COPY_POLLS)) {
            errs |= ERRBIT_TIMEOUT;
            net_copy_wait(&bar, NET_COPY_POLLS);
        }
        __syncthreads();
        net_guess_rows(N.W, N.feat, N.guess, kThreads, a.gamma, a.net_sc);
        __syncthreads();
        guess = N.guess[threadIdx.x];
    }
    float lmax = 0.0f;
    if (act) {
        if (SYS == 0) {
            ne_primitives32(a.gamma, u, P);
        } else {
            errs |= sr_prims_mixed(a.gamma, a.gamma_d, a.kappa_sw, a.d_atm, a.tau_atm, u, sl.Un + e * 5 * a.nn + q,
                                   a.nn, guess, P);
            if (sl.pout) sl.pout[g] = P[3];
            if (sl.Pout)
#pragma unroll
                for (int c = 0; c < NPRIM; ++c) sl.Pout[(e * NPRIM + c) * a.nn + q] = P[c];
        }
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            float lo, hi;
            speeds_axis32<SYS>(a.gamma, u, P, ax, lo, hi);
            lmax = fmaxf(lmax, fmaxf(fabsf(lo), fabsf(hi)));
        }
    }
    if (errs) atomicOr(sl.err, errs);
    __shared__ float red[kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lmax;
    __syncthreads();
    if (threadIdx.x == 0) {
        float mx = red[0];
        for (int w = 1; w < kThreads / 32; ++w) mx = fmaxf(mx, red[w]);
        atomicMax(sl.lam, (unsigned long long)__double_as_longlong(f32_to_f64(mx)));
    }
}

}  // namespace

CflArgs cfl_args(const dg_mesh *m, float kappa_sw)
{
    CflArgs a;
    std::memset(&a, 0, sizeof(a));
    a.one.err = m->err;
    a.one.lam = m->lam;
    a.one.nodes = m->E * m->nn;
    a.nslots = 1;
    a.nn = m->nn;
    a.gamma = (float)m->d.gamma;
    a.gamma_d = m->d.gamma;
    a.kappa_sw = kappa_sw;
    a.d_atm = m->d.d_atm;
    a.tau_atm = m->d.tau_atm;
    if (m->d.system == 1 && m->net != nullptr) {
        const void *img = nullptr;
        net_device_view(m->net, &img, a.net_sc);
        a.netImg = static_cast<const NetWeightsSmem *>(img);
    }
    return a;
}

cudaError_t launch_cfl_batch(int system, const CflArgs &a, long long nchunks, cudaStream_t s)
{
    if (nchunks <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)nchunks;
    if (system == 0) {
        k_cfl_mixed<0, 0><<<grid, kThreads, 0, s>>>(a);
    } else if (a.netImg == nullptr) {
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

cudaError_t launch_cfl_mixed(const dg_mesh *m, const double *Un, const float *pin, float *pout, float *Pout,
                             float kappa_sw, cudaStream_t s)
{
    CflArgs a = cfl_args(m, kappa_sw);
    a.one.Un = Un;
    a.one.pin = pin;
    a.one.pout = pout;
    a.one.Pout = Pout;
    return launch_cfl_batch(m->d.system, a, (a.one.nodes + kThreads - 1) / kThreads, s);
}

}  // namespace dg
