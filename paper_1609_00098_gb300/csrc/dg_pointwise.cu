// dg_pointwise.cu -- node-wise kernels: primitive recovery with the fused SR fix
// and the CFL wave-speed maximum, the SR fix alone, the CFL step, node
// coordinates, primitive->conserved, and standalone con2prim.
#include "dg_internal.h"
#include "dg_physics.cuh"

namespace dg {

namespace {

constexpr int kThreads = 256;

unsigned grid_for(long long count, int threads)
{
    long long b = (count + threads - 1) / threads;
    if (b > 152LL * 64) b = 152LL * 64;  // grid-stride beyond 64 CTAs per SM
    return (unsigned)(b < 1 ? 1 : b);
}

struct PrimArgs {
    const double *U;
    double *Ufix;  // SR fix target (== U) or nullptr
    double *P;
    unsigned long long *lam;
    unsigned int *err;
    long long total;
    int nn;
    double gamma, d_atm, tau_atm;
};

// One thread per node: (optional SR fix of the node in place), primitives
// (vx, vy, vz, p) into P[e][c][node], and the block-reduced largest wave speed
// folded into *lam with an integer atomicMax on the bit pattern (exact and
// independent of order for non-negative doubles).
template <int SYS>
__global__ void __launch_bounds__(kThreads) k_primitives(const PrimArgs a)
{
    double lmax = 0.0;
    unsigned errs = 0;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < a.total;
         g += (long long)gridDim.x * blockDim.x) {
        const long long e = g / a.nn;
        const int q = (int)(g - e * a.nn);
        double u[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) u[v] = a.U[(e * 5 + v) * a.nn + q];
        if (SYS == 1 && a.Ufix) {
            double f[5] = {u[0], u[1], u[2], u[3], u[4]};
            if (sr_fix(a.d_atm, a.tau_atm, f)) {
#pragma unroll
                for (int v = 0; v < 5; ++v) {
                    if (f[v] != u[v]) a.Ufix[(e * 5 + v) * a.nn + q] = f[v];
                    u[v] = f[v];
                }
            }
        }
        double P[4];
        if (node_primitives<SYS>(a.gamma, u, P)) errs |= ERRBIT_C2P;
#pragma unroll
        for (int c = 0; c < 4; ++c) a.P[(e * 4 + c) * a.nn + q] = P[c];
        if (a.lam) lmax = fmax(lmax, max_speed<SYS>(a.gamma, u, P));
    }
    if (errs) atomicOr(a.err, errs);
    if (a.lam) {
        __shared__ double red[kThreads / 32];
        for (int o = 16; o > 0; o >>= 1) lmax = fmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lmax;
        __syncthreads();
        if (threadIdx.x == 0) {
            double m = red[0];
            for (int w = 1; w < kThreads / 32; ++w) m = fmax(m, red[w]);
            atomicMax(a.lam, (unsigned long long)__double_as_longlong(m));
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_fix(double *U, long long total, int nn, double d_atm, double tau_atm)
{
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        const long long e = g / nn;
        const int q = (int)(g - e * nn);
        double u[5], f[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) f[v] = u[v] = U[(e * 5 + v) * nn + q];
        if (sr_fix(d_atm, tau_atm, f)) {
#pragma unroll
            for (int v = 0; v < 5; ++v)
                if (f[v] != u[v]) U[(e * 5 + v) * nn + q] = f[v];
        }
    }
}

// U <- U + dt ((c0 L0 - c1 L1) + c2 L2), the third-order Adams-Bashforth
// combination (Sec. 3.4) with c = (23, 16, 5)/12, in the oracle's operation order.
__global__ void __launch_bounds__(kThreads) k_ab3(double *U, const double *L0, const double *L1, const double *L2,
                                                  double dt, double c0, double c1, double c2, long long count)
{
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < count;
         g += (long long)gridDim.x * blockDim.x)
        U[g] = U[g] + dt * ((c0 * L0[g] - c1 * L1[g]) + c2 * L2[g]);
}

__global__ void k_dt(const unsigned long long *lam, double cfl, double dxmin, double *dt)
{
    const double l = __longlong_as_double((long long)*lam);
    *dt = cfl * dxmin / l;
}

__global__ void __launch_bounds__(kThreads) k_coords(double *xyz, long long total, int n, int K0, int K1,
                                                     double lo0, double lo1, double lo2, double dx0,
                                                     double dx1, double dx2, Tables T)
{
    const int nn = n * n * n;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        const long long e = g / nn;
        const int q = (int)(g - e * nn);
        const int id[3] = {q % n, (q / n) % n, q / (n * n)};
        const int ec[3] = {(int)(e % K0), (int)((e / K0) % K1), (int)(e / ((long long)K0 * K1))};
        const double lo[3] = {lo0, lo1, lo2}, dx[3] = {dx0, dx1, dx2};
        for (int a = 0; a < 3; ++a) {
            // eq:AffineMap with a^k = lo + ec dx and b^k = a^k + dx
            const double ak = lo[a] + ec[a] * dx[a];
            const double bk = ak + dx[a];
            xyz[a * total + g] = ak + 0.5 * (1.0 + T.x[id[a]]) * (bk - ak);
        }
    }
}

template <int SYS>
__global__ void __launch_bounds__(kThreads) k_prim2con(const double *prim, double *U, long long total, int nn,
                                                       double g)
{
    for (long long gi = (long long)blockIdx.x * blockDim.x + threadIdx.x; gi < total;
         gi += (long long)gridDim.x * blockDim.x) {
        const long long e = gi / nn;
        const int q = (int)(gi - e * nn);
        const double rho = prim[gi], vx = prim[total + gi], vy = prim[2 * total + gi];
        const double vz = prim[3 * total + gi], p = prim[4 * total + gi];
        const double v2 = vx * vx + vy * vy + vz * vz;
        double u[5];
        if (SYS == 0) {
            u[0] = rho;
            u[1] = rho * vx;
            u[2] = rho * vy;
            u[3] = rho * vz;
            u[4] = p / (g - 1.0) + 0.5 * rho * v2;
        } else {
            // tau = rho W (W-1) + rho eps W^2 + p (W^2-1), with W-1 = W^2 v^2/(W+1)
            const double W = 1.0 / sqrt(1.0 - v2);
            const double W2v2 = W * W * v2;
            const double rhoeps = p / (g - 1.0);
            const double rhoh = rho + rhoeps + p;
            u[0] = rho * W;
            u[1] = rhoh * W * W * vx;
            u[2] = rhoh * W * W * vy;
            u[3] = rhoh * W * W * vz;
            u[4] = rho * W * (W2v2 / (W + 1.0)) + rhoeps * W * W + p * W2v2;
        }
        for (int v = 0; v < 5; ++v) U[(e * 5 + v) * nn + q] = u[v];
    }
}

__global__ void __launch_bounds__(kThreads) k_con2prim(long long count, double gamma, const double *cons,
                                                       double *prim, const double *guess, int *iters,
                                                       int *status)
{
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < count;
         g += (long long)gridDim.x * blockDim.x) {
        double u[5], pr[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) u[v] = cons[v * count + g];
        int it;
        const int st = sr_con2prim(gamma, u, guess ? guess[g] : -1.0, pr, &it);
#pragma unroll
        for (int v = 0; v < 5; ++v) prim[v * count + g] = pr[v];
        if (iters) iters[g] = it;
        if (status) status[g] = st;
    }
}

__global__ void k_set(double *p, double v) { *p = v; }

}  // namespace

cudaError_t launch_set(double *p, double v, cudaStream_t s)
{
    k_set<<<1, 1, 0, s>>>(p, v);
    return cudaGetLastError();
}

cudaError_t launch_primitives(const dg_mesh *m, const double *U, double *P, int fix, double *Ufix,
                              unsigned long long *lam, cudaStream_t s)
{
    PrimArgs a;
    a.U = U;
    a.Ufix = fix ? Ufix : nullptr;
    a.P = P;
    a.lam = lam;
    a.err = m->err;
    a.total = m->E * m->nn;
    a.nn = m->nn;
    a.gamma = m->d.gamma;
    a.d_atm = m->d.d_atm;
    a.tau_atm = m->d.tau_atm;
    const unsigned grid = grid_for(a.total, kThreads);
    if (m->d.system == 0) k_primitives<0><<<grid, kThreads, 0, s>>>(a);
    else k_primitives<1><<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_fix(const dg_mesh *m, double *U, cudaStream_t s)
{
    const long long total = m->E * m->nn;
    k_fix<<<grid_for(total, kThreads), kThreads, 0, s>>>(U, total, m->nn, m->d.d_atm, m->d.tau_atm);
    return cudaGetLastError();
}

cudaError_t launch_ab3_combine(double *U, const double *L0, const double *L1, const double *L2, double dt,
                               long long count, cudaStream_t s)
{
    k_ab3<<<grid_for(count, kThreads), kThreads, 0, s>>>(U, L0, L1, L2, dt, 23.0 / 12.0, 16.0 / 12.0, 5.0 / 12.0,
                                                         count);
    return cudaGetLastError();
}

cudaError_t launch_dt(const dg_mesh *m, double cfl, double *dt, cudaStream_t s)
{
    k_dt<<<1, 1, 0, s>>>(m->lam, cfl, m->dxmin, dt);
    return cudaGetLastError();
}

cudaError_t launch_coords(const dg_mesh *m, double *xyz, cudaStream_t s)
{
    const long long total = m->E * m->nn;
    k_coords<<<grid_for(total, kThreads), kThreads, 0, s>>>(xyz, total, m->d.n, m->d.K[0], m->d.K[1],
                                                            m->d.lo[0], m->d.lo[1], m->d.lo[2], m->dx[0],
                                                            m->dx[1], m->dx[2], m->T);
    return cudaGetLastError();
}

cudaError_t launch_prim2con(const dg_mesh *m, const double *prim, double *U, cudaStream_t s)
{
    const long long total = m->E * m->nn;
    if (m->d.system == 0)
        k_prim2con<0><<<grid_for(total, kThreads), kThreads, 0, s>>>(prim, U, total, m->nn, m->d.gamma);
    else
        k_prim2con<1><<<grid_for(total, kThreads), kThreads, 0, s>>>(prim, U, total, m->nn, m->d.gamma);
    return cudaGetLastError();
}

cudaError_t launch_con2prim(long long count, double gamma, const double *cons, double *prim,
                            const double *guess, int *iters, int *status, cudaStream_t s)
{
    k_con2prim<<<grid_for(count, kThreads), kThreads, 0, s>>>(count, gamma, cons, prim, guess, iters, status);
    return cudaGetLastError();
}

}  // namespace dg
