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

// Moment limiter of Moe, Rossmanith and Seal (Sec. 3.3.3, eq:MRSSol), Newtonian
// system, with the oracle's operations: per element T = (U0[5], w0[5], w_max[5],
// w_min[5]), w = (rho, vx, vy, vz, p) the node primitives and w0 those of the
// LGL cell average U0 (summaries S[e][v][0]).  One warp per element.
template <int NP>
__global__ void __launch_bounds__(256) k_mrs_prepare(const double *U, const double *S, double *T, long long E,
                                                     double g)
{
    constexpr int NN = NP * NP * NP;
    const long long e = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (e >= E) return;
    double wmax[5], wmin[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        wmax[c] = -INFINITY;
        wmin[c] = INFINITY;
    }
    for (int q = lane; q < NN; q += 32) {
        double u[5], P[4];
#pragma unroll
        for (int v = 0; v < 5; ++v) u[v] = U[(e * 5 + v) * NN + q];
        ne_primitives(g, u, P);
        const double w[5] = {u[0], P[0], P[1], P[2], P[3]};
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            wmax[c] = fmax(wmax[c], w[c]);
            wmin[c] = fmin(wmin[c], w[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < 5; ++c)
        for (int o = 16; o > 0; o >>= 1) {
            wmax[c] = fmax(wmax[c], __shfl_xor_sync(0xffffffffu, wmax[c], o));
            wmin[c] = fmin(wmin[c], __shfl_xor_sync(0xffffffffu, wmin[c], o));
        }
    if (lane == 0) {
        double *Te = T + 20 * e;
        double u0[5], P0[4];
#pragma unroll
        for (int v = 0; v < 5; ++v) u0[v] = Te[v] = S[(e * 5 + v) * 10];
        ne_primitives(g, u0, P0);
        Te[5] = u0[0];
#pragma unroll
        for (int c = 0; c < 4; ++c) Te[6 + c] = P0[c];
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            Te[10 + c] = wmax[c];
            Te[15 + c] = wmin[c];
        }
    }
}

// Theta = min over components of min(1, |(M - w0)/(w_max - w0)|, |(m - w0)/(w_min - w0)|)
// with [m, M] the face neighbours' w0 widened to w0 -+ wid (wid = alpha~ h^{3/2}), a
// ratio counting 1 when its denominator is within 1e-12 |w0|; then U -> U0 + Theta (U - U0).
template <int NP>
__global__ void __launch_bounds__(256) k_mrs_limit(double *U, const double *T, unsigned char *troubled, long long E,
                                                   int K0, int K1, int K2, double wid)
{
    constexpr int NN = NP * NP * NP;
    const long long e = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (e >= E) return;
    const double *Te = T + 20 * e;
    double theta = 1.0;
    if (lane < 5) {
        const int c = lane;
        const int K[3] = {K0, K1, K2};
        const double w0 = Te[5 + c];
        double M = w0 + wid, mm = w0 - wid;
        for (int a = 0; a < 3; ++a)
            for (int sd = -1; sd <= 1; sd += 2) {
                const double *Tn = T + 20 * elem_neighbour(e, K, a, sd);
                M = fmax(M, Tn[5 + c]);
                mm = fmin(mm, Tn[5 + c]);
            }
        const double dmax = Te[10 + c] - w0, dmin = Te[15 + c] - w0;
        const double tiny = 1e-12 * fabs(w0);
        if (fabs(dmax) > tiny) theta = fmin(theta, fabs((M - w0) / dmax));
        if (fabs(dmin) > tiny) theta = fmin(theta, fabs((mm - w0) / dmin));
    }
    for (int o = 16; o > 0; o >>= 1) theta = fmin(theta, __shfl_xor_sync(0xffffffffu, theta, o));
    if (lane == 0 && troubled) troubled[e] = theta < 1.0 ? 0x1f : 0;
    if (!(theta < 1.0)) return;
    for (int v = 0; v < 5; ++v) {
        const double U0 = Te[v];
        for (int q = lane; q < NN; q += 32) {
            double *x = U + (e * 5 + v) * NN + q;
            *x = U0 + theta * (*x - U0);
        }
    }
}

// Exterior states of the analytic outer faces (Sec. 3.4): the isentropic vortex
// (eq:isen_vortex, P = rho^gamma, par = beta, X0, Y0, U, V, W) at time
// *t + ct dt and at the coordinates of the interior trace node (eq:AffineMap),
// conserved and with its FP64 primitives, on ghost face node r of ghost gi.
__global__ void __launch_bounds__(kThreads) k_exterior(double *gU, double *gP, Ghosts gh, long long total, int n,
                                                     int K0, int K1, int K2, double lo0, double lo1, double lo2,
                                                     double dx0, double dx1, double dx2, Tables T, double g,
                                                     double b0, double b1, double b2, double b3, double b4,
                                                     double b5, const double *t, double ct, const double *dt_ptr,
                                                     double dt_val)
{
    const double pi = 3.14159265358979323846;
    const int nf = n * n, nn = n * n * n;
    const int K[3] = {K0, K1, K2};
    const double lo[3] = {lo0, lo1, lo2}, dx[3] = {dx0, dx1, dx2};
    const double dt = dt_ptr ? *dt_ptr : dt_val;
    const double ts = *t + ct * dt;
    for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < total;
         w += (long long)gridDim.x * blockDim.x) {
        const long long gi = w / nf;
        const int r = (int)(w - gi * nf);
        int a = -1, s = 0;
        for (int aa = 0; aa < 3 && a < 0; ++aa) {
            if (!((gh.mask >> aa) & 1)) continue;
            const long long cnt = (long long)K[(aa + 1) % 3] * K[(aa + 2) % 3];
            for (int ss = 0; ss < 2; ++ss)
                if (gi >= gh.base[aa][ss] && gi < gh.base[aa][ss] + cnt) {
                    a = aa;
                    s = ss;
                }
        }
        if (a < 0) continue;
        const int b = (a + 1) % 3, c = (a + 2) % 3;
        const long long fi = gi - gh.base[a][s];
        int ec[3], id[3];
        ec[b] = (int)(fi % K[b]);
        ec[c] = (int)(fi / K[b]);
        ec[a] = s ? K[a] - 1 : 0;
        id[b] = r % n;
        id[c] = r / n;
        id[a] = s ? n - 1 : 0;
        double x[3];
        for (int d = 0; d < 3; ++d) {
            const double ak = lo[d] + ec[d] * dx[d];
            const double bk = ak + dx[d];
            x[d] = ak + 0.5 * (1.0 + T.x[id[d]]) * (bk - ak);
        }
        const double beta = b0;
        const double xt = x[0] - b1 - b3 * ts;
        const double yt = x[1] - b2 - b4 * ts;
        const double r2 = xt * xt + yt * yt;
        const double rho = pow(1.0 - (g - 1.0) * beta * beta / (8.0 * g * pi * pi) * exp(1.0 - r2), 1.0 / (g - 1.0));
        const double f = beta / (2.0 * pi) * exp(0.5 * (1.0 - r2));
        const double vx = b3 - yt * f, vy = b4 + xt * f, vz = b5;
        const double p = pow(rho, g);
        const double v2 = vx * vx + vy * vy + vz * vz;
        double u[5], P[4];
        u[0] = rho;
        u[1] = rho * vx;
        u[2] = rho * vy;
        u[3] = rho * vz;
        u[4] = p / (g - 1.0) + 0.5 * rho * v2;
        ne_primitives(g, u, P);
        id[a] = s ? 0 : n - 1;  // the ghost's node facing the mesh
        const int qn = id[0] + n * (id[1] + n * id[2]);
        for (int v = 0; v < 5; ++v) gU[(gi * 5 + v) * nn + qn] = u[v];
        for (int k = 0; k < 4; ++k) gP[(gi * 4 + k) * nn + qn] = P[k];
    }
}

__global__ void k_time_add(double *t, const double *dt_ptr, double dt)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *t = *t + (dt_ptr ? *dt_ptr : dt);
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

template <int NP>
cudaError_t launch_mrs_np(const dg_mesh *m, double *U, unsigned char *troubled, cudaStream_t s)
{
    const unsigned grid = (unsigned)((m->E * 32 + 255) / 256);
    k_mrs_prepare<NP><<<grid, 256, 0, s>>>(U, m->S, m->mrsT, m->E, m->d.gamma);
    double h = 0.0;
    for (int a = 0; a < 3; ++a) h = fmax(h, m->dx[a]);
    const double wid = m->d.mrs_alpha * h * sqrt(h);
    k_mrs_limit<NP><<<grid, 256, 0, s>>>(U, m->mrsT, troubled, m->E, m->d.K[0], m->d.K[1], m->d.K[2], wid);
    return cudaGetLastError();
}

// MRS pass over a state whose summaries S are current (the stage kernel's, or
// dg_limiter_summaries').
cudaError_t launch_mrs(const dg_mesh *m, double *U, unsigned char *troubled, cudaStream_t s)
{
    switch (m->d.n) {
    case 2: return launch_mrs_np<2>(m, U, troubled, s);
    case 3: return launch_mrs_np<3>(m, U, troubled, s);
    case 4: return launch_mrs_np<4>(m, U, troubled, s);
    case 5: return launch_mrs_np<5>(m, U, troubled, s);
    case 6: return launch_mrs_np<6>(m, U, troubled, s);
    case 7: return launch_mrs_np<7>(m, U, troubled, s);
    case 8: return launch_mrs_np<8>(m, U, troubled, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_exterior(const dg_mesh *m, double ct, const double *dt_ptr, double dt, cudaStream_t s)
{
    if (!m->gh.mask) return cudaSuccess;
    const long long total = m->nghost * m->d.n * m->d.n;
    const double *b = m->d.exact_par;
    k_exterior<<<grid_for(total, kThreads), kThreads, 0, s>>>(
        const_cast<double *>(m->gh.U), const_cast<double *>(m->gh.P), m->gh, total, m->d.n, m->d.K[0], m->d.K[1],
        m->d.K[2], m->d.lo[0], m->d.lo[1], m->d.lo[2], m->dx[0], m->dx[1], m->dx[2], m->T, m->d.gamma, b[0], b[1],
        b[2], b[3], b[4], b[5], m->t, ct, dt_ptr, dt);
    return cudaGetLastError();
}

cudaError_t launch_time_add(double *t, const double *dt_ptr, double dt, cudaStream_t s)
{
    k_time_add<<<1, 32, 0, s>>>(t, dt_ptr, dt);
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
