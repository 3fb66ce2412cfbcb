// dg_stage_fp64.cuh -- FP64 element kernels of the DG stage (templated on the
// number of LGL nodes per axis NP):
//   k_stage_fp64  : volume term + lifted surface term of eq:411, the SSP-RK3
//                   stage combination (Sec. 3.4) and the limiter summaries;
//   k_summaries   : the limiter summaries alone;
//   k_limit       : the MinModN / MinMod decision and linear replacement (Sec. 3.3).
// One CTA per element, one thread per node; the element's fluxes live in shared
// memory for the three tensor-product contractions (eq:405).  This file is
// compiled without floating-point contraction and every sum runs in a fixed
// order, so that the FP64 path reproduces a plain sequential evaluation of the
// same formulas operation for operation.
#pragma once

#include "dg_internal.h"
#include "dg_physics.cuh"

namespace dg {

// Mean over the face nodes of axis `a` at index ia along a, weighted by the LGL
// weights of the two other axes (divided by the reference face area 4).
template <int NP>
__device__ __forceinline__ double face_mean(const double *Uv, const double *sW, int a, int ia)
{
    const int b = (a + 1) % 3, c = (a + 2) % 3;
    double s = 0.0;
    for (int t1 = 0; t1 < NP; ++t1)
        for (int t0 = 0; t0 < NP; ++t0) {
            int id[3];
            id[a] = ia;
            id[b] = t0;
            id[c] = t1;
            s = s + sW[t0] * sW[t1] * Uv[id[0] + NP * (id[1] + NP * id[2])];
        }
    return s / 4.0;
}

// Limiter summaries of one element from its state in shared memory:
// S[v][0] cell mean (LGL quadrature / 8), S[v][1+2a], S[v][2+2a] lower / upper
// face means along a, S[v][7+a] Legendre P1 coefficient along a of the mean over
// the other axes.  The block's threads produce the 50 entries, strided.
template <int NP>
__device__ __forceinline__ void element_summaries(const double *sU, const double *sW, const double *sRow1,
                                                  double *Sout, int t)
{
    constexpr int NN = NP * NP * NP;
    for (int id = t; id < 50; id += blockDim.x) {
    const int v = id / 10, kind = id % 10;
    const double *Uv = sU + v * NN;
    double r;
    if (kind == 0) {
        double s = 0.0;
        for (int k = 0; k < NP; ++k)
            for (int j = 0; j < NP; ++j)
                for (int i = 0; i < NP; ++i)
                    s = s + sW[i] * sW[j] * sW[k] * Uv[i + NP * (j + NP * k)];
        r = s / 8.0;
    } else if (kind <= 6) {
        const int a = (kind - 1) / 2;
        r = face_mean<NP>(Uv, sW, a, ((kind - 1) % 2) ? NP - 1 : 0);
    } else {
        const int a = kind - 7;
        double c1 = 0.0;
        for (int ia = 0; ia < NP; ++ia) c1 = c1 + sRow1[ia] * face_mean<NP>(Uv, sW, a, ia);
        r = c1;
    }
    Sout[v * 10 + kind] = r;
    }
}

template <int NP, int SYS, int FLX>
__global__ void __launch_bounds__(round_up32(NP *NP *NP)) k_stage_fp64(const StageArgs a)
{
    constexpr int NN = NP * NP * NP;
    extern __shared__ double smem_stage[];
    double *sF = smem_stage;            // fluxes F^a_v per node [3][5][NN]; later the new state
    double *sR = smem_stage + 15 * NN;  // right-hand side per node [5][NN]
    __shared__ double sD[NP * NP];
    __shared__ double sW[NP], sRow1[NP];
    __shared__ long long sNb[6];

    const int t = threadIdx.x;
    const long long e = blockIdx.x;
    for (int i = t; i < NP * NP; i += blockDim.x) sD[i] = a.T.D[i];
    if (t < NP) {
        sW[t] = a.T.w[t];
        sRow1[t] = a.T.row1[t];
    }
    if (t < 6) sNb[t] = SYS == 0 ? elem_neighbour_bc(e, a.K, t >> 1, (t & 1) ? 1 : -1, a.gh)
                                 : elem_neighbour(e, a.K, t >> 1, (t & 1) ? 1 : -1);

    double u[5], P[4];
    if (t < NN) {
#pragma unroll
        for (int v = 0; v < 5; ++v) u[v] = a.Us[(e * 5 + v) * NN + t];
#pragma unroll
        for (int c = 0; c < 4; ++c) P[c] = a.P[(e * 4 + c) * NN + t];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            double f[5];
            flux_axis(u, P, ax, f);
#pragma unroll
            for (int v = 0; v < 5; ++v) sF[(ax * 5 + v) * NN + t] = f[v];
        }
    }
    __syncthreads();

    // volume term: -sum_a (2/dx_a) sum_l D_{i_a l} F^a_l
    if (t < NN) {
        const int i = t % NP, j = (t / NP) % NP, k = t / (NP * NP);
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            const double *Fx = sF + (0 * 5 + v) * NN;
            const double *Fy = sF + (1 * 5 + v) * NN;
            const double *Fz = sF + (2 * 5 + v) * NN;
            double sx = 0.0, sy = 0.0, sz = 0.0;
#pragma unroll
            for (int l = 0; l < NP; ++l) {
                sx = sx + sD[i * NP + l] * Fx[l + NP * (j + NP * k)];
                sy = sy + sD[j * NP + l] * Fy[i + NP * (l + NP * k)];
                sz = sz + sD[k * NP + l] * Fz[i + NP * (j + NP * l)];
            }
            double acc = a.g[0] * sx;
            acc = acc + a.g[1] * sy;
            acc = acc + a.g[2] * sz;
            sR[v * NN + t] = -acc;
        }
    }
    __syncthreads();

    // surface terms, one axis after another (within an axis no node is hit twice)
    for (int ax = 0; ax < 3; ++ax) {
        for (int fp = t; fp < 2 * NP * NP; fp += blockDim.x) {
            const int side = fp / (NP * NP);
            const int rem = fp % (NP * NP);
            int id[3];
            id[ax] = side ? NP - 1 : 0;
            id[(ax + 1) % 3] = rem % NP;
            id[(ax + 2) % 3] = rem / NP;
            const int q = id[0] + NP * (id[1] + NP * id[2]);
            id[ax] = side ? 0 : NP - 1;
            const int qn = id[0] + NP * (id[1] + NP * id[2]);
            long long en = sNb[2 * ax + side];
            // a negative neighbour is a ghost holding the analytic exterior state
            const double *Ub = a.Us, *Pb = a.P;
            if (SYS == 0 && en < 0) {
                Ub = a.gh.U;
                Pb = a.gh.P;
                en = -1 - en;
            }
            double uo[5], Po[4], un[5], Pn[4];
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                uo[v] = a.Us[(e * 5 + v) * NN + q];
                un[v] = Ub[(en * 5 + v) * NN + qn];
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                Po[c] = a.P[(e * 4 + c) * NN + q];
                Pn[c] = Pb[(en * 4 + c) * NN + qn];
            }
            double Fs[5], FL[5], FR[5];
            if (side) {
                num_flux<SYS, FLX>(a.gamma, ax, uo, Po, un, Pn, Fs, FL, FR);
#pragma unroll
                for (int v = 0; v < 5; ++v) sR[v * NN + q] = sR[v * NN + q] - a.liftN[ax] * (Fs[v] - FL[v]);
            } else {
                num_flux<SYS, FLX>(a.gamma, ax, un, Pn, uo, Po, Fs, FL, FR);
#pragma unroll
                for (int v = 0; v < 5; ++v) sR[v * NN + q] = sR[v * NN + q] + a.lift0[ax] * (Fs[v] - FR[v]);
            }
        }
        __syncthreads();
    }

    // stage combination (or the bare RHS)
    bool bad = false;
    if (t < NN) {
        const double dt = a.dt_ptr ? *a.dt_ptr : a.dt;
        double un[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            const double R = sR[v * NN + t];
            double val;
            if (a.mode == 0) {
                val = R;
            } else {
                const double y = u[v] + dt * R;
                val = a.first ? y : a.ca * a.Un[(e * 5 + v) * NN + t] + a.cb * y;
            }
            a.out[(e * 5 + v) * NN + t] = val;
            sF[v * NN + t] = val;
            un[v] = val;
        }
        if (SYS == 1) bad = sr_unphysical(un);
    }
    if (a.S == nullptr) return;
    const int anybad = __syncthreads_or(bad);
    element_summaries<NP>(sF, sW, sRow1, a.S + e * 50, t);
    if (SYS == 1 && t == 0 && a.unphys) a.unphys[e] = anybad ? 1 : 0;
}

template <int NP>
__global__ void __launch_bounds__(round_up32(NP *NP *NP)) k_summaries(const SummaryArgs a)
{
    constexpr int NN = NP * NP * NP;
    __shared__ double sU[5 * NN];
    __shared__ double sW[NP], sRow1[NP];
    const int t = threadIdx.x;
    const long long e = blockIdx.x;
    if (t < NP) {
        sW[t] = a.T.w[t];
        sRow1[t] = a.T.row1[t];
    }
    bool bad = false;
    if (t < NN) {
        double u[5];
        for (int v = 0; v < 5; ++v) sU[v * NN + t] = u[v] = a.U[(e * 5 + v) * NN + t];
        bad = sr_unphysical(u);
    }
    const int anybad = __syncthreads_or(bad);
    element_summaries<NP>(sU, sW, sRow1, a.S + e * 50, t);
    if (t == 0 && a.unphys) a.unphys[e] = anybad ? 1 : 0;
}

// One warp per element.  Lanes 0..4 decide for one conserved variable each:
// MinModN tests the six face conditions of Sec. 3.3.2 (tolerance 1e-8, M = 0);
// MinMod always limits; SR elements with an unphysical node limit every
// variable.  A limited variable becomes U0 + sum_a m_B(U_a, dU+/(dx/beta),
// dU-/(dx/beta); M)(x_a - x_a0) (eq:MinModSol) at every node.
template <int NP>
__global__ void __launch_bounds__(256) k_limit(const LimitArgs a)
{
    constexpr int NN = NP * NP * NP;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= a.E) return;
    const long long e = warp;
    int flag = 0;
    double sl[3] = {0.0, 0.0, 0.0};
    double U0 = 0.0;
    if (lane < 5) {
        const int v = lane;
        const double *Se = a.S + (e * 5 + v) * 10;
        U0 = Se[0];
        flag = (a.limiter == 2);
        for (int ax = 0; ax < 3; ++ax) {
            const double U0m = a.S[(elem_neighbour(e, a.K, ax, -1) * 5 + v) * 10];
            const double U0p = a.S[(elem_neighbour(e, a.K, ax, +1) * 5 + v) * 10];
            const double ulo = Se[1 + 2 * ax], uhi = Se[2 + 2 * ax];
            if (a.limiter == 1) {
                const double vl = U0 - minmodB(U0 - ulo, U0 - U0m, U0p - U0, 0.0, a.dx[ax]);
                const double vr = U0 + minmodB(uhi - U0, U0 - U0m, U0p - U0, 0.0, a.dx[ax]);
                if (fabs(vl - ulo) > 1e-8 || fabs(vr - uhi) > 1e-8) flag = 1;
            }
            const double h = a.dx[ax] / a.beta;
            sl[ax] = minmodB(2.0 * Se[7 + ax] / a.dx[ax], (U0p - U0) / h, (U0 - U0m) / h, a.tvb_M, a.dx[ax]);
        }
    }
    unsigned mask = __ballot_sync(0xffffffffu, flag) & 0x1fu;
    if (a.unphys && a.unphys[e]) mask = 0x1fu;
    if (lane == 0 && a.troubled) a.troubled[e] = (unsigned char)mask;
    if (!mask) return;
    double hx[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) hx[i] = a.T.x[i];
    for (int v = 0; v < 5; ++v) {
        const double m0 = __shfl_sync(0xffffffffu, U0, v);
        const double s0 = __shfl_sync(0xffffffffu, sl[0], v);
        const double s1 = __shfl_sync(0xffffffffu, sl[1], v);
        const double s2 = __shfl_sync(0xffffffffu, sl[2], v);
        if (!(mask & (1u << v))) continue;
        for (int q = lane; q < NN; q += 32) {
            const int i = q % NP, j = (q / NP) % NP, k = q / (NP * NP);
            double val = m0;
            val = val + s0 * (0.5 * a.dx[0] * hx[i]);
            val = val + s1 * (0.5 * a.dx[1] * hx[j]);
            val = val + s2 * (0.5 * a.dx[2] * hx[k]);
            a.U[(e * 5 + v) * NN + q] = val;
        }
    }
}

// Dispatch helpers instantiated once per NP in dg_stage_fp64_n*.cu.
template <int NP>
cudaError_t launch_stage_np(int system, int flux, const StageArgs &a, long long E, cudaStream_t s)
{
    const dim3 grid((unsigned)E), block(round_up32(NP * NP * NP));
    const size_t smem = sizeof(double) * 20 * NP * NP * NP;
    void (*kern)(const StageArgs);
    if (system == 0 && flux == 2) kern = k_stage_fp64<NP, 0, 2>;
    else if (system == 0 && flux == 0) kern = k_stage_fp64<NP, 0, 0>;
    else if (system == 0) kern = k_stage_fp64<NP, 0, 1>;
    else if (flux == 0) kern = k_stage_fp64<NP, 1, 0>;
    else kern = k_stage_fp64<NP, 1, 1>;
    if (smem > 48 * 1024) {
        cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
    }
    kern<<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
}

template <int NP>
cudaError_t launch_summaries_np(const SummaryArgs &a, long long E, cudaStream_t s)
{
    k_summaries<NP><<<(unsigned)E, round_up32(NP * NP * NP), 0, s>>>(a);
    return cudaGetLastError();
}

template <int NP>
cudaError_t launch_limit_np(const LimitArgs &a, cudaStream_t s)
{
    const long long threads = a.E * 32;
    k_limit<NP><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace dg

#define DG_INSTANTIATE_STAGE(NP)                                                                      \
    namespace dg {                                                                                    \
    cudaError_t launch_stage_fp64_n##NP(int system, int flux, const StageArgs &a, long long E,         \
                                        cudaStream_t s)                                               \
    {                                                                                                 \
        return launch_stage_np<NP>(system, flux, a, E, s);                                            \
    }                                                                                                 \
    cudaError_t launch_summaries_n##NP(const SummaryArgs &a, long long E, cudaStream_t s)             \
    {                                                                                                 \
        return launch_summaries_np<NP>(a, E, s);                                                      \
    }                                                                                                 \
    cudaError_t launch_limit_n##NP(const LimitArgs &a, cudaStream_t s) { return launch_limit_np<NP>(a, s); } \
    }
