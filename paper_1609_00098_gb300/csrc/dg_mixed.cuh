// dg_mixed.cuh -- mixed-precision DG stage kernels (templated on the number of
// LGL nodes per axis NP).
//
// State and accumulation stay FP64: U^n is read in FP64 and U^{n+1} = U^n + D3 is
// formed in FP64 once per step.  Inside a step the SSP-RK3 stages (Sec. 3.4) are
// carried as FP32 increments of U^n:
//   D1 = dt L(U^n),  D2 = (D1 + dt L(U^n + D1)) / 4,  D3 = 2/3 (D2 + dt L(U^n + D2)),
// which is the Shu-Osher form rewritten about U^n (U1 = U^n + D1, U2 = U^n + D2,
// U^{n+1} = U^n + D3).  Fluxes, the tensor-product contraction (eq:405), the
// numerical fluxes (eq:LLF, eq:HLL) and the lift (eq:411) run in FP32.  SR
// con2prim runs in FP32 from the previous pass's pressure; where the conditioning
// estimate tau/(rho eps) exceeds kappa_sw the pressure is polished by FP64 Newton
// on the FP64 conserved state.  The limiter's cell and face means are the FP64
// means of U^n (computed at stage 1) plus FP32 means of the increment, so the
// 1e-8 detector of Sec. 3.3.2 and conservation by the limiter keep FP64 anchors.
// FP64<->FP32 conversions are done with integer operations: on this GPU the
// conversion instructions issue at the FP64 rate.
#pragma once

#include "dg_internal.h"
#include "dg_physics.cuh"

namespace dg {

// ---------------------------------------------------------------------------
// FP64 <-> FP32 by integer operations (normal range; |x| < 2^-126 flushes to 0).

__device__ __forceinline__ float f64_to_f32(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned sign = hi & 0x80000000u;
    const unsigned ef = (hi >> 20) & 0x7ffu;
    if (ef == 0x7ffu) return __uint_as_float(sign | 0x7f800000u | ((((hi & 0xfffffu) | lo) != 0u) ? 0x400000u : 0u));
    const int e = (int)ef - 896;
    if (e <= 0) return __uint_as_float(sign);
    if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
    unsigned bits = sign | ((unsigned)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    bits += (lo >> 28) & 1u;  // round half away from zero; a carry into the exponent is exact
    return __uint_as_float(bits);
}

__device__ __forceinline__ double f32_to_f64(float f)
{
    const unsigned b = __float_as_uint(f);
    const unsigned sign = b & 0x80000000u, ef = (b >> 23) & 0xffu, m = b & 0x7fffffu;
    if (ef == 0u) return __hiloint2double((int)sign, 0);
    const unsigned he = (ef == 0xffu) ? 0x7ffu : ef + 896u;
    return __hiloint2double((int)(sign | (he << 20) | (m >> 3)), (int)(m << 29));
}

// ---------------------------------------------------------------------------
// FP32 physics (same formulas as the FP64 path)

__device__ __forceinline__ void flux_axis32(const float u[5], const float P[4], int a, float F[5])
{
    const float va = P[a], p = P[3];
    F[0] = u[0] * va;
    F[1] = u[1] * va;
    F[2] = u[2] * va;
    F[3] = u[3] * va;
    F[1 + a] += p;
    F[4] = (u[4] + p) * va;
}

// Same operations and the same treatment of negative or NaN intermediate values
// as the FP64 path (a negative pressure gives NaN speeds, which fmin/fmax then
// ignore), so both paths agree on states that leave the physical range.
template <int SYS>
__device__ __forceinline__ void speeds_axis32(float g, const float u[5], const float P[4], int a, float &lmin,
                                              float &lmax)
{
    const float va = P[a], p = P[3];
    if (SYS == 0) {
        const float c = sqrtf(g * p / u[0]);
        lmin = va - c;
        lmax = va + c;
        return;
    }
    const float v2 = P[0] * P[0] + P[1] * P[1] + P[2] * P[2];
    const float rhoh = (u[4] + u[0] + p) * (1.0f - v2);
    const float cs2 = g * p / rhoh;
    const float cs = sqrtf(cs2);
    float disc = (1.0f - v2) * (1.0f - v2 * cs2 - va * va * (1.0f - cs2));
    if (disc < 0.0f) disc = 0.0f;
    const float root = cs * sqrtf(disc);
    const float inv = 1.0f / (1.0f - v2 * cs2);
    lmin = (va * (1.0f - cs2) - root) * inv;
    lmax = (va * (1.0f - cs2) + root) * inv;
}

// Numerical flux along +e_a minus each side's physical flux, in jump form:
// with dF = F(U_R) - F(U_L) and dU = U_R - U_L,
//   HLL (eq:HLL):  F* - F_L = -cmin dF/(cmax-cmin) + cmin cmax/(cmax-cmin) dU,
//                  F* - F_R = -cmax dF/(cmax-cmin) + cmin cmax/(cmax-cmin) dU;
//   LLF (eq:LLF):  F* - F_L =  dF/2 - alpha dU/2,  F* - F_R = -dF/2 - alpha dU/2.
// Algebraically the eq:LLF / eq:HLL fluxes; in FP32 the differences are taken
// before they are scaled, so equal states give exactly zero.
template <int SYS, int FLX>
__device__ __forceinline__ void num_flux_jump32(float g, int a, const float uL[5], const float PL[4],
                                                const float uR[5], const float PR[4], float dL[5], float dR[5])
{
    float FL[5], FR[5], lminL, lmaxL, lminR, lmaxR;
    flux_axis32(uL, PL, a, FL);
    flux_axis32(uR, PR, a, FR);
    speeds_axis32<SYS>(g, uL, PL, a, lminL, lmaxL);
    speeds_axis32<SYS>(g, uR, PR, a, lminR, lmaxR);
    if (FLX == 0) {
        const float hal = 0.5f * fmaxf(fmaxf(fabsf(lminL), fabsf(lmaxL)), fmaxf(fabsf(lminR), fabsf(lmaxR)));
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            const float dF = FR[v] - FL[v], dU = uR[v] - uL[v];
            dL[v] = 0.5f * dF - hal * dU;
            dR[v] = -0.5f * dF - hal * dU;
        }
    } else {
        const float cmin = fminf(fminf(lminL, lminR), 0.0f);
        const float cmax = fmaxf(fmaxf(lmaxL, lmaxR), 0.0f);
        const float den = cmax - cmin;
        if (den > 0.0f) {
            const float inv = 1.0f / den;
            const float cc = cmin * cmax * inv, wl = -cmin * inv, wr = -cmax * inv;
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                const float dF = FR[v] - FL[v], dU = uR[v] - uL[v];
                dL[v] = wl * dF + cc * dU;
                dR[v] = wr * dF + cc * dU;
            }
        } else {
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                const float dF = FR[v] - FL[v];
                dL[v] = 0.5f * dF;
                dR[v] = -0.5f * dF;
            }
        }
    }
}

__device__ __forceinline__ void ne_primitives32(float g, const float u[5], float P[4])
{
    const float inv = 1.0f / u[0];
    P[0] = u[1] * inv;
    P[1] = u[2] * inv;
    P[2] = u[3] * inv;
    P[3] = (g - 1.0f) * (u[4] - 0.5f * (u[1] * P[0] + u[2] * P[1] + u[3] * P[2]));
}

// FP32 SR con2prim: the safeguarded Newton of the FP64 path in FP32, stopping
// when the step is below 2^-21 p or the residual is at the FP32 noise level of
// its terms.  Returns 0 ok, 1 unphysical in FP32, 2 no convergence; kappa gets
// tau/(rho eps), the amplification of input rounding into p.
__device__ __forceinline__ int sr_con2prim32(float g, const float u[5], float guess, float P[4], float &kappa)
{
    const float D = u[0], tau = u[4];
    const float s2 = u[1] * u[1] + u[2] * u[2] + u[3] * u[3];
    if (!(D > 0.0f) || !(tau > 0.0f) || !(s2 < tau * (tau + 2.0f * D))) return 1;
    const float E = tau + D;
    float plo = fmaxf(sqrtf(s2) - E, 0.0f);
    float phi = (g - 1.0f) * tau;
    float p = (guess >= 0.0f) ? fminf(fmaxf(guess, plo), phi) : phi;
    float rhoeps = tau;
    int status = 2;
    for (int it = 0; it < 60; ++it) {
        const float Ep = E + p;
        const float v2 = s2 / (Ep * Ep);
        const float W = rsqrtf(1.0f - v2);
        const float DW = D * W;
        rhoeps = tau - v2 * (Ep - DW / (W + 1.0f));
        const float f = p - (g - 1.0f) * rhoeps;
        const float df = 1.0f - (g - 1.0f) * v2 * (1.0f - DW / Ep);
        const float noise = 6.0e-7f * (p + (g - 1.0f) * (tau + v2 * Ep));
        if (fabsf(f) <= noise) { status = 0; break; }
        if (f > 0.0f) phi = p; else plo = p;
        float pn = p - f / df;
        if (!(pn > plo && pn < phi)) pn = 0.5f * (plo + phi);
        const float dp = fabsf(pn - p);
        p = pn;
        if (dp <= 4.8e-7f * p || !(phi > plo)) { status = 0; break; }
    }
    const float Ep = E + p;
    const float inv = 1.0f / Ep;
    P[0] = u[1] * inv;
    P[1] = u[2] * inv;
    P[2] = u[3] * inv;
    P[3] = p;
    kappa = tau / fmaxf(rhoeps, 1e-30f);
    return status;
}

// FP64 Newton on the pressure from a starting value p0 (the FP32 result, or the
// standard guess when p0 < 0), on the FP64 conserved state u: the bracket and
// step rules of the FP64 con2prim, stopping when the step is below 2^-40 p or
// the residual is at the FP64 rounding level of its terms.  That level is
// reached in a few steps even where tau/(rho eps) is huge, so the cost stays
// bounded on cold states at the conserved-fix bound.
__device__ __forceinline__ int sr_polish64(double g, const double u[5], double p0, double Pd[4])
{
    const double D = u[0], tau = u[4];
    const double s2 = u[1] * u[1] + u[2] * u[2] + u[3] * u[3];
    if (!(D > 0.0) || !(tau > 0.0) || !(s2 < tau * (tau + 2.0 * D))) {
        for (int c = 0; c < 4; ++c) Pd[c] = __longlong_as_double(0x7ff8000000000000LL);
        return 1;
    }
    const double E = tau + D;
    double plo = fmax(sqrt(s2) - E, 0.0), phi = (g - 1.0) * tau;
    double p = (p0 >= 0.0) ? fmin(fmax(p0, plo), phi) : phi;
    int status = 2;
    for (int it = 0; it < 60; ++it) {
        const double Ep = E + p;
        const double v2 = s2 / (Ep * Ep);
        const double W = 1.0 / sqrt(1.0 - v2);
        const double DW = D * W;
        const double rhoeps = tau - v2 * (Ep - DW / (W + 1.0));
        const double f = p - (g - 1.0) * rhoeps;
        const double df = 1.0 - (g - 1.0) * v2 * (1.0 - DW / Ep);
        if (fabs(f) <= 0x1p-50 * (p + (g - 1.0) * (tau + v2 * Ep))) { status = 0; break; }
        if (f > 0.0) phi = p; else plo = p;
        double pn = p - f / df;
        if (!(pn > plo && pn < phi)) pn = 0.5 * (plo + phi);
        const double dp = fabs(pn - p);
        p = pn;
        if (dp <= 0x1p-40 * p || !(phi > plo)) { status = 0; break; }
    }
    const double Ep = E + p;
    Pd[0] = u[1] / Ep;
    Pd[1] = u[2] / Ep;
    Pd[2] = u[3] / Ep;
    Pd[3] = p;
    return status;
}

// ---------------------------------------------------------------------------

struct MixedArgs {
    const double *Un;       // U^n (state layout)
    const float *Din;       // increment of the stage input (nullptr: the input is U^n)
    float *Dout;            // increment of the stage output (nullptr: RHS-only mode writes R)
    float *Rout;            // RHS output (RHS-only mode) or nullptr
    const float *pin;       // SR pressures of the previous pass [e][node] (guesses), or nullptr
    float *pout;            // SR pressures of this stage's input [e][node]
    double *Sn;             // FP64 means of U^n, [e][5][7]: written when write_Sn, read otherwise
    double *S;              // limiter summaries of the output [e][5][10], or nullptr
    unsigned char *unphys;  // SR: per-element unphysical flag of the output, or nullptr
    unsigned int *err;
    const double *dt_ptr;
    double dt;
    float cD;               // Dout = cD (Din + dt R)
    int write_Sn;
    int K[3];
    float gamma;
    double gamma_d;
    float g[3], lift0[3], liftN[3];
    float kappa_sw;
    double d_atm, tau_atm;
    float D32[MAXN * MAXN], w32[MAXN], row1_32[MAXN];
    double wd[MAXN];
};

// Primitives of one node of the stage input (FP32), with the FP64 polish or the
// FP64 fall-back (fix of a local copy, full FP64 con2prim) where FP32 is not enough.
template <int NP, int SYS>
__device__ __forceinline__ void node_prims_mixed(const MixedArgs &a, long long e, int q, const float u[5], float P[4],
                                                 unsigned &errs)
{
    constexpr int NN = NP * NP * NP;
    if (SYS == 0) {
        ne_primitives32(a.gamma, u, P);
        return;
    }
    const float guess = a.pin ? a.pin[e * NN + q] : -1.0f;
    float kappa = 1.0f;
    const int st = sr_con2prim32(a.gamma, u, guess, P, kappa);
    if (st == 0 && kappa <= a.kappa_sw) return;
    // FP64 conserved state of the node
    double u64[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        u64[v] = a.Un[(e * 5 + v) * NN + q];
        if (a.Din) u64[v] += f32_to_f64(a.Din[(e * 5 + v) * NN + q]);
    }
    double Pd[4];
    int st64 = 1;
    if (st == 0) st64 = sr_polish64(a.gamma_d, u64, f32_to_f64(P[3]), Pd);
    if (st64 != 0) {
        // unphysical in FP32 or in FP64: recover from the fixed FP64 state,
        // starting from the previous pass's pressure
        sr_fix(a.d_atm, a.tau_atm, u64);
        st64 = sr_polish64(a.gamma_d, u64, guess >= 0.0f ? f32_to_f64(guess) : -1.0, Pd);
    }
    if (st64) errs |= ERRBIT_C2P;
#pragma unroll
    for (int c = 0; c < 4; ++c) P[c] = f64_to_f32(Pd[c]);
}

template <int NP, int SYS, int FLX>
__global__ void __launch_bounds__(round_up32(NP *NP *NP)) k_stage_mixed(const MixedArgs a)
{
    constexpr int NN = NP * NP * NP;
    extern __shared__ float smem_mixed[];
    float *sF = smem_mixed;     // [3][5][NN] fluxes, later the output increment [5][NN]
    float *sR = sF + 15 * NN;   // [5][NN] right-hand side
    float *sU = sR + 5 * NN;    // [5][NN] stage input state, later the output state
    float *sP = sU + 5 * NN;    // [4][NN] primitives of the input
    __shared__ float sD[NP * NP], sW[NP], sRow1[NP];
    __shared__ double sSn[35];
    __shared__ long long sNb[6];

    const int t = threadIdx.x;
    const long long e = blockIdx.x;
    for (int i = t; i < NP * NP; i += blockDim.x) sD[i] = a.D32[i];
    if (t < NP) {
        sW[t] = a.w32[t];
        sRow1[t] = a.row1_32[t];
    }
    if (t < 6) sNb[t] = elem_neighbour(e, a.K, t >> 1, (t & 1) ? 1 : -1);
    unsigned errs = 0;

    if (t < NN) {
        float u[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            u[v] = f64_to_f32(a.Un[(e * 5 + v) * NN + t]);
            if (a.Din) u[v] += a.Din[(e * 5 + v) * NN + t];
            sU[v * NN + t] = u[v];
        }
        float P[4];
        node_prims_mixed<NP, SYS>(a, e, t, u, P, errs);
        if (SYS == 1 && a.pout) a.pout[e * NN + t] = P[3];
#pragma unroll
        for (int c = 0; c < 4; ++c) sP[c * NN + t] = P[c];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            float f[5];
            flux_axis32(u, P, ax, f);
#pragma unroll
            for (int v = 0; v < 5; ++v) sF[(ax * 5 + v) * NN + t] = f[v];
        }
    }
    // FP64 cell and face means of U^n (stage 1), or their stored values
    if (a.S) {
        for (int id = t; id < 35; id += blockDim.x) {
            const int v = id / 7, kind = id % 7;
            double r;
            if (a.write_Sn) {
                const double *Uv = a.Un + (e * 5 + v) * NN;
                if (kind == 0) {
                    double s = 0.0;
                    for (int k = 0; k < NP; ++k)
                        for (int j = 0; j < NP; ++j)
                            for (int i = 0; i < NP; ++i) s += a.wd[i] * a.wd[j] * a.wd[k] * Uv[i + NP * (j + NP * k)];
                    r = s * 0.125;
                } else {
                    const int ax = (kind - 1) / 2, ia = ((kind - 1) % 2) ? NP - 1 : 0;
                    const int b = (ax + 1) % 3, c = (ax + 2) % 3;
                    double s = 0.0;
                    for (int t1 = 0; t1 < NP; ++t1)
                        for (int t0 = 0; t0 < NP; ++t0) {
                            int id3[3];
                            id3[ax] = ia;
                            id3[b] = t0;
                            id3[c] = t1;
                            s += a.wd[t0] * a.wd[t1] * Uv[id3[0] + NP * (id3[1] + NP * id3[2])];
                        }
                    r = s * 0.25;
                }
                a.Sn[e * 35 + id] = r;
            } else {
                r = a.Sn[e * 35 + id];
            }
            sSn[id] = r;
        }
    }
    __syncthreads();
    // Subtract node 0's flux per axis and variable: D annihilates constants, so
    // the contraction is unchanged in exact arithmetic, and in FP32 its rounding
    // scales with the flux variation inside the element instead of its size.
    {
        float ref[15];
#pragma unroll
        for (int c = 0; c < 15; ++c) ref[c] = sF[c * NN];
        __syncthreads();
        if (t < NN)
#pragma unroll
            for (int c = 0; c < 15; ++c) sF[c * NN + t] -= ref[c];
    }
    __syncthreads();

    // volume term in FP32
    if (t < NN) {
        const int i = t % NP, j = (t / NP) % NP, k = t / (NP * NP);
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            const float *Fx = sF + (0 * 5 + v) * NN;
            const float *Fy = sF + (1 * 5 + v) * NN;
            const float *Fz = sF + (2 * 5 + v) * NN;
            float sx = 0.0f, sy = 0.0f, sz = 0.0f;
#pragma unroll
            for (int l = 0; l < NP; ++l) {
                sx = fmaf(sD[i * NP + l], Fx[l + NP * (j + NP * k)], sx);
                sy = fmaf(sD[j * NP + l], Fy[i + NP * (l + NP * k)], sy);
                sz = fmaf(sD[k * NP + l], Fz[i + NP * (j + NP * l)], sz);
            }
            sR[v * NN + t] = -(a.g[0] * sx + a.g[1] * sy + a.g[2] * sz);
        }
    }
    __syncthreads();

    // surface terms; the neighbour's face node is recovered here from U^n + Din
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
            const long long en = sNb[2 * ax + side];
            float uo[5], Po[4], un[5], Pn[4];
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                uo[v] = sU[v * NN + q];
                un[v] = f64_to_f32(a.Un[(en * 5 + v) * NN + qn]);
                if (a.Din) un[v] += a.Din[(en * 5 + v) * NN + qn];
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) Po[c] = sP[c * NN + q];
            node_prims_mixed<NP, SYS>(a, en, qn, un, Pn, errs);
            float dL[5], dR[5];
            if (side) {
                num_flux_jump32<SYS, FLX>(a.gamma, ax, uo, Po, un, Pn, dL, dR);
#pragma unroll
                for (int v = 0; v < 5; ++v) sR[v * NN + q] -= a.liftN[ax] * dL[v];
            } else {
                num_flux_jump32<SYS, FLX>(a.gamma, ax, un, Pn, uo, Po, dL, dR);
#pragma unroll
                for (int v = 0; v < 5; ++v) sR[v * NN + q] += a.lift0[ax] * dR[v];
            }
        }
        __syncthreads();
    }
    if (errs) atomicOr(a.err, errs);

    // stage increment and FP32 output state.  The limiter summaries and the
    // unphysical flag see the output before the conserved fix (Sec. 3.3: limit,
    // then fix); the stored increment carries the fix, which is exact for elements
    // the limiter leaves alone, and the limiter re-applies it where it rewrites.
    bool bad = false, needfix = false;
    if (t < NN) {
        const float dt = (float)(a.dt_ptr ? *a.dt_ptr : a.dt);
        float d[5], un[5], dfix[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            const float R = sR[v * NN + t];
            if (a.Rout) a.Rout[(e * 5 + v) * NN + t] = R;
            const float din = a.Din ? a.Din[(e * 5 + v) * NN + t] : 0.0f;
            d[v] = a.cD * (din + dt * R);
            un[v] = f64_to_f32(a.Un[(e * 5 + v) * NN + t]) + d[v];
            dfix[v] = d[v];
        }
        if (SYS == 1) {
            // decided on the FP64 state wherever FP32 cannot rule the bounds out
            const float s2 = un[1] * un[1] + un[2] * un[2] + un[3] * un[3];
            if (!(un[0] > 2.0f * (float)a.d_atm) || !(un[4] > 2.0f * (float)a.tau_atm * un[0]) ||
                !(s2 < 0.999f * un[4] * (un[4] + 2.0f * un[0]))) {
                double u64[5], f64v[5];
#pragma unroll
                for (int v = 0; v < 5; ++v) {
                    u64[v] = a.Un[(e * 5 + v) * NN + t] + f32_to_f64(d[v]);
                    f64v[v] = u64[v];
                }
                bad = sr_unphysical(u64);
                if (a.Dout && sr_fix(a.d_atm, a.tau_atm, f64v)) {
                    needfix = true;
#pragma unroll
                    for (int v = 0; v < 5; ++v)
                        if (f64v[v] != u64[v]) dfix[v] = f64_to_f32(f64v[v] - a.Un[(e * 5 + v) * NN + t]);
                }
            }
        }
        // with the limiter on, the fix waits for it (flagged elements only)
        const bool defer = a.S != nullptr;
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            if (a.Dout) a.Dout[(e * 5 + v) * NN + t] = defer ? d[v] : dfix[v];
            sF[v * NN + t] = d[v];
            sU[v * NN + t] = un[v];
        }
    }
    if (a.S == nullptr) return;
    const int anybad = __syncthreads_or(bad);
    const int anyfix = __syncthreads_or(needfix);
    // summaries: FP64 means of U^n + FP32 means of the increment; FP32 slopes
    for (int id = t; id < 50; id += blockDim.x) {
        const int v = id / 10, kind = id % 10;
        const float *Dv = sF + v * NN;
        double r;
        if (kind == 0) {
            float s = 0.0f;
            for (int k = 0; k < NP; ++k)
                for (int j = 0; j < NP; ++j)
                    for (int i = 0; i < NP; ++i) s = fmaf(sW[i] * sW[j] * sW[k], Dv[i + NP * (j + NP * k)], s);
            r = sSn[v * 7] + f32_to_f64(s * 0.125f);
        } else if (kind <= 6) {
            const int ax = (kind - 1) / 2, ia = ((kind - 1) % 2) ? NP - 1 : 0;
            const int b = (ax + 1) % 3, c = (ax + 2) % 3;
            float s = 0.0f;
            for (int t1 = 0; t1 < NP; ++t1)
                for (int t0 = 0; t0 < NP; ++t0) {
                    int id3[3];
                    id3[ax] = ia;
                    id3[b] = t0;
                    id3[c] = t1;
                    s = fmaf(sW[t0] * sW[t1], Dv[id3[0] + NP * (id3[1] + NP * id3[2])], s);
                }
            r = sSn[v * 7 + kind] + f32_to_f64(s * 0.25f);
        } else {
            const int ax = kind - 7;
            const int b = (ax + 1) % 3, c = (ax + 2) % 3;
            const float *Uv = sU + v * NN;
            float c1 = 0.0f;
            for (int ia = 0; ia < NP; ++ia) {
                float s = 0.0f;
                for (int t1 = 0; t1 < NP; ++t1)
                    for (int t0 = 0; t0 < NP; ++t0) {
                        int id3[3];
                        id3[ax] = ia;
                        id3[b] = t0;
                        id3[c] = t1;
                        s = fmaf(sW[t0] * sW[t1], Uv[id3[0] + NP * (id3[1] + NP * id3[2])], s);
                    }
                c1 = fmaf(sRow1[ia], s * 0.25f, c1);
            }
            r = f32_to_f64(c1);
        }
        a.S[e * 50 + id] = r;
    }
    // bit 0: an unphysical node (limit every variable); bit 1: a node needs the fix
    if (SYS == 1 && t == 0 && a.unphys) a.unphys[e] = (anybad ? 1 : 0) | (anyfix ? 2 : 0);
}

// ---------------------------------------------------------------------------
// Limiter of the mixed path, one warp per element (decision as in k_limit).
// final_pass == 0: stage outputs held as increments; troubled variables get
//   D = (U0 + sum_a slope_a (x_a - x_a0)) - U^n.
// final_pass == 1: U^{n+1} = U^n + D3 at every node (FP64), the linear
//   replacement in troubled variables, then the SR fix in FP64, in place.
struct LimitMixedArgs {
    double *U;              // U^n in, U^{n+1} out (final pass)
    float *Dv;              // increments of the stage output
    const double *S;
    const unsigned char *unphys;
    unsigned char *troubled;
    long long E;
    int K[3];
    int limiter;
    int final_pass;
    double tvb_M, beta;
    double dx[3];
    double d_atm, tau_atm;
    double x[MAXN];
};

// FP32 screen of the conserved-fix bounds; nodes that fail it are decided in FP64.
__device__ __forceinline__ bool sr_fix_screen32(const float u[5], float d_atm, float tau_atm)
{
    const float s2 = u[1] * u[1] + u[2] * u[2] + u[3] * u[3];
    return !(u[0] > 2.0f * d_atm) || !(u[4] > 2.0f * tau_atm * u[0]) ||
           !(s2 < 0.999f * u[4] * (u[4] + 2.0f * u[0]));
}

template <int NP, int SYS>
__global__ void __launch_bounds__(256) k_limit_mixed(const LimitMixedArgs a)
{
    constexpr int NN = NP * NP * NP;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= a.E) return;
    const long long e = warp;
    int flag = 0;
    double sl[3] = {0.0, 0.0, 0.0};
    double U0 = 0.0;
    if (lane < 5 && a.limiter != 0) {
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
    const unsigned char uf = (a.limiter != 0 && a.unphys) ? a.unphys[e] : 0;
    if (uf & 1) mask = 0x1fu;
    if (lane == 0 && a.troubled) a.troubled[e] = (unsigned char)mask;
    if (!mask && !(uf & 2) && !a.final_pass) return;
    // the replacement U0 + sum_a slope_a (x_a - x_a0) (eq:MinModSol) is formed as an
    // FP32 increment of U^n about the FP64 anchor U0 - U^n
    double m0[5];
    float s0[5], s1[5], s2[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        m0[v] = __shfl_sync(0xffffffffu, U0, v);
        s0[v] = f64_to_f32(__shfl_sync(0xffffffffu, sl[0], v));
        s1[v] = f64_to_f32(__shfl_sync(0xffffffffu, sl[1], v));
        s2[v] = f64_to_f32(__shfl_sync(0xffffffffu, sl[2], v));
    }
    const float hx0 = f64_to_f32(0.5 * a.dx[0]), hx1 = f64_to_f32(0.5 * a.dx[1]), hx2 = f64_to_f32(0.5 * a.dx[2]);
    for (int q = lane; q < NN; q += 32) {
        const int i = q % NP, j = (q / NP) % NP, k = q / (NP * NP);
        const float xi = f64_to_f32(a.x[i]) * hx0, xj = f64_to_f32(a.x[j]) * hx1, xk = f64_to_f32(a.x[k]) * hx2;
        double un[5];
        float d[5], u32[5];
        unsigned nm = mask;
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            const long long ix = (e * 5 + v) * NN + q;
            un[v] = a.U[ix];
            if (mask & (1u << v))
                d[v] = f64_to_f32(m0[v] - un[v]) + (s0[v] * xi + s1[v] * xj + s2[v] * xk);
            else
                d[v] = a.Dv[ix];
            u32[v] = f64_to_f32(un[v]) + d[v];
        }
        double u64[5];
        bool exact = false;
        if (SYS == 1 && sr_fix_screen32(u32, (float)a.d_atm, (float)a.tau_atm)) {
            // the conserved fix after the replacement (Sec. 2.1.4, Sec. 3.3), in FP64
#pragma unroll
            for (int v = 0; v < 5; ++v) u64[v] = un[v] + f32_to_f64(d[v]);
            double w[5] = {u64[0], u64[1], u64[2], u64[3], u64[4]};
            if (sr_fix(a.d_atm, a.tau_atm, w)) {
                exact = a.final_pass != 0;
#pragma unroll
                for (int v = 0; v < 5; ++v)
                    if (w[v] != u64[v]) {
                        nm |= 1u << v;
                        d[v] = f64_to_f32(w[v] - un[v]);
                        u64[v] = w[v];
                    }
            }
        }
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            const long long ix = (e * 5 + v) * NN + q;
            if (a.final_pass)
                a.U[ix] = exact ? u64[v] : un[v] + f32_to_f64(d[v]);
            else if (nm & (1u << v))
                a.Dv[ix] = d[v];
        }
    }
}

template <int NP>
cudaError_t launch_stage_mixed_np(int system, int flux, const MixedArgs &a, long long E, cudaStream_t s)
{
    const dim3 grid((unsigned)E), block(round_up32(NP * NP * NP));
    const size_t smem = sizeof(float) * 29 * NP * NP * NP;
    void (*kern)(const MixedArgs);
    if (system == 0 && flux == 0) kern = k_stage_mixed<NP, 0, 0>;
    else if (system == 0) kern = k_stage_mixed<NP, 0, 1>;
    else if (flux == 0) kern = k_stage_mixed<NP, 1, 0>;
    else kern = k_stage_mixed<NP, 1, 1>;
    if (smem > 48 * 1024) {
        cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
    }
    kern<<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
}

template <int NP>
cudaError_t launch_limit_mixed_np(int system, const LimitMixedArgs &a, cudaStream_t s)
{
    const long long threads = a.E * 32;
    const unsigned grid = (unsigned)((threads + 255) / 256);
    if (system == 0) k_limit_mixed<NP, 0><<<grid, 256, 0, s>>>(a);
    else k_limit_mixed<NP, 1><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace dg

#define DG_INSTANTIATE_MIXED(NP)                                                                       \
    namespace dg {                                                                                     \
    cudaError_t launch_stage_mixed_n##NP(int system, int flux, const MixedArgs &a, long long E,         \
                                         cudaStream_t s)                                               \
    {                                                                                                  \
        return launch_stage_mixed_np<NP>(system, flux, a, E, s);                                       \
    }                                                                                                  \
    cudaError_t launch_limit_mixed_n##NP(int system, const LimitMixedArgs &a, cudaStream_t s)           \
    {                                                                                                  \
        return launch_limit_mixed_np<NP>(system, a, s);                                                \
    }                                                                                                  \
    }
