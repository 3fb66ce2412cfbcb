// dg_physics.cuh -- point-wise physics of the two conservation laws, FP64,
// device side (Sec. 2.1.1 Newtonian Euler, Sec. 2.1.2 SR hydro in flat space,
// Sec. 3.2 numerical fluxes, Sec. 2.1.4 conserved-variable fix).
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace dg {

// Status bits of the per-mesh device status word.
enum : unsigned { ERRBIT_C2P = 1u, ERRBIT_UNPHYSICAL = 2u, ERRBIT_TIMEOUT = 4u };

// ---------------------------------------------------------------------------
// Newtonian Euler: U = [rho, rho v_i, E], E = rho eps + rho v^2/2, p = (g-1) rho eps.
__device__ __forceinline__ void ne_primitives(double g, const double u[5], double P[4])
{
    const double inv = 1.0 / u[0];
    P[0] = u[1] * inv;
    P[1] = u[2] * inv;
    P[2] = u[3] * inv;
    P[3] = (g - 1.0) * (u[4] - 0.5 * (u[1] * P[0] + u[2] * P[1] + u[3] * P[2]));
}

// ---------------------------------------------------------------------------
// SR con2prim.  With E = tau + D and s = |S|, the pressure is the root of
//   f(p) = p - (g-1) rho eps(p),  v = s/(E+p), W = (1-v^2)^(-1/2), rho = D/W,
//   rho eps = tau - v^2 [(E+p) - D W/(W+1)]   (from the definitions of D, S, tau),
//   f'(p) = 1 - (g-1) v^2 (1 - D W/(E+p)),
// bracketed by [max(0, s-E), (g-1) tau]; Newton steps that leave the bracket
// become bisections, except a step landing exactly on an end that is still its
// a-priori bound (at v = 0 the root is (g-1) tau itself); the bracket follows
// the sign of f; stop once
// |dp| <= 2^-48 p and take one more Newton step.
struct C2PEval {
    double f, df;
};

__device__ __forceinline__ C2PEval sr_c2p_eval(double g, double D, double s2, double tau, double p)
{
    C2PEval r;
    const double Ep = tau + D + p;
    const double v2 = s2 / (Ep * Ep);
    const double W = 1.0 / sqrt(1.0 - v2);
    const double rhoeps = tau - v2 * (Ep - D * W / (W + 1.0));
    r.f = p - (g - 1.0) * rhoeps;
    r.df = 1.0 - (g - 1.0) * v2 * (1.0 - D * W / Ep);
    return r;
}

__device__ __forceinline__ bool sr_unphysical(const double u[5])
{
    const double s2 = u[1] * u[1] + u[2] * u[2] + u[3] * u[3];
    return !(u[0] > 0.0) || !(u[4] > 0.0) || !(s2 < u[4] * (u[4] + 2.0 * u[0]));
}

// Returns 0 ok, 1 unphysical input, 2 no convergence.  prim = (rho, vx, vy, vz, p).
// guess < 0 selects the standard guess (g-1) tau.
__device__ __forceinline__ int sr_con2prim(double g, const double u[5], double guess, double prim[5],
                                           int *iters)
{
    const double D = u[0], tau = u[4];
    const double s2 = u[1] * u[1] + u[2] * u[2] + u[3] * u[3];
    *iters = 0;
    if (!(D > 0.0) || !(tau > 0.0) || !(s2 < tau * (tau + 2.0 * D))) {
        for (int v = 0; v < 5; ++v) prim[v] = __longlong_as_double(0x7ff8000000000000LL);
        return 1;
    }
    const double E = tau + D;
    double plo = sqrt(s2) - E;
    if (plo < 0.0) plo = 0.0;
    double phi = (g - 1.0) * tau;
    double p = (guess >= 0.0) ? guess : phi;
    if (p < plo) p = plo;
    if (p > phi) p = phi;
    int status = 2;
    bool lo_moved = false, hi_moved = false;  // an end still at its a-priori bound may be landed on
    int it = 0;
    for (; it < 200; ++it) {
        const C2PEval r = sr_c2p_eval(g, D, s2, tau, p);
        if (r.f == 0.0) { status = 0; break; }
        if (r.f > 0.0) { phi = p; hi_moved = true; } else { plo = p; lo_moved = true; }
        double pn = p - r.f / r.df;
        if (!((pn > plo && pn < phi) || (pn == phi && !hi_moved) || (pn == plo && !lo_moved)))
            pn = 0.5 * (plo + phi);
        const double dp = fabs(pn - p);
        p = pn;
        if (dp <= 0x1p-48 * p) {
            const C2PEval r2 = sr_c2p_eval(g, D, s2, tau, p);
            p = p - r2.f / r2.df;
            it += 1;
            status = 0;
            break;
        }
        if (phi - plo <= 0.0) { status = 0; break; }
    }
    *iters = it + 1;
    const double Ep = E + p;
    prim[0] = D * sqrt(1.0 - s2 / (Ep * Ep));
    prim[1] = u[1] / Ep;
    prim[2] = u[2] / Ep;
    prim[3] = u[3] / Ep;
    prim[4] = p;
    return status;
}

// Flux-relevant primitives (vx, vy, vz, p) of either system; returns c2p status.
template <int SYS>
__device__ __forceinline__ int node_primitives(double g, const double u[5], double P[4])
{
    if (SYS == 0) {
        ne_primitives(g, u, P);
        return 0;
    }
    double pr[5];
    int it;
    const int st = sr_con2prim(g, u, -1.0, pr, &it);
    P[0] = pr[1];
    P[1] = pr[2];
    P[2] = pr[3];
    P[3] = pr[4];
    return st;
}

// ---------------------------------------------------------------------------
// Physical flux along axis a, common to both systems with alpha = 1, beta = 0:
// F = [U0 v_a, S_i v_a + p delta_ia, (U4 + p) v_a].
__device__ __forceinline__ void flux_axis(const double u[5], const double P[4], int a, double F[5])
{
    const double va = P[a], p = P[3];
    F[0] = u[0] * va;
    F[1] = u[1] * va;
    F[2] = u[2] * va;
    F[3] = u[3] * va;
    F[1 + a] = F[1 + a] + p;
    F[4] = (u[4] + p) * va;
}

// Extreme characteristic speeds along axis a (eq:CharDecomp).
template <int SYS>
__device__ __forceinline__ void speeds_axis(double g, const double u[5], const double P[4], int a,
                                            double &lmin, double &lmax)
{
    const double va = P[a], p = P[3];
    if (SYS == 0) {
        const double c = sqrt(g * p / u[0]);
        lmin = va - c;
        lmax = va + c;
        return;
    }
    const double v2 = P[0] * P[0] + P[1] * P[1] + P[2] * P[2];
    const double rhoh = (u[4] + u[0] + p) * (1.0 - v2);
    const double cs2 = g * p / rhoh;
    const double cs = sqrt(cs2);
    double disc = (1.0 - v2) * (1.0 - v2 * cs2 - va * va * (1.0 - cs2));
    if (disc < 0.0) disc = 0.0;
    const double root = cs * sqrt(disc);
    const double den = 1.0 - v2 * cs2;
    lmin = (va * (1.0 - cs2) - root) / den;
    lmax = (va * (1.0 - cs2) + root) / den;
}

// Numerical flux along +e_a between the lower state L and the upper state R:
// FLX = 0 local Lax-Friedrichs (eq:LLF), 1 HLL with Davis speeds (eq:HLL).
// Roe dissipation D = sum_i alpha_i |lambda_i| e_i of eq:Roe for the Newtonian
// ideal gas (Sec. 3.2.3): the flux Jacobian along e_a at the Roe averages
// (eq:RoeAverages) of the velocity and of h = (E + p)/rho, eigenvalues u_n - c,
// u_n (x3), u_n + c with c^2 = (g-1)(h - |v|^2/2), wave strengths from the jump on
// the left eigenvectors in the frame (normal, t1, t2) = (a, a+1, a+2).
__device__ __forceinline__ void roe_dissipation(double g, int a, const double uL[5], const double PL[4],
                                                const double uR[5], const double PR[4], double D[5])
{
    const double sl = sqrt(uL[0]), sr = sqrt(uR[0]);
    const double wsum = sl + sr;
    double vh[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) vh[i] = (sl * PL[i] + sr * PR[i]) / wsum;
    const double hL = (uL[4] + PL[3]) / uL[0], hR = (uR[4] + PR[3]) / uR[0];
    const double hh = (sl * hL + sr * hR) / wsum;
    const double q2 = vh[0] * vh[0] + vh[1] * vh[1] + vh[2] * vh[2];
    const double c2 = (g - 1.0) * (hh - 0.5 * q2);
    const double c = sqrt(c2);
    const int b = (a + 1) % 3, d = (a + 2) % 3;
    const double un = vh[a], ut1 = vh[b], ut2 = vh[d];
    const double j1 = uR[0] - uL[0], jn = uR[1 + a] - uL[1 + a];
    const double jt1 = uR[1 + b] - uL[1 + b], jt2 = uR[1 + d] - uL[1 + d], j5 = uR[4] - uL[4];
    const double al3 = jt1 - ut1 * j1;
    const double al4 = jt2 - ut2 * j1;
    const double j5b = j5 - al3 * ut1 - al4 * ut2;
    const double al2 = (g - 1.0) / c2 * (j1 * (hh - un * un) + un * jn - j5b);
    const double al1 = (j1 * (un + c) - jn - c * al2) / (2.0 * c);
    const double al5 = j1 - (al1 + al2);
    const double w1 = fabs(un - c) * al1, w2 = fabs(un) * al2, w5 = fabs(un + c) * al5;
    const double w3 = fabs(un) * al3, w4 = fabs(un) * al4;
    D[0] = w1 + w2 + w5;
    D[1 + a] = w1 * (un - c) + w2 * un + w5 * (un + c);
    D[1 + b] = (w1 + w2 + w5) * ut1 + w3;
    D[1 + d] = (w1 + w2 + w5) * ut2 + w4;
    D[4] = w1 * (hh - un * c) + w2 * (0.5 * q2) + w3 * ut1 + w4 * ut2 + w5 * (hh + un * c);
}

template <int SYS, int FLX>
__device__ __forceinline__ void num_flux(double g, int a, const double uL[5], const double PL[4],
                                         const double uR[5], const double PR[4], double Fs[5],
                                         double FL[5], double FR[5])
{
    double lminL, lmaxL, lminR, lmaxR;
    flux_axis(uL, PL, a, FL);
    flux_axis(uR, PR, a, FR);
    if (FLX == 2) {  // Roe (Newtonian only)
        double D[5];
        roe_dissipation(g, a, uL, PL, uR, PR, D);
#pragma unroll
        for (int v = 0; v < 5; ++v) Fs[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * D[v];
        return;
    }
    speeds_axis<SYS>(g, uL, PL, a, lminL, lmaxL);
    speeds_axis<SYS>(g, uR, PR, a, lminR, lmaxR);
    if (FLX == 0) {
        const double al = fmax(fmax(fabs(lminL), fabs(lmaxL)), fmax(fabs(lminR), fabs(lmaxR)));
#pragma unroll
        for (int v = 0; v < 5; ++v) Fs[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * al * (uR[v] - uL[v]);
    } else {
        const double cmin = fmin(fmin(lminL, lminR), 0.0);
        const double cmax = fmax(fmax(lmaxL, lmaxR), 0.0);
        const double den = cmax - cmin;
        if (den > 0.0) {
#pragma unroll
            for (int v = 0; v < 5; ++v)
                Fs[v] = (cmax * FL[v] - cmin * FR[v]) / den + (cmin * cmax / den) * (uR[v] - uL[v]);
        } else {
#pragma unroll
            for (int v = 0; v < 5; ++v) Fs[v] = 0.5 * (FL[v] + FR[v]);
        }
    }
}

// Largest |characteristic speed| over the three axes.
template <int SYS>
__device__ __forceinline__ double max_speed(double g, const double u[5], const double P[4])
{
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double lo, hi;
        speeds_axis<SYS>(g, u, P, a, lo, hi);
        s = fmax(s, fmax(fabs(lo), fabs(hi)));
    }
    return s;
}

// SR conserved-variable fix (Sec. 2.1.4): D >= d_atm, tau >= tau_atm D and
// S^2 <= (1 - 1e-12) tau (tau + 2D).  Returns the variables it set, as a bit
// mask (bit v for u[v]; the three momenta together), 0 if u is unchanged.
__device__ __forceinline__ unsigned sr_fix(double d_atm, double tau_atm, double u[5])
{
    unsigned ch = 0;
    if (!(u[0] >= d_atm)) { u[0] = d_atm; ch |= 1u; }
    const double tmin = tau_atm * u[0];
    if (!(u[4] >= tmin)) { u[4] = tmin; ch |= 16u; }
    const double s2 = u[1] * u[1] + u[2] * u[2] + u[3] * u[3];
    const double s2max = (1.0 - 1e-12) * (u[4] * (u[4] + 2.0 * u[0]));
    if (s2 > s2max) {
        const double f = sqrt(s2max / s2);
        u[1] *= f;
        u[2] *= f;
        u[3] *= f;
        ch |= 14u;
    }
    return ch;
}

// minmod of three slopes (eq:MinMod) and the TVB-bounded m_B (eq:MinModB).
__device__ __forceinline__ double minmod3(double a1, double a2, double a3)
{
    if (a1 > 0.0 && a2 > 0.0 && a3 > 0.0) return fmin(a1, fmin(a2, a3));
    if (a1 < 0.0 && a2 < 0.0 && a3 < 0.0) return fmax(a1, fmax(a2, a3));
    return 0.0;
}

__device__ __forceinline__ double minmodB(double a1, double a2, double a3, double M, double h)
{
    if (fabs(a1) <= M * h * h) return a1;
    return minmod3(a1, a2, a3);
}

}  // namespace dg
