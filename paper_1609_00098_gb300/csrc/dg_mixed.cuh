// dg_mixed.cuh -- mixed-precision DG stage kernels (templated on the number of
// LGL nodes per axis NP).
//
// The state and every SSP-RK3 stage state stay FP64 (Sec. 3.4), and so do the
// limiter's replacement and the conserved fix acting on them; the right-hand side
// (eq:411) is evaluated in FP32: SR con2prim from the previous pass's pressure,
// fluxes, the tensor-product contraction (eq:405), the numerical fluxes (eq:LLF,
// eq:HLL) and the lift.  The stage update adds an FP32 increment to the FP64 state,
// U_{s+1} = U_s + [ca (U^n - U_s) + cb dt R].  FP64 work is kept warp-uniform
// (a warp-wide FP64 instruction costs the whole SM's FP64 pipe for ~17 cycles on
// this GPU, with or without inactive lanes); FP64<->FP32 conversions use integer
// operations because the conversion instructions issue at the FP64 rate.
#pragma once

#include "dg_c2p_net.cuh"
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
// Split-BF16x3 products on the tensor cores: x = x_hi + x_mid + x_lo with each
// part the BF16 rounding of what the previous parts leave (24 significant bits in
// all), and a product kept as the six partial products of order >= 2^-16
// (lo.hi, hi.lo, mid.mid, mid.hi, hi.mid, hi.hi, smallest first) accumulated in
// FP32 by mma.sync m16n8k8.

__device__ __forceinline__ void split_bf16x3(float x, float part[3])
{
    const float h = __bfloat162float(__float2bfloat16_rn(x));
    const float r = x - h;
    const float m = __bfloat162float(__float2bfloat16_rn(r));
    part[0] = h;
    part[1] = m;
    part[2] = r - m;  // rounded to BF16 when packed
}

__device__ __forceinline__ uint32_t pack2_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ void mma_bf16_k8(float c[4], uint32_t a0, uint32_t a1, uint32_t b)
{
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(b));
}

// ---------------------------------------------------------------------------
// FP32 physics.  Node primitives are held as P = (vx, vy, vz, p, 1 - v^2); the
// last entry is 1 for the Newtonian system.  1 - v^2 comes from FP64 wherever the
// Lorentz factor is large enough for FP32 to lose it (see sr_prims_mixed).

constexpr int NPRIM = 5;

__device__ __forceinline__ void flux_axis32(const float u[5], const float P[NPRIM], int a, float F[5])
{
    const float va = P[a], p = P[3];
    F[0] = u[0] * va;
    F[1] = u[1] * va;
    F[2] = u[2] * va;
    F[3] = u[3] * va;
    F[1 + a] += p;
    F[4] = (u[4] + p) * va;
}

// Wave speeds along axis a: Newtonian v_a -+ c_s; SR the eigenvalues of Sec. 2.1.2
//   lambda = [v_a (1 - cs^2) -+ cs sqrt((1 - v^2)(1 - v^2 cs^2 - v_a^2 (1 - cs^2)))] / (1 - v^2 cs^2),
// with the two factors that cancel as v -> 1 rewritten as sums of non-negative terms,
//   1 - v^2 cs^2 = (1 - v^2) + v^2 (1 - cs^2),
//   1 - v^2 cs^2 - v_a^2 (1 - cs^2) = (1 - v^2) + (1 - cs^2)(v_b^2 + v_c^2),
// so the FP32 speeds keep their accuracy at large Lorentz factors.  A negative
// pressure gives NaN speeds, as in the FP64 path, which fmin/fmax then ignore.
template <int SYS>
__device__ __forceinline__ void speeds_axis32(float g, const float u[5], const float P[NPRIM], int a, float &lmin,
                                              float &lmax)
{
    const float va = P[a], p = P[3];
    if (SYS == 0) {
        const float c = sqrtf(g * p / u[0]);
        lmin = va - c;
        lmax = va + c;
        return;
    }
    const float w2i = P[4];
    const float vb = P[a == 0 ? 1 : 0], vc = P[a == 2 ? 1 : 2];
    const float v2 = P[0] * P[0] + P[1] * P[1] + P[2] * P[2];
    const float rhoh = (u[4] + u[0] + p) * w2i;
    const float cs2 = g * p / rhoh;
    const float cs = sqrtf(cs2);
    const float om = 1.0f - cs2;
    float disc = w2i * (w2i + om * (vb * vb + vc * vc));
    if (disc < 0.0f) disc = 0.0f;
    const float root = cs * sqrtf(disc);
    const float inv = 1.0f / (w2i + v2 * om);
    lmin = (va * om - root) * inv;
    lmax = (va * om + root) * inv;
}

// Numerical flux along +e_a minus each side's physical flux, in jump form:
// with dF = F(U_R) - F(U_L) and dU = U_R - U_L,
//   HLL (eq:HLL):  F* - F_L = -cmin dF/(cmax-cmin) + cmin cmax/(cmax-cmin) dU,
//                  F* - F_R = -cmax dF/(cmax-cmin) + cmin cmax/(cmax-cmin) dU;
//   LLF (eq:LLF):  F* - F_L =  dF/2 - alpha dU/2,  F* - F_R = -dF/2 - alpha dU/2.
// Algebraically the eq:LLF / eq:HLL fluxes; in FP32 the differences are taken
// before they are scaled, so equal states give exactly zero.
template <int SYS, int FLX>
__device__ __forceinline__ void num_flux_jump32(float g, int a, const float uL[5], const float PL[NPRIM],
                                                const float uR[5], const float PR[NPRIM], float dL[5], float dR[5])
{
    float FL[5], FR[5], lminL, lmaxL, lminR, lmaxR;
    flux_axis32(uL, PL, a, FL);
    flux_axis32(uR, PR, a, FR);
    if (FLX == 2) {
        // Roe (eq:Roe, Newtonian): F* - F_L = dF/2 - D/2, F* - F_R = -dF/2 - D/2,
        // with the dissipation D = sum_i alpha_i |lambda_i| e_i at the Roe averages;
        // the wave strengths come from the jump, so equal states give D = 0.
        const float sl = sqrtf(uL[0]), sr = sqrtf(uR[0]);
        const float inv = 1.0f / (sl + sr);
        float vh[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) vh[i] = (sl * PL[i] + sr * PR[i]) * inv;
        const float hL = (uL[4] + PL[3]) / uL[0], hR = (uR[4] + PR[3]) / uR[0];
        const float hh = (sl * hL + sr * hR) * inv;
        const float q2 = vh[0] * vh[0] + vh[1] * vh[1] + vh[2] * vh[2];
        const float c2 = (g - 1.0f) * (hh - 0.5f * q2);
        const float c = sqrtf(c2);
        const int b = a == 0 ? 1 : (a == 1 ? 2 : 0), d = a == 0 ? 2 : (a == 1 ? 0 : 1);
        const float un = vh[a], ut1 = vh[b], ut2 = vh[d];
        const float j1 = uR[0] - uL[0], jn = uR[1 + a] - uL[1 + a];
        const float jt1 = uR[1 + b] - uL[1 + b], jt2 = uR[1 + d] - uL[1 + d], j5 = uR[4] - uL[4];
        const float al3 = jt1 - ut1 * j1;
        const float al4 = jt2 - ut2 * j1;
        const float j5b = j5 - al3 * ut1 - al4 * ut2;
        const float al2 = (g - 1.0f) / c2 * (j1 * (hh - un * un) + un * jn - j5b);
        const float al1 = (j1 * (un + c) - jn - c * al2) / (2.0f * c);
        const float al5 = j1 - (al1 + al2);
        const float w1 = fabsf(un - c) * al1, w2 = fabsf(un) * al2, w5 = fabsf(un + c) * al5;
        const float w3 = fabsf(un) * al3, w4 = fabsf(un) * al4;
        float D[5];
        D[0] = w1 + w2 + w5;
        D[1 + a] = w1 * (un - c) + w2 * un + w5 * (un + c);
        D[1 + b] = (w1 + w2 + w5) * ut1 + w3;
        D[1 + d] = (w1 + w2 + w5) * ut2 + w4;
        D[4] = w1 * (hh - un * c) + w2 * (0.5f * q2) + w3 * ut1 + w4 * ut2 + w5 * (hh + un * c);
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            const float dF = FR[v] - FL[v];
            dL[v] = 0.5f * dF - 0.5f * D[v];
            dR[v] = -0.5f * dF - 0.5f * D[v];
        }
        return;
    }
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

// Node-index stride of axis x (1, NP, NP^2) and a component chosen by a runtime
// axis, both by selection: indexing a register array with a runtime value would
// move it to local memory.
template <int NP>
__device__ __forceinline__ int axis_stride(int x)
{
    return x == 0 ? 1 : (x == 1 ? NP : NP * NP);
}
__device__ __forceinline__ float pick3(int k, float x0, float x1, float x2) { return k == 0 ? x0 : (k == 1 ? x1 : x2); }

__device__ __forceinline__ void ne_primitives32(float g, const float u[5], float P[NPRIM])
{
    const float inv = 1.0f / u[0];
    P[0] = u[1] * inv;
    P[1] = u[2] * inv;
    P[2] = u[3] * inv;
    P[3] = (g - 1.0f) * (u[4] - 0.5f * (u[1] * P[0] + u[2] * P[1] + u[3] * P[2]));
    P[4] = 1.0f;
}

// FP32 SR con2prim: the safeguarded Newton of the FP64 path in FP32 (with
// geometric bisection across wide brackets), stopping when the step is below
// 2^-21 p or the residual is at the FP32 noise level of its terms.  Returns 0 ok, 1 unphysical in FP32, 2 no convergence; kappa gets
// tau/(rho eps), the amplification of input rounding into p.
__device__ __forceinline__ int sr_con2prim32(float g, const float u[5], float guess, float P[NPRIM], float &kappa)
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
    bool lo_moved = false, hi_moved = false;
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
        if (f > 0.0f) { phi = p; hi_moved = true; } else { plo = p; lo_moved = true; }
        float pn = p - f / df;
        // Newton steps that leave the bracket become bisections: geometric while the
        // bracket spans more than a factor 4 (a cold state's pressure can sit many
        // decades below the bracket's top, (g-1) tau, where halving needs ~20 steps),
        // arithmetic below that
        if (!((pn > plo && pn < phi) || (pn == phi && !hi_moved) || (pn == plo && !lo_moved)))
            pn = phi > 4.0f * plo ? sqrtf(fmaxf(plo, 0x1p-40f * phi) * phi) : 0.5f * (plo + phi);
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
    P[4] = 1.0f - (P[0] * P[0] + P[1] * P[1] + P[2] * P[2]);
    kappa = tau / fmaxf(rhoeps, 1e-30f);
    return status;
}

// FP64 Newton on the pressure from a starting value p0 (the FP32 result, or the
// standard guess when p0 < 0), on the FP64 conserved state u: the bracket and
// step rules of sr_con2prim32 in FP64, stopping when the step is below 2^-40 p or
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
    bool lo_moved = false, hi_moved = false;
    for (int it = 0; it < 60; ++it) {
        const double Ep = E + p;
        const double v2 = s2 / (Ep * Ep);
        const double W = 1.0 / sqrt(1.0 - v2);
        const double DW = D * W;
        const double rhoeps = tau - v2 * (Ep - DW / (W + 1.0));
        const double f = p - (g - 1.0) * rhoeps;
        const double df = 1.0 - (g - 1.0) * v2 * (1.0 - DW / Ep);
        if (fabs(f) <= 0x1p-50 * (p + (g - 1.0) * (tau + v2 * Ep))) { status = 0; break; }
        if (f > 0.0) { phi = p; hi_moved = true; } else { plo = p; lo_moved = true; }
        double pn = p - f / df;
        if (!((pn > plo && pn < phi) || (pn == phi && !hi_moved) || (pn == plo && !lo_moved)))
            pn = phi > 4.0 * plo ? sqrt(fmax(plo, 0x1p-40 * phi) * phi) : 0.5 * (plo + phi);
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
// Per-mesh part of a stage launch.  A launch advances one mesh (its slot passed
// inline) or a ragged batch of meshes that share n, the system, the flux, the
// limiter setting and the guess mode (slot table and element offsets in device
// memory; each CTA finds its mesh by binary search over the offsets).
struct MeshSlot {
    const double *Us;       // stage input (state layout, FP64)
    const double *Un;       // U^n (stages 2, 3)
    double *out;            // stage output U_{s+1} (mode 1) or dU/dt (mode 0)
    const float *pin;       // SR pressures of the previous pass [e][node] (guesses), or nullptr
    float *pout;            // SR pressures of this stage's input [e][node], or nullptr
    const float *Pin;       // SR: FP32 primitives [e][NPRIM][node] of U_s already solved (the
                            // CFL pass's, for stage 1), or nullptr: no con2prim then
    double *S;              // limiter summaries of the output [e][5][10], or nullptr
    unsigned char *flags;   // SR: bit 0 unphysical node, bit 1 a node needs the fix (limiter on)
    unsigned int *err;
    const double *dt_ptr;
    double dt;
    int K[3];
    Ghosts gh;              // analytic boundaries (Newtonian; mask 0: periodic)
    float g[3], lift0[3], liftN[3];
};

struct MixedArgs {
    MeshSlot one;                    // the mesh of a single-mesh launch
    const MeshSlot *slots;           // batch: per-mesh slots, or nullptr
    const long long *elem0;          // batch: first element of each mesh in the launch (nslots entries)
    int nslots;
    long long nelem;                 // elements in the launch
    int epb;                         // elements per CTA
    int lim;                         // limiter on: write summaries and flags, leave the SR fix to it
    float ca, cb;           // U_{s+1} = ca U^n + cb (U_s + dt R) = U_s + ca (U^n - U_s) + cb dt R
    int first;              // first stage: U_{s+1} = U_s + dt R
    int mode;               // 0: dU/dt, 1: stage update
    float gamma;
    double gamma_d;
    float kappa_sw;
    double d_atm, tau_atm;
    int tc;                          // volume contraction: 1 split-BF16x3 tensor cores, 0 FP32 FMA
    const NetWeightsSmem *netImg;    // learned-guess network: its shared-memory image, or nullptr
    float net_sc[6];                 // its feature scales
    float D32[MAXN * MAXN];
    double w64[MAXN], row1_64[MAXN];
};

constexpr int CFL_CHUNK = 256;  // nodes per CTA of the CFL pass

// Per-mesh part of a CFL launch; a launch covers one mesh or a ragged batch of
// meshes with the same n and system, in chunks of CFL_CHUNK nodes (a chunk never
// spans two meshes, so the block maximum goes to one mesh's slot).
struct CflSlot {
    const double *Un;
    const float *pin;              // previous pass's pressures (guesses), or nullptr
    float *pout;                   // this pass's pressures, or nullptr
    float *Pout;                   // SR: this pass's FP32 primitives [e][NPRIM][node], or nullptr
    unsigned long long *lam;
    unsigned int *err;
    long long nodes;
};

struct CflArgs {
    CflSlot one;
    const CflSlot *slots;          // batch: per-mesh slots, or nullptr
    const long long *chunk0;       // batch: first chunk of each mesh
    int nslots;
    int nn;
    float gamma;
    double gamma_d;
    float kappa_sw;
    double d_atm, tau_atm;
    const NetWeightsSmem *netImg;  // learned-guess network: its shared-memory image, or nullptr
    float net_sc[6];
};

__device__ __forceinline__ int find_slot(const long long *elem0, int nslots, long long ge)
{
    int lo = 0, hi = nslots - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (elem0[mid] <= ge) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// SR primitives of one node, u the FP32 copy of the FP64 state Ub[v * stride]:
// FP32 con2prim from `guess`; where the conditioning estimate tau/(rho eps)
// exceeds kappa_sw (this covers every large Lorentz factor too:
// tau/(rho eps) = W(W-1)/eps + W^2 + (gamma-1)(W^2-1) >= W^2), or FP32 cannot
// resolve physicality, FP64
// Newton on the FP64 state finishes it and 1 - v^2 is formed in FP64.  Cold
// states whose pressure bracket (gamma-1) tau is below 2^-20 E keep the FP32
// value: any pressure in that bracket leaves the fluxes unchanged at FP32
// accuracy, and such states have v^2 < 2 tau / D, so 1 - v^2 is exact enough.
// Returns ERRBIT_C2P where FP64 Newton fails too, else 0.
__device__ __forceinline__ unsigned sr_prims_mixed(float g, double gd, float kappa_sw, double d_atm, double tau_atm,
                                                   const float u[5], const double *Ub, long long stride, float guess,
                                                   float P[NPRIM])
{
    float kappa = 1.0f;
    const int st = sr_con2prim32(g, u, guess, P, kappa);
    if (st == 0 && kappa <= kappa_sw) return 0u;
    if ((g - 1.0f) * u[4] <= 0x1p-20f * (u[4] + u[0]) && u[0] > 0.0f && u[4] >= 0.0f) {
        if (st != 0) {
            // cold and unresolved in FP32: mid-bracket pressure, v = S/(E+p)
            const float p = 0.5f * (g - 1.0f) * u[4];
            const float inv = 1.0f / (u[4] + u[0] + p);
            P[0] = u[1] * inv;
            P[1] = u[2] * inv;
            P[2] = u[3] * inv;
            P[3] = p;
            P[4] = 1.0f - (P[0] * P[0] + P[1] * P[1] + P[2] * P[2]);
        }
        return 0u;
    }
    double u64[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) u64[v] = Ub[v * stride];
    double Pd[4];
    int st64 = 1;
    if (st == 0) st64 = sr_polish64(gd, u64, f32_to_f64(P[3]), Pd);
    if (st64 != 0) {
        // unphysical in FP32 or in FP64: recover from the fixed FP64 state,
        // starting from the previous pass's pressure
        sr_fix(d_atm, tau_atm, u64);
        st64 = sr_polish64(gd, u64, guess >= 0.0f ? f32_to_f64(guess) : -1.0, Pd);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) P[c] = f64_to_f32(Pd[c]);
    P[4] = f64_to_f32(1.0 - (Pd[0] * Pd[0] + Pd[1] * Pd[1] + Pd[2] * Pd[2]));
    return st64 ? ERRBIT_C2P : 0u;
}
// Threads per element and the largest CTA of k_stage_mixed<NP>.
template <int NP>
struct StageShape {
    static constexpr int NN = NP * NP * NP;
    // threads per element: one per node; for n = 5 one more warp, so that the 150
    // face points take one pass of the face loop (measured 4-5 % faster per stage
    // than 128 threads)
    static constexpr int TPE = round_up32(NN) + (NP == 5 ? 32 : 0);
    static constexpr int MAXT = NP == 5 ? 2 * TPE : (TPE > 256 ? TPE : 256);
    static constexpr int MAX_EPB = MAXT / TPE;
    // CTAs of MAXT threads that must fit on an SM: this caps the registers at 64
    // per thread (56 for n = 7).  Spills, but occupancy matters more: at n = 5 a
    // 90-96 register build was 4-8 % slower, and capping n = 6, 7, 8 (they used
    // 92-114) made the 256-mesh ensemble step 26 % faster.
    static constexpr int MIN_CTAS = NP == 5 ? 3 : (NN <= 128 ? 4 : (NP == 6 ? 4 : (NP == 7 ? 3 : 2)));
};

// Shared memory of k_stage_mixed: per element (stride ELEM) the main arrays,
// the neighbour face nodes (later the summaries' partial sums), the plane sums,
// the neighbour indices, two flags, the element index and the mesh slot; then (learned guess only) the network's weights, and the features
// and guesses of all the CTA's nodes.
template <int NP>
struct MixedSmem {
    static constexpr int NN = NP * NP * NP;
    static constexpr int NF = 6 * NP * NP;                           // face points (both sides, 3 axes)
    static constexpr size_t MAIN = sizeof(float) * (25 + NPRIM) * NN;
    // neighbour face-node states [5][NF] and guesses [NF] (face phase), later the
    // summaries' partial sums [3][NP][NP][5] (FP64)
    static constexpr size_t FACE = (MAIN + 15) / 16 * 16;
    // (the guess array holds max(NF, NN) floats: the learned variant puts its
    // nodes' guesses there, and for n >= 7 an element has more nodes than face points)
    static constexpr size_t FACE_FLOATS = 5 * NF + (NF > NN ? NF : NN);
    static constexpr size_t FACE_BYTES = sizeof(float) * FACE_FLOATS > sizeof(double) * 15 * NP * NP
                                             ? sizeof(float) * FACE_FLOATS : sizeof(double) * 15 * NP * NP;
    static constexpr size_t Q = (FACE + FACE_BYTES + 15) / 16 * 16;
    static constexpr size_t NB = Q + sizeof(double) * 3 * NP * 5;
    static constexpr size_t FLAG = NB + sizeof(long long) * 7;      // 6 neighbours + element index
    static constexpr size_t SLOT = (FLAG + 2 * sizeof(int) + 15) / 16 * 16;
    static constexpr size_t ELEM = (SLOT + sizeof(MeshSlot) + 15) / 16 * 16;
    // Learned guess: the network's weights (one copy per CTA), and per element the
    // features [NN][6] of its nodes.  They are dead once the network has run, before
    // the element's MAIN region is first written, so where MAIN has room (n >= 5)
    // they live inside it: the weights and element 0's features in element 0's
    // MAIN, element s's features in element s's.  Otherwise they follow the
    // elements.  The guesses go to the element's face-guess array (FACE + 5 NF
    // floats), which the learned variant does not otherwise use.
    static constexpr size_t NET_BYTES = (sizeof(NetWeightsSmem) + 15) / 16 * 16;
    static constexpr size_t FEAT_BYTES = sizeof(float) * 6 * NN;
    static constexpr bool NET_IN_MAIN = NET_BYTES + FEAT_BYTES <= MAIN;
    __host__ __device__ static size_t net(int epb) { return NET_IN_MAIN ? 0 : ELEM * epb; }
    __host__ __device__ static size_t feat(int epb, int s)
    {
        return NET_IN_MAIN ? ELEM * s + (s == 0 ? NET_BYTES : 0) : ELEM * epb + NET_BYTES + FEAT_BYTES * s;
    }
    __host__ __device__ static size_t guess(int s) { return ELEM * s + FACE + sizeof(float) * 5 * NF; }
    __host__ __device__ static size_t total(int epb, bool learned)
    {
        return learned && !NET_IN_MAIN ? ELEM * epb + NET_BYTES + FEAT_BYTES * epb : ELEM * epb;
    }
};

// Physicality (bit 0 set if unphysical, as sr_unphysical) and whether the conserved
// fix of Sec. 2.1.4 would change u (bit 1, as a nonzero sr_fix), from one FP64
// evaluation of S^2 and tau (tau + 2D), without the fix's rescaling.
__device__ __forceinline__ unsigned sr_check64(double d_atm, double tau_atm, const double u[5])
{
    const double s2 = u[1] * u[1] + u[2] * u[2] + u[3] * u[3];
    const double tt = u[4] * (u[4] + 2.0 * u[0]);
    const bool bad = !(u[0] > 0.0) || !(u[4] > 0.0) || !(s2 < tt);
    const bool fix = !(u[0] >= d_atm) || !(u[4] >= tau_atm * u[0]) || s2 > (1.0 - 1e-12) * tt;
    return (bad ? 1u : 0u) | (fix ? 2u : 0u);
}

// FP32 screen of the bounds of the conserved fix (Sec. 2.1.4) and of physicality;
// nodes that fail it are decided in FP64.
__device__ __forceinline__ bool sr_screen32(const float u[5], float d_atm, float tau_atm)
{
    const float s2 = u[1] * u[1] + u[2] * u[2] + u[3] * u[3];
    return !(u[0] > 2.0f * d_atm) || !(u[4] > 2.0f * tau_atm * u[0]) ||
           !(s2 < 0.999f * u[4] * (u[4] + 2.0f * u[0]));
}
template <int NP, int SYS, int FLX, int GUESS>
__global__ void __launch_bounds__(StageShape<NP>::MAXT, StageShape<NP>::MIN_CTAS) k_stage_mixed(const MixedArgs a)
{
    constexpr int NN = NP * NP * NP;
    constexpr int TPE = StageShape<NP>::TPE;
    using SM = MixedSmem<NP>;
    extern __shared__ __align__(16) unsigned char smem_mixed[];
    const int sub = threadIdx.x / TPE, t = threadIdx.x % TPE;
    unsigned char *base = smem_mixed + SM::ELEM * sub;
    float *sF = reinterpret_cast<float *>(base);  // [3][5][NN] fluxes (later the FP64 output)
    float *sR = sF + 15 * NN;                      // [5][NN] right-hand side
    float *sU = sR + 5 * NN;                       // [5][NN] stage input state (FP32)
    float *sP = sU + 5 * NN;                       // [NPRIM][NN] primitives of the input
    double *sQ = reinterpret_cast<double *>(base + SM::Q);
    constexpr int NF = SM::NF;
    float *sFU = reinterpret_cast<float *>(base + SM::FACE);  // [5][NF] neighbour face-node states
    float *sFG = sFU + 5 * NF;                                // [NF] their con2prim guesses (warm start)
    double *sPart = reinterpret_cast<double *>(base + SM::FACE);
    long long *sNb = reinterpret_cast<long long *>(base + SM::NB);
    int *sFlag = reinterpret_cast<int *>(base + SM::FLAG);
    MeshSlot &sl = *reinterpret_cast<MeshSlot *>(base + SM::SLOT);
    __shared__ float sD[NP * NP];
    __shared__ double sW64[NP], sRow164[NP];
    __shared__ uint64_t sNetBar;  // completion of the network weights' bulk copy

    const long long ge = (long long)blockIdx.x * a.epb + sub;
    const bool live = sub < a.epb && ge < a.nelem;  // uniform within the element's warps
    if (t == 0) {
        sFlag[0] = sFlag[1] = 0;
        if (live) {
            const int m = a.slots ? find_slot(a.elem0, a.nslots, ge) : 0;
            sl = a.slots ? a.slots[m] : a.one;
            sNb[6] = a.slots ? ge - a.elem0[m] : ge;
        }
    }
    if (GUESS && threadIdx.x == 0) net_bar_init(&sNetBar);
    for (int i = threadIdx.x; i < NP * NP; i += blockDim.x) sD[i] = a.D32[i];
    if (threadIdx.x < NP) {
        sW64[threadIdx.x] = a.w64[threadIdx.x];
        sRow164[threadIdx.x] = a.row1_64[threadIdx.x];
    }
    __syncthreads();
    // the network's weights travel by one bulk asynchronous copy while the face
    // nodes and the features load
    if (GUESS && threadIdx.x == 0)
        net_copy_issue(reinterpret_cast<NetWeightsSmem *>(smem_mixed + SM::net(a.epb)), a.netImg, &sNetBar);
    const long long e = live ? sNb[6] : 0;
    if (live && t < 6) sNb[t] = elem_neighbour(e, sl.K, t >> 1, (t & 1) ? 1 : -1);
    const bool own = live && t < NN;  // this thread holds node t of a live element
    unsigned errs = 0;

    // Neighbour face nodes of all three axes (point f = 2 NP^2 ax + NP^2 side + rem):
    // their FP32 states and guesses, staged first so that the loads overlap the
    // network's phase and the element's own loads.
    for (int f = t; live && f < NF; f += TPE) {
        const int ax = f / (2 * NP * NP), fpa = f % (2 * NP * NP);
        const int side = fpa / (NP * NP), rem = fpa % (NP * NP);
        const int b = ax == 2 ? 0 : ax + 1, c = ax == 0 ? 2 : ax - 1;
        const int qn = (side ? 0 : NP - 1) * axis_stride<NP>(ax) + (rem % NP) * axis_stride<NP>(b) +
                       (rem / NP) * axis_stride<NP>(c);
        if (SYS == 0) {
            // a negative neighbour is a ghost holding the analytic exterior state
            const long long en = elem_neighbour_bc(e, sl.K, ax, side ? 1 : -1, sl.gh);
            const double *src = en >= 0 ? sl.Us + en * 5 * NN : sl.gh.U + (-1 - en) * 5 * NN;
#pragma unroll
            for (int v = 0; v < 5; ++v) sFU[v * NF + f] = f64_to_f32(src[v * NN + qn]);
            sFG[f] = -1.0f;
        } else {
            const long long en = elem_neighbour(e, sl.K, ax, side ? 1 : -1);
#pragma unroll
            for (int v = 0; v < 5; ++v) sFU[v * NF + f] = f64_to_f32(sl.Us[(en * 5 + v) * NN + qn]);
            if (!GUESS) sFG[f] = sl.pin ? sl.pin[en * NN + qn] : -1.0f;
        }
    }

    // Learned con2prim guesses for the CTA's nodes (the network runs on the tensor
    // cores over 16-row tiles, all warps of the CTA on each element's rows in turn).
    // The neighbours' face nodes in the face loop start from the pressure of this
    // element's node at the same point (the other side of the trace), solved by then.
    if (GUESS) {
        const NetWeightsSmem &W = *reinterpret_cast<const NetWeightsSmem *>(smem_mixed + SM::net(a.epb));
        if (t < NN) {
            float u[5] = {1.0f, 0.0f, 0.0f, 0.0f, 1.0f};
            if (own)
#pragma unroll
                for (int v = 0; v < 5; ++v) u[v] = f64_to_f32(sl.Us[(e * 5 + v) * NN + t]);
            net_features(u, a.net_sc, reinterpret_cast<float(*)[6]>(smem_mixed + SM::feat(a.epb, sub))[t]);
        }
        if (!net_copy_wait(&sNetBar, NET_COPY_POLLS)) {
            // flag it, and give the copy one more bounded wait before its region is reused
            errs |= ERRBIT_TIMEOUT;
            net_copy_wait(&sNetBar, NET_COPY_POLLS);
        }
        __syncthreads();
        for (int s2 = 0; s2 < a.epb; ++s2)
            net_guess_rows(W, reinterpret_cast<const float(*)[6]>(smem_mixed + SM::feat(a.epb, s2)),
                           reinterpret_cast<float *>(smem_mixed + SM::guess(s2)), NN, a.gamma, a.net_sc);
        __syncthreads();  // the guesses are in sFG; the network's regions are dead from here on
    }

    if (own) {
        float u[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            u[v] = f64_to_f32(sl.Us[(e * 5 + v) * NN + t]);
            sU[v * NN + t] = u[v];
        }
        float P[NPRIM];
        const float guess = GUESS ? sFG[t] : (sl.pin ? sl.pin[e * NN + t] : -1.0f);
        if (SYS == 0) {
            ne_primitives32(a.gamma, u, P);
        } else if (sl.Pin) {
#pragma unroll
            for (int c = 0; c < NPRIM; ++c) P[c] = sl.Pin[(e * NPRIM + c) * NN + t];
        } else {
            errs |= sr_prims_mixed(a.gamma, a.gamma_d, a.kappa_sw, a.d_atm, a.tau_atm, u, sl.Us + e * 5 * NN + t,
                                   NN, guess, P);
        }
        if (SYS == 1 && sl.pout) sl.pout[e * NN + t] = P[3];
#pragma unroll
        for (int c = 0; c < NPRIM; ++c) sP[c * NN + t] = P[c];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            float f[5];
            flux_axis32(u, P, ax, f);
#pragma unroll
            for (int v = 0; v < 5; ++v) sF[(ax * 5 + v) * NN + t] = f[v];
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
        if (own)
#pragma unroll
            for (int c = 0; c < 15; ++c) sF[c * NN + t] -= ref[c];
    }
    __syncthreads();

    // Volume term (eq:405), per axis a and variable v the contraction
    // sum_l D_il (F_v^a - F_ref)_l along axis a, scaled by -2/dx_a.
    if (a.tc) {
        // Tensor cores: for axis a the products R^T = F^T D^T, with rows (v, line)
        // -- the 5 NP^2 lines of nodes along a -- K = l and N = i padded to 8.
        const int lane = t & 31, warp = t >> 5, nwarps = TPE >> 5;
        const int g = lane >> 2, tq = lane & 3;
        uint32_t bfr[3];  // B = D^T: this lane holds B[2tq][g], B[2tq+1][g] = D[g][2tq], D[g][2tq+1]
        {
            float d0[3], d1[3];
            split_bf16x3((g < NP && 2 * tq < NP) ? sD[g * NP + 2 * tq] : 0.0f, d0);
            split_bf16x3((g < NP && 2 * tq + 1 < NP) ? sD[g * NP + 2 * tq + 1] : 0.0f, d1);
#pragma unroll
            for (int p = 0; p < 3; ++p) bfr[p] = pack2_bf16(d0[p], d1[p]);
        }
        constexpr int ROWS = 5 * NP * NP, TILES = (ROWS + 15) / 16;
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            // node of line c at position l along axis ax
            auto node_of = [=](int c, int l) {
                return ax == 0 ? l + NP * c : (ax == 1 ? (c % NP) + NP * (l + NP * (c / NP)) : c + NP * NP * l);
            };
            const float gax = live ? sl.g[ax] : 0.0f;
            for (int tile = warp; live && tile < TILES; tile += nwarps) {
                const int ra = tile * 16 + g, rb = ra + 8;
                float va[2], vb[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int l = 2 * tq + h;
                    va[h] = (ra < ROWS && l < NP) ? sF[(ax * 5 + ra / (NP * NP)) * NN + node_of(ra % (NP * NP), l)] : 0.0f;
                    vb[h] = (rb < ROWS && l < NP) ? sF[(ax * 5 + rb / (NP * NP)) * NN + node_of(rb % (NP * NP), l)] : 0.0f;
                }
                float pa0[3], pa1[3], pb0[3], pb1[3];
                split_bf16x3(va[0], pa0);
                split_bf16x3(va[1], pa1);
                split_bf16x3(vb[0], pb0);
                split_bf16x3(vb[1], pb1);
                uint32_t a0[3], a1[3];
#pragma unroll
                for (int p = 0; p < 3; ++p) {
                    a0[p] = pack2_bf16(pa0[p], pa1[p]);
                    a1[p] = pack2_bf16(pb0[p], pb1[p]);
                }
                float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                mma_bf16_k8(acc, a0[2], a1[2], bfr[0]);
                mma_bf16_k8(acc, a0[0], a1[0], bfr[2]);
                mma_bf16_k8(acc, a0[1], a1[1], bfr[1]);
                mma_bf16_k8(acc, a0[1], a1[1], bfr[0]);
                mma_bf16_k8(acc, a0[0], a1[0], bfr[1]);
                mma_bf16_k8(acc, a0[0], a1[0], bfr[0]);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int r = (c < 2) ? ra : rb, i = 2 * tq + (c & 1);
                    if (r < ROWS && i < NP) {
                        float *dst = sR + (r / (NP * NP)) * NN + node_of(r % (NP * NP), i);
                        *dst = (ax == 0) ? -gax * acc[c] : *dst - gax * acc[c];
                    }
                }
            }
            __syncthreads();
        }
    } else {
        if (own) {
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
                sR[v * NN + t] = -(sl.g[0] * sx + sl.g[1] * sy + sl.g[2] * sz);
            }
        }
        __syncthreads();
    }

    // Surface terms (eq:411: each face taken once along +e_a, the lower element
    // lifting -(2/dx_a)(F* - F_L)/w_N, the upper +(2/dx_a)(F* - F_R)/w_0) for the
    // face points of all three axes at once; the neighbour's face node is
    // recovered here from its staged state.  Each axis's lift goes to its own
    // array (over the flux arrays, no longer read): within an axis a node lies on
    // at most one face, so there are no write conflicts, and the three are summed
    // in a fixed order afterwards.
    // (sA[ax] is written only at the nodes on an ax-face; the sum below reads it
    // only there, so nothing needs clearing first)
    float *sA = sF;  // [3][5][NN]
    for (int f = t; live && f < NF; f += TPE) {
        const int ax = f / (2 * NP * NP), fpa = f % (2 * NP * NP);
        const int side = fpa / (NP * NP), rem = fpa % (NP * NP);
        // the face's normal axis and its tangential axes b, c in cyclic order
        const int b = ax == 2 ? 0 : ax + 1, c = ax == 0 ? 2 : ax - 1;
        const int sa = axis_stride<NP>(ax);
        const int tq = (rem % NP) * axis_stride<NP>(b) + (rem / NP) * axis_stride<NP>(c);
        const int q = (side ? NP - 1 : 0) * sa + tq;
        const int qn = (side ? 0 : NP - 1) * sa + tq;
        // Both traces in the face frame (normal, b, c components): the flux routines
        // then run with axis 0 and keep their arrays in registers.  The neighbour's
        // con2prim works in the mesh frame, its result is rotated after.
        float uo[5], Po[NPRIM], um[5], Pm[NPRIM];
        uo[0] = sU[q];
        uo[1] = sU[(1 + ax) * NN + q];
        uo[2] = sU[(1 + b) * NN + q];
        uo[3] = sU[(1 + c) * NN + q];
        uo[4] = sU[4 * NN + q];
        Po[0] = sP[ax * NN + q];
        Po[1] = sP[b * NN + q];
        Po[2] = sP[c * NN + q];
        Po[3] = sP[3 * NN + q];
        Po[4] = sP[4 * NN + q];
#pragma unroll
        for (int v = 0; v < 5; ++v) um[v] = sFU[v * NF + f];
        const float gn = GUESS ? Po[3] : sFG[f];
        if (SYS == 0) {
            ne_primitives32(a.gamma, um, Pm);
        } else if (sl.Pin) {
            const long long en = sNb[2 * ax + side];
#pragma unroll
            for (int k = 0; k < NPRIM; ++k) Pm[k] = sl.Pin[(en * NPRIM + k) * NN + qn];
        } else {
            const long long en = sNb[2 * ax + side];
            errs |= sr_prims_mixed(a.gamma, a.gamma_d, a.kappa_sw, a.d_atm, a.tau_atm, um,
                                   sl.Us + en * 5 * NN + qn, NN, gn, Pm);
        }
        const float un[5] = {um[0], pick3(ax, um[1], um[2], um[3]), pick3(b, um[1], um[2], um[3]),
                             pick3(c, um[1], um[2], um[3]), um[4]};
        const float Pn[NPRIM] = {pick3(ax, Pm[0], Pm[1], Pm[2]), pick3(b, Pm[0], Pm[1], Pm[2]),
                                 pick3(c, Pm[0], Pm[1], Pm[2]), Pm[3], Pm[4]};
        float dL[5], dR[5], o[5];
        if (side) {
            num_flux_jump32<SYS, FLX>(a.gamma, 0, uo, Po, un, Pn, dL, dR);
            const float lN = sl.liftN[ax];
#pragma unroll
            for (int v = 0; v < 5; ++v) o[v] = -lN * dL[v];
        } else {
            num_flux_jump32<SYS, FLX>(a.gamma, 0, un, Pn, uo, Po, dL, dR);
            const float l0 = sl.lift0[ax];
#pragma unroll
            for (int v = 0; v < 5; ++v) o[v] = l0 * dR[v];
        }
        float *acc = sA + ax * 5 * NN + q;
        acc[0] = o[0];
        acc[(1 + ax) * NN] = o[1];
        acc[(1 + b) * NN] = o[2];
        acc[(1 + c) * NN] = o[3];
        acc[4 * NN] = o[4];
    }
    __syncthreads();
    if (own) {
        const int i = t % NP, j = (t / NP) % NP, k = t / (NP * NP);
        const bool fx = i == 0 || i == NP - 1, fy = j == 0 || j == NP - 1, fz = k == 0 || k == NP - 1;
#pragma unroll
        for (int v = 0; v < 5; ++v)
            sR[v * NN + t] += ((fx ? sA[v * NN + t] : 0.0f) + (fy ? sA[(5 + v) * NN + t] : 0.0f)) +
                              (fz ? sA[(10 + v) * NN + t] : 0.0f);
    }
    if (errs) atomicOr(sl.err, errs);

    // Stage update in FP64: U_{s+1} = U_s + [ca (U^n - U_s) + cb dt R], the bracket
    // in FP32 (it carries the FP32 RHS), the accumulation in FP64.  The limiter
    // summaries and the SR flags see the output before the conserved fix (Sec. 3.3:
    // limit, then fix); with the limiter on the fix is left to the limiter pass,
    // which visits the flagged elements.
    double val[5];
    bool bad = false, needfix = false;
    if (own) {
        const float dt = (float)(sl.dt_ptr ? *sl.dt_ptr : sl.dt);
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            const long long ix = (e * 5 + v) * NN + t;
            const float R = sR[v * NN + t];
            if (a.mode == 0) {
                sl.out[ix] = f32_to_f64(R);
                continue;
            }
            const double us = sl.Us[ix];
            float inc;
            if (a.first) {
                inc = dt * R;
            } else {
                const float dn = f64_to_f32(sl.Un[ix] - us);
                inc = a.ca * dn + a.cb * (dt * R);
            }
            val[v] = us + f32_to_f64(inc);
        }
    }
    if (a.mode == 0) return;
    if (own && SYS == 1) {
        float u32[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) u32[v] = f64_to_f32(val[v]);
        if (sr_screen32(u32, (float)a.d_atm, (float)a.tau_atm)) {
            if (a.lim) {
                // the limiter runs the fix; here only its decision and physicality
                const unsigned c = sr_check64(a.d_atm, a.tau_atm, val);
                bad = c & 1u;
                needfix = c & 2u;
            } else {
                sr_fix(a.d_atm, a.tau_atm, val);
            }
        }
    }
    if (own)
#pragma unroll
        for (int v = 0; v < 5; ++v) sl.out[(e * 5 + v) * NN + t] = val[v];
    if (!a.lim) return;

    // Limiter summaries of the output in FP64 (the limiter's decisions and its
    // replacement, and through them the conserved fix at the replaced nodes, are
    // sensitive to them at the FP64 level).  Plane sums
    //   Q_a[i][v] = sum_{t0,t1} w_t0 w_t1 U_v(node with index i along axis a)
    // give the cell mean sum_i w_i Q_0[i] / 8, the face means Q_a[0] / 4 and
    // Q_a[NP-1] / 4, and the P1 coefficients sum_i row1_i Q_a[i] / 4.  The FP64 copy
    // of the output overlays the flux array, which is no longer read.
    double *sV = reinterpret_cast<double *>(base);
    if (own)
#pragma unroll
        for (int v = 0; v < 5; ++v) sV[v * NN + t] = val[v];
    if (bad) atomicOr(&sFlag[0], 1);
    if (needfix) atomicOr(&sFlag[1], 1);
    __syncthreads();
    // Line sums P_a[ia][t1] = sum_t0 w_t0 U (axis a at index ia, t0 along the next
    // axis, t1 along the one after) for a = x (sums over y) and a = z (sums over x),
    // then Q_x and Q_z over t1; the planes across y reuse the x sums:
    // Q_y[j] = sum_k w_k P_z[k][j].  Two FP64 FMAs per node and variable.
    for (int id = t; live && id < 10 * NP * NP; id += TPE) {
        const int v = id % 5, t1 = (id / 5) % NP, ia = (id / (5 * NP)) % NP, ax = id < 5 * NP * NP ? 0 : 2;
        const int b = (ax + 1) % 3, c = (ax + 2) % 3;
        const double *Vv = sV + v * NN;
        double r = 0.0;
        const int base_node = ia * axis_stride<NP>(ax) + t1 * axis_stride<NP>(c), st0 = axis_stride<NP>(b);
        for (int t0 = 0; t0 < NP; ++t0) r = fma(sW64[t0], Vv[base_node + t0 * st0], r);
        sPart[((ax * NP + ia) * NP + t1) * 5 + v] = r;
    }
    __syncthreads();
    for (int id = t; live && id < 15 * NP; id += TPE) {
        const int ax = id / (5 * NP), ia = (id / 5) % NP, v = id % 5;
        double q = 0.0;
        if (ax == 1)
            for (int k = 0; k < NP; ++k) q = fma(sW64[k], sPart[((2 * NP + k) * NP + ia) * 5 + v], q);
        else
            for (int t1 = 0; t1 < NP; ++t1) q = fma(sW64[t1], sPart[((ax * NP + ia) * NP + t1) * 5 + v], q);
        sQ[(ax * NP + ia) * 5 + v] = q;
    }
    __syncthreads();
    for (int id = t; live && id < 50; id += TPE) {
        const int v = id / 10, kind = id % 10;
        double r;
        if (kind == 0) {
            double s = 0.0;
            for (int i = 0; i < NP; ++i) s = fma(sW64[i], sQ[i * 5 + v], s);
            r = s * 0.125;
        } else if (kind <= 6) {
            const int ax = (kind - 1) / 2, ia = ((kind - 1) % 2) ? NP - 1 : 0;
            r = sQ[(ax * NP + ia) * 5 + v] * 0.25;
        } else {
            const int ax = kind - 7;
            double s = 0.0;
            for (int i = 0; i < NP; ++i) s = fma(sRow164[i], sQ[(ax * NP + i) * 5 + v], s);
            r = s * 0.25;
        }
        sl.S[e * 50 + id] = r;
    }
    if (SYS == 1 && live && t == 0 && sl.flags) sl.flags[e] = (sFlag[0] ? 1 : 0) | (sFlag[1] ? 2 : 0);
}

template <int NP>
cudaError_t launch_stage_mixed_np(int system, int flux, const MixedArgs &a, cudaStream_t s)
{
    using SS = StageShape<NP>;
    if (a.epb < 1 || a.epb > SS::MAX_EPB) return cudaErrorInvalidValue;
    if (a.nelem <= 0) return cudaSuccess;
    const long long blocks = (a.nelem + a.epb - 1) / a.epb;
    const dim3 grid((unsigned)blocks), block(SS::TPE * a.epb);
    const bool learned = system == 1 && a.netImg != nullptr;
    const size_t smem = MixedSmem<NP>::total(a.epb, learned);
    void (*kern)(const MixedArgs);
    if (system == 0 && flux == 2) kern = k_stage_mixed<NP, 0, 2, 0>;
    else if (system == 0 && flux == 0) kern = k_stage_mixed<NP, 0, 0, 0>;
    else if (system == 0) kern = k_stage_mixed<NP, 0, 1, 0>;
    else if (flux == 0) kern = learned ? k_stage_mixed<NP, 1, 0, 1> : k_stage_mixed<NP, 1, 0, 0>;
    else kern = learned ? k_stage_mixed<NP, 1, 1, 1> : k_stage_mixed<NP, 1, 1, 0>;
    if (smem > 48 * 1024) {
        cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
    }
    kern<<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
}

// Largest elements-per-CTA of the stage kernel for n nodes per axis.
inline int stage_max_epb(int n)
{
    const int nn = n * n * n, tpe = round_up32(nn) + (n == 5 ? 32 : 0);
    const int maxt = n == 5 ? 2 * tpe : (tpe > 256 ? tpe : 256);
    return maxt / tpe;
}

}  // namespace dg

// the limiter of the mixed path
#include "dg_limit_mixed.cuh"
// the Newtonian delta-form step
#include "dg_ne_mixed.cuh"

#define DG_INSTANTIATE_MIXED(NP)                                                                       \
    namespace dg {                                                                                     \
    cudaError_t launch_stage_mixed_n##NP(int system, int flux, const MixedArgs &a, cudaStream_t s)      \
    {                                                                                                  \
        return launch_stage_mixed_np<NP>(system, flux, a, s);                                          \
    }                                                                                                  \
    cudaError_t launch_limit_mixed_n##NP(int system, const LimitMixedArgs &a, cudaStream_t s)           \
    {                                                                                                  \
        return launch_limit_mixed_np<NP>(system, a, s);                                                \
    }                                                                                                  \
    cudaError_t launch_ne_stage_n##NP(int flux, int stage, const NeArgs &a, cudaStream_t s)             \
    {                                                                                                  \
        return launch_ne_stage_np<NP>(flux, stage, a, s);                                              \
    }                                                                                                  \
    cudaError_t launch_ne_decide_n##NP(int final_pass, const NeDecideArgs &a, cudaStream_t s)           \
    {                                                                                                  \
        return launch_ne_decide_np<NP>(final_pass, a, s);                                              \
    }                                                                                                  \
    }
