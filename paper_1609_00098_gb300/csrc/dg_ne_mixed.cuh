// dg_ne_mixed.cuh -- the Newtonian mixed-precision SSP-RK3 step in delta form
// (templated on the number of LGL nodes per axis NP).
//
// The state U^n stays FP64 and is written once per step; the SSP-RK3 stage states
// (Sec. 3.4) are held as FP32 differences from it,
//   U^1 = U^n + D1,  D1 = dt R(U^n),
//   U^2 = U^n + D2,  D2 = (D1 + dt R(U^1)) / 4,
//   U^3 = U^n + D3,  D3 = 2 (D2 + dt R(U^2)) / 3,
// which is the Shu-Osher form with ca + cb = 1 written for the differences, and the
// step ends with U^{n+1} = U^n + D3 added in FP64.  A difference carries the FP32
// rounding of the stage's change only, as the FP32 increments of a stage update on
// FP64 stage states would.  Stage 1 stores R(U^n) itself (dt is not known until its
// CFL maximum is complete) and stage 2 scales it.
//
// The limiter (Sec. 3.3) acts on U^s after every stage.  Its decisions are taken
// per element from summaries of U^s (cell mean, six face means, three P1
// coefficients, as the other paths use) by k_ne_decide, which writes for every
// limited variable the replacement U0 + sum_a s_a (x_a - x_a0) (eq:MinModSol) as
// parameters: the FP64 mean and three FP32 slopes times dx_a/2.  The next stage
// kernel evaluates the replacement where it reads U^s, so a limited stage state is
// never written node by node; only U^{n+1} is, by the last pass.
//
// Summaries of U^s = U^n + D are S(U^n) + S(D): S(U^n) is formed once per step by
// stage 1 from U^n shifted by a per-element reference, as double-float (compensated
// FP32) sums where the limiter's face tests need them (mean and face means), the
// reference added in FP64; S(D) in FP32.  The limiter's face tests are then taken
// in FP64 on those summaries, its slope candidates from FP64 differences rounded to
// FP32 (the precision the replacement stores).
//
// Work split of k_ne_stage: one thread per x-line (j, k) of an element, NP nodes;
// a CTA holds NeShape<NP>::EPB consecutive elements.  For even NP each element's
// U^n (and in stages 2 and 3 its difference and replacement parameters, and its
// neighbours' replacement parameters) arrive in shared memory by bulk asynchronous
// copies issued at the start of the kernel, on a transaction barrier per element.
// The x derivative is taken in registers (node pairs in paired FP32 FMAs for even
// NP); the y and z derivatives read fluxes of other threads' lines from shared
// memory.  Face points are split evenly: at its face position (j, k) a thread takes
// one point of every (axis, side), the neighbours' traces staged first so that the
// flux phase runs without divergence.
#pragma once

#include "dg_internal.h"

namespace dg {

// ---------------------------------------------------------------------------
// FP64 -> FP32 hi/lo parts by integer operations.  hi = the double rounded to FP32
// (half away from zero; |x| < 2^-126 gives a signed zero, overflow inf, NaN stays
// NaN); lo = x - hi as FP32 (exact up to the rounding of 30 bits to 24, i.e. within
// 2^-47 |x|; 0 for |x| < 2^-74).

__device__ __forceinline__ float ne_hi(double x)
{
    const unsigned H = (unsigned)__double2hiint(x), L = (unsigned)__double2loint(x);
    const unsigned mag = H & 0x7fffffffu;
    unsigned bits = __funnelshift_l(L, mag - (896u << 20), 3) + ((L >> 28) & 1u);
    bits = mag < (897u << 20) ? 0u : bits;
    const bool nan = (mag > 0x7ff00000u) | ((mag == 0x7ff00000u) & (L != 0u));
    bits = mag >= (1151u << 20) ? (nan ? 0x7fc00000u : 0x7f800000u) : bits;
    return __uint_as_float(bits | (H & 0x80000000u));
}

__device__ __forceinline__ float ne_lo(double x)
{
    const unsigned H = (unsigned)__double2hiint(x), L = (unsigned)__double2loint(x);
    const unsigned e = (H >> 20) & 0x7ffu;
    // remainder below the FP32 rounding point, in units of 2^(e-1075), signed
    const int r = (int)(L & 0x1fffffffu) - (int)(((L >> 28) & 1u) << 29);
    const float sc = __uint_as_float((e - 948u) << 23);
    const float lo = __int2float_rn(r) * sc;
    const float v = (e >= 949u && e <= 1150u) ? lo : 0.0f;
    return (H & 0x80000000u) ? -v : v;
}

__device__ __forceinline__ double ne_f32_to_f64(float f)
{
    const unsigned b = __float_as_uint(f);
    const unsigned sign = b & 0x80000000u, ef = (b >> 23) & 0xffu, m = b & 0x7fffffu;
    if (ef == 0u) return __hiloint2double((int)sign, 0);
    const unsigned he = (ef == 0xffu) ? 0x7ffu : ef + 896u;
    return __hiloint2double((int)(sign | (he << 20) | (m >> 3)), (int)(m << 29));
}

// ---------------------------------------------------------------------------
// Launch shape: elements per CTA (EPB), threads per CTA and CTAs per SM the
// registers are sized for, for NP nodes per axis, and the shared-memory layout of
// one element (floats, regions 16-byte aligned):
//   U   stage state sU[5][NN]                     phase 1 .. face fluxes
//   HF  neighbour face traces sH[6][L][5]         halo staging .. face fluxes,
//       then the flux buffers sF[2][2][NN] (y, z; double-buffered over the variables)
//   LF  y/z face lifts sL[2][2][L][5]             face fluxes .. volume term
// The S(U^n) reduction of stage 1 works in HF + LF before the halo staging, the
// reduction of the output's summaries in U + HF after the volume term.
template <int NP>
struct NeShape {
    static constexpr int L = NP * NP;        // x-lines (threads) per element
    static constexpr int NN = NP * NP * NP;
    static constexpr int EPB = NP == 2 ? 32 : NP == 3 ? 16 : NP == 4 ? 8 : NP == 5 ? 6 : NP == 6 ? 7 : NP == 7 ? 3 : 2;
    static constexpr int THREADS = (EPB * L + 31) / 32 * 32;
    static constexpr int MINB = NP == 6 ? 2 : 3;
    static constexpr int R4(int v) { return (v + 3) / 4 * 4; }
    static constexpr int SN_NEED = 35 * L + 60 * NP;  // S(U^n): line partials, then per-(v, k) sums
    static constexpr int SD_NEED = 20 * L + 35 * NP;  // S(output): the same in FP32
    static constexpr int HF = R4(30 * L > 4 * NN ? 30 * L : 4 * NN);
    static constexpr int F_U = 0;
    static constexpr int F_H = R4(5 * NN);
    static constexpr int F_F = F_H;
    static constexpr int F_L = F_H + HF + (SN_NEED > HF + 20 * L ? R4(SN_NEED - (HF + 20 * L)) : 0);
    // stages 2, 3: the element's U^n (FP64) lands by one bulk copy at F_H, over the
    // halo, flux and lift arrays (free until phase 1 has read it), its difference by
    // another over U; the copies move whole elements, 16-byte multiples for even NP
    static constexpr bool STAGE = NP % 2 == 0;
    static constexpr int F_S = F_H;
    static constexpr int ELEM_BASE = F_L + R4(20 * L);
    static constexpr int ELEM_FLOATS = STAGE && F_S + 10 * NN > ELEM_BASE ? F_S + 10 * NN : ELEM_BASE;
    static_assert(SD_NEED <= F_L, "output-summary scratch must fit in U + HF");
    static_assert(!STAGE || (40 * NN) % 16 == 0 && (ELEM_FLOATS * 4) % 16 == 0 && (F_S * 4) % 16 == 0,
                  "bulk copies need 16-byte sizes and addresses");
    static constexpr size_t SMEM = sizeof(float) * (size_t)ELEM_FLOATS * EPB;
};

// Elements per CTA of k_ne_stage for n nodes per axis (NeShape<n>::EPB).
inline int ne_epb(int n)
{
    return n == 2 ? 32 : n == 3 ? 16 : n == 4 ? 8 : n == 5 ? 6 : n == 6 ? 7 : n == 7 ? 3 : 2;
}

// Error-free FP32 steps for the double-float sums of S(U^n): s + e = a + b exactly
// (Knuth's two-sum), and acc += w * p for double-float w = wh + wl, p = ph + pl,
// the product's rounding error taken exactly by an FMA.
__device__ __forceinline__ void ne_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

__device__ __forceinline__ void ne_df_fma(float &h, float &l, float wh, float wl, float ph, float pl)
{
    const float p = __fmul_rn(wh, ph);
    const float pe = fmaf(wh, ph, -p);
    float sum, err;
    ne_two_sum(h, p, sum, err);
    h = sum;
    l = __fadd_rn(l, __fadd_rn(__fadd_rn(pe, err), fmaf(wh, pl, __fmul_rn(wl, ph))));
}

// Per-mesh part of a Newtonian delta-form stage launch.  A launch advances one
// mesh (its slot passed inline) or a ragged batch of meshes with the same n,
// flux, gamma and limiter setting (slot table and element offsets in device
// memory; each element finds its mesh by binary search over the offsets).
struct NeSlot {
    const double *Un;          // U^n [e][5][NN]
    const float *Din;          // stage 2: R(U^n) (scaled by dt here); stage 3: D2; [e][5][NN]
    float *Dout;               // stage 1: R(U^n); stage 2: D2; stage 3: D3
    double *rhs;               // right-hand-side mode: dU/dt (FP64) [e][5][NN]
    const unsigned char *mask; // stages 2, 3 with a limiter: limited variables of U^s (bit v), else nullptr
    const float4 *SH;          // [e][5] {f32(U0), s_x dx/2, s_y dy/2, s_z dz/2} of the limited variables
    const double *M0;          // [e][5] FP64 cell means U0 of the limited variables
    double *SN;                // stage 1 with a limiter: S(U^n) [e][5][10] (FP64), else nullptr
    float *SD;                 // with a limiter: S of Dout [e][5][10] (FP32), else nullptr
    unsigned long long *lam;   // stage 1 with CFL: max wave speed (bits of a double), else nullptr
    unsigned int *err;         // the mesh's sticky status word (ERRBIT_TIMEOUT)
    const double *dt_ptr;      // device dt, or nullptr (host dt)
    double dt;
    int K[3];
    Ghosts gh;                 // analytic boundaries (mask 0: periodic)
    float g[3], lift0[3], liftN[3];
};

// Per-launch arguments of the Newtonian delta-form stage kernel.
struct NeArgs {
    NeSlot one;                // the mesh of a single-mesh launch
    const NeSlot *slots;       // batch: per-mesh slots, or nullptr
    const long long *elem0;    // batch: first element of each mesh in the launch
    int nslots;
    long long nelem;           // elements in the launch
    float cb;                  // D_{s+1} = cb (D_s + dt R)
    float gamma;
    float D[MAXN * MAXN];      // differentiation matrix, D[i * NP + l]
    alignas(8) float DT[MAXN * MAXN];  // its transpose, DT[l * NP + i] (node pairs as 64-bit words)
    float x[MAXN], w[MAXN], row1[MAXN];
    float wh[MAXN], wl[MAXN];  // LGL weights as FP32 pairs (w = wh + wl to ~2^-48)
};

// Per-mesh part of a decision pass.
struct NeDecideSlot {
    const double *SN;          // S(U^n) [e][5][10]
    const float *SD;           // S(D) [e][5][10]
    const double *dt_ptr;      // S(U^s) = SN + c SD with c = dt (stage 1, SD = S(R)) or 1
    double dt;
    unsigned char *mask;       // out: limited variables (bit v)
    double *M0;                // out: FP64 means
    float4 *SH;                // out: {f32(U0), slopes times dx/2}
    unsigned char *troubled;   // optional copy of the mask (last stage)
    double *U;                 // final pass: U^{n+1} = U^n + D3 (in place), replaced where limited
    const float *D3;
    int K[3];
    float tvb_f[3], two_inv_dx_f[3], beta_dx_f[3], hdx_f[3];  // M dx^2, 2/dx, beta/dx, dx/2
};

// minmod of three FP32 values: the one of least magnitude if all have one sign, else 0
__device__ __forceinline__ float ne_minmod3f(float a1, float a2, float a3)
{
    const bool pos = (a1 > 0.0f) & (a2 > 0.0f) & (a3 > 0.0f);
    const bool neg = (a1 < 0.0f) & (a2 < 0.0f) & (a3 < 0.0f);
    const float m = fminf(fabsf(a1), fminf(fabsf(a2), fabsf(a3)));
    return pos ? m : neg ? -m : 0.0f;
}

// Per-launch arguments of the decision pass.
struct NeDecideArgs {
    NeDecideSlot one;
    const NeDecideSlot *slots;
    const long long *elem0;
    int nslots;
    long long nelem;
    int scale_dt;
    int limiter;               // 0 none (final pass only), 1 MinModN, 2 MinMod
    float x[MAXN];
};

__device__ __forceinline__ int ne_find_slot(const long long *elem0, int nslots, long long ge)
{
    int lo = 0, hi = nslots - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (elem0[mid] <= ge) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// Face fluxes in the face frame (normal component first), jump form as in the
// other mixed kernels: dL = F* - F(U_L), dR = F* - F(U_R) along the normal.

__device__ __forceinline__ void ne_prims(float g, const float u[5], float &vn, float &vb, float &vc, float &p)
{
    const float inv = 1.0f / u[0];
    vn = u[1] * inv;
    vb = u[2] * inv;
    vc = u[3] * inv;
    p = (g - 1.0f) * (u[4] - 0.5f * (u[1] * vn + u[2] * vb + u[3] * vc));
}

template <int FLX>
__device__ __forceinline__ void ne_face_flux(float g, const float uL[5], const float uR[5], float dL[5], float dR[5])
{
    float vL, bL, cL, pL, vR, bR, cR, pR;
    ne_prims(g, uL, vL, bL, cL, pL);
    ne_prims(g, uR, vR, bR, cR, pR);
    float dF[5];
    dF[0] = uR[1] - uL[1];
    dF[1] = (uR[1] * vR + pR) - (uL[1] * vL + pL);
    dF[2] = uR[2] * vR - uL[2] * vL;
    dF[3] = uR[3] * vR - uL[3] * vL;
    dF[4] = (uR[4] + pR) * vR - (uL[4] + pL) * vL;
    if (FLX == 2) {
        // Roe (eq:Roe): dissipation sum_i alpha_i |lambda_i| e_i at the Roe averages
        const float sl = sqrtf(uL[0]), sr = sqrtf(uR[0]);
        const float inv = 1.0f / (sl + sr);
        const float un = (sl * vL + sr * vR) * inv, ut1 = (sl * bL + sr * bR) * inv, ut2 = (sl * cL + sr * cR) * inv;
        const float hL = (uL[4] + pL) / uL[0], hR = (uR[4] + pR) / uR[0];
        const float hh = (sl * hL + sr * hR) * inv;
        const float q2 = un * un + ut1 * ut1 + ut2 * ut2;
        const float c2 = (g - 1.0f) * (hh - 0.5f * q2);
        const float c = sqrtf(c2);
        const float j1 = uR[0] - uL[0], jn = uR[1] - uL[1], jt1 = uR[2] - uL[2], jt2 = uR[3] - uL[3];
        const float j5 = uR[4] - uL[4];
        const float al3 = jt1 - ut1 * j1, al4 = jt2 - ut2 * j1;
        const float j5b = j5 - al3 * ut1 - al4 * ut2;
        const float al2 = (g - 1.0f) / c2 * (j1 * (hh - un * un) + un * jn - j5b);
        const float al1 = (j1 * (un + c) - jn - c * al2) / (2.0f * c);
        const float al5 = j1 - (al1 + al2);
        const float w1 = fabsf(un - c) * al1, w2 = fabsf(un) * al2, w5 = fabsf(un + c) * al5;
        const float w3 = fabsf(un) * al3, w4 = fabsf(un) * al4;
        float Dd[5];
        Dd[0] = w1 + w2 + w5;
        Dd[1] = w1 * (un - c) + w2 * un + w5 * (un + c);
        Dd[2] = (w1 + w2 + w5) * ut1 + w3;
        Dd[3] = (w1 + w2 + w5) * ut2 + w4;
        Dd[4] = w1 * (hh - un * c) + w2 * (0.5f * q2) + w3 * ut1 + w4 * ut2 + w5 * (hh + un * c);
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            dL[v] = 0.5f * dF[v] - 0.5f * Dd[v];
            dR[v] = -0.5f * dF[v] - 0.5f * Dd[v];
        }
        return;
    }
    const float csL = sqrtf(g * pL / uL[0]), csR = sqrtf(g * pR / uR[0]);
    if (FLX == 0) {
        // LLF (eq:LLF)
        const float hal = 0.5f * fmaxf(fmaxf(fabsf(vL - csL), fabsf(vL + csL)), fmaxf(fabsf(vR - csR), fabsf(vR + csR)));
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            const float dU = uR[v] - uL[v];
            dL[v] = 0.5f * dF[v] - hal * dU;
            dR[v] = -0.5f * dF[v] - hal * dU;
        }
        return;
    }
    // HLL (eq:HLL)
    const float cmin = fminf(fminf(vL - csL, vR - csR), 0.0f);
    const float cmax = fmaxf(fmaxf(vL + csL, vR + csR), 0.0f);
    const float den = cmax - cmin;
    if (den > 0.0f) {
        const float inv = 1.0f / den;
        const float cc = cmin * cmax * inv, wl = -cmin * inv, wr = -cmax * inv;
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            const float dU = uR[v] - uL[v];
            dL[v] = wl * dF[v] + cc * dU;
            dR[v] = wr * dF[v] + cc * dU;
        }
    } else {
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            dL[v] = 0.5f * dF[v];
            dR[v] = -0.5f * dF[v];
        }
    }
}

// One x-line (NP floats, 8-byte aligned for even NP) to / from shared memory: 64-bit
// accesses for even NP, whose 24-byte line stride is free of bank conflicts.
template <int NP>
__device__ __forceinline__ void ne_st_line(float *p, const float v[NP])
{
    if (NP % 2 == 0) {
#pragma unroll
        for (int h = 0; h < NP / 2; ++h) reinterpret_cast<float2 *>(p)[h] = make_float2(v[2 * h], v[2 * h + 1]);
    } else {
#pragma unroll
        for (int i = 0; i < NP; ++i) p[i] = v[i];
    }
}

template <int NP>
__device__ __forceinline__ void ne_ld_line(const float *p, float v[NP])
{
    if (NP % 2 == 0) {
#pragma unroll
        for (int h = 0; h < NP / 2; ++h) {
            const float2 q = reinterpret_cast<const float2 *>(p)[h];
            v[2 * h] = q.x;
            v[2 * h + 1] = q.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < NP; ++i) v[i] = p[i];
    }
}

// One-shot transaction barrier in shared memory for the element's bulk copies: one
// thread initialises it (arrival count `count`), issues the copies, each with its
// byte count, and arrives; every thread of the element polls its first phase.
__device__ __forceinline__ void ne_bar_init(uint64_t *bar, unsigned count)
{
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(b), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void ne_bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(b),
                 "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(d),
                 "l"(src), "r"(bytes), "r"(b)
                 : "memory");
}

__device__ __forceinline__ void ne_bar_arrive(uint64_t *bar)
{
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(b) : "memory");
}

// Poll the first phase at most `limit` times; false if it has not completed.
__device__ __forceinline__ bool ne_bar_wait(uint64_t *bar, int limit)
{
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
    for (int i = 0; i < limit; ++i) {
        uint32_t ok;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(ok)
                     : "r"(b)
                     : "memory");
        if (ok) return true;
    }
    return false;
}
constexpr int NE_COPY_POLLS = 1 << 20;

// Bulk prefetch of [p, p + bytes) into L2 (a hint: no data reaches the SM).  The
// range is shrunk to 16-byte boundaries so that nothing outside it is touched.
__device__ __forceinline__ void ne_prefetch_l2(const void *p, unsigned long long bytes)
{
    unsigned long long a;
    asm("cvta.to.global.u64 %0, %1;" : "=l"(a) : "l"(p));
    const unsigned long long lo = (a + 15ull) & ~15ull, hi = (a + bytes) & ~15ull;
    if (hi > lo)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo), "r"((unsigned)(hi - lo)) : "memory");
}

// Linear part of a limited variable's replacement at LGL coordinates (x, y, z),
// sh = {f32(U0), s_x dx/2, s_y dy/2, s_z dz/2}: one fixed rounding sequence, so that
// every place that evaluates it (own nodes, neighbours' face nodes) gets the same bits.
__device__ __forceinline__ float ne_lin(const float4 sh, float x, float y, float z)
{
    return __fmaf_rn(sh.y, x, __fmaf_rn(sh.z, y, __fmul_rn(sh.w, z)));
}

// Node index of the point at face position (p0, p1) on the face normal to axis ax
// at layer `lay` (0 or NP-1): x-faces (lay, p0, p1), y-faces (p0, lay, p1),
// z-faces (p0, p1, lay).  Consecutive p0 are consecutive in memory for y and z.
template <int NP>
__device__ __forceinline__ int ne_face_node(int ax, int lay, int p0, int p1)
{
    return ax == 0 ? lay + NP * (p0 + NP * p1) : ax == 1 ? p0 + NP * (lay + NP * p1) : p0 + NP * (p1 + NP * lay);
}

// Physical fluxes of the NE system at one node along the three axes, variable V.
template <int V>
__device__ __forceinline__ void ne_flux3(float uv, float vx, float vy, float vz, float p, float &fx, float &fy,
                                         float &fz)
{
    if (V == 4) {
        const float h = uv + p;
        fx = h * vx;
        fy = h * vy;
        fz = h * vz;
    } else {
        fx = uv * vx + (V == 1 ? p : 0.0f);
        fy = uv * vy + (V == 2 ? p : 0.0f);
        fz = uv * vz + (V == 3 ? p : 0.0f);
    }
}

__device__ __forceinline__ void ne_flux3v(int v, float uv, float vx, float vy, float vz, float p, float &fx,
                                          float &fy, float &fz)
{
    switch (v) {
    case 0: ne_flux3<0>(uv, vx, vy, vz, p, fx, fy, fz); break;
    case 1: ne_flux3<1>(uv, vx, vy, vz, p, fx, fy, fz); break;
    case 2: ne_flux3<2>(uv, vx, vy, vz, p, fx, fy, fz); break;
    case 3: ne_flux3<3>(uv, vx, vy, vz, p, fx, fy, fz); break;
    default: ne_flux3<4>(uv, vx, vy, vz, p, fx, fy, fz); break;
    }
}

// Summaries of one element and variable from its per-(v, k) sums (second pass of
// the separable reduction): A0 = sum_j w_j L0(j, k), A1 = sum_j row1_j L0(j, k),
// AX0 / AXN = sum_j w_j X_0 / X_N (j, k), A4 = sum_j w_j L1(j, k), A5 / A6 = L0(0 /
// N, k), where the line partials of the line (j, k) are L0 = sum_i w_i X_i,
// L1 = sum_i row1_i X_i and the end values X_0, X_N.  Kind 0 mean, 1-6 face means
// (x lo/hi, y lo/hi, z lo/hi), 7-9 P1 coefficients (x, y, z).
template <int NP, class Q>
__device__ __forceinline__ float ne_final_sum(const NeArgs &a, int kind, Q q)
{
    float s = 0.0f;
    if (kind == 5 || kind == 6) return q(kind == 5 ? 0 : NP - 1, 0) * 0.25f;
    const int src = kind == 0 ? 0 : kind == 1 ? 2 : kind == 2 ? 3 : kind == 3 ? 5 : kind == 4 ? 6 : kind == 7 ? 4 : kind == 8 ? 1 : 0;
#pragma unroll
    for (int kk = 0; kk < NP; ++kk) s = fmaf(kind == 9 ? a.row1[kk] : a.w[kk], q(kk, src), s);
    return kind == 0 ? s * 0.125f : s * 0.25f;
}

// ---------------------------------------------------------------------------
// One stage of the delta-form step (ST = 1, 2, 3), or the right-hand side
// dU/dt = R(U^n) alone (ST = 0).  Sec. 3.1, eq:411 (volume term eq:405, surface
// terms with each face taken along +e_a, the lower element lifting
// -(2/dx_a)(F* - F_L)/w_N, the upper +(2/dx_a)(F* - F_R)/w_0); eq:LLF, eq:HLL,
// eq:Roe; Sec. 3.4 (SSP-RK3 in the difference form above, CFL maximum).
template <int NP, int FLX, int ST>
__global__ void __launch_bounds__(NeShape<NP>::THREADS, NeShape<NP>::MINB) k_ne_stage(const __grid_constant__ NeArgs a)
{
    using SH = NeShape<NP>;
    constexpr int L = SH::L, NN = SH::NN, EPB = SH::EPB, N1 = NP - 1;
    extern __shared__ __align__(16) float ne_smem[];
    __shared__ long long sNb[EPB][6];
    __shared__ unsigned sMask[EPB][7];  // neighbours' limited variables (1 + 2 ax + side)
    __shared__ unsigned sLamE[EPB];  // per element: max wave speed (bits of a non-negative float)
    __shared__ float4 sNbSH[EPB][6][5];  // the neighbours' replacement parameters (limited variables)
    __shared__ NeSlot sSlot[EPB];
    __shared__ long long sLoc[EPB];
    __shared__ uint64_t sBar[EPB];  // the element's bulk copies (stages 2, 3, even NP)
    __shared__ float4 sOwnSH[EPB][5];  // the element's own replacement parameters (staged stages)
    __shared__ double sOwnM0[EPB][5];
    // (U^n and the differences are 16-byte aligned: the library allocates the
    // differences, and its entry points refuse a caller's U that is not)
    constexpr bool STAGED = ST >= 1 && SH::STAGE;

    const int t = threadIdx.x;
    const int sub_raw = t / L, ln = t % L, j = ln % NP, k = ln / NP;
    const int sub = sub_raw < EPB ? sub_raw : EPB - 1;
    const long long e0 = (long long)blockIdx.x * EPB;  // first element of the CTA (launch numbering)
    const long long ge = e0 + sub;
    const bool live = sub_raw < EPB && ge < a.nelem;
    // Every element of the CTA gets its mesh's slot in shared memory (past the last
    // element: the first mesh's, so that per-slot settings, the same for all meshes
    // of a launch, are read consistently by every thread).  Single-mesh and batch
    // launches run this one code path, so they give the same bits.
    if (sub_raw < EPB) {
        // (the slot is copied word by word across the element's threads)
        constexpr int W = (int)(sizeof(NeSlot) / sizeof(unsigned long long));
        static_assert(sizeof(NeSlot) % sizeof(unsigned long long) == 0, "slot words");
        const int m = (a.slots && live) ? ne_find_slot(a.elem0, a.nslots, ge) : 0;
        const unsigned long long *src = reinterpret_cast<const unsigned long long *>(a.slots ? &a.slots[m] : &a.one);
        unsigned long long *dst = reinterpret_cast<unsigned long long *>(&sSlot[sub]);
        for (int w = ln; w < W; w += L) dst[w] = src[w];
        if (ln == 0) sLoc[sub] = live ? (a.slots ? ge - a.elem0[m] : ge) : 0;
        // nine arrivals: three from the staging thread, one per neighbour
        if (STAGED && ln == L - 1) ne_bar_init(&sBar[sub], 9);
    }
    if (t < EPB) sLamE[t] = 0u;
    __syncthreads();
    const NeSlot &sl = sSlot[sub];
    const long long e = sLoc[sub];                              // element index within its mesh
    const long long gofs = ge - e;                              // launch index of the mesh's element 0
    float *const eb = ne_smem + SH::ELEM_FLOATS * sub;
    float *const sU = eb + SH::F_U;
    float *const sH = eb + SH::F_H;
    float *const sF = eb + SH::F_F;
    float *const sL = eb + SH::F_L;
    const bool lim_in = ST >= 2 && sl.mask != nullptr;
    const bool do_sn = ST == 1 && sl.SN != nullptr;
    const float dtf = (ST >= 2 && live) ? (float)(sl.dt_ptr ? *sl.dt_ptr : sl.dt) : 0.0f;
    const float xj = a.x[j], xk = a.x[k];

    if (live && ln == L - 1) {
        if (STAGED) {
            // stages 2, 3: the element's U^n, its own replacement parameters and,
            // unless every variable is limited, its difference, into shared memory
            // by bulk copies that run while the neighbour tables are built; the
            // means U0 (40 bytes, not a bulk-copy size) by plain loads before the
            // last arrival, which publishes them
            ne_bulk_load(eb + SH::F_S, sl.Un + e * 5 * NN, 40u * NN, &sBar[sub]);
            if (lim_in) ne_bulk_load(&sOwnSH[sub][0], sl.SH + e * 5, 5u * sizeof(float4), &sBar[sub]);
            else ne_bar_arrive(&sBar[sub]);
            const unsigned mo = lim_in ? sl.mask[e] : 0u;
            if (lim_in)
#pragma unroll
                for (int v = 0; v < 5; ++v) sOwnM0[sub][v] = sl.M0[e * 5 + v];
            if (ST >= 2 && mo != 0x1fu) ne_bulk_load(eb + SH::F_U, sl.Din + e * 5 * NN, 20u * NN, &sBar[sub]);
            else ne_bar_arrive(&sBar[sub]);
        } else {
            // the element's U^n on its way to L2 while the neighbour tables are built
            ne_prefetch_l2(sl.Un + e * 5 * NN, sizeof(double) * 5 * NN);
        }
    }
    // The neighbour table and masks are read in the halo staging, after the barrier
    // that ends phase 1; phase 1 itself needs only the element's own mask, which
    // every thread loads (staged stages: while the copies are in flight).
    for (int q = ln; live && q < 7; q += L) {
        if (q == 6) {
            if (ST >= 2 && !STAGED && lim_in && sl.mask[e] != 0x1fu)
                ne_prefetch_l2(sl.Din + e * 5 * NN, sizeof(float) * 5 * NN);
        } else {
            const int ax = q >> 1, side = q & 1;
            const long long en = elem_neighbour_bc(e, sl.K, ax, side ? 1 : -1, sl.gh);
            sNb[sub][q] = en;
            if (STAGED) {
                // the neighbour's replacement parameters (all five; the masks say
                // which are read) on the element's barrier
                if (lim_in && en >= 0) ne_bulk_load(&sNbSH[sub][q][0], sl.SH + en * 5, 5u * sizeof(float4), &sBar[sub]);
                else ne_bar_arrive(&sBar[sub]);
            }
            sMask[sub][1 + q] = (lim_in && en >= 0) ? sl.mask[en] : 0u;
        }
    }
    const unsigned mask = (live && lim_in) ? sl.mask[e] : 0u;
    if (!STAGED) __syncthreads();  // the loop below reads the neighbour table
    // the neighbours' replacement parameters, once per element (read in the halo
    // staging, after the next barrier)
    for (int q = ln; !STAGED && lim_in && live && q < 30; q += L) {
        const int m = q / 5, v = q % 5;
        const long long en = sNb[sub][m];
        if (en >= 0 && ((sMask[sub][1 + m] >> v) & 1u)) sNbSH[sub][m][v] = sl.SH[en * 5 + v];
    }

    // ---- phase 1: the stage state of the thread's line: FP32 values for the
    // right-hand side (sU), the accurate difference d = U^s - U^n for the update;
    // stage 1 with a limiter: line partials of S(U^n) on U^n - c (c = the element's
    // node-0 value rounded to FP32), as double-float pairs where the limiter's
    // tests need them (L0 and the end values), FP32 for L1
    if (STAGED && live && !ne_bar_wait(&sBar[sub], NE_COPY_POLLS)) {
        // flag it, and give the copies one more bounded wait before their regions are reused
        atomicOr(sl.err, ERRBIT_TIMEOUT);
        ne_bar_wait(&sBar[sub], NE_COPY_POLLS);
    }
    // stage 1 with a limiter: the reference values c_v (node 0 of the element,
    // rounded to FP32), all five loads at once
    float cref[5];
#pragma unroll
    for (int v = 0; v < 5; ++v)
        cref[v] = (do_sn && live) ? ne_hi(STAGED ? reinterpret_cast<const double *>(eb + SH::F_S)[v * NN]
                                                 : sl.Un[(e * 5 + v) * NN])
                                  : 0.0f;
    // staged stage 1: the S(U^n) line partials wait in registers until every line
    // has read its U^n (their scratch lies over the staged copy)
    float snp[STAGED && ST == 1 ? 5 : 1][7];
    float d[5][NP];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        float uv[NP];
        const long long base = (e * 5 + v) * NN + (long long)ln * NP;
        double un[NP];
        if (live && STAGED) {
            const double2 *p2 = reinterpret_cast<const double2 *>(eb + SH::F_S) + (v * NN + ln * NP) / 2;
#pragma unroll
            for (int h = 0; h < NP / 2; ++h) {
                const double2 q = p2[h];
                un[2 * h] = q.x;
                un[2 * h + 1] = q.y;
            }
        } else if (live) {
            if (NP % 2 == 0) {
                const double2 *p2 = reinterpret_cast<const double2 *>(sl.Un + base);
#pragma unroll
                for (int h = 0; h < NP / 2; ++h) {
                    const double2 q = p2[h];
                    un[2 * h] = q.x;
                    un[2 * h + 1] = q.y;
                }
            } else {
#pragma unroll
                for (int i = 0; i < NP; ++i) un[i] = sl.Un[base + i];
            }
        } else {
#pragma unroll
            for (int i = 0; i < NP; ++i) un[i] = v == 0 ? 1.0 : (v == 4 ? 2.5 : 0.0);
        }
        float uh[NP];
        if (!(ST >= 2 && ((mask >> v) & 1u)))
#pragma unroll
            for (int i = 0; i < NP; ++i) uh[i] = ne_hi(un[i]);
        if (do_sn) {
            const float c = cref[v];
            float ah[NP], al[NP];
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                float err;
                ne_two_sum(uh[i], -c, ah[i], err);
                al[i] = __fadd_rn(err, ne_lo(un[i]));
            }
            float l0h = 0.0f, l0l = 0.0f, l1 = 0.0f;
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                ne_df_fma(l0h, l0l, a.wh[i], a.wl[i], ah[i], al[i]);
                l1 = fmaf(a.row1[i], ah[i] + al[i], l1);
            }
            if (STAGED) {
                float *q = snp[STAGED && ST == 1 ? v : 0];
                q[0] = l0h;
                q[1] = l0l;
                q[2] = l1;
                q[3] = ah[0];
                q[4] = al[0];
                q[5] = ah[N1];
                q[6] = al[N1];
            } else if (live) {
                float *P = sF + v * 7 * L + ln;
                P[0 * L] = l0h;
                P[1 * L] = l0l;
                P[2 * L] = l1;
                P[3 * L] = ah[0];
                P[4 * L] = al[0];
                P[5 * L] = ah[N1];
                P[6 * L] = al[N1];
            }
        }
        if (ST >= 2 && ((mask >> v) & 1u)) {
            // replaced: U^s = U0 + lin, so d = (U0 - U^n) + lin with U0 - U^n in FP64
            // (the FP64 pipe is otherwise idle here), rounded once to FP32
            const float4 sh = STAGED ? sOwnSH[sub][v] : sl.SH[e * 5 + v];
            const double m0 = STAGED ? sOwnM0[sub][v] : sl.M0[e * 5 + v];
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                const float lin = ne_lin(sh, a.x[i], xj, xk);
                uv[i] = __fadd_rn(sh.x, lin);
                d[v][i] = __fadd_rn(ne_hi(m0 - un[i]), lin);
            }
        } else if (ST >= 2) {
            float dv[NP];
            // staged: the difference sits where this line's stage state goes
            const float *src = STAGED ? sU + v * NN + ln * NP : sl.Din + base;
            if (live) {
                if (NP % 2 == 0) {
                    const float2 *p2 = reinterpret_cast<const float2 *>(src);
#pragma unroll
                    for (int h = 0; h < NP / 2; ++h) {
                        const float2 q = p2[h];
                        dv[2 * h] = q.x;
                        dv[2 * h + 1] = q.y;
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < NP; ++i) dv[i] = src[i];
                }
            } else {
#pragma unroll
                for (int i = 0; i < NP; ++i) dv[i] = 0.0f;
            }
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                d[v][i] = ST == 2 ? __fmul_rn(dtf, dv[i]) : dv[i];
                uv[i] = __fadd_rn(uh[i], d[v][i]);
            }
        } else {
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                d[v][i] = 0.0f;
                uv[i] = uh[i];
            }
        }
        if (live) ne_st_line<NP>(sU + v * NN + ln * NP, uv);
    }

    // CFL maximum of U^n (stage 1): max over nodes and axes of |v_a| + c, per
    // element in shared memory, then one atomic per run of elements of one mesh
    if (ST == 1 && sl.lam && live) {
        float lmax = 0.0f;
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            float w[5];
#pragma unroll
            for (int v = 0; v < 5; ++v) w[v] = sU[v * NN + ln * NP + i];
            float vx, vy, vz, p;
            ne_prims(a.gamma, w, vx, vy, vz, p);
            const float c = sqrtf(a.gamma * p / w[0]);
            lmax = fmaxf(lmax, fmaxf(fabsf(vx), fmaxf(fabsf(vy), fabsf(vz))) + c);
        }
        atomicMax(&sLamE[sub], __float_as_uint(lmax));
    }
    __syncthreads();
    if (ST == 1 && t == 0) {
        unsigned long long *cur = nullptr;
        float mx = 0.0f;
        for (int s0 = 0; s0 < EPB && e0 + s0 < a.nelem; ++s0) {
            const NeSlot &m = sSlot[s0];
            if (m.lam != cur) {
                if (cur) atomicMax(cur, (unsigned long long)__double_as_longlong(ne_f32_to_f64(mx)));
                cur = m.lam;
                mx = 0.0f;
            }
            mx = fmaxf(mx, __uint_as_float(sLamE[s0]));
        }
        if (cur) atomicMax(cur, (unsigned long long)__double_as_longlong(ne_f32_to_f64(mx)));
    }

    // ---- S(U^n) (stage 1 with a limiter), second pass: per (v, k) sums over j
    float *const sQn = sF + 35 * L;  // [5][NP][12]
    if (STAGED && ST == 1 && do_sn) {
        if (live)
#pragma unroll
            for (int v = 0; v < 5; ++v)
#pragma unroll
                for (int q = 0; q < 7; ++q) sF[v * 7 * L + q * L + ln] = snp[STAGED && ST == 1 ? v : 0][q];
        __syncthreads();
    }
    if (do_sn) {
        for (int r = ln; live && r < 5 * NP; r += L) {
            const int v = r / NP, kk = r % NP;
            const float *P = sF + v * 7 * L + NP * kk;
            float a0h = 0.0f, a0l = 0.0f, x0h = 0.0f, x0l = 0.0f, xnh = 0.0f, xnl = 0.0f, a1 = 0.0f, a4 = 0.0f;
#pragma unroll
            for (int jj = 0; jj < NP; ++jj) {
                const float l0h = P[jj], l0l = P[L + jj];
                ne_df_fma(a0h, a0l, a.wh[jj], a.wl[jj], l0h, l0l);
                ne_df_fma(x0h, x0l, a.wh[jj], a.wl[jj], P[3 * L + jj], P[4 * L + jj]);
                ne_df_fma(xnh, xnl, a.wh[jj], a.wl[jj], P[5 * L + jj], P[6 * L + jj]);
                a1 = fmaf(a.row1[jj], l0h + l0l, a1);
                a4 = fmaf(a.w[jj], P[2 * L + jj], a4);
            }
            float *Q = sQn + r * 12;
            Q[0] = a0h;
            Q[1] = a0l;
            Q[2] = x0h;
            Q[3] = x0l;
            Q[4] = xnh;
            Q[5] = xnl;
            Q[6] = P[0];            // L0(0, k)
            Q[7] = P[L];
            Q[8] = P[N1];           // L0(N, k)
            Q[9] = P[L + N1];
            Q[10] = a1;
            Q[11] = a4;
        }
        __syncthreads();
    }
    // third pass: the 50 summaries, the reference c added in FP64 (mean and face
    // means of a constant are the constant, its P1 coefficient is zero)
    if (do_sn) {
        // kind-major over the element's lines: the double-float kinds 0-4 all in the
        // first round, and neighbouring lanes on the same kind
        for (int t3 = ln; live && t3 < 50; t3 += L) {
            const int kind = t3 / 5, v = t3 % 5, o = v * 10 + kind;
            const float *Q = sQn + v * NP * 12;
            float h = 0.0f, l = 0.0f;
            if (kind == 5 || kind == 6) {
                const int kk = kind == 5 ? 0 : N1;
                h = Q[kk * 12] * 0.25f;
                l = Q[kk * 12 + 1] * 0.25f;
            } else if (kind <= 4) {
                const int src = kind == 0 ? 0 : kind == 1 ? 2 : kind == 2 ? 4 : kind == 3 ? 6 : 8;
#pragma unroll
                for (int kk = 0; kk < NP; ++kk)
                    ne_df_fma(h, l, a.wh[kk], a.wl[kk], Q[kk * 12 + src], Q[kk * 12 + src + 1]);
                const float sc = kind == 0 ? 0.125f : 0.25f;
                h *= sc;
                l *= sc;
            } else {
#pragma unroll
                for (int kk = 0; kk < NP; ++kk) {
                    const float val = kind == 7 ? Q[kk * 12 + 11] : kind == 8 ? Q[kk * 12 + 10] : Q[kk * 12] + Q[kk * 12 + 1];
                    h = fmaf(kind == 9 ? a.row1[kk] : a.w[kk], val, h);
                }
                h *= 0.25f;
            }
            const float cf = v == 0 ? cref[0] : v == 1 ? cref[1] : v == 2 ? cref[2] : v == 3 ? cref[3] : cref[4];
            const double cv = ne_f32_to_f64(cf);
            sl.SN[e * 50 + o] = (kind <= 6 ? cv : 0.0) + (ne_f32_to_f64(h) + ne_f32_to_f64(l));
        }
        __syncthreads();  // the scratch overlaps the halo and face-lift arrays
    }

    // ---- halo staging: the neighbours' traces at this thread's six face points,
    // from shared memory (elements of this CTA), a ghost's exterior state, or
    // global memory (U^n + D, or a limited variable's replacement)
    if (live) {
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            const int ax = m >> 1, side = m & 1, layn = side ? 0 : N1;
            const int qn = ne_face_node<NP>(ax, layn, j, k);
            const long long en = sNb[sub][m];
            const long long sn = en + gofs - e0;
            float w[5];
            if (en >= 0 && sn >= 0 && sn < EPB && en + gofs < a.nelem) {
                const float *nU = ne_smem + SH::ELEM_FLOATS * sn + SH::F_U;
#pragma unroll
                for (int v = 0; v < 5; ++v) w[v] = nU[v * NN + qn];
            } else if (en < 0) {
#pragma unroll
                for (int v = 0; v < 5; ++v) w[v] = ne_hi(sl.gh.U[((-1 - en) * 5 + v) * NN + qn]);
            } else {
                const unsigned nmask = sMask[sub][1 + m];
                // the face node's (x, y, z) LGL coordinates in the neighbour
                const float cx = ax == 0 ? a.x[layn] : xj;
                const float cy = ax == 0 ? xj : ax == 1 ? a.x[layn] : xk;
                const float cz = ax == 2 ? a.x[layn] : xk;
#pragma unroll
                for (int v = 0; v < 5; ++v) {
                    const long long ix = (en * 5 + v) * NN + qn;
                    if (ST >= 2 && ((nmask >> v) & 1u)) {
                        const float4 sh = sNbSH[sub][m][v];
                        w[v] = __fadd_rn(sh.x, ne_lin(sh, cx, cy, cz));
                    } else {
                        // the same roundings as the neighbour's own phase 1
                        w[v] = ne_hi(sl.Un[ix]);
                        if (ST >= 2) w[v] = __fadd_rn(w[v], ST == 2 ? __fmul_rn(dtf, sl.Din[ix]) : sl.Din[ix]);
                    }
                }
            }
#pragma unroll
            for (int v = 0; v < 5; ++v) sH[(m * L + ln) * 5 + v] = w[v];
        }
    }
    // (no barrier: each thread reads back only its own halo entries, and the face
    // fluxes write only lifts that are read after the next barrier)

    // ---- face fluxes at the thread's six face points.  x-face lifts belong to the
    // thread's own line and stay in registers; y and z lifts go to sL for the lines
    // that own them.
    float liftx[2][5];
    if (live) {
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            const int ax = m >> 1, side = m & 1;
            const int q = ne_face_node<NP>(ax, side ? N1 : 0, j, k);
            float wo[5], wn[5];
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                wo[v] = sU[v * NN + q];
                wn[v] = sH[(m * L + ln) * 5 + v];
            }
            // both traces in the face frame (normal, then the other two axes)
            const float uo[5] = {wo[0], ax == 0 ? wo[1] : ax == 1 ? wo[2] : wo[3], ax == 0 ? wo[2] : wo[1],
                                 ax == 2 ? wo[2] : wo[3], wo[4]};
            const float um[5] = {wn[0], ax == 0 ? wn[1] : ax == 1 ? wn[2] : wn[3], ax == 0 ? wn[2] : wn[1],
                                 ax == 2 ? wn[2] : wn[3], wn[4]};
            float dL[5], dR[5], o[5];
            if (side) {
                ne_face_flux<FLX>(a.gamma, uo, um, dL, dR);
#pragma unroll
                for (int v = 0; v < 5; ++v) o[v] = -sl.liftN[ax] * dL[v];
            } else {
                ne_face_flux<FLX>(a.gamma, um, uo, dL, dR);
#pragma unroll
                for (int v = 0; v < 5; ++v) o[v] = sl.lift0[ax] * dR[v];
            }
            // back to the mesh frame
            const float r[5] = {o[0], ax == 0 ? o[1] : o[2], ax == 0 ? o[2] : ax == 1 ? o[1] : o[3],
                                ax == 2 ? o[1] : o[3], o[4]};
            if (ax == 0) {
#pragma unroll
                for (int v = 0; v < 5; ++v) liftx[side][v] = r[v];
            } else {
                float *dst = sL + ((ax - 1) * 2 + side) * L * 5 + ln * 5;
#pragma unroll
                for (int v = 0; v < 5; ++v) dst[v] = r[v];
            }
        }
    }
    __syncthreads();

    // ---- volume term per variable: fluxes of the line minus the element's node-0
    // flux (D annihilates constants, so the FP32 rounding scales with the flux
    // variation inside the element), the x derivative in registers, the y and z
    // derivatives through shared memory (sF double-buffered over v)
    // (the state of the thread's own line and the element's node 0 come from sU;
    // from iteration v on, variable v's part of sU holds the summary partials)
    constexpr bool PART_IN_U = 4 * L <= NN;
    float vx[NP], vy[NP], vz[NP], pr[NP];
    {
        float ul[5][NP];
#pragma unroll
        for (int v = 0; v < 5; ++v) ne_ld_line<NP>(sU + v * NN + ln * NP, ul[v]);
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            float w[5];
#pragma unroll
            for (int v = 0; v < 5; ++v) w[v] = ul[v][i];
            ne_prims(a.gamma, w, vx[i], vy[i], vz[i], pr[i]);
        }
    }
    float vx0, vy0, vz0, pr0, u0[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) u0[v] = sU[v * NN];
    ne_prims(a.gamma, u0, vx0, vy0, vz0, pr0);
    float Dj[NP], Dk[NP];
#pragma unroll
    for (int l = 0; l < NP; ++l) {
        Dj[l] = a.D[j * NP + l];
        Dk[l] = a.D[k * NP + l];
    }
    float part[PART_IN_U ? 1 : 5][4];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        float *bF = sF + (v & 1) * 2 * NN;
        float rx, ry, rz;
        ne_flux3v(v, u0[v], vx0, vy0, vz0, pr0, rx, ry, rz);
        float uv[NP];
        ne_ld_line<NP>(sU + v * NN + ln * NP, uv);
        float fx[NP], fy[NP], fz[NP];
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            float f0, f1, f2;
            ne_flux3v(v, uv[i], vx[i], vy[i], vz[i], pr[i], f0, f1, f2);
            fx[i] = f0 - rx;
            fy[i] = f1 - ry;
            fz[i] = f2 - rz;
        }
        if (live) {
            ne_st_line<NP>(bF + ln * NP, fy);
            ne_st_line<NP>(bF + NN + ln * NP, fz);
        }
        float R[NP];
        if constexpr (NP % 2 == 0) {
            // node pairs (i, i + 1) in paired FP32 FMAs: the same per-node FMA chain
            float2 s2[NP / 2];
#pragma unroll
            for (int h = 0; h < NP / 2; ++h) s2[h] = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int l = 0; l < NP; ++l) {
                const float2 f2 = make_float2(fx[l], fx[l]);
#pragma unroll
                for (int h = 0; h < NP / 2; ++h)
                    s2[h] = __ffma2_rn(*reinterpret_cast<const float2 *>(&a.DT[l * NP + 2 * h]), f2, s2[h]);
            }
#pragma unroll
            for (int h = 0; h < NP / 2; ++h) {
                R[2 * h] = -sl.g[0] * s2[h].x;
                R[2 * h + 1] = -sl.g[0] * s2[h].y;
            }
        } else {
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                float s = 0.0f;
#pragma unroll
                for (int l = 0; l < NP; ++l) s = fmaf(a.D[i * NP + l], fx[l], s);
                R[i] = -sl.g[0] * s;
            }
        }
        __syncthreads();
        if (live) {
            float sy[NP], sz[NP];
            if constexpr (NP % 2 == 0) {
                // node pairs in paired FP32 FMAs, straight from the 64-bit line loads
                float2 sy2[NP / 2], sz2[NP / 2];
#pragma unroll
                for (int h = 0; h < NP / 2; ++h) sy2[h] = sz2[h] = make_float2(0.0f, 0.0f);
#pragma unroll
                for (int l = 0; l < NP; ++l) {
                    const float2 *gy2 = reinterpret_cast<const float2 *>(bF + NP * (l + NP * k));       // F^y(., l, k)
                    const float2 *gz2 = reinterpret_cast<const float2 *>(bF + NN + NP * (j + NP * l));  // F^z(., j, l)
                    const float2 dj2 = make_float2(Dj[l], Dj[l]), dk2 = make_float2(Dk[l], Dk[l]);
#pragma unroll
                    for (int h = 0; h < NP / 2; ++h) {
                        sy2[h] = __ffma2_rn(dj2, gy2[h], sy2[h]);
                        sz2[h] = __ffma2_rn(dk2, gz2[h], sz2[h]);
                    }
                }
#pragma unroll
                for (int h = 0; h < NP / 2; ++h) {
                    sy[2 * h] = sy2[h].x;
                    sy[2 * h + 1] = sy2[h].y;
                    sz[2 * h] = sz2[h].x;
                    sz[2 * h + 1] = sz2[h].y;
                }
            } else {
#pragma unroll
                for (int i = 0; i < NP; ++i) sy[i] = sz[i] = 0.0f;
#pragma unroll
                for (int l = 0; l < NP; ++l) {
                    float gy[NP], gz[NP];
                    ne_ld_line<NP>(bF + NP * (l + NP * k), gy);       // F^y(., l, k)
                    ne_ld_line<NP>(bF + NN + NP * (j + NP * l), gz);  // F^z(., j, l)
#pragma unroll
                    for (int i = 0; i < NP; ++i) {
                        sy[i] = fmaf(Dj[l], gy[i], sy[i]);
                        sz[i] = fmaf(Dk[l], gz[i], sz[i]);
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < NP; ++i) R[i] -= sl.g[1] * sy[i] + sl.g[2] * sz[i];
            // surface terms
            R[0] += liftx[0][v];
            R[N1] += liftx[1][v];
            if (j == 0 || j == N1) {
                const float *Ly = sL + (j == N1 ? 1 : 0) * L * 5;
#pragma unroll
                for (int i = 0; i < NP; ++i) R[i] += Ly[(i + NP * k) * 5 + v];
            }
            if (k == 0 || k == N1) {
                const float *Lz = sL + (2 + (k == N1 ? 1 : 0)) * L * 5;
#pragma unroll
                for (int i = 0; i < NP; ++i) R[i] += Lz[(i + NP * j) * 5 + v];
            }
            // output
            const long long base = (e * 5 + v) * NN + (long long)ln * NP;
            float X[NP];
            if (ST == 0) {
#pragma unroll
                for (int i = 0; i < NP; ++i) sl.rhs[base + i] = ne_f32_to_f64(R[i]);
            } else {
#pragma unroll
                for (int i = 0; i < NP; ++i) X[i] = ST == 1 ? R[i] : a.cb * (d[v][i] + dtf * R[i]);
                if (NP % 2 == 0) {
                    float2 *p2 = reinterpret_cast<float2 *>(sl.Dout + base);
#pragma unroll
                    for (int h = 0; h < NP / 2; ++h) p2[h] = make_float2(X[2 * h], X[2 * h + 1]);
                } else {
#pragma unroll
                    for (int i = 0; i < NP; ++i) sl.Dout[base + i] = X[i];
                }
                float l0 = 0.0f, l1 = 0.0f;
#pragma unroll
                for (int i = 0; i < NP; ++i) {
                    l0 = fmaf(a.w[i], X[i], l0);
                    l1 = fmaf(a.row1[i], X[i], l1);
                }
                if (PART_IN_U) {
                    // variable v's stage state is no longer read (after this iteration's barrier)
                    float *P = sU + v * NN + ln;
                    P[0] = l0;
                    P[L] = l1;
                    P[2 * L] = X[0];
                    P[3 * L] = X[N1];
                } else {
                    part[PART_IN_U ? 0 : v][0] = l0;
                    part[PART_IN_U ? 0 : v][1] = l1;
                    part[PART_IN_U ? 0 : v][2] = X[0];
                    part[PART_IN_U ? 0 : v][3] = X[N1];
                }
            }
        }
    }
    if (ST == 0 || !sl.SD) return;

    // ---- summaries S(Dout) in FP32: line partials (to U + H, last read before the
    // volume term's barriers), per-(v, k) sums, then the 50 values
    // partials of variable v at sU + v * NN (PART_IN_U), else [5][4][L] from U on
    float *const sP = eb + SH::F_U;
    constexpr int PSTR = PART_IN_U ? NN : 4 * L;
    float *const sQ = PART_IN_U ? sF : sL;    // [5][NP][7]; sF and sL are dead by now
    if (!PART_IN_U) {
        __syncthreads();  // (small n: the partials reach the flux buffers)
        if (live)
#pragma unroll
            for (int v = 0; v < 5; ++v)
#pragma unroll
                for (int q = 0; q < 4; ++q) sP[(v * 4 + q) * L + ln] = part[PART_IN_U ? 0 : v][q];
    }
    __syncthreads();
    for (int r = ln; live && r < 5 * NP; r += L) {
        const int v = r / NP, kk = r % NP;
        const float *P = sP + v * PSTR + NP * kk;
        float a0 = 0.0f, a1 = 0.0f, ax0 = 0.0f, axn = 0.0f, a4 = 0.0f;
#pragma unroll
        for (int jj = 0; jj < NP; ++jj) {
            a0 = fmaf(a.w[jj], P[jj], a0);
            a1 = fmaf(a.row1[jj], P[jj], a1);
            a4 = fmaf(a.w[jj], P[L + jj], a4);
            ax0 = fmaf(a.w[jj], P[2 * L + jj], ax0);
            axn = fmaf(a.w[jj], P[3 * L + jj], axn);
        }
        float *Q = sQ + r * 7;
        Q[0] = a0;
        Q[1] = a1;
        Q[2] = ax0;
        Q[3] = axn;
        Q[4] = a4;
        Q[5] = P[0];
        Q[6] = P[N1];
    }
    __syncthreads();
    for (int t3 = ln; live && t3 < 50; t3 += L) {  // kind-major: neighbouring lanes on one kind
        const int kind = t3 / 5, v = t3 % 5, o = v * 10 + kind;
        const float *Q = sQ + v * NP * 7;
        sl.SD[e * 50 + o] = ne_final_sum<NP>(a, kind, [&](int kk, int src) { return Q[kk * 7 + src]; });
    }
}

// ---------------------------------------------------------------------------
// Limiter decisions of the Newtonian delta-form step (Sec. 3.3.1-3.3.2), two
// elements per warp: lane 16 h + 3 v + a (v < 5, a < 3) decides variable v along
// axis a of element 2 w + h from S(U^s) = SN + c SD (FP64), as the other mixed
// limiter: the MinModN face tests (tolerance 1e-8, M = 0 in the detector), the
// m_B slope (eq:MinModB).  Limited variables get the replacement parameters of
// eq:MinModSol.  FINAL: the last pass of a step also writes U^{n+1} in place,
// U^n + D3 where not limited, else the replacement, in FP64.
template <int NP, int FINAL>
__global__ void __launch_bounds__(128) k_ne_decide(const __grid_constant__ NeDecideArgs a)
{
    constexpr int NN = NP * NP * NP;
    __shared__ float sx[MAXN];  // LGL nodes, for the final pass's per-lane coordinates
    if (FINAL) {
        if (threadIdx.x < MAXN) sx[threadIdx.x] = a.x[threadIdx.x];
        __syncthreads();
    }
    const int lane = threadIdx.x & 31, half = lane >> 4, h = lane & 15;
    const long long ge = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 4;
    const bool live = ge < a.nelem;
    // one code path for single-mesh and batch launches (the same bits either way)
    const int slot = (a.slots && live) ? ne_find_slot(a.elem0, a.nslots, ge) : 0;
    const NeDecideSlot &sl = a.slots ? a.slots[slot] : a.one;
    const long long e = live ? (a.slots ? ge - a.elem0[slot] : ge) : 0;
    const double c = a.scale_dt ? (sl.dt_ptr ? *sl.dt_ptr : sl.dt) : 1.0;
    int flag = 0;
    double U0 = 0.0;
    float shl = 0.0f;
    if (live && h < 15 && a.limiter) {
        const int v = h / 3, ax = h % 3;
        auto S = [&](long long el, int kind) {
            const long long ix = (el * 5 + v) * 10 + kind;
            return fma(c, ne_f32_to_f64(sl.SD[ix]), sl.SN[ix]);
        };
        U0 = S(e, 0);
        const double U0m = S(elem_neighbour(e, sl.K, ax, -1), 0);
        const double U0p = S(elem_neighbour(e, sl.K, ax, +1), 0);
        const double dm = U0 - U0m, dp = U0p - U0;
        flag = a.limiter == 2;
        if (a.limiter == 1) {
            // the face tests in FP64 (tolerance 1e-8 on O(U) values)
            // (|U0 - m - ulo| with a = U0 - ulo is |a - minmod(a, ...)|: zero when the
            // minmod keeps a, one FP64 difference otherwise; likewise at the upper face)
            const double al = U0 - S(e, 1 + 2 * ax), au = S(e, 2 + 2 * ax) - U0;
            if (abs_gt(al - minmod3_bits(al, dm, dp), 1e-8) || abs_gt(au - minmod3_bits(au, dm, dp), 1e-8)) flag = 1;
        }
        // the slope candidates of eq:MinModB from their FP64 differences, rounded to
        // FP32 (the replacement's slopes are FP32): the products and the pick on the
        // FP32 pipe
        const float s1 = ne_hi(S(e, 7 + ax)) * sl.two_inv_dx_f[ax];
        const float slope = fabsf(s1) <= sl.tvb_f[ax]
                                ? s1
                                : ne_minmod3f(s1, ne_hi(dp) * sl.beta_dx_f[ax], ne_hi(dm) * sl.beta_dx_f[ax]);
        shl = slope * sl.hdx_f[ax];
    }
    const unsigned fb = (__ballot_sync(0xffffffffu, flag) >> (16 * half)) & 0x7fffu;
    unsigned mask = 0;
#pragma unroll
    for (int v = 0; v < 5; ++v)
        if ((fb >> (3 * v)) & 7u) mask |= 1u << v;
    // replacement parameters: lane 3 v of the half gathers the slopes of v
    const float s1v = __shfl_down_sync(0xffffffffu, shl, 1);
    const float s2v = __shfl_down_sync(0xffffffffu, shl, 2);
    if (live && a.limiter) {
        if (h == 0) {
            sl.mask[e] = (unsigned char)mask;
            if (sl.troubled) sl.troubled[e] = (unsigned char)mask;
        }
        if (h < 15 && h % 3 == 0 && ((mask >> (h / 3)) & 1u)) {
            const int v = h / 3;
            sl.M0[e * 5 + v] = U0;
            sl.SH[e * 5 + v] = make_float4(ne_hi(U0), shl, s1v, s2v);
        }
    } else if (live && h == 0 && sl.troubled) {
        sl.troubled[e] = 0;
    }
    if (!FINAL) return;
    // U^{n+1} of the warp's two elements: 2 x NP^2 x-lines x 5 variables, each
    // (line, variable) a task of NP nodes, dealt to the 32 lanes in turn (U^n + D3,
    // or the replacement); the FP64 pipe then runs with nearly all lanes busy
    constexpr int TASKS = 2 * NP * NP * 5;
    __shared__ double sM0[4][2][5];  // per warp of the CTA: the two elements' parameters
    __shared__ float sSHp[4][2][5][3];
    __shared__ unsigned sMk[4][2];
    __shared__ long long sE[4][2];
    __shared__ int sLive[4][2];
    __shared__ double *sUp[4][2];      // the elements' meshes (a batch may mix meshes)
    __shared__ const float *sD3p[4][2];
    const int w = threadIdx.x >> 5;
    if (h < 15 && h % 3 == 0) {
        const int v = h / 3;
        sM0[w][half][v] = U0;
        sSHp[w][half][v][0] = shl;
        sSHp[w][half][v][1] = s1v;
        sSHp[w][half][v][2] = s2v;
    }
    if (h == 0) {
        sMk[w][half] = mask;
        sE[w][half] = e;
        sLive[w][half] = live ? 1 : 0;
        sUp[w][half] = sl.U;
        sD3p[w][half] = sl.D3;
    }
    __syncwarp();
    for (int tk = lane; tk < TASKS; tk += 32) {
        const int el = tk / (NP * NP * 5), rem = tk % (NP * NP * 5);
        const int v = rem / (NP * NP), ln = rem % (NP * NP);  // consecutive lanes: consecutive lines
        if (!sLive[w][el]) continue;
        const long long base = (sE[w][el] * 5 + v) * NN + (long long)ln * NP;
        double *const Ue = sUp[w][el];
        const float *const D3e = sD3p[w][el];
        double val[NP];
        if ((sMk[w][el] >> v) & 1u) {
            const float4 sh = make_float4(0.0f, sSHp[w][el][v][0], sSHp[w][el][v][1], sSHp[w][el][v][2]);
            const float xj = sx[ln % NP], xk = sx[ln / NP];
            const double m0 = sM0[w][el][v];
#pragma unroll
            for (int i = 0; i < NP; ++i) val[i] = m0 + ne_f32_to_f64(ne_lin(sh, a.x[i], xj, xk));
        } else {
#pragma unroll
            for (int i = 0; i < NP; ++i) val[i] = Ue[base + i] + ne_f32_to_f64(D3e[base + i]);
        }
        if (NP % 2 == 0) {
            double2 *p2 = reinterpret_cast<double2 *>(Ue + base);
#pragma unroll
            for (int q = 0; q < NP / 2; ++q) p2[q] = make_double2(val[2 * q], val[2 * q + 1]);
        } else {
#pragma unroll
            for (int i = 0; i < NP; ++i) Ue[base + i] = val[i];
        }
    }
}

template <int NP>
cudaError_t launch_ne_stage_np(int flux, int stage, const NeArgs &a, cudaStream_t s)
{
    using SH = NeShape<NP>;
    if (a.nelem <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)((a.nelem + SH::EPB - 1) / SH::EPB);
    void (*kern)(const NeArgs) = nullptr;
#define DG_NE_PICK(F)                                                                                 \
    kern = stage == 0 ? k_ne_stage<NP, F, 0> : stage == 1 ? k_ne_stage<NP, F, 1>                        \
         : stage == 2 ? k_ne_stage<NP, F, 2> : k_ne_stage<NP, F, 3>
    if (flux == 0) DG_NE_PICK(0);
    else if (flux == 1) DG_NE_PICK(1);
    else DG_NE_PICK(2);
#undef DG_NE_PICK
    // static + dynamic shared memory exceed 48 KB for every n: opt in
    const cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SH::SMEM);
    if (err != cudaSuccess) return err;
    kern<<<grid, SH::THREADS, SH::SMEM, s>>>(a);
    return cudaGetLastError();
}

template <int NP>
cudaError_t launch_ne_decide_np(int final_pass, const NeDecideArgs &a, cudaStream_t s)
{
    if (a.nelem <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)((a.nelem + 7) / 8);  // 8 elements per 128-thread CTA
    if (final_pass) k_ne_decide<NP, 1><<<grid, 128, 0, s>>>(a);
    else k_ne_decide<NP, 0><<<grid, 128, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace dg
