// dg_limit_mixed.cuh -- limiter of the mixed-precision path (templated on the
// number of LGL nodes per axis NP).  Included at the end of dg_mixed.cuh, whose
// helpers it uses (mesh slots, FP32 screens, FP64<->FP32 conversions).
#pragma once

namespace dg {

// Sign tests, minmod (eq:MinMod) and magnitude comparisons of doubles done on
// their bit patterns, on the integer ALU instead of the FP64 pipe (which bounds
// this kernel).  They decide exactly as the floating-point forms, NaN included:
// - a double is > 0 iff its bits, read as a signed integer, lie in (0, +inf];
// - it is < 0 iff its sign bit is set and its magnitude bits lie in (0, inf]
//   (-0 is not negative);
// - doubles of one sign are ordered like their bits, reversed for negatives, so
//   among three positive or three negative doubles the one closest to 0 (the
//   minmod pick) has the smallest bit pattern as a signed integer;
// - |x| > c and |x| <= c for a finite c >= 0 compare the magnitude bits with c's.
constexpr long long kMagBits = 0x7fffffffffffffffLL;
constexpr long long kInfBits = 0x7ff0000000000000LL;

__device__ __forceinline__ bool bits_pos(long long b) { return b > 0 && b <= kInfBits; }
__device__ __forceinline__ bool bits_neg(long long b)
{
    const long long m = b & kMagBits;
    return b < 0 && m != 0 && m <= kInfBits;
}

__device__ __forceinline__ double minmod3_bits(double a1, double a2, double a3)
{
    const long long b1 = __double_as_longlong(a1), b2 = __double_as_longlong(a2), b3 = __double_as_longlong(a3);
    const bool pos = bits_pos(b1) & bits_pos(b2) & bits_pos(b3);
    const bool neg = bits_neg(b1) & bits_neg(b2) & bits_neg(b3);
    return (pos | neg) ? __longlong_as_double(min(b1, min(b2, b3))) : 0.0;
}

// |x| > c, for finite c >= 0
__device__ __forceinline__ bool abs_gt(double x, double c)
{
    const long long m = __double_as_longlong(x) & kMagBits;
    return m > __double_as_longlong(c) && m <= kInfBits;
}

// |x| <= c, for finite c >= 0
__device__ __forceinline__ bool abs_le(double x, double c)
{
    return (__double_as_longlong(x) & kMagBits) <= __double_as_longlong(c);
}

// ---------------------------------------------------------------------------
// Limiter of the mixed path on FP64 stage states, one warp per element.  Lane
// 3v + a (v < 5, a < 3) decides variable v along axis a: the MinModN face tests
// of Sec. 3.3.2 (tolerance 1e-8, M = 0) and the m_B slope (eq:MinModB) in FP64,
// with the divisions by dx and dx/beta taken as products with host reciprocals.
// A limited variable becomes U0 + sum_a slope_a (x_a - x_a0) (eq:MinModSol) in
// FP64; then (SR) the conserved fix of Sec. 2.1.4 runs in FP64 on every node that
// an FP32 screen of its bounds does not clear (such nodes are gathered, so the
// FP64 fix runs in as few warp passes as possible).  Elements that are neither
// troubled nor flagged by the stage kernel as needing the fix are left alone.
// Like the stage kernel, a launch covers one mesh or a ragged batch of meshes.
struct LimitSlot {
    double *U;
    const double *S;
    const unsigned char *flags;
    unsigned char *troubled;
    int K[3];
    double tvb[3];          // M dx_a^2
    double inv_dx[3];       // 1 / dx_a
    double beta_dx[3];      // beta / dx_a
    double hdx[3];          // dx_a / 2
};

struct LimitMixedArgs {
    LimitSlot one;
    const LimitSlot *slots;
    const long long *elem0;
    int nslots;
    long long E;            // elements in the launch
    int limiter;
    double d_atm, tau_atm;
    double x[MAXN];         // LGL nodes
};

// Warps (elements) per CTA of the limiter: small CTAs spread a one-wave launch
// evenly over the SMs (with 8 warps per CTA, 4,096 elements left some SMs a third
// more work than others).
constexpr int kLimitWarps = 4;

template <int NP, int SYS>
__global__ void __launch_bounds__(32 * kLimitWarps) k_limit_mixed(const LimitMixedArgs a)
{
    constexpr int NN = NP * NP * NP;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= a.E) return;
    long long e = warp;
    const LimitSlot *slp = &a.one;
    if (a.slots) {
        const int m = find_slot(a.elem0, a.nslots, warp);
        slp = a.slots + m;
        e = warp - a.elem0[m];
    }
    const LimitSlot &sl = *slp;
    int flag = 0;
    double slope = 0.0, U0 = 0.0;
    if (lane < 15) {
        const int v = lane / 3, ax = lane % 3;
        const double *Se = sl.S + (e * 5 + v) * 10;
        U0 = Se[0];
        const double U0m = sl.S[(elem_neighbour(e, sl.K, ax, -1) * 5 + v) * 10];
        const double U0p = sl.S[(elem_neighbour(e, sl.K, ax, +1) * 5 + v) * 10];
        flag = (a.limiter == 2);
        if (a.limiter == 1) {
            const double ulo = Se[1 + 2 * ax], uhi = Se[2 + 2 * ax];
            const double vl = U0 - minmod3_bits(U0 - ulo, U0 - U0m, U0p - U0);
            const double vr = U0 + minmod3_bits(uhi - U0, U0 - U0m, U0p - U0);
            if (abs_gt(vl - ulo, 1e-8) || abs_gt(vr - uhi, 1e-8)) flag = 1;
        }
        const double s1 = 2.0 * Se[7 + ax] * sl.inv_dx[ax];
        slope = abs_le(s1, sl.tvb[ax]) ? s1
                                       : minmod3_bits(s1, (U0p - U0) * sl.beta_dx[ax], (U0 - U0m) * sl.beta_dx[ax]);
    }
    const unsigned fb = __ballot_sync(0xffffffffu, flag);
    unsigned mask = 0;
#pragma unroll
    for (int v = 0; v < 5; ++v)
        if ((fb >> (3 * v)) & 7u) mask |= 1u << v;
    const unsigned char fl = sl.flags ? sl.flags[e] : 0;
    if (fl & 1) mask = 0x1fu;
    if (lane == 0 && sl.troubled) sl.troubled[e] = (unsigned char)mask;
    if (!mask && !(fl & 2)) return;
    // The replacement m0 + s0 h0(i) + s1 h1(j) + s2 h2(k) (h_a = (dx_a/2) xbar): the
    // part m0 + s0 h0(i) + s1 h1(j) is built once per (i, j) plane point and
    // variable, so a node costs one FP64 FMA per limited variable.
    __shared__ double sAB[kLimitWarps][5][NP * NP];  // per warp of the CTA
    __shared__ double sH2[kLimitWarps][NP];
    const int wl = threadIdx.x >> 5;
    double s2[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) s2[v] = __shfl_sync(0xffffffffu, slope, 3 * v + 2);
    if (mask) {
        double m0[5], s0[5], s1[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            m0[v] = __shfl_sync(0xffffffffu, U0, 3 * v);
            s0[v] = __shfl_sync(0xffffffffu, slope, 3 * v);
            s1[v] = __shfl_sync(0xffffffffu, slope, 3 * v + 1);
        }
        for (int ij = lane; ij < NP * NP; ij += 32) {
            const double h0 = sl.hdx[0] * a.x[ij % NP], h1 = sl.hdx[1] * a.x[ij / NP];
#pragma unroll
            for (int v = 0; v < 5; ++v) sAB[wl][v][ij] = fma(s1[v], h1, fma(s0[v], h0, m0[v]));
        }
        if (lane < NP) sH2[wl][lane] = sl.hdx[2] * a.x[lane];
        __syncwarp();
    }
    // Node values: the replacement of the limited variables, else the stage state.
    auto node = [&](int q, double u[5]) {
        const int ij = q % (NP * NP), k = q / (NP * NP);
        const double h2 = mask ? sH2[wl][k] : 0.0;
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            const long long ix = (e * 5 + v) * NN + q;
            u[v] = (mask & (1u << v)) ? fma(s2[v], h2, sAB[wl][v][ij]) : sl.U[ix];
        }
    };
    // Nodes the FP32 screen does not clear are listed and fixed afterwards in full
    // warps: a warp-wide FP64 instruction costs the same with one lane active.
    __shared__ unsigned short sFix[kLimitWarps][NN];
    int nfix = 0;
    for (int q0 = 0; q0 < NN; q0 += 32) {
        const int q = q0 + lane;
        bool need = false;
        if (q < NN) {
            double u[5];
            node(q, u);
            if (SYS == 1) {
                float u32[5];
#pragma unroll
                for (int v = 0; v < 5; ++v) u32[v] = f64_to_f32(u[v]);
                need = sr_screen32(u32, (float)a.d_atm, (float)a.tau_atm);
            }
            if (!need)
#pragma unroll
                for (int v = 0; v < 5; ++v)
                    if (mask & (1u << v)) sl.U[(e * 5 + v) * NN + q] = u[v];
        }
        if (SYS == 1) {
            const unsigned b = __ballot_sync(0xffffffffu, need);
            if (need) sFix[wl][nfix + __popc(b & ((1u << lane) - 1u))] = (unsigned short)q;
            nfix += __popc(b);
        }
    }
    if (SYS == 1 && nfix) {
        __syncwarp();
        for (int r = lane; r < nfix; r += 32) {
            const int q = sFix[wl][r];
            double u[5];
            node(q, u);
            const unsigned nm = mask | sr_fix(a.d_atm, a.tau_atm, u);
#pragma unroll
            for (int v = 0; v < 5; ++v)
                if (nm & (1u << v)) sl.U[(e * 5 + v) * NN + q] = u[v];
        }
    }
}

template <int NP>
cudaError_t launch_limit_mixed_np(int system, const LimitMixedArgs &a, cudaStream_t s)
{
    if (a.E <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)((a.E + kLimitWarps - 1) / kLimitWarps);  // one warp per element
    if (system == 0) k_limit_mixed<NP, 0><<<grid, 32 * kLimitWarps, 0, s>>>(a);
    else k_limit_mixed<NP, 1><<<grid, 32 * kLimitWarps, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace dg
