// dg_c2p_net.cuh -- pieces of the learned con2prim starting guess (an addition to
// the SR con2prim of Sec. 2.1.2) shared by the standalone MLP kernels and the
// mixed-precision stage kernel: parameter layout, activations, the BF16
// tensor-core fragment helpers, and a CTA-wide inference routine for a batch of
// rows whose features sit in shared memory.
//
// Network: 3 -> 64 -> 64 -> 1 with SiLU activations.  Parameters (flat, FP32):
// W1[64][3], b1[64], W2[64][64], b2[64], W3[64], b3 (W[j][i] maps input i to
// output j).  Features (E = tau + D, s = |S|): x1 = 2 (log10(tau/D) - lo1)/(hi1 - lo1) - 1,
// x2 = 2 s/E - 1, x3 = 2 (log10 D - lo3)/(hi3 - lo3) - 1; the output y maps to the
// pressure E 10^(y y_scale + y_shift), clamped into con2prim's bracket
// [max(0, s - E), (gamma - 1) tau]; scales = (lo1, hi1, lo3, hi3, y_shift, y_scale).
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

namespace dg {

constexpr int NET_PARAMS = 4481;
constexpr int OFF_W1 = 0, OFF_B1 = 192, OFF_W2 = 256, OFF_B2 = 4352, OFF_W3 = 4416, OFF_B3 = 4480;
constexpr int NET_TILE = 128;  // samples per CTA of the standalone kernels, 32 per warp
constexpr int NET_PARTIAL = NET_PARAMS + 1;  // gradient + loss per CTA

struct NetTileArgs {
    const float *P;              // FP32 parameters
    const __nv_bfloat16 *W2b;    // W2 [j][i] in BF16
    const __nv_bfloat16 *W2tb;   // W2 transposed [i][j] in BF16
    const double *cons;          // 5 rows of `count`
    const double *p;             // true pressures (training) or nullptr
    double *guess;               // output guesses (inference) or nullptr
    float *partial;              // [gridDim.x][NET_PARTIAL] gradient partials (training)
    long long count;             // rows of cons
    long long first;             // first sample of this launch
    long long nsamp;             // samples in this launch (batch)
    float inv_batch;             // 1 / batch
    float gamma;
    float sc[6];
};

__device__ __forceinline__ float silu(float z) { return z * __fdividef(1.0f, 1.0f + __expf(-z)); }

__device__ __forceinline__ float dsilu(float z)
{
    const float s = __fdividef(1.0f, 1.0f + __expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], const uint32_t b[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// A fragment (16 x 16) of a row-major BF16 matrix M (leading dimension ld) at (r0, c0).
__device__ __forceinline__ void load_a(uint32_t a[4], const __nv_bfloat16 *M, int ld, int r0, int c0, int lane)
{
    const int g = lane >> 2, tq = lane & 3;
    a[0] = *reinterpret_cast<const uint32_t *>(M + (r0 + g) * ld + c0 + 2 * tq);
    a[1] = *reinterpret_cast<const uint32_t *>(M + (r0 + g + 8) * ld + c0 + 2 * tq);
    a[2] = *reinterpret_cast<const uint32_t *>(M + (r0 + g) * ld + c0 + 2 * tq + 8);
    a[3] = *reinterpret_cast<const uint32_t *>(M + (r0 + g + 8) * ld + c0 + 2 * tq + 8);
}

// B fragment (16 x 8, k x n) from the row-major transpose Bt[n][k] at (k0, n0).
__device__ __forceinline__ void load_b(uint32_t b[2], const __nv_bfloat16 *Bt, int ld, int k0, int n0, int lane)
{
    const int g = lane >> 2, tq = lane & 3;
    b[0] = *reinterpret_cast<const uint32_t *>(Bt + (n0 + g) * ld + k0 + 2 * tq);
    b[1] = *reinterpret_cast<const uint32_t *>(Bt + (n0 + g) * ld + k0 + 2 * tq + 8);
}

// In-kernel inference evaluates SiLU on halved pre-activations z' = z/2 (the image
// below stores W1, b1, W2, b2 halved, an exact scaling): silu(z) = z sigma(z) =
// z' (1 + tanh z'), one hardware tanh and one FMA.  tanh.approx has a relative
// error near 2^-11, far below the BF16 rounding of layer 2's inputs.
__device__ __forceinline__ float silu_half(float zh)
{
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(zh));
    return fmaf(zh, t, zh);
}

// The same for two values, packed as the BF16 pair that layer 2 takes as its A
// operand: (lo, hi) -> BF16x2 of (silu(2 lo), silu(2 hi)), tanh and FMA in BF16x2.
__device__ __forceinline__ uint32_t silu_half_bf16x2(float lo, float hi)
{
    uint32_t z, t, h;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(z) : "f"(hi), "f"(lo));
    asm("tanh.approx.bf16x2 %0, %1;" : "=r"(t) : "r"(z));
    asm("fma.rn.bf16x2 %0, %1, %2, %1;" : "=r"(h) : "r"(z), "r"(t));
    return h;
}

// TF32 rounding (round to nearest, ties away) of an FP32 value, as an FP32 bit pattern.
__device__ __forceinline__ uint32_t to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// D = A B + D for one m16n8k8 TF32 tile whose A has columns 4-7 zero (a2 = a3 = 0)
// and whose B has rows 4-7 zero (b1 = 0): a K = 4 product on the tensor cores.
__device__ __forceinline__ void mma_tf32_k4(float d[4], uint32_t a0, uint32_t a1, uint32_t b0)
{
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%6}, {%7,%6}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(0u), "r"(b0));
}

// Four 8 x 8 BF16 matrices from shared memory; this lane gives the address of one
// row (lanes 8m..8m+7: the rows of matrix m).
__device__ __forceinline__ void ldmatrix_x4(uint32_t r[4], const void *row)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(row);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a)
                 : "memory");
}

// Network weights for in-kernel inference, laid out as they sit in shared memory.
// The library keeps this image in device memory (refreshed whenever the
// parameters change) and each CTA fetches it with one bulk asynchronous copy.
// W2's rows are padded to 72 BF16 (144 bytes): the eight rows an ldmatrix touches
// then fall in different banks.  W1, b1, W2, b2 are stored halved (see silu_half).
constexpr int NET_W2_LD = 72;
struct NetWeightsSmem {
    __nv_bfloat16 W2h[64][NET_W2_LD];  // W2 / 2, [j][i]: the B^T operand of layer 2
    float4 W1b1h[64];                   // (W1[j][0], W1[j][1], W1[j][2], b1[j]) / 2, TF32-rounded
    float b2h[64];                      // b2 / 2
    float W3[64];
    float b3, pad[3];
};
static_assert(sizeof(NetWeightsSmem) % 16 == 0, "bulk copies move multiples of 16 bytes");

// The bulk copy: one thread initialises the barrier before a __syncthreads, one
// thread issues the copy after it, and every thread waits before reading.
__device__ __forceinline__ void net_bar_init(uint64_t *bar)
{
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void net_copy_issue(NetWeightsSmem *dst, const NetWeightsSmem *src, uint64_t *bar)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
    constexpr uint32_t bytes = sizeof(NetWeightsSmem);
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(b),
                 "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(d),
                 "l"(src), "r"(bytes), "r"(b)
                 : "memory");
}

// Poll the barrier's first phase at most `limit` times; false if the copy has not
// landed by then.
__device__ __forceinline__ bool net_copy_wait(uint64_t *bar, int limit)
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
constexpr int NET_COPY_POLLS = 1 << 20;

// Features and bracket data of one SR state, FP32: f = (x1, x2, x3, E, s, tau).
// log10 x = log2 x * log10 2 with the hardware log2 (relative error ~2^-22).
__device__ __forceinline__ void net_features(const float u[5], const float sc[6], float f[6])
{
    const float D = u[0], tau = u[4];
    const float E = tau + D;
    const float smag = sqrtf(u[1] * u[1] + u[2] * u[2] + u[3] * u[3]);
    constexpr float LOG10_2 = 0.30102999566398120f;
    f[0] = 2.0f * (__log2f(tau / D) * LOG10_2 - sc[0]) / (sc[1] - sc[0]) - 1.0f;
    f[1] = 2.0f * smag / E - 1.0f;
    f[2] = 2.0f * (__log2f(D) * LOG10_2 - sc[2]) / (sc[3] - sc[2]) - 1.0f;
    f[3] = E;
    f[4] = smag;
    f[5] = tau;
}

// Pressure guesses for `rows` states whose features sF[r][6] (net_features) sit in
// shared memory; writes sG[r].  Each warp takes 16-row tiles.  Layer 1 runs as
// TF32 mma.sync m16n8k8 with K = 4 (the three features and a constant 1 for the
// bias); its accumulator fragments are laid out as layer 2's A fragments, which
// the BF16x2 SiLU packs directly.  Layer 2 runs as mma.sync m16n8k16 (BF16 in, FP32
// accumulate, starting from the bias) with its B fragments loaded by ldmatrix, and
// layer 3 is a per-row dot product reduced over the four lanes of a row.  States with non-finite
// features (unphysical or non-positive D, tau) get -1, which con2prim reads as "no
// guess".
__device__ __forceinline__ void net_guess_rows(const NetWeightsSmem &W, const float (*sF)[6], float *sG, int rows,
                                               float gamma, const float sc[6])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int g = lane >> 2, tq = lane & 3;
    // this lane's ldmatrix row within a 16 (n) x 16 (k) block of W2h: matrices
    // (n 0-7, k 0-7), (n 0-7, k 8-15), (n 8-15, k 0-7), (n 8-15, k 8-15)
    const int lr_n = (lane & 7) + 8 * (lane >> 4), lr_k = 8 * ((lane >> 3) & 1);
    for (int r0 = warp * 16; r0 < rows; r0 += nwarps * 16) {
        const int ra = min(r0 + g, rows - 1), rb = min(r0 + g + 8, rows - 1);
        // layer 1's A fragment: column tq of rows ra, rb is feature tq (tq < 3) or 1
        const uint32_t fa = to_tf32(tq < 3 ? sF[ra][tq] : 1.0f), fb = to_tf32(tq < 3 ? sF[rb][tq] : 1.0f);
        const float *w1 = reinterpret_cast<const float *>(W.W1b1h);  // [64][4]
        float acc[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const float2 b = *reinterpret_cast<const float2 *>(&W.b2h[nt * 8 + 2 * tq]);
            acc[nt][0] = b.x;
            acc[nt][1] = b.y;
            acc[nt][2] = b.x;
            acc[nt][3] = b.y;
        }
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            // halved pre-activations of hidden units 16 kk .. 16 kk + 15 (two n-tiles)
            float z0[4] = {0.0f, 0.0f, 0.0f, 0.0f}, z1[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            mma_tf32_k4(z0, fa, fb, __float_as_uint(w1[(16 * kk + g) * 4 + tq]));
            mma_tf32_k4(z1, fa, fb, __float_as_uint(w1[(16 * kk + 8 + g) * 4 + tq]));
            uint32_t af[4];  // rows (g, g+8) x hidden units (16 kk + 2tq, +1 | +8, +9)
            af[0] = silu_half_bf16x2(z0[0], z0[1]);
            af[1] = silu_half_bf16x2(z0[2], z0[3]);
            af[2] = silu_half_bf16x2(z1[0], z1[1]);
            af[3] = silu_half_bf16x2(z1[2], z1[3]);
#pragma unroll
            for (int nt2 = 0; nt2 < 4; ++nt2) {
                uint32_t bq[4];
                ldmatrix_x4(bq, &W.W2h[nt2 * 16 + lr_n][kk * 16 + lr_k]);
                mma_bf16(acc[2 * nt2], af, bq);
                mma_bf16(acc[2 * nt2 + 1], af, bq + 2);
            }
        }
        float ya = 0.0f, yb = 0.0f;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const float2 w3 = *reinterpret_cast<const float2 *>(&W.W3[nt * 8 + 2 * tq]);
            ya = fmaf(w3.x, silu_half(acc[nt][0]), ya);
            ya = fmaf(w3.y, silu_half(acc[nt][1]), ya);
            yb = fmaf(w3.x, silu_half(acc[nt][2]), yb);
            yb = fmaf(w3.y, silu_half(acc[nt][3]), yb);
        }
        ya += __shfl_xor_sync(0xffffffffu, ya, 1);
        ya += __shfl_xor_sync(0xffffffffu, ya, 2);
        yb += __shfl_xor_sync(0xffffffffu, yb, 1);
        yb += __shfl_xor_sync(0xffffffffu, yb, 2);
        if (tq == 0) {
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
                const int r = r0 + g + 8 * h2;
                if (r >= rows) continue;
                const float y = (h2 ? yb : ya) + W.b3;
                const float E = sF[r][3], smag = sF[r][4], tau = sF[r][5];
                float pg = E * exp10f(y * sc[5] + sc[4]);
                pg = fminf(fmaxf(pg, fmaxf(smag - E, 0.0f)), (gamma - 1.0f) * tau);
                const bool ok = isfinite(sF[r][0]) && isfinite(sF[r][2]) && isfinite(pg) && pg >= 0.0f;
                sG[r] = ok ? pg : -1.0f;
            }
        }
    }
}

}  // namespace dg
