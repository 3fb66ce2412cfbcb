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

// SiLU for in-kernel inference: z sigma(z) = z (1 + tanh(z/2)) / 2 with the
// hardware tanh approximation (one MUFU operation instead of an exponential and
// a reciprocal; relative error ~2^-11, far below the BF16 rounding of layer 2).
__device__ __forceinline__ float silu_fast(float z)
{
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(0.5f * z));
    const float hz = 0.5f * z;
    return fmaf(hz, t, hz);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// Network weights staged in shared memory for in-kernel inference.  W2's rows
// are padded to 72 BF16 (144 bytes): the eight rows a B-fragment load touches then
// fall in different banks.
constexpr int NET_W2_LD = 72;
struct NetWeightsSmem {
    __nv_bfloat16 W2[64][NET_W2_LD];  // [j][i]: the B^T operand of layer 2
    float W1[64][3], b1[64], b2[64], W3[64], b3;
};

// Stage the weights (all threads of the CTA take part; the caller synchronises).
// W2 moves as 16-byte vectors, all loads issued before the stores, so a CTA
// waits about one L2 round trip rather than one per element.
__device__ __forceinline__ void net_stage_weights(NetWeightsSmem &W, const float *P, const __nv_bfloat16 *W2b)
{
    constexpr int NV = 64 * 64 * 2 / 16;  // uint4 vectors of W2, 8 per row
    const uint4 *src = reinterpret_cast<const uint4 *>(W2b);
    for (int k0 = 0; k0 < NV; k0 += 4 * (int)blockDim.x) {
        uint4 r[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int k = k0 + j * blockDim.x + threadIdx.x;
            if (k < NV) r[j] = __ldg(src + k);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int k = k0 + j * blockDim.x + threadIdx.x;
            if (k < NV) *reinterpret_cast<uint4 *>(&W.W2[k >> 3][(k & 7) * 8]) = r[j];
        }
    }
    for (int k = threadIdx.x; k < 192 + 64; k += blockDim.x) {
        const float w1 = __ldg(P + OFF_W1 + k);  // W1 and b1 are contiguous
        if (k < 192) (&W.W1[0][0])[k] = w1;
        else W.b1[k - 192] = w1;
    }
    for (int k = threadIdx.x; k < 64; k += blockDim.x) {
        W.b2[k] = __ldg(P + OFF_B2 + k);
        W.W3[k] = __ldg(P + OFF_W3 + k);
    }
    if (threadIdx.x == 0) W.b3 = __ldg(P + OFF_B3);
}

// Features and bracket data of one SR state, FP32: f = (x1, x2, x3, E, s, tau).
__device__ __forceinline__ void net_features(const float u[5], const float sc[6], float f[6])
{
    const float D = u[0], tau = u[4];
    const float E = tau + D;
    const float smag = sqrtf(u[1] * u[1] + u[2] * u[2] + u[3] * u[3]);
    f[0] = 2.0f * (log10f(tau / D) - sc[0]) / (sc[1] - sc[0]) - 1.0f;
    f[1] = 2.0f * smag / E - 1.0f;
    f[2] = 2.0f * (log10f(D) - sc[2]) / (sc[3] - sc[2]) - 1.0f;
    f[3] = E;
    f[4] = smag;
    f[5] = tau;
}

// Pressure guesses for `rows` states whose features sF[r][6] (net_features) sit in
// shared memory; writes sG[r].  Each warp takes 16-row tiles: layer 1 is evaluated
// straight into the A fragments of layer 2 (every hidden value belongs to exactly
// one lane), layer 2 runs as mma.sync m16n8k16 (BF16 in, FP32 accumulate), and
// layer 3 is a per-row dot product reduced over the four lanes of a row.  States
// with non-finite features (unphysical or non-positive D, tau) get -1, which
// con2prim reads as "no guess".
__device__ __forceinline__ void net_guess_rows(const NetWeightsSmem &W, const float (*sF)[6], float *sG, int rows,
                                               float gamma, const float sc[6])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int g = lane >> 2, tq = lane & 3;
    for (int r0 = warp * 16; r0 < rows; r0 += nwarps * 16) {
        const int ra = min(r0 + g, rows - 1), rb = min(r0 + g + 8, rows - 1);
        const float xa0 = sF[ra][0], xa1 = sF[ra][1], xa2 = sF[ra][2];
        const float xb0 = sF[rb][0], xb1 = sF[rb][1], xb2 = sF[rb][2];
        float acc[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[nt][c] = 0.0f;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            float h[2][4];  // [row a/b][col 2tq, 2tq+1, 2tq+8, 2tq+9]
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int j = kk * 16 + 2 * tq + (q & 1) + 8 * (q >> 1);
                h[0][q] = silu_fast(W.W1[j][0] * xa0 + W.W1[j][1] * xa1 + W.W1[j][2] * xa2 + W.b1[j]);
                h[1][q] = silu_fast(W.W1[j][0] * xb0 + W.W1[j][1] * xb1 + W.W1[j][2] * xb2 + W.b1[j]);
            }
            uint32_t af[4];
            af[0] = pack_bf16(h[0][0], h[0][1]);
            af[1] = pack_bf16(h[1][0], h[1][1]);
            af[2] = pack_bf16(h[0][2], h[0][3]);
            af[3] = pack_bf16(h[1][2], h[1][3]);
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                uint32_t bf[2];
                load_b(bf, &W.W2[0][0], NET_W2_LD, kk * 16, nt * 8, lane);
                mma_bf16(acc[nt], af, bf);
            }
        }
        float ya = 0.0f, yb = 0.0f;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int col = nt * 8 + 2 * tq + (c & 1);
                const float v = W.W3[col] * silu_fast(acc[nt][c] + W.b2[col]);
                if (c < 2) ya += v;
                else yb += v;
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
