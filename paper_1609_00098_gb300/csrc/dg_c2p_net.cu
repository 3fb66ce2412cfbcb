// dg_c2p_net.cu -- learned starting guess for the SR con2prim Newton solve
// (Sec. 2.1.2): a 3 -> 64 -> 64 -> 1 SiLU MLP mapping scaled invariants of the
// conserved state to a scaled log pressure, with its own inference, gradient and
// Adam training kernels.  The 64 x 64 layer runs on the tensor cores
// (mma.sync m16n8k16, BF16 operands, FP32 accumulation) in the forward pass and
// in both backward products; the rest is FP32.  Reductions run in a fixed order,
// so training is deterministic.
//
// Parameters (flat, FP32): W1[64][3], b1[64], W2[64][64], b2[64], W3[64], b3.
// Features (E = tau + D, s = |S|): x1 = 2 (log10(tau/D) - lo1)/(hi1 - lo1) - 1,
// x2 = 2 s/E - 1, x3 = 2 (log10 D - lo3)/(hi3 - lo3) - 1; target
// y = (log10(p/E) - y_shift)/y_scale; scales = (lo1, hi1, lo3, hi3, y_shift, y_scale).
#include <cuda_bf16.h>

#include <cstdint>
#include <cstring>

#include "dg_c2p_net.cuh"
#include "dg_mixed.cuh"

namespace dg {

// Shared memory of one tile.  Inference needs only the first block of members.
struct NetSmemFwd {
    float x[NET_TILE][3];
    float t[NET_TILE];
    int ok[NET_TILE];                   // finite features (and target): takes part in the loss
    __nv_bfloat16 h1[NET_TILE][64];     // A of layer 2
    __nv_bfloat16 W2[64][64];           // B^T of layer 2
    float W1[64][3], b1[64], b2[64], W3[64];
};
struct NetSmem : NetSmemFwd {
    float z1[NET_TILE][64];
    __nv_bfloat16 h1t[64][NET_TILE];    // B^T of dW2
    __nv_bfloat16 dz2[NET_TILE][64];    // A of dh1
    __nv_bfloat16 dz2t[64][NET_TILE];   // A of dW2
    __nv_bfloat16 W2t[64][64];          // B^T of dh1
    float red[4][64 * 3 + 64 + 64 + 64 + 2];  // per-warp partial sums
};

template <bool TRAIN>
__global__ void __launch_bounds__(NET_TILE) k_net_tile(const NetTileArgs a)
{
    extern __shared__ __align__(16) unsigned char net_smem_raw[];
    // inference touches only the NetSmemFwd part and is launched with its size
    NetSmem &S = *reinterpret_cast<NetSmem *>(net_smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, tq = lane & 3;

    for (int k = tid; k < 64 * 64; k += NET_TILE) {
        (&S.W2[0][0])[k] = a.W2b[k];
        if (TRAIN) (&S.W2t[0][0])[k] = a.W2tb[k];
    }
    for (int k = tid; k < 192; k += NET_TILE) (&S.W1[0][0])[k] = a.P[OFF_W1 + k];
    if (tid < 64) {
        S.b1[tid] = a.P[OFF_B1 + tid];
        S.b2[tid] = a.P[OFF_B2 + tid];
        S.W3[tid] = a.P[OFF_W3 + tid];
    }
    const float b3 = a.P[OFF_B3];

    // features of this thread's sample
    const long long sloc = (long long)blockIdx.x * NET_TILE + tid;  // index within the launch
    const bool valid = sloc < a.nsamp;
    const long long gs = a.first + sloc;
    float E32 = 1.0f, smag = 0.0f, tau32 = 1.0f;
    {
        float x0 = 0.f, x1 = 0.f, x2 = 0.f, t = 0.f;
        if (valid) {
            const float D = f64_to_f32(a.cons[gs]);
            const float Sx = f64_to_f32(a.cons[a.count + gs]), Sy = f64_to_f32(a.cons[2 * a.count + gs]);
            const float Sz = f64_to_f32(a.cons[3 * a.count + gs]);
            tau32 = f64_to_f32(a.cons[4 * a.count + gs]);
            E32 = tau32 + D;
            smag = sqrtf(Sx * Sx + Sy * Sy + Sz * Sz);
            x0 = 2.0f * (log10f(tau32 / D) - a.sc[0]) / (a.sc[1] - a.sc[0]) - 1.0f;
            x1 = 2.0f * smag / E32 - 1.0f;
            x2 = 2.0f * (log10f(D) - a.sc[2]) / (a.sc[3] - a.sc[2]) - 1.0f;
            if (TRAIN) t = (log10f(f64_to_f32(a.p[gs]) / E32) - a.sc[4]) / a.sc[5];
        }
        // states whose features or target are not finite (D or tau not positive,
        // a pressure below the FP32 range) enter neither the loss nor the gradient
        const bool fin = valid && isfinite(x0) && isfinite(x1) && isfinite(x2) && isfinite(t);
        if (!fin) x0 = x1 = x2 = t = 0.0f;
        S.x[tid][0] = x0;
        S.x[tid][1] = x1;
        S.x[tid][2] = x2;
        S.t[tid] = t;
        S.ok[tid] = fin ? 1 : 0;
    }
    __syncthreads();

    // layer 1 (FP32) for the thread's own sample
    for (int j = 0; j < 64; ++j) {
        const float z = S.W1[j][0] * S.x[tid][0] + S.W1[j][1] * S.x[tid][1] + S.W1[j][2] * S.x[tid][2] + S.b1[j];
        const float h = silu(z);
        S.h1[tid][j] = __float2bfloat16_rn(h);
        if (TRAIN) {
            S.z1[tid][j] = z;
            S.h1t[j][tid] = __float2bfloat16_rn(h);
        }
    }
    __syncthreads();

    // layer 2 on the tensor cores: z2[s][j] = sum_i h1[s][i] W2[j][i]
    const int r0 = warp * 32;
    float acc[2][8][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[mt][nt][c] = 0.0f;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        uint32_t af[2][4];
        load_a(af[0], &S.h1[0][0], 64, r0, kk * 16, lane);
        load_a(af[1], &S.h1[0][0], 64, r0 + 16, kk * 16, lane);
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            uint32_t bf[2];
            load_b(bf, &S.W2[0][0], 64, kk * 16, nt * 8, lane);
            mma_bf16(acc[0][nt], af[0], bf);
            mma_bf16(acc[1][nt], af[1], bf);
        }
    }
    // layer 3: y = W3 . silu(z2 + b2) + b3; thread holds rows (g, g+8) of each m-tile
    float ypart[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int col = nt * 8 + 2 * tq + (c & 1);
                const float z = acc[mt][nt][c] + S.b2[col];
                acc[mt][nt][c] = z;  // keep z2
                ypart[mt][c >> 1] += S.W3[col] * silu(z);
            }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float v = ypart[mt][h];
            v += __shfl_xor_sync(0xffffffffu, v, 1);
            v += __shfl_xor_sync(0xffffffffu, v, 2);
            ypart[mt][h] = v + b3;
        }

    if (!TRAIN) {
        if (tq == 0) {
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int row = r0 + mt * 16 + g + 8 * h;
                    const long long sl = (long long)blockIdx.x * NET_TILE + row;
                    if (sl < a.nsamp) {
                        const long long gi = a.first + sl;
                        const float D = f64_to_f32(a.cons[gi]);
                        const float tau = f64_to_f32(a.cons[4 * a.count + gi]);
                        const float Sx = f64_to_f32(a.cons[a.count + gi]), Sy = f64_to_f32(a.cons[2 * a.count + gi]);
                        const float Sz = f64_to_f32(a.cons[3 * a.count + gi]);
                        const float E = tau + D;
                        float pg = E * exp10f(ypart[mt][h] * a.sc[5] + a.sc[4]);
                        pg = fminf(fmaxf(pg, fmaxf(sqrtf(Sx * Sx + Sy * Sy + Sz * Sz) - E, 0.0f)), (a.gamma - 1.0f) * tau);
                        a.guess[gi] = (S.ok[row] && isfinite(pg)) ? f32_to_f64(pg) : -1.0;
                    }
                }
        }
        return;
    }

    // ---- backward ----
    float *red = S.red[warp];
    float dy[2][2], loss_part = 0.0f, db3_part = 0.0f;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int row = r0 + mt * 16 + g + 8 * h;
            const bool ok = (long long)blockIdx.x * NET_TILE + row < a.nsamp && S.ok[row];
            const float r = ok ? ypart[mt][h] - S.t[row] : 0.0f;
            dy[mt][h] = 2.0f * r * a.inv_batch;
            if (tq == 0) {
                loss_part += r * r;
                db3_part += dy[mt][h];
            }
        }
    // dW3[col] = sum_s dy h2; db2[col] = sum_s dz2; dz2 = dy W3 silu'(z2)
    float w3p[8][2], b2p[8][2];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int e2 = 0; e2 < 2; ++e2) {
            w3p[nt][e2] = 0.0f;
            b2p[nt][e2] = 0.0f;
        }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int col = nt * 8 + 2 * tq + (c & 1);
                const int row = r0 + mt * 16 + g + 8 * (c >> 1);
                const float z = acc[mt][nt][c];
                const float d = dy[mt][c >> 1];
                w3p[nt][c & 1] += d * silu(z);
                const float dz = d * S.W3[col] * dsilu(z);
                b2p[nt][c & 1] += dz;
                const __nv_bfloat16 dzb = __float2bfloat16_rn(dz);
                S.dz2[row][col] = dzb;
                S.dz2t[col][row] = dzb;
            }
    // reduce over the 8 row groups (lanes with the same tq)
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int e2 = 0; e2 < 2; ++e2) {
            float v = w3p[nt][e2], u = b2p[nt][e2];
            for (int o = 4; o < 32; o <<= 1) {
                v += __shfl_xor_sync(0xffffffffu, v, o);
                u += __shfl_xor_sync(0xffffffffu, u, o);
            }
            if (g == 0) {
                red[192 + 64 + 64 + nt * 8 + 2 * tq + e2] = v;  // W3
                red[192 + 64 + nt * 8 + 2 * tq + e2] = u;       // b2
            }
        }
    for (int o = 1; o < 32; o <<= 1) {
        loss_part += __shfl_xor_sync(0xffffffffu, loss_part, o);
        db3_part += __shfl_xor_sync(0xffffffffu, db3_part, o);
    }
    if (lane == 0) {
        red[192 + 64 + 64 + 64] = db3_part;
        red[192 + 64 + 64 + 64 + 1] = loss_part;
    }
    __syncthreads();

    // dW2[j][i] = sum_s dz2[s][j] h1[s][i]: warp w takes rows j in [16w, 16w+16), all 128 samples
    {
        float gacc[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int c = 0; c < 4; ++c) gacc[nt][c] = 0.0f;
#pragma unroll
        for (int kk = 0; kk < NET_TILE / 16; ++kk) {
            uint32_t af[4];
            load_a(af, &S.dz2t[0][0], NET_TILE, warp * 16, kk * 16, lane);
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                uint32_t bf[2];
                load_b(bf, &S.h1t[0][0], NET_TILE, kk * 16, nt * 8, lane);
                mma_bf16(gacc[nt], af, bf);
            }
        }
        float *out = a.partial + (long long)blockIdx.x * NET_PARTIAL + OFF_W2;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int j = warp * 16 + g + 8 * (c >> 1);
                const int i = nt * 8 + 2 * tq + (c & 1);
                out[j * 64 + i] = gacc[nt][c];
            }
    }
    // dh1[s][i] = sum_j dz2[s][j] W2[j][i], then dz1 = dh1 silu'(z1); dW1, db1
    {
        float hacc[2][8][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 8; ++nt)
#pragma unroll
                for (int c = 0; c < 4; ++c) hacc[mt][nt][c] = 0.0f;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            uint32_t af[2][4];
            load_a(af[0], &S.dz2[0][0], 64, r0, kk * 16, lane);
            load_a(af[1], &S.dz2[0][0], 64, r0 + 16, kk * 16, lane);
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                uint32_t bf[2];
                load_b(bf, &S.W2t[0][0], 64, kk * 16, nt * 8, lane);
                mma_bf16(hacc[0][nt], af[0], bf);
                mma_bf16(hacc[1][nt], af[1], bf);
            }
        }
        float w1p[8][2][3], b1p[8][2];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int e2 = 0; e2 < 2; ++e2) {
                b1p[nt][e2] = 0.0f;
                w1p[nt][e2][0] = w1p[nt][e2][1] = w1p[nt][e2][2] = 0.0f;
            }
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 8; ++nt)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int i = nt * 8 + 2 * tq + (c & 1);
                    const int row = r0 + mt * 16 + g + 8 * (c >> 1);
                    const float dz = hacc[mt][nt][c] * dsilu(S.z1[row][i]);
                    b1p[nt][c & 1] += dz;
                    w1p[nt][c & 1][0] += dz * S.x[row][0];
                    w1p[nt][c & 1][1] += dz * S.x[row][1];
                    w1p[nt][c & 1][2] += dz * S.x[row][2];
                }
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int e2 = 0; e2 < 2; ++e2) {
                float v0 = w1p[nt][e2][0], v1 = w1p[nt][e2][1], v2 = w1p[nt][e2][2], u = b1p[nt][e2];
                for (int o = 4; o < 32; o <<= 1) {
                    v0 += __shfl_xor_sync(0xffffffffu, v0, o);
                    v1 += __shfl_xor_sync(0xffffffffu, v1, o);
                    v2 += __shfl_xor_sync(0xffffffffu, v2, o);
                    u += __shfl_xor_sync(0xffffffffu, u, o);
                }
                if (g == 0) {
                    const int i = nt * 8 + 2 * tq + e2;
                    red[i * 3 + 0] = v0;
                    red[i * 3 + 1] = v1;
                    red[i * 3 + 2] = v2;
                    red[192 + i] = u;
                }
            }
    }
    __syncthreads();
    // CTA partial of everything but W2: sum the four warps in order
    float *out = a.partial + (long long)blockIdx.x * NET_PARTIAL;
    for (int k = tid; k < 192 + 64 + 64 + 64 + 2; k += NET_TILE) {
        const float v = S.red[0][k] + S.red[1][k] + S.red[2][k] + S.red[3][k];
        int dst;
        if (k < 192) dst = OFF_W1 + k;
        else if (k < 256) dst = OFF_B1 + (k - 192);
        else if (k < 320) dst = OFF_B2 + (k - 256);
        else if (k < 384) dst = OFF_W3 + (k - 320);
        else if (k == 384) dst = OFF_B3;
        else dst = NET_PARAMS;  // loss
        out[dst] = v;
    }
}

// Sum the CTA partials in order; optionally take one Adam step (Kingma & Ba) and
// refresh the BF16 copies of W2.  One thread per parameter (+1 for the loss).
__global__ void k_net_reduce(const float *partial, int nblocks, float *grad, float *P, float *m, float *v,
                             __nv_bfloat16 *W2b, __nv_bfloat16 *W2tb, float lr, float bc1, float bc2, int adam,
                             float *loss_acc, float loss_scale)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > NET_PARAMS) return;
    float s = 0.0f;
    for (int b = 0; b < nblocks; ++b) s += partial[(long long)b * NET_PARTIAL + k];
    if (k == NET_PARAMS) {
        if (loss_acc) *loss_acc += s * loss_scale;
        return;
    }
    if (grad) grad[k] = s;
    if (!adam) return;
    const float mk = 0.9f * m[k] + 0.1f * s;
    const float vk = 0.999f * v[k] + 0.001f * s * s;
    m[k] = mk;
    v[k] = vk;
    const float pk = P[k] - lr * (mk / bc1) / (sqrtf(vk / bc2) + 1e-8f);
    P[k] = pk;
    if (k >= OFF_W2 && k < OFF_W2 + 4096) {
        const int j = (k - OFF_W2) / 64, i = (k - OFF_W2) % 64;
        W2b[j * 64 + i] = __float2bfloat16_rn(pk);
        W2tb[i * 64 + j] = __float2bfloat16_rn(pk);
    }
}

__global__ void k_net_bf16(const float *P, __nv_bfloat16 *W2b, __nv_bfloat16 *W2tb)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 4096) return;
    const int j = k / 64, i = k % 64;
    W2b[j * 64 + i] = __float2bfloat16_rn(P[OFF_W2 + k]);
    W2tb[i * 64 + j] = __float2bfloat16_rn(P[OFF_W2 + k]);
}

// The shared-memory image of the weights for in-kernel inference (NetWeightsSmem)
// from the FP32 parameters: W2 in BF16 with padded rows; W1, b1, W2, b2 halved.
__global__ void k_net_image(const float *P, NetWeightsSmem *img)
{
    for (int k = threadIdx.x; k < 64 * NET_W2_LD; k += blockDim.x) {
        const int j = k / NET_W2_LD, i = k % NET_W2_LD;
        img->W2h[j][i] = __float2bfloat16_rn(i < 64 ? 0.5f * P[OFF_W2 + j * 64 + i] : 0.0f);
    }
    for (int j = threadIdx.x; j < 64; j += blockDim.x) {
        img->W1b1h[j] = make_float4(__uint_as_float(to_tf32(0.5f * P[OFF_W1 + 3 * j])),
                                    __uint_as_float(to_tf32(0.5f * P[OFF_W1 + 3 * j + 1])),
                                    __uint_as_float(to_tf32(0.5f * P[OFF_W1 + 3 * j + 2])),
                                    __uint_as_float(to_tf32(0.5f * P[OFF_B1 + j])));
        img->b2h[j] = 0.5f * P[OFF_B2 + j];
        img->W3[j] = P[OFF_W3 + j];
    }
    if (threadIdx.x == 0) {
        img->b3 = P[OFF_B3];
        img->pad[0] = img->pad[1] = img->pad[2] = 0.0f;
    }
}

}  // namespace dg

// ---------------------------------------------------------------------------

struct dg_c2p_net {
    int device;
    float *P, *m, *v, *grad, *partial;
    __nv_bfloat16 *W2b, *W2tb;
    dg::NetWeightsSmem *img;  // weights for in-kernel inference
    long long partial_blocks;
    long long step;
    float sc[6];
};

namespace {

cudaError_t net_smem_attr(size_t bytes)
{
    cudaError_t e = cudaFuncSetAttribute(dg::k_net_tile<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(dg::k_net_tile<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

namespace dg {

dg_status set_error(dg_status st, const char *msg);

cudaError_t net_launch_tile(dg_c2p_net *n, bool train, const double *cons, const double *p, double *guess,
                            long long count, long long first, long long nsamp, float gamma, cudaStream_t s)
{
    NetTileArgs a;
    std::memset(&a, 0, sizeof(a));
    a.P = n->P;
    a.W2b = n->W2b;
    a.W2tb = n->W2tb;
    a.cons = cons;
    a.p = p;
    a.guess = guess;
    a.partial = n->partial;
    a.count = count;
    a.first = first;
    a.nsamp = nsamp;
    a.inv_batch = 1.0f / (float)nsamp;
    a.gamma = gamma;
    for (int i = 0; i < 6; ++i) a.sc[i] = n->sc[i];
    const unsigned grid = (unsigned)((nsamp + NET_TILE - 1) / NET_TILE);
    const size_t smem = train ? sizeof(NetSmem) : sizeof(NetSmemFwd);
    cudaError_t e = net_smem_attr(sizeof(NetSmem));
    if (e != cudaSuccess) return e;
    if (train) k_net_tile<true><<<grid, NET_TILE, smem, s>>>(a);
    else k_net_tile<false><<<grid, NET_TILE, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace dg

namespace dg {

void net_device_view(const dg_c2p_net *n, const void **img, float sc[6])
{
    *img = n->img;
    for (int i = 0; i < 6; ++i) sc[i] = n->sc[i];
}

}  // namespace dg

using namespace dg;

#define NET_CUDA(expr)                                                                                   \
    do {                                                                                                 \
        cudaError_t e_ = (expr);                                                                         \
        if (e_ != cudaSuccess) return set_error(DG_ERR_CUDA, cudaGetErrorString(e_));                    \
    } while (0)

extern "C" {

dg_status dg_c2p_net_create(const float *params, const double *scales, dg_c2p_net **out)
{
    if (!params || !scales || !out) return set_error(DG_ERR_ARG, "params, scales and out must not be NULL");
    *out = nullptr;
    if (!(scales[1] > scales[0]) || !(scales[3] > scales[2]) || !(scales[5] != 0.0))
        return set_error(DG_ERR_ARG, "invalid feature scales");
    dg_c2p_net *n = new dg_c2p_net;
    std::memset(n, 0, sizeof(*n));
    cudaGetDevice(&n->device);
    for (int i = 0; i < 6; ++i) n->sc[i] = (float)scales[i];
    cudaError_t e = cudaSuccess;
    e = e ? e : cudaMalloc(&n->P, sizeof(float) * NET_PARAMS);
    e = e ? e : cudaMalloc(&n->m, sizeof(float) * NET_PARAMS);
    e = e ? e : cudaMalloc(&n->v, sizeof(float) * NET_PARAMS);
    e = e ? e : cudaMalloc(&n->grad, sizeof(float) * NET_PARAMS);
    e = e ? e : cudaMalloc(&n->W2b, sizeof(__nv_bfloat16) * 4096);
    e = e ? e : cudaMalloc(&n->W2tb, sizeof(__nv_bfloat16) * 4096);
    e = e ? e : cudaMalloc(&n->img, sizeof(NetWeightsSmem));
    if (e == cudaSuccess) e = cudaMemcpy(n->P, params, sizeof(float) * NET_PARAMS, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(n->m, 0, sizeof(float) * NET_PARAMS);
    if (e == cudaSuccess) e = cudaMemset(n->v, 0, sizeof(float) * NET_PARAMS);
    if (e == cudaSuccess) {
        k_net_bf16<<<16, 256>>>(n->P, n->W2b, n->W2tb);
        k_net_image<<<1, 256>>>(n->P, n->img);
        e = cudaDeviceSynchronize();
    }
    if (e != cudaSuccess) {
        dg_c2p_net_destroy(n);
        return set_error(e == cudaErrorMemoryAllocation ? DG_ERR_NOMEM : DG_ERR_CUDA, cudaGetErrorString(e));
    }
    *out = n;
    return DG_OK;
}

void dg_c2p_net_destroy(dg_c2p_net *n)
{
    if (!n) return;
    cudaDeviceSynchronize();
    cudaFree(n->P);
    cudaFree(n->m);
    cudaFree(n->v);
    cudaFree(n->grad);
    cudaFree(n->partial);
    cudaFree(n->W2b);
    cudaFree(n->W2tb);
    cudaFree(n->img);
    delete n;
}

dg_status dg_c2p_net_get_params(const dg_c2p_net *n, float *params)
{
    if (!n || !params) return set_error(DG_ERR_ARG, "net and params must not be NULL");
    NET_CUDA(cudaDeviceSynchronize());
    NET_CUDA(cudaMemcpy(params, n->P, sizeof(float) * NET_PARAMS, cudaMemcpyDeviceToHost));
    return DG_OK;
}

dg_status dg_c2p_net_guess(dg_c2p_net *n, long long count, double gamma, const double *cons, double *p_guess,
                           void *stream)
{
    if (!n || count < 0) return set_error(DG_ERR_ARG, "net must not be NULL and count >= 0");
    if (count == 0) return DG_OK;
    if (!cons || !p_guess) return set_error(DG_ERR_ARG, "cons and p_guess must not be NULL");
    NET_CUDA(net_launch_tile(n, false, cons, nullptr, p_guess, count, 0, count, (float)gamma, (cudaStream_t)stream));
    return DG_OK;
}

static dg_status ensure_partial(dg_c2p_net *n, long long blocks)
{
    if (blocks <= n->partial_blocks) return DG_OK;
    cudaFree(n->partial);
    n->partial = nullptr;
    NET_CUDA(cudaMalloc(&n->partial, sizeof(float) * NET_PARTIAL * blocks));
    n->partial_blocks = blocks;
    return DG_OK;
}

dg_status dg_c2p_net_grad(dg_c2p_net *n, long long count, const double *cons, const double *p, float *grad,
                          float *loss, void *stream)
{
    if (!n || count <= 0 || !cons || !p || !grad || !loss)
        return set_error(DG_ERR_ARG, "net, cons, p, grad, loss must not be NULL and count > 0");
    const long long blocks = (count + NET_TILE - 1) / NET_TILE;
    if (dg_status st = ensure_partial(n, blocks)) return st;
    cudaStream_t s = (cudaStream_t)stream;
    NET_CUDA(cudaMemsetAsync(loss, 0, sizeof(float), s));
    NET_CUDA(net_launch_tile(n, true, cons, p, nullptr, count, 0, count, 0.0f, s));
    k_net_reduce<<<(NET_PARAMS + 256) / 256, 256, 0, s>>>(n->partial, (int)blocks, grad, n->P, n->m, n->v, n->W2b,
                                                           n->W2tb, 0.0f, 1.0f, 1.0f, 0, loss, 1.0f / (float)count);
    NET_CUDA(cudaGetLastError());
    return DG_OK;
}

dg_status dg_c2p_net_train(dg_c2p_net *n, long long count, const double *cons, const double *p, int epochs,
                           int batch, float lr, float *loss_per_epoch, void *stream)
{
    if (!n || count <= 0 || !cons || !p || epochs <= 0 || batch <= 0 || !(lr > 0.0f))
        return set_error(DG_ERR_ARG, "invalid training arguments");
    const long long blocks = ((long long)batch + NET_TILE - 1) / NET_TILE;
    if (dg_status st = ensure_partial(n, blocks)) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const long long nb = (count + batch - 1) / batch;
    if (loss_per_epoch) NET_CUDA(cudaMemsetAsync(loss_per_epoch, 0, sizeof(float) * epochs, s));
    for (int ep = 0; ep < epochs; ++ep) {
        for (long long b = 0; b < nb; ++b) {
            const long long first = b * batch;
            const long long ns = (first + batch <= count) ? batch : count - first;
            NET_CUDA(net_launch_tile(n, true, cons, p, nullptr, count, first, ns, 0.0f, s));
            n->step += 1;
            const float bc1 = 1.0f - powf(0.9f, (float)n->step);
            const float bc2 = 1.0f - powf(0.999f, (float)n->step);
            const int nblk = (int)((ns + NET_TILE - 1) / NET_TILE);
            k_net_reduce<<<(NET_PARAMS + 256) / 256, 256, 0, s>>>(
                n->partial, nblk, nullptr, n->P, n->m, n->v, n->W2b, n->W2tb, lr, bc1, bc2, 1,
                loss_per_epoch ? loss_per_epoch + ep : nullptr, 1.0f / (float)count);
            NET_CUDA(cudaGetLastError());
        }
    }
    k_net_image<<<1, 256, 0, s>>>(n->P, n->img);
    NET_CUDA(cudaGetLastError());
    return DG_OK;
}

}  // extern "C"
