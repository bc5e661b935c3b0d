// Transport-data surrogate: a 2 -> 128 -> 128 -> 6 network with tanh hidden
// units (the flux transport data of Sec. 2.2.4 as a function of log10 E/N and
// the O2 fraction), trained by full-batch Adam (Kingma & Ba 2015) on swarm
// results and evaluated on query points.
//
// The 128 x 128 layer is the only dense contraction: its forward product,
// the backpropagated product and the weight gradient run on the tensor cores
// in BF16 with FP32 accumulation (mma.sync m16n8k16).  The 2 -> 128 and
// 128 -> 6 layers, tanh, the loss and Adam run in FP32 on the CUDA cores.
// Reductions over points are per-block partial sums added in a fixed order
// (deterministic).
//
// Parameters (float32, one vector): W1[128][2], b1[128], W2[128][128], b2[128],
// W3[6][128], b3[6]; W[o][i] multiplies input i of unit o.
#include <cuda_bf16.h>
#include <stdint.h>

#include "common.cuh"
#include "../../include/picmcc.h"

namespace mlp {

using pic::kFull;

constexpr int NI = MLP_NI, NH = MLP_NH, NO = MLP_NO;
constexpr int OFF_W1 = 0, OFF_B1 = NH * NI, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH, OFF_W3 = OFF_B2 + NH,
              OFF_B3 = OFF_W3 + NO * NH, NP = OFF_B3 + NO;
static_assert(NP == MLP_NPARAMS, "parameter count");

__device__ __forceinline__ float tanh_fast(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

// D = A B + C for one 16 x 8 x 16 tile (A row-major, B column-major, BF16
// inputs, FP32 accumulate).  Fragments: with g = lane / 4, t = lane % 4,
// a0 = A[g][2t, 2t+1], a1 = A[g+8][2t, 2t+1], a2 = A[g][2t+8, 2t+9],
// a3 = A[g+8][2t+8, 2t+9]; b0 = B[2t, 2t+1][g], b1 = B[2t+8, 2t+9][g];
// c0, c1 = C[g][2t, 2t+1], c2, c3 = C[g+8][2t, 2t+1].
__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// ------------------------------------------------------------------ GEMM
// C_part[z] = A[M][K-slice z] B[N][K-slice z]^T (both operands K-contiguous
// BF16), FP32 out.  CTA tile 64 x 64, four warps of 32 x 32, K staged in
// chunks of 32.  M, N multiples of 64; K a multiple of 32 * splits.
constexpr int GT = 64, GK = 32, GPAD = 8;
__global__ void __launch_bounds__(128) k_gemm_nt(const __nv_bfloat16* __restrict__ A,
                                                 const __nv_bfloat16* __restrict__ B, float* __restrict__ C, int M,
                                                 int N, int K, int k_per_split) {
    __shared__ __align__(16) __nv_bfloat16 As[GT][GK + GPAD];
    __shared__ __align__(16) __nv_bfloat16 Bs[GT][GK + GPAD];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT, kz0 = blockIdx.z * k_per_split;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    float acc[2][4][4] = {};
    for (int k0 = kz0; k0 < kz0 + k_per_split; k0 += GK) {
        // 64 rows x 32 bf16 = 256 chunks of 16 B per operand: two per thread
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int q = tid + u * 128, r = q >> 2, c8 = (q & 3) * 8;
            *reinterpret_cast<uint4*>(&As[r][c8]) =
                *reinterpret_cast<const uint4*>(A + (size_t)(m0 + r) * K + k0 + c8);
            *reinterpret_cast<uint4*>(&Bs[r][c8]) =
                *reinterpret_cast<const uint4*>(B + (size_t)(n0 + r) * K + k0 + c8);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; kk += 16) {
            uint32_t a[2][4], b[4][2];
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                const int r = wm + mi * 16 + g;
                a[mi][0] = *reinterpret_cast<const uint32_t*>(&As[r][kk + 2 * t]);
                a[mi][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][kk + 2 * t]);
                a[mi][2] = *reinterpret_cast<const uint32_t*>(&As[r][kk + 2 * t + 8]);
                a[mi][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][kk + 2 * t + 8]);
            }
#pragma unroll
            for (int ni = 0; ni < 4; ++ni) {
                const int r = wn + ni * 8 + g;
                b[ni][0] = *reinterpret_cast<const uint32_t*>(&Bs[r][kk + 2 * t]);
                b[ni][1] = *reinterpret_cast<const uint32_t*>(&Bs[r][kk + 2 * t + 8]);
            }
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni)
                    mma_bf16(acc[mi][ni], a[mi][0], a[mi][1], a[mi][2], a[mi][3], b[ni][0], b[ni][1]);
        }
        __syncthreads();
    }
    float* Cz = C + (size_t)blockIdx.z * M * N;
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) {
            const int r = m0 + wm + mi * 16 + g, c = n0 + wn + ni * 8 + 2 * t;
            *reinterpret_cast<float2*>(Cz + (size_t)r * N + c) = make_float2(acc[mi][ni][0], acc[mi][ni][1]);
            *reinterpret_cast<float2*>(Cz + (size_t)(r + 8) * N + c) = make_float2(acc[mi][ni][2], acc[mi][ni][3]);
        }
}

// ------------------------------------------------------------------ training kernels
// BF16 copies of W2 ([o][i] and its transpose [i][o]).
__global__ void k_prep(const float* __restrict__ th, __nv_bfloat16* __restrict__ w2b, __nv_bfloat16* __restrict__ w2t) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < NH * NH) {
        const int o = k / NH, i = k % NH;
        const __nv_bfloat16 v = __float2bfloat16_rn(th[OFF_W2 + k]);
        w2b[k] = v;
        w2t[i * NH + o] = v;
    }
}

// h1 = tanh(W1 x + b1): FP32 [n][128], BF16 [n][128] and BF16 transposed [128][n].
__global__ void k_layer1(const float* __restrict__ th, const float* __restrict__ x, int n, float* __restrict__ h1,
                         __nv_bfloat16* __restrict__ h1b, __nv_bfloat16* __restrict__ h1t) {
    const int p = blockIdx.x, u = threadIdx.x;
    if (p >= n) return;
    const float z = fmaf(th[OFF_W1 + u * NI + 1], x[p * NI + 1], fmaf(th[OFF_W1 + u * NI], x[p * NI], th[OFF_B1 + u]));
    const float h = tanh_fast(z);
    h1[(size_t)p * NH + u] = h;
    const __nv_bfloat16 hb = __float2bfloat16_rn(h);
    h1b[(size_t)p * NH + u] = hb;
    h1t[(size_t)u * n + p] = hb;
}

// Output layer, loss and the first backward steps.  One warp per point (lane
// l holds hidden units l, l+32, l+64, l+96), kHeadPts points per block.
// Per-block partial sums: gW3[6][128], gb3[6], gb2[128], loss.
constexpr int kHeadWarps = 8, kHeadPts = 64, kHeadPart = NO * NH + NO + NH + 1;
__global__ void __launch_bounds__(kHeadWarps * 32) k_head(const float* __restrict__ th, const float* __restrict__ z2,
                                                          const float* __restrict__ tgt, int n, float inv6n,
                                                          __nv_bfloat16* __restrict__ dz2b,
                                                          __nv_bfloat16* __restrict__ dz2t, float* __restrict__ part) {
    __shared__ float sW3[NO * NH], sgW3[kHeadWarps][NO * NH], sgb2[kHeadWarps][NH], sgb3[kHeadWarps][NO],
        sloss[kHeadWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < NO * NH; k += blockDim.x) sW3[k] = th[OFF_W3 + k];
    for (int k = lane; k < NO * NH; k += 32) sgW3[warp][k] = 0.0f;
    for (int k = lane; k < NH; k += 32) sgb2[warp][k] = 0.0f;
    if (lane < NO) sgb3[warp][lane] = 0.0f;
    if (lane == 0) sloss[warp] = 0.0f;
    __syncthreads();
    float b2[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) b2[q] = th[OFF_B2 + lane + 32 * q];
    for (int pp = warp; pp < kHeadPts; pp += kHeadWarps) {
        const int p = blockIdx.x * kHeadPts + pp;
        if (p >= n) break;
        float h2[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) h2[q] = tanh_fast(z2[(size_t)p * NH + lane + 32 * q] + b2[q]);
        float dy[NO];
        float lsum = 0.0f;
#pragma unroll
        for (int o = 0; o < NO; ++o) {
            float s = 0.0f;
#pragma unroll
            for (int q = 0; q < 4; ++q) s = fmaf(sW3[o * NH + lane + 32 * q], h2[q], s);
            for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(kFull, s, off);
            const float y = s + th[OFF_B3 + o];
            const float d = y - tgt[(size_t)p * NO + o];
            lsum = fmaf(d, d, lsum);
            dy[o] = 2.0f * d * inv6n;
        }
        if (lane == 0) sloss[warp] += lsum;
        if (lane < NO) {
            float v = 0.0f;
#pragma unroll
            for (int o = 0; o < NO; ++o) v = lane == o ? dy[o] : v;
            sgb3[warp][lane] += v;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int u = lane + 32 * q;
            float dh = 0.0f;
#pragma unroll
            for (int o = 0; o < NO; ++o) {
                sgW3[warp][o * NH + u] += dy[o] * h2[q];
                dh = fmaf(sW3[o * NH + u], dy[o], dh);
            }
            const float dz = dh * (1.0f - h2[q] * h2[q]);
            sgb2[warp][u] += dz;
            const __nv_bfloat16 db = __float2bfloat16_rn(dz);
            dz2b[(size_t)p * NH + u] = db;
            dz2t[(size_t)u * n + p] = db;
        }
    }
    __syncthreads();
    float* out = part + (size_t)blockIdx.x * kHeadPart;
    for (int k = threadIdx.x; k < kHeadPart; k += blockDim.x) {
        float s = 0.0f;
        for (int w = 0; w < kHeadWarps; ++w) {
            if (k < NO * NH) s += sgW3[w][k];
            else if (k < NO * NH + NO) s += sgb3[w][k - NO * NH];
            else if (k < NO * NH + NO + NH) s += sgb2[w][k - NO * NH - NO];
            else s += sloss[w];
        }
        out[k] = s;
    }
}

// dz1 = dh1 (1 - h1^2); per-block partials of gW1[128][2] and gb1[128] over
// kL1Pts points (thread = hidden unit).
constexpr int kL1Pts = 64, kL1Part = NH * NI + NH;
__global__ void __launch_bounds__(NH) k_layer1_back(const float* __restrict__ dh1, const float* __restrict__ h1,
                                                    const float* __restrict__ x, int n, float* __restrict__ part) {
    const int u = threadIdx.x;
    float g0 = 0.0f, g1 = 0.0f, gb = 0.0f;
    for (int pp = 0; pp < kL1Pts; ++pp) {
        const int p = blockIdx.x * kL1Pts + pp;
        if (p >= n) break;
        const float h = h1[(size_t)p * NH + u];
        const float dz = dh1[(size_t)p * NH + u] * (1.0f - h * h);
        g0 = fmaf(dz, x[p * NI], g0);
        g1 = fmaf(dz, x[p * NI + 1], g1);
        gb += dz;
    }
    float* out = part + (size_t)blockIdx.x * kL1Part;
    out[u * NI] = g0;
    out[u * NI + 1] = g1;
    out[NH * NI + u] = gb;
}

struct Parts {
    const float* gw2;   // [splits][128][128]
    const float* head;  // [n_head][kHeadPart]
    const float* l1;    // [n_l1][kL1Part]
    int splits, n_head, n_l1;
};

// Gradient of parameter k from the partial sums, added in a fixed order.
__device__ float grad_of(const Parts& P, int k) {
    float s = 0.0f;
    if (k < OFF_W2) {
        const int j = k;  // W1 then b1: same order as the l1 partial layout
        for (int b = 0; b < P.n_l1; ++b) s += P.l1[(size_t)b * kL1Part + j];
    } else if (k < OFF_B2) {
        for (int z = 0; z < P.splits; ++z) s += P.gw2[(size_t)z * NH * NH + (k - OFF_W2)];
    } else {
        int j;
        if (k < OFF_W3) j = NO * NH + NO + (k - OFF_B2);        // b2
        else if (k < OFF_B3) j = k - OFF_W3;                      // W3
        else j = NO * NH + (k - OFF_B3);                          // b3
        for (int b = 0; b < P.n_head; ++b) s += P.head[(size_t)b * kHeadPart + j];
    }
    return s;
}

__global__ void k_grad_out(Parts P, float* __restrict__ grad, float* __restrict__ loss, float inv6n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < NP) grad[k] = grad_of(P, k);
    if (k == 0 && loss) {
        float s = 0.0f;
        for (int b = 0; b < P.n_head; ++b) s += P.head[(size_t)b * kHeadPart + kHeadPart - 1];
        *loss = s * inv6n;
    }
}

// Adam (Kingma & Ba 2015, Algorithm 1) on every parameter, then the BF16
// copies of W2 for the next step.  step_dev holds the step count (t >= 1
// after the increment here, done by thread 0 of block 0 at the end).
__global__ void k_adam(Parts P, float* __restrict__ th, float* __restrict__ m, float* __restrict__ v,
                       int* __restrict__ step_dev, float lr, float beta1, float beta2, float eps,
                       __nv_bfloat16* __restrict__ w2b, __nv_bfloat16* __restrict__ w2t, float* __restrict__ loss,
                       float inv6n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int step = *step_dev + 1;
    if (k < NP) {
        const float gk = grad_of(P, k);
        const float mk = beta1 * m[k] + (1.0f - beta1) * gk;
        const float vk = beta2 * v[k] + (1.0f - beta2) * gk * gk;
        m[k] = mk;
        v[k] = vk;
        const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
        const float nt = th[k] - lr * (mk / c1) / (sqrtf(vk / c2) + eps);
        th[k] = nt;
        if (k >= OFF_W2 && k < OFF_B2) {
            const int o = (k - OFF_W2) / NH, i = (k - OFF_W2) % NH;
            const __nv_bfloat16 b = __float2bfloat16_rn(nt);
            w2b[o * NH + i] = b;
            w2t[i * NH + o] = b;
        }
    }
    if (k == 0 && loss) {
        float s = 0.0f;
        for (int b = 0; b < P.n_head; ++b) s += P.head[(size_t)b * kHeadPart + kHeadPart - 1];
        *loss = s * inv6n;
    }
}

__global__ void k_step_inc(int* step_dev) { *step_dev += 1; }

// ------------------------------------------------------------------ inference
// Fused forward pass.  Four warps per block; each warp takes 16 points at a
// time: layer 1 on the CUDA cores into a BF16 tile in shared memory, the
// 128 x 128 layer by mma.sync against W2 (BF16, resident in shared memory),
// tanh and the 128 -> 6 layer in the accumulator registers, reduced over the
// four lanes that share a row.
constexpr int kInfWarps = 4, kRowPad = NH + 8;
struct InfSmem {
    __nv_bfloat16 w2[NH][kRowPad];
    __nv_bfloat16 h1[kInfWarps][16][kRowPad];
    float w1[NH * NI], b1[NH], b2[NH], w3[NO * NH], b3[NO];
};

__global__ void __launch_bounds__(kInfWarps * 32) k_infer(const float* __restrict__ th,
                                                          const __nv_bfloat16* __restrict__ w2b,
                                                          const float* __restrict__ x, float* __restrict__ y,
                                                          long long n) {
    extern __shared__ __align__(16) unsigned char inf_raw[];
    InfSmem& S = *reinterpret_cast<InfSmem*>(inf_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    for (int k = tid; k < NH * NH / 2; k += blockDim.x) {
        const int o = (2 * k) / NH, i = (2 * k) % NH;
        *reinterpret_cast<uint32_t*>(&S.w2[o][i]) = reinterpret_cast<const uint32_t*>(w2b)[k];
    }
    for (int k = tid; k < NH * NI; k += blockDim.x) S.w1[k] = th[OFF_W1 + k];
    for (int k = tid; k < NH; k += blockDim.x) {
        S.b1[k] = th[OFF_B1 + k];
        S.b2[k] = th[OFF_B2 + k];
    }
    for (int k = tid; k < NO * NH; k += blockDim.x) S.w3[k] = th[OFF_W3 + k];
    if (tid < NO) S.b3[tid] = th[OFF_B3 + tid];
    __syncthreads();
    const long long n_tiles = (n + 15) / 16;
    for (long long tile = (long long)blockIdx.x * kInfWarps + warp; tile < n_tiles;
         tile += (long long)gridDim.x * kInfWarps) {
        const long long p0 = tile * 16;
        // inputs of the 16 points (lanes 0..15 load, everyone reads by shuffle)
        float x0 = 0.0f, x1 = 0.0f;
        if (lane < 16 && p0 + lane < n) {
            x0 = x[(p0 + lane) * NI];
            x1 = x[(p0 + lane) * NI + 1];
        }
        // layer 1: lane covers units lane + 32 q for all 16 points
#pragma unroll 4
        for (int r = 0; r < 16; ++r) {
            const float a0 = __shfl_sync(kFull, x0, r), a1 = __shfl_sync(kFull, x1, r);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int u = lane + 32 * q;
                const float z = fmaf(S.w1[u * NI + 1], a1, fmaf(S.w1[u * NI], a0, S.b1[u]));
                S.h1[warp][r][u] = __float2bfloat16_rn(tanh_fast(z));
            }
        }
        __syncwarp();
        // layer 2 on the tensor cores: acc[nt] covers output units 8 nt .. 8 nt + 7
        float acc[NH / 8][4];
#pragma unroll
        for (int nt = 0; nt < NH / 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.0f;
#pragma unroll
        for (int kk = 0; kk < NH; kk += 16) {
            const uint32_t a0 = *reinterpret_cast<const uint32_t*>(&S.h1[warp][g][kk + 2 * t]);
            const uint32_t a1 = *reinterpret_cast<const uint32_t*>(&S.h1[warp][g + 8][kk + 2 * t]);
            const uint32_t a2 = *reinterpret_cast<const uint32_t*>(&S.h1[warp][g][kk + 2 * t + 8]);
            const uint32_t a3 = *reinterpret_cast<const uint32_t*>(&S.h1[warp][g + 8][kk + 2 * t + 8]);
#pragma unroll
            for (int nt = 0; nt < NH / 8; ++nt) {
                const uint32_t b0 = *reinterpret_cast<const uint32_t*>(&S.w2[nt * 8 + g][kk + 2 * t]);
                const uint32_t b1 = *reinterpret_cast<const uint32_t*>(&S.w2[nt * 8 + g][kk + 2 * t + 8]);
                mma_bf16(acc[nt], a0, a1, a2, a3, b0, b1);
            }
        }
        __syncwarp();
        // tanh and the output layer for rows g and g + 8
        float ya[NO], yb[NO];
#pragma unroll
        for (int o = 0; o < NO; ++o) ya[o] = yb[o] = 0.0f;
#pragma unroll
        for (int nt = 0; nt < NH / 8; ++nt) {
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int u = nt * 8 + 2 * t + e;
                const float ha = tanh_fast(acc[nt][e] + S.b2[u]);
                const float hb = tanh_fast(acc[nt][2 + e] + S.b2[u]);
#pragma unroll
                for (int o = 0; o < NO; ++o) {
                    ya[o] = fmaf(S.w3[o * NH + u], ha, ya[o]);
                    yb[o] = fmaf(S.w3[o * NH + u], hb, yb[o]);
                }
            }
        }
#pragma unroll
        for (int o = 0; o < NO; ++o) {
            ya[o] += __shfl_xor_sync(kFull, ya[o], 1);
            ya[o] += __shfl_xor_sync(kFull, ya[o], 2);
            yb[o] += __shfl_xor_sync(kFull, yb[o], 1);
            yb[o] += __shfl_xor_sync(kFull, yb[o], 2);
        }
        if (t == 0) {
            const long long pa = p0 + g, pb = p0 + g + 8;
            if (pa < n)
#pragma unroll
                for (int o = 0; o < NO; ++o) y[pa * NO + o] = ya[o] + S.b3[o];
            if (pb < n)
#pragma unroll
                for (int o = 0; o < NO; ++o) y[pb * NO + o] = yb[o] + S.b3[o];
        }
    }
}

}  // namespace mlp

// ------------------------------------------------------------------ C ABI
using namespace mlp;

namespace {

size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

struct TrainWs {
    __nv_bfloat16 *w2b, *w2t, *h1b, *h1t, *dz2b, *dz2t;
    float *h1, *z2, *dh1, *gw2, *head, *l1, *loss;
    int* step;
    int splits, n_head, n_l1;
};

// Layout of the workspace for n points (base null: sizes only).
size_t carve(void* base, int n, TrainWs* w) {
    uintptr_t p = (uintptr_t)base;
    const uintptr_t p0 = p;
    auto take = [&](size_t b) {
        void* r = (void*)p;
        p += al256(b);
        return r;
    };
    const size_t nh = (size_t)n * NH;
    w->splits = n >= 256 ? n / 256 : 1;
    w->n_head = (n + kHeadPts - 1) / kHeadPts;
    w->n_l1 = (n + kL1Pts - 1) / kL1Pts;
    w->w2b = (__nv_bfloat16*)take(NH * NH * 2);
    w->w2t = (__nv_bfloat16*)take(NH * NH * 2);
    w->h1 = (float*)take(nh * 4);
    w->h1b = (__nv_bfloat16*)take(nh * 2);
    w->h1t = (__nv_bfloat16*)take(nh * 2);
    w->z2 = (float*)take(nh * 4);
    w->dz2b = (__nv_bfloat16*)take(nh * 2);
    w->dz2t = (__nv_bfloat16*)take(nh * 2);
    w->dh1 = (float*)take(nh * 4);
    w->gw2 = (float*)take((size_t)w->splits * NH * NH * 4);
    w->head = (float*)take((size_t)w->n_head * kHeadPart * 4);
    w->l1 = (float*)take((size_t)w->n_l1 * kL1Part * 4);
    w->loss = (float*)take(64);
    w->step = (int*)take(64);
    return (size_t)(p - p0);
}

Parts parts_of(const TrainWs& w) {
    Parts P;
    P.gw2 = w.gw2;
    P.head = w.head;
    P.l1 = w.l1;
    P.splits = w.splits;
    P.n_head = w.n_head;
    P.n_l1 = w.n_l1;
    return P;
}

// Forward and backward over the batch: leaves the partial sums in the workspace.
void backprop(const float* th, const float* x, const float* t, int n, const TrainWs& w, cudaStream_t s) {
    const float inv6n = 1.0f / (6.0f * (float)n);
    k_layer1<<<n, NH, 0, s>>>(th, x, n, w.h1, w.h1b, w.h1t);
    k_gemm_nt<<<dim3(NH / GT, n / GT, 1), 128, 0, s>>>(w.h1b, w.w2b, w.z2, n, NH, NH, NH);
    k_head<<<w.n_head, kHeadWarps * 32, 0, s>>>(th, w.z2, t, n, inv6n, w.dz2b, w.dz2t, w.head);
    k_gemm_nt<<<dim3(NH / GT, n / GT, 1), 128, 0, s>>>(w.dz2b, w.w2t, w.dh1, n, NH, NH, NH);
    k_layer1_back<<<w.n_l1, NH, 0, s>>>(w.dh1, w.h1, x, n, w.l1);
    k_gemm_nt<<<dim3(NH / GT, NH / GT, w.splits), 128, 0, s>>>(w.dz2t, w.h1t, w.gw2, NH, NH, n, n / w.splits);
}

bool train_size_ok(int n) { return n >= 64 && n % 64 == 0 && (n < 256 || n % 256 == 0); }

}  // namespace

extern "C" size_t mlp_workspace_bytes(int n_max) {
    if (n_max < 0 || (n_max > 0 && !train_size_ok(n_max))) return 0;
    TrainWs w;
    return carve(nullptr, n_max > 0 ? n_max : 64, &w);
}

extern "C" int mlp_forward(const float* params, const float* x, float* y, long long n, void* ws, size_t ws_bytes,
                           pic_stream_t stream) {
    if (!params || !x || !y || n < 0 || !ws || ((uintptr_t)ws & 255) || ws_bytes < mlp_workspace_bytes(0))
        return PIC_ERR_ARG;
    if (n == 0) return PIC_OK;
    cudaStream_t s = (cudaStream_t)stream;
    TrainWs w;
    carve(ws, 64, &w);
    k_prep<<<(NH * NH + 255) / 256, 256, 0, s>>>(params, w.w2b, w.w2t);
    static bool attr = false;
    const int smem = (int)sizeof(InfSmem);
    if (!attr) {
        if (cudaFuncSetAttribute(k_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
            return PIC_ERR_CUDA;
        attr = true;
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_infer, kInfWarps * 32, smem);
    const long long tiles = (n + 15) / 16;
    long long blocks = (long long)sms * (per_sm > 0 ? per_sm : 1);
    if (blocks * kInfWarps > tiles) blocks = (tiles + kInfWarps - 1) / kInfWarps;
    k_infer<<<(unsigned)blocks, kInfWarps * 32, smem, s>>>(params, w.w2b, x, y, n);
    return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ERR_CUDA;
}

extern "C" int mlp_loss_grad(const float* params, const float* x, const float* t, int n, float* grad, float* loss,
                             void* ws, size_t ws_bytes, pic_stream_t stream) {
    if (!params || !x || !t || !grad || !ws || ((uintptr_t)ws & 255) || !train_size_ok(n) ||
        ws_bytes < mlp_workspace_bytes(n))
        return PIC_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    TrainWs w;
    carve(ws, n, &w);
    k_prep<<<(NH * NH + 255) / 256, 256, 0, s>>>(params, w.w2b, w.w2t);
    backprop(params, x, t, n, w, s);
    k_grad_out<<<(NP + 255) / 256, 256, 0, s>>>(parts_of(w), grad, loss, 1.0f / (6.0f * (float)n));
    return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ERR_CUDA;
}

extern "C" int mlp_train(float* params, float* m, float* v, int step0, const float* x, const float* t, int n,
                         int n_steps, float lr, float beta1, float beta2, float eps, float* loss, void* ws,
                         size_t ws_bytes, pic_stream_t stream) {
    if (!params || !m || !v || !x || !t || !ws || ((uintptr_t)ws & 255) || !train_size_ok(n) || n_steps < 0 ||
        step0 < 0 || !(lr > 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0) ||
        ws_bytes < mlp_workspace_bytes(n))
        return PIC_ERR_ARG;
    if (n_steps == 0) return PIC_OK;
    cudaStream_t s = (cudaStream_t)stream;
    TrainWs w;
    carve(ws, n, &w);
    const float inv6n = 1.0f / (6.0f * (float)n);
    if (cudaMemcpyAsync(w.step, &step0, sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess) return PIC_ERR_CUDA;
    k_prep<<<(NH * NH + 255) / 256, 256, 0, s>>>(params, w.w2b, w.w2t);
    auto one_step = [&](cudaStream_t q) {
        backprop(params, x, t, n, w, q);
        k_adam<<<(NP + 255) / 256, 256, 0, q>>>(parts_of(w), params, m, v, w.step, lr, beta1, beta2, eps, w.w2b,
                                               w.w2t, loss, inv6n);
        k_step_inc<<<1, 1, 0, q>>>(w.step);
    };
    if (n_steps < 8) {
        for (int k = 0; k < n_steps; ++k) one_step(s);
        return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ERR_CUDA;
    }
    // longer runs: one step captured as a graph on a private stream, replayed on s
    cudaStream_t cap = nullptr;
    cudaGraph_t gr = nullptr;
    cudaGraphExec_t ge = nullptr;
    int rc = PIC_OK;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return PIC_ERR_CUDA;
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = PIC_ERR_CUDA;
    if (rc == PIC_OK) {
        one_step(cap);
        if (cudaStreamEndCapture(cap, &gr) != cudaSuccess) rc = PIC_ERR_CUDA;
    }
    if (rc == PIC_OK && cudaGraphInstantiate(&ge, gr, 0) != cudaSuccess) rc = PIC_ERR_CUDA;
    for (int k = 0; rc == PIC_OK && k < n_steps; ++k)
        if (cudaGraphLaunch(ge, s) != cudaSuccess) rc = PIC_ERR_CUDA;
    if (ge) cudaGraphExecDestroy(ge);
    if (gr) cudaGraphDestroy(gr);
    cudaStreamDestroy(cap);
    if (rc == PIC_OK && cudaGetLastError() != cudaSuccess) rc = PIC_ERR_CUDA;
    return rc;
}
