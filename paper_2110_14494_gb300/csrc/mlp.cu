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
#include <math.h>
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
    // training batches are multiples of kHeadPts (train_size_ok): every point
    // of the block exists; the next point's z2 row is loaded ahead
    float zn[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) zn[q] = z2[(size_t)(blockIdx.x * kHeadPts + warp) * NH + lane + 32 * q];
    for (int pp = warp; pp < kHeadPts; pp += kHeadWarps) {
        const int p = blockIdx.x * kHeadPts + pp;
        float h2[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) h2[q] = tanh_fast(zn[q] + b2[q]);
        if (pp + kHeadWarps < kHeadPts) {
#pragma unroll
            for (int q = 0; q < 4; ++q) zn[q] = z2[(size_t)(p + kHeadWarps) * NH + lane + 32 * q];
        }
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
// kL1Pts points (thread = hidden unit).  Training batches are multiples of
// kL1Pts (train_size_ok), so every block has all of its points; the loop is
// unrolled so that the loads of several points are in flight together (the
// sums still run over the points in order).
constexpr int kL1Pts = 64, kL1Part = NH * NI + NH;
__global__ void __launch_bounds__(NH) k_layer1_back(const float* __restrict__ dh1, const float* __restrict__ h1,
                                                    const float* __restrict__ x, int n, float* __restrict__ part) {
    (void)n;
    const int u = threadIdx.x;
    float g0 = 0.0f, g1 = 0.0f, gb = 0.0f;
#pragma unroll 16
    for (int pp = 0; pp < kL1Pts; ++pp) {
        const int p = blockIdx.x * kL1Pts + pp;
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

// ------------------------------------------------------------------ inference on tcgen05
// Fused forward pass on the fifth-generation tensor cores.  A block of 256
// threads takes 128 points at a time (thread t: point t % 128, hidden units
// 64 (t / 128) .. 64 (t / 128) + 63):
//   1. layer 1 in FP32, tanh in packed BF16, written as the A operand (128
//      points x 128 units) in shared memory;
//   2. one thread issues eight 128 x 128 x 16 MMAs (A: h1, B: W2 resident in
//      shared memory) into a 128-column FP32 accumulator in tensor memory;
//   3. the accumulator rows are read back (row = point = TMEM lane), bias and
//      tanh applied, and h2 written over the A operand;
//   4. eight 128 x 16 x 16 MMAs against W3 (padded to 16 outputs) into the
//      first 16 accumulator columns; the first half of the threads read the
//      six outputs back, add b3 and store.
// Operands use the canonical K-major layout without swizzle: core matrices
// of 8 rows x 16 bytes stored contiguously, the next core matrix along K at
// +128 bytes, the next 8-row group at +2048 bytes (the same strides for the
// 16-row W3 tile, 4 KB).  Every MMA reads at most start + 15 x 2048 + 255
// bytes, inside its 32 KB (4 KB) tile.  Waits on the MMA completion barrier are
// bounded; on expiry the block writes NaN outputs, records the error and
// leaves, releasing its tensor memory.
constexpr int kTcThreads = 256, kTcRows = 128;
constexpr uint32_t kTile = kTcRows * NH * 2;   // one 128 x 128 BF16 operand: 32 KB
constexpr uint32_t kLbo = 128, kSbo = 2048;    // core-matrix strides (bytes) along K and along M/N
constexpr uint32_t kB2Bytes = 16 * NH * 2;     // W3 padded to 16 rows: 4 KB
constexpr long long kWaitLimit = 1ll << 26;

struct TcSmem {
    alignas(1024) unsigned char w2[kTile];   // B of layer 2: row o (output unit), K = input unit
    alignas(1024) unsigned char a[kTile];    // A: row = point, K = unit (h1, then h2)
    alignas(1024) unsigned char w3[kB2Bytes];
    float w1[NH * NI], b1[NH], b2[NH], b3[NO];
    alignas(8) unsigned long long bar;
    uint32_t tmem;
    int abort;
};

// byte offset of element (row r, k) in a K-major no-swizzle operand
__host__ __device__ constexpr uint32_t kmajor_off(uint32_t r, uint32_t k) {
    return (r >> 3) * kSbo + (k >> 3) * kLbo + (r & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading (K) and stride
// (M/N) byte offsets in 16-byte units, the fixed version bits 46-47 = 1,
// no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16
// A and B (bits 7-9 = 1, 10-12 = 1), both K-major, N / 8 in bits 17-22,
// M / 16 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(uint32_t m, uint32_t n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((m >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                 : "memory");
}

// Bounded wait for the barrier phase with the given parity; false on expiry.
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
    for (long long it = 0; it < kWaitLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,"
        "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = __uint_as_float(r[q]);
}

// tanh of two floats as packed BF16 (hardware approximation)
__device__ __forceinline__ uint32_t tanh_bf16x2(float lo, float hi) {
    uint32_t in = pack_bf16(lo, hi), out;
    asm("tanh.approx.bf16x2 %0, %1;" : "=r"(out) : "r"(in));
    return out;
}

__global__ void __launch_bounds__(kTcThreads) k_infer_tc(const float* __restrict__ th,
                                                         const __nv_bfloat16* __restrict__ w2b,
                                                         const float* __restrict__ x, float* __restrict__ y,
                                                         long long n, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    // align the operand tiles to 1024 bytes
    TcSmem& S = *reinterpret_cast<TcSmem*>(tc_raw + ((1024 - (smem_u32(tc_raw) & 1023)) & 1023));
    const int tid = threadIdx.x, warp = tid >> 5;
    const int row = tid & (kTcRows - 1), half = tid >> 7;
    // operands and parameters
    for (int k = tid; k < NH * NH; k += kTcThreads) {
        const int o = k / NH, i = k % NH;
        *reinterpret_cast<__nv_bfloat16*>(S.w2 + kmajor_off(o, i)) = w2b[k];
    }
    for (int k = tid; k < 16 * NH; k += kTcThreads) {
        const int o = k / NH, i = k % NH;
        *reinterpret_cast<__nv_bfloat16*>(S.w3 + kmajor_off(o, i)) =
            __float2bfloat16_rn(o < NO ? th[OFF_W3 + o * NH + i] : 0.0f);
    }
    for (int k = tid; k < NH * NI; k += kTcThreads) S.w1[k] = th[OFF_W1 + k];
    for (int k = tid; k < NH; k += kTcThreads) {
        S.b1[k] = th[OFF_B1 + k];
        S.b2[k] = th[OFF_B2 + k];
    }
    if (tid < NO) S.b3[tid] = th[OFF_B3 + tid];
    const uint32_t bar = smem_u32(&S.bar);
    if (tid == 0) {
        S.abort = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&S.tmem)),
                     "r"(128)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem;
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    const uint32_t a_addr = smem_u32(S.a), w2_addr = smem_u32(S.w2), w3_addr = smem_u32(S.w3);
    uint32_t parity = 0;
    const long long n_tiles = (n + kTcRows - 1) / kTcRows;
    // this thread's point of the next tile is loaded one tile ahead
    float xn0 = 0.0f, xn1 = 0.0f;
    {
        const long long p0 = (long long)blockIdx.x * kTcRows + row;
        if (p0 < n) { xn0 = x[p0 * NI]; xn1 = x[p0 * NI + 1]; }
    }
    for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const long long p = tile * kTcRows + row;
        const bool valid = p < n;
        const float x0 = xn0, x1 = xn1;
        {
            const long long pn = (tile + gridDim.x) * kTcRows + row;
            if (pn < n) { xn0 = x[pn * NI]; xn1 = x[pn * NI + 1]; }
        }
        // 1. layer 1 into the A operand (this thread: 64 units of its point)
        {
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int u0 = half * 64 + c * 8;
                uint32_t w[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int u = u0 + 2 * e;
                    const float z0 = fmaf(S.w1[u * NI + 1], x1, fmaf(S.w1[u * NI], x0, S.b1[u]));
                    const float z1 = fmaf(S.w1[(u + 1) * NI + 1], x1, fmaf(S.w1[(u + 1) * NI], x0, S.b1[u + 1]));
                    w[e] = tanh_bf16x2(z0, z1);
                }
                *reinterpret_cast<uint4*>(S.a + kmajor_off(row, u0)) = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        fence_async_smem();
        __syncthreads();
        // 2. h1 W2^T into the accumulator
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int kk = 0; kk < NH / 16; ++kk)
                tc_mma(tmem, sdesc(a_addr + kk * 2 * kLbo, kLbo, kSbo), sdesc(w2_addr + kk * 2 * kLbo, kLbo, kSbo),
                       idesc_bf16(128, 128), kk > 0 ? 1u : 0u);
            tc_commit(bar);
        }
        if (!bar_wait(bar, parity)) S.abort = 1;
        parity ^= 1;
        tc_fence_after();
        __syncthreads();
        if (S.abort) break;
        // 3. bias, tanh, h2 over the A operand
#pragma unroll
        for (int ch = 0; ch < 2; ++ch) {
            const int c0 = half * 64 + ch * 32;
            float acc[32];
            tmem_ld32(tmem + lane_base + (uint32_t)c0, acc);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                uint32_t w[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int q = c * 8 + 2 * e;
                    w[e] = tanh_bf16x2(acc[q] + S.b2[c0 + q], acc[q + 1] + S.b2[c0 + q + 1]);
                }
                *reinterpret_cast<uint4*>(S.a + kmajor_off(row, c0 + c * 8)) = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        tc_fence_before();
        fence_async_smem();
        __syncthreads();
        // 4. h2 W3^T (16 padded outputs) into accumulator columns 0..15
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int kk = 0; kk < NH / 16; ++kk)
                tc_mma(tmem, sdesc(a_addr + kk * 2 * kLbo, kLbo, kSbo), sdesc(w3_addr + kk * 2 * kLbo, kLbo, kSbo),
                       idesc_bf16(128, 16), kk > 0 ? 1u : 0u);
            tc_commit(bar);
        }
        if (!bar_wait(bar, parity)) S.abort = 1;
        parity ^= 1;
        tc_fence_after();
        __syncthreads();
        if (S.abort) break;
        if (half == 0) {
            float o8[8];
            tmem_ld8(tmem + lane_base, o8);
            if (valid)
#pragma unroll
                for (int o = 0; o < NO; ++o) y[p * NO + o] = o8[o] + S.b3[o];
        }
        tc_fence_before();
        __syncthreads();
    }
    if (S.abort) {
        // a wait expired: mark this block's remaining outputs and report
        if (tid == 0) atomicOr(err, 1);
        for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
            const long long p = tile * kTcRows + row;
            if (half == 0 && p < n)
                for (int o = 0; o < NO; ++o) y[p * NO + o] = __int_as_float(0x7fc00000);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(128) : "memory");
    }
}

// ------------------------------------------------------------------ standardization
// The caller's affine standardizations folded into the parameters (one
// thread per parameter, float64 arithmetic rounded once): inputs x_std =
// (x - xm) / xs enter layer 1, outputs y = y_std ys + ym leave layer 3.
struct Affine {
    double xm[NI], xs[NI], ym[NO], ys[NO];
};
__global__ void k_fold(const float* __restrict__ th, Affine a, float* __restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= NP) return;
    double v = (double)th[k];
    if (k < OFF_B1) {
        v /= a.xs[k % NI];
    } else if (k < OFF_W2) {
        const int o = k - OFF_B1;
        for (int i = 0; i < NI; ++i) v -= (double)th[OFF_W1 + o * NI + i] * a.xm[i] / a.xs[i];
    } else if (k >= OFF_W3 && k < OFF_B3) {
        v *= a.ys[(k - OFF_W3) / NH];
    } else if (k >= OFF_B3) {
        const int o = k - OFF_B3;
        v = v * a.ys[o] + a.ym[o];
    }
    out[k] = (float)v;
}

// The network's inputs of transport-data queries: log10(E/N in Td) and the
// O2 fraction, in float32 (the network's input precision; a float64
// logarithm would run on this GPU's slow float64 units).
__global__ void k_features(const double* __restrict__ en, const double* __restrict__ f, float* __restrict__ x,
                           long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        reinterpret_cast<float2*>(x)[i] = make_float2(log10f((float)en[i]), (float)f[i]);
}

}  // namespace mlp

// ------------------------------------------------------------------ C ABI
using namespace mlp;

namespace {

size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

struct TrainWs {
    __nv_bfloat16 *w2b, *w2t, *h1b, *h1t, *dz2b, *dz2t;
    float *h1, *z2, *dh1, *gw2, *head, *l1, *loss;
    int *step, *err;
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
    w->err = (int*)take(64);
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

extern "C" int mlp_forward_variant(const float* params, const float* x, float* y, long long n, int variant,
                                   void* ws, size_t ws_bytes, pic_stream_t stream) {
    if (!params || !x || !y || n < 0 || !ws || ((uintptr_t)ws & 255) || ws_bytes < mlp_workspace_bytes(0) ||
        (variant != 0 && variant != 1))
        return PIC_ERR_ARG;
    if (n == 0) return PIC_OK;
    cudaStream_t s = (cudaStream_t)stream;
    TrainWs w;
    carve(ws, 64, &w);
    k_prep<<<(NH * NH + 255) / 256, 256, 0, s>>>(params, w.w2b, w.w2t);
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (variant == 0) {
        const int smem = (int)sizeof(TcSmem) + 1024;
        if (cudaFuncSetAttribute(k_infer_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
            return PIC_ERR_CUDA;
        // blocks per SM from the shared memory each needs (plus the 1 KB the
        // runtime reserves per block); each block also holds 128 of the 512
        // tensor-memory columns, so at most 4
        int smem_sm = 0;
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        per_sm = smem_sm / (smem + 1024);
        per_sm = per_sm < 1 ? 1 : (per_sm > 4 ? 4 : per_sm);
        const long long tiles = (n + kTcRows - 1) / kTcRows;
        long long blocks = (long long)sms * per_sm;
        if (blocks > tiles) blocks = tiles;
        k_infer_tc<<<(unsigned)blocks, kTcThreads, smem, s>>>(params, w.w2b, x, y, n, w.err);
    } else {
        const int smem = (int)sizeof(InfSmem);
        if (cudaFuncSetAttribute(k_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
            return PIC_ERR_CUDA;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_infer, kInfWarps * 32, smem);
        const long long tiles = (n + 15) / 16;
        long long blocks = (long long)sms * (per_sm > 0 ? per_sm : 1);
        if (blocks * kInfWarps > tiles) blocks = (tiles + kInfWarps - 1) / kInfWarps;
        k_infer<<<(unsigned)blocks, kInfWarps * 32, smem, s>>>(params, w.w2b, x, y, n);
    }
    return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ERR_CUDA;
}

extern "C" int mlp_fold_standardization(const float* params, const double x_mean[2], const double x_scale[2],
                                        const double y_mean[6], const double y_scale[6], float* out,
                                        pic_stream_t stream) {
    if (!params || !out || params == out || !x_mean || !x_scale || !y_mean || !y_scale) return PIC_ERR_ARG;
    mlp::Affine a;
    for (int i = 0; i < mlp::NI; ++i) {
        if (!(x_scale[i] != 0.0) || !isfinite(x_scale[i]) || !isfinite(x_mean[i])) return PIC_ERR_ARG;
        a.xm[i] = x_mean[i];
        a.xs[i] = x_scale[i];
    }
    for (int o = 0; o < mlp::NO; ++o) {
        if (!isfinite(y_scale[o]) || !isfinite(y_mean[o])) return PIC_ERR_ARG;
        a.ym[o] = y_mean[o];
        a.ys[o] = y_scale[o];
    }
    mlp::k_fold<<<(mlp::NP + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, a, out);
    return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ERR_CUDA;
}

extern "C" int mlp_features(const double* EN_Td, const double* f_o2, float* x, long long n, pic_stream_t stream) {
    if (n < 0 || (n > 0 && (!EN_Td || !f_o2 || !x))) return PIC_ERR_ARG;
    if (n == 0) return PIC_OK;
    long long g = (n + 255) / 256;
    if (g > 65535) g = 65535;
    mlp::k_features<<<(unsigned)g, 256, 0, (cudaStream_t)stream>>>(EN_Td, f_o2, x, n);
    return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ERR_CUDA;
}

extern "C" int mlp_forward(const float* params, const float* x, float* y, long long n, void* ws, size_t ws_bytes,
                           pic_stream_t stream) {
    return mlp_forward_variant(params, x, y, n, 0, ws, ws_bytes, stream);
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
