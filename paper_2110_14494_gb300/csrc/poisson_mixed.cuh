// Mixed-precision Poisson kernels (included by poisson.cu inside its
// anonymous namespace).
//
// The potential is held as an unevaluated sum of two floats (hi + lo, about
// 48 significant bits), so the outer residual b - A phi and the field
// -grad(phi) are formed without float64 arithmetic: the stencil only ever
// needs differences of neighbouring potentials, and those come out of the
// float pairs exactly up to one rounding of the small difference.  The
// correction delta with A delta = r is found by flexible CG in float32 (the
// same float32 V-cycle preconditioner), then added to phi in the pair
// format.  When the float32 residual has dropped by kRefineDrop and the
// tolerance is not met yet, the correction is committed and the residual is
// re-formed from phi (iterative refinement).
//
// Reductions are deterministic: each block stores its partial sums, and the
// last block to finish (an atomic counter) adds the partials in a fixed order
// and updates the CG scalars, so no separate scalar kernels are launched.

constexpr int ZC = 4;            // z planes per thread in the stencil kernels
constexpr int kFlatPer = 2;      // float4 groups per thread in the flat kernels
constexpr int kFlatBlock = 256;
constexpr double kRefineDrop = 1e-4;

// ---------------------------------------------------------------- float pairs
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// hi + lo of a - b, both pairs; the result is renormalised
__device__ __forceinline__ float2 df_sub(float2 a, float2 b) {
    float t, e;
    two_sum(a.x, -b.x, t, e);
    const float l = e + (a.y - b.y);
    const float s = t + l;
    return make_float2(s, l - (s - t));
}

__device__ __forceinline__ float2 df_add_f(float2 a, float d) {
    float t, e;
    two_sum(a.x, d, t, e);
    const float l = e + a.y;
    const float s = t + l;
    return make_float2(s, l - (s - t));
}

// a - b rounded to one float
__device__ __forceinline__ float df_diff(float2 a, float2 b) {
    float t, e;
    two_sum(a.x, -b.x, t, e);
    return t + (e + (a.y - b.y));
}

__device__ __forceinline__ float2 ld_df(const float* hi, const float* lo, int c) { return make_float2(hi[c], lo[c]); }

// Running float-pair sum.
struct DFAcc {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add(float2 d) {
        float s, e;
        two_sum(hi, d.x, s, e);
        hi = s;
        lo += e + d.y;
    }
    __device__ __forceinline__ void add(float d) {
        float s, e;
        two_sum(hi, d, s, e);
        hi = s;
        lo += e;
    }
    __device__ __forceinline__ float value() const { return hi + lo; }
};

// ---------------------------------------------------------------- reductions
// Sums NV per-thread float values over the grid.  Every block stores its sums
// in part[NV * block + q]; the last block to arrive adds all partials in a
// fixed order, leaves the totals in tot[] (all its threads) and returns true;
// the others return false.  The counter is reset for the next launch.
template <int NV>
__device__ bool grid_sums(const float (&v)[NV], double* part, unsigned* ctr, double (&tot)[NV]) {
    __shared__ double red[NV][32];
    __shared__ int last;
    const int nthr = blockDim.x * blockDim.y;
    const int t = threadIdx.x + threadIdx.y * blockDim.x;
    const int lane = t & 31, w = t >> 5, nw = nthr >> 5;
    const unsigned b = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const unsigned nb = gridDim.x * gridDim.y * gridDim.z;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        float x = v[q];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
        if (lane == 0) red[q][w] = (double)x;
    }
    __syncthreads();
    if (t == 0) {
        for (int q = 0; q < NV; ++q) {
            double s = 0.0;
            for (int x = 0; x < nw; ++x) s += red[q][x];
            part[(size_t)b * NV + q] = s;
        }
        __threadfence();
        last = atomicAdd(ctr, 1u) == nb - 1 ? 1 : 0;
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        // sixteen independent loads per round (one round trip covers the
        // partials of up to 16 blocks per thread), added in a fixed order
        double s = 0.0;
        for (unsigned x0 = t; x0 < nb; x0 += 16u * nthr) {
            double a[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const unsigned x = x0 + u * nthr;
                a[u] = x < nb ? __ldcg(part + (size_t)x * NV + q) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) a[u] += a[u + 8];
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] += a[u + 4];
            s += (a[0] + a[1]) + (a[2] + a[3]);
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
        __syncthreads();
        if (lane == 0) red[q][w] = s;
        __syncthreads();
        double a = 0.0;
        for (int x = 0; x < nw; ++x) a += red[q][x];
        tot[q] = a;
    }
    if (t == 0) *ctr = 0u;
    return true;
}

#define MX_CELLS_BEGIN                                                     \
    const int i = blockIdx.x * BX + threadIdx.x;                          \
    const int j = blockIdx.y * BY + threadIdx.y;                          \
    const bool in_xy = i < nx && j < ny;                                  \
    _Pragma("unroll") for (int dz = 0; dz < ZC; ++dz) {                   \
        const int k = blockIdx.z * ZC + dz;                               \
        if (!in_xy || k >= nz) continue;                                  \
        const int c = lin(i, j, k, nx, ny);
#define MX_CELLS_END }

// ---------------------------------------------------------------- kernels
struct MxBoundary {
    float2 v_lo, v_hi, v_mask;  // plate and electrode potentials as float pairs
};

// Electrode cells take the electrode potential (run once per potential
// buffer: the correction is zero there, so later solves keep it).
__global__ void k_mx_fix_mask(const uint8_t* __restrict__ mask, float* __restrict__ hi, float* __restrict__ lo, int n,
                              float2 v_mask) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n && mask[c]) {
        hi[c] = v_mask.x;
        lo[c] = v_mask.y;
    }
}

// Adds the face difference (neighbour - centre) of an interior face; an
// electrode neighbour stands for v_mask.
__device__ __forceinline__ void face_add(DFAcc& s, int& nmask, float2 nb, uint8_t m_nb, float2 pc, float2 vm) {
    if (m_nb) {
        ++nmask;
        s.add(df_sub(vm, pc));
    } else {
        s.add(df_sub(nb, pc));
    }
}

// r = b - A phi from the float-pair potential (r = 0 on electrode cells,
// whose potential must already be v_mask); b = h^2 rho / eps0 + plate and
// electrode terms.  rho is h^2 rho / eps0 in float (RHO = float) or rho in
// float64 (RHO = double, scaled by h2e here).  Sums ||b||^2 and ||r||^2 into
// sc[S_B2], sc[S_R2].  Loads as in the other stencil kernels (column, y
// neighbours, x from the adjacent lanes).  Issue-bound (the pair
// arithmetic): registers capped for eight blocks per SM.
template <class RHO>
__global__ void __launch_bounds__(BX * BY, 8) k_mx_resid(const RHO* __restrict__ rho, double h2e,
                                                      const uint8_t* __restrict__ mask,
                                                      const float* __restrict__ phi_hi,
                                                      const float* __restrict__ phi_lo, int nx, int ny, int nz,
                                                      MxBoundary bc, float* __restrict__ r, double* part,
                                                      unsigned* ctr, double* sc) {
    const int lane = threadIdx.x;
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k0 = blockIdx.z * ZC;
    const bool in = i < nx && j < ny;
    const int pl = nx * ny;
    const int c0 = in ? lin(i, j, 0, nx, ny) : 0;
    float2 col[ZC + 2];
    uint8_t cm[ZC + 2];
#pragma unroll
    for (int d = 0; d < ZC + 2; ++d) {
        const int k = k0 - 1 + d;
        const bool ok = in && k >= 0 && k < nz;
        const int c = c0 + (ok ? k : 0) * pl;
        col[d] = ok ? ld_df(phi_hi, phi_lo, c) : make_float2(0.0f, 0.0f);
        cm[d] = ok ? mask[c] : 0;
    }
    float2 ym[ZC], yp[ZC], xe[ZC];
    uint8_t mym[ZC], myp[ZC], mxe[ZC];
    float2 hr[ZC];
#pragma unroll
    for (int d = 0; d < ZC; ++d) {
        const int k = k0 + d;
        const bool ok = in && k < nz;
        const int c = c0 + (ok ? k : 0) * pl;
        const bool a = ok && j > 0, b = ok && j < ny - 1;
        ym[d] = a ? ld_df(phi_hi, phi_lo, c - nx) : make_float2(0.0f, 0.0f);
        mym[d] = a ? mask[c - nx] : 0;
        yp[d] = b ? ld_df(phi_hi, phi_lo, c + nx) : make_float2(0.0f, 0.0f);
        myp[d] = b ? mask[c + nx] : 0;
        xe[d] = make_float2(0.0f, 0.0f);
        mxe[d] = 0;
        const int xq = lane == 0 ? c - 1 : c + 1;
        if (ok && ((lane == 0 && i > 0) || (lane == BX - 1 && i < nx - 1))) {
            xe[d] = ld_df(phi_hi, phi_lo, xq);
            mxe[d] = mask[xq];
        }
        if (ok) {
            if (sizeof(RHO) == 8) {
                const double x = h2e * (double)rho[c];
                hr[d].x = (float)x;
                hr[d].y = (float)(x - (double)hr[d].x);
            } else {
                hr[d] = make_float2((float)rho[c], 0.0f);
            }
        } else {
            hr[d] = make_float2(0.0f, 0.0f);
        }
    }
    float acc[2] = {0.0f, 0.0f};
#pragma unroll
    for (int d = 0; d < ZC; ++d) {
        const int k = k0 + d;
        const float2 pc = col[d + 1];
        const uint8_t mc = cm[d + 1];
        float2 xm = make_float2(__shfl_up_sync(kFull, pc.x, 1), __shfl_up_sync(kFull, pc.y, 1));
        float2 xp = make_float2(__shfl_down_sync(kFull, pc.x, 1), __shfl_down_sync(kFull, pc.y, 1));
        uint8_t mxm = (uint8_t)__shfl_up_sync(kFull, (int)mc, 1), mxp = (uint8_t)__shfl_down_sync(kFull, (int)mc, 1);
        if (lane == 0) { xm = xe[d]; mxm = mxe[d]; }
        if (lane == BX - 1) { xp = xe[d]; mxp = mxe[d]; }
        if (!in || k >= nz) continue;
        const int c = c0 + k * pl;
        if (mc) {
            r[c] = 0.0f;
            continue;
        }
        DFAcc s;
        int nmask = 0;
        float bsum = hr[d].x;
        if (i > 0) face_add(s, nmask, xm, mxm, pc, bc.v_mask);
        if (i < nx - 1) face_add(s, nmask, xp, mxp, pc, bc.v_mask);
        if (j > 0) face_add(s, nmask, ym[d], mym[d], pc, bc.v_mask);
        if (j < ny - 1) face_add(s, nmask, yp[d], myp[d], pc, bc.v_mask);
        if (k > 0) face_add(s, nmask, col[d], cm[d], pc, bc.v_mask);
        else { const float2 t = df_sub(bc.v_lo, pc); s.add(make_float2(2.0f * t.x, 2.0f * t.y)); bsum += 2.0f * bc.v_lo.x; }
        if (k < nz - 1) face_add(s, nmask, col[d + 2], cm[d + 2], pc, bc.v_mask);
        else { const float2 t = df_sub(bc.v_hi, pc); s.add(make_float2(2.0f * t.x, 2.0f * t.y)); bsum += 2.0f * bc.v_hi.x; }
        s.add(hr[d]);
        const float rr = s.value();
        bsum += (float)nmask * bc.v_mask.x;
        r[c] = rr;
        acc[0] += bsum * bsum;
        acc[1] += rr * rr;
    }
    double tot[2];
    if (grid_sums<2>(acc, part, ctr, tot) && threadIdx.x == 0 && threadIdx.y == 0) {
        sc[S_B2] = tot[0];
        sc[S_R2] = tot[1];
    }
}

// Flat kernels: each thread takes kFlatPer groups of four cells as float4
// (all loads issued before any use); a remainder of n % 4 cells goes to the
// first threads of block 0.
#define FLAT4_LOOP(BODY4, BODY1)                                              \
    {                                                                         \
        const int n4 = n >> 2;                                                \
        const int base = blockIdx.x * (kFlatBlock * kFlatPer) + threadIdx.x;  \
        _Pragma("unroll") for (int u = 0; u < kFlatPer; ++u) {                \
            const int v4 = base + u * kFlatBlock;                             \
            if (v4 < n4) { BODY4 }                                            \
        }                                                                     \
        if (blockIdx.x == 0 && threadIdx.x < (n & 3)) {                       \
            const int c = (n4 << 2) + threadIdx.x;                            \
            BODY1                                                             \
        }                                                                     \
    }

__device__ __forceinline__ float dot4(float4 a, float4 b) { return ((a.x * b.x + a.y * b.y) + a.z * b.z) + a.w * b.w; }
__device__ __forceinline__ float4 fma4(float a, float4 x, float4 y) {
    return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}
__device__ __forceinline__ float4 ld4(const float* p, int v4) { return reinterpret_cast<const float4*>(p)[v4]; }
__device__ __forceinline__ void st4(float* p, int v4, float4 v) { reinterpret_cast<float4*>(p)[v4] = v; }

// One flexible-CG iteration takes two kernels.  With z = M r, the new
// direction p = z + beta p_prev and q = A p = A z + beta q_prev, so A z and
// the three sums z.r, z.q_prev, z.(A z) can be formed in one stencil pass
// before p exists: with A symmetric, p.q = z.Az + 2 beta z.q_prev + beta^2
// p_prev.q_prev (p_prev.Az = q_prev.z), where p_prev.q_prev is the previous
// iteration's gamma.  The second pass forms p and q and updates delta and r.

// The scalars of the iteration from the three sums: beta = -alpha_prev
// (z.q_prev) / rho_prev (flexible CG), rho = z.r, gamma = p.q, alpha = rho /
// gamma.  First iteration of a pass: beta = 0, gamma = z.Az.
__device__ __forceinline__ void cg_scalars(const double (&tot)[3], int first, double* sc) {
    const double rho_old = sc[S_RHO];
    const double beta = (first || rho_old == 0.0) ? 0.0 : -sc[S_ALPHA] * tot[1] / rho_old;
    const double gam = first ? tot[2] : tot[2] + beta * (2.0 * tot[1] + beta * sc[S_GAM]);
    sc[S_BETA] = beta;
    sc[S_RHO] = tot[0];
    sc[S_GAM] = gam;
    sc[S_ALPHA] = gam > 0.0 ? tot[0] / gam : 0.0;
}

// Stencil kernels walk ZC planes per thread and load everything first: the
// centre column from k0 - 1 to k0 + ZC (reused as the z neighbours), the y
// neighbours by plane, and the x neighbours from the adjacent lanes (a warp
// is one row of 32 consecutive x), loading only at the warp's ends.
__device__ __forceinline__ float lane_xm(float v, int lane) { return __shfl_up_sync(kFull, v, 1); }
__device__ __forceinline__ float lane_xp(float v, int lane) { return __shfl_down_sync(kFull, v, 1); }

// w = A z (0 on electrode cells) with the sums z.r, z.q_prev, z.w, then the
// iteration's scalars (last block).  q_prev is not read when first is set.
__global__ void __launch_bounds__(BX * BY) k_mx_apply(const float* __restrict__ z, const float* __restrict__ r,
                                                      const float* __restrict__ q_prev, float* __restrict__ w,
                                                      const uint8_t* __restrict__ mask, int nx, int ny, int nz,
                                                      int first, double* part, unsigned* ctr, double* sc) {
    pdl_wait();
    const int lane = threadIdx.x;
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k0 = blockIdx.z * ZC;
    const bool in = i < nx && j < ny;
    const int pl = nx * ny;
    const int c0 = in ? lin(i, j, 0, nx, ny) : 0;
    float col[ZC + 2], ym[ZC], yp[ZC], xe[ZC], rv[ZC], qv[ZC];
    uint8_t mk[ZC];
#pragma unroll
    for (int d = 0; d < ZC + 2; ++d) {
        const int k = k0 - 1 + d;
        col[d] = (in && k >= 0 && k < nz) ? __ldg(z + c0 + k * pl) : 0.0f;
    }
#pragma unroll
    for (int d = 0; d < ZC; ++d) {
        const int k = k0 + d;
        const bool ok = in && k < nz;
        const int c = c0 + (ok ? k : 0) * pl;
        ym[d] = ok && j > 0 ? __ldg(z + c - nx) : 0.0f;
        yp[d] = ok && j < ny - 1 ? __ldg(z + c + nx) : 0.0f;
        // the warp's end lanes fetch their outer x neighbour
        xe[d] = 0.0f;
        if (ok && lane == 0 && i > 0) xe[d] = __ldg(z + c - 1);
        if (ok && lane == BX - 1 && i < nx - 1) xe[d] = __ldg(z + c + 1);
        mk[d] = ok ? mask[c] : 1;
        rv[d] = ok ? __ldg(r + c) : 0.0f;
        qv[d] = ok && !first ? __ldg(q_prev + c) : 0.0f;
    }
    float acc[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int d = 0; d < ZC; ++d) {
        const int k = k0 + d;
        const float zc = col[d + 1];
        float xm = lane_xm(zc, lane), xp = lane_xp(zc, lane);
        if (lane == 0) xm = xe[d];
        if (lane == BX - 1) xp = xe[d];
        if (!in || k >= nz) continue;
        if (i == 0) xm = 0.0f;
        if (i == nx - 1) xp = 0.0f;
        const float zm = col[d], zp = col[d + 2];
        const float diag =
            6.0f - (float)((i == 0) + (i == nx - 1) + (j == 0) + (j == ny - 1)) + (float)((k == 0) + (k == nz - 1));
        float ww = diag * zc - (((((xm + xp) + ym[d]) + yp[d]) + zm) + zp);
        if (mk[d]) ww = 0.0f;
        w[c0 + k * pl] = ww;
        acc[0] += zc * rv[d];
        acc[1] += zc * qv[d];
        acc[2] += zc * ww;
    }
    double tot[3];
    if (grid_sums<3>(acc, part, ctr, tot) && threadIdx.x == 0 && threadIdx.y == 0) cg_scalars(tot, first, sc);
}

// The same for nx % 4 == 0, with four consecutive x cells per thread
// (16-byte loads and stores): lane l of a warp holds x = 4 (32 b + l) .. + 3
// of one row; the x neighbours across float4 boundaries come from the
// adjacent lanes, and the warp's end lanes load them.  Each cell's w is the
// scalar kernel's (same operations in the same order); the partial sums
// group the cells differently.
__device__ __forceinline__ float4 ld4g(const float* p, int c) { return __ldg(reinterpret_cast<const float4*>(p + c)); }
__device__ __forceinline__ float f4c(const float4& v, int e) { return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w)); }

// Registers capped for six blocks per SM (latency-bound: more warps in flight).
__global__ void __launch_bounds__(BX * BY, 6) k_mx_apply4(const float* __restrict__ z, const float* __restrict__ r,
                                                       const float* __restrict__ q_prev, float* __restrict__ w,
                                                       const uint8_t* __restrict__ mask, int nx, int ny, int nz,
                                                       int first, double* part, unsigned* ctr, double* sc) {
    pdl_wait();
    const int lane = threadIdx.x;
    const int i0 = 4 * (blockIdx.x * BX + threadIdx.x), j = blockIdx.y * BY + threadIdx.y, k0 = blockIdx.z * ZC;
    const bool in = i0 < nx && j < ny;
    const int pl = nx * ny;
    const int c0 = in ? lin(i0, j, 0, nx, ny) : 0;
    float4 col[ZC + 2], ym[ZC], yp[ZC];
    float xl[ZC], xr[ZC];
    uchar4 mk[ZC];
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int d = 0; d < ZC + 2; ++d) {
        const int k = k0 - 1 + d;
        col[d] = (in && k >= 0 && k < nz) ? ld4g(z, c0 + k * pl) : zero4;
    }
#pragma unroll
    for (int d = 0; d < ZC; ++d) {
        const int k = k0 + d;
        const bool ok = in && k < nz;
        const int c = c0 + (ok ? k : 0) * pl;
        ym[d] = ok && j > 0 ? ld4g(z, c - nx) : zero4;
        yp[d] = ok && j < ny - 1 ? ld4g(z, c + nx) : zero4;
        xl[d] = ok && lane == 0 && i0 > 0 ? __ldg(z + c - 1) : 0.0f;
        xr[d] = ok && lane == BX - 1 && i0 + 4 < nx ? __ldg(z + c + 4) : 0.0f;
        mk[d] = ok ? *reinterpret_cast<const uchar4*>(mask + c) : make_uchar4(1, 1, 1, 1);
    }
    float acc[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int d = 0; d < ZC; ++d) {
        const int k = k0 + d;
        const float4 zc = col[d + 1];
        float left = __shfl_up_sync(kFull, zc.w, 1), right = __shfl_down_sync(kFull, zc.x, 1);
        if (lane == 0) left = xl[d];
        if (lane == BX - 1) right = xr[d];
        if (!in || k >= nz) continue;
        const float fz = (float)((k == 0) + (k == nz - 1));
        const float fy = (float)((j == 0) + (j == ny - 1));
        const unsigned char mm[4] = {mk[d].x, mk[d].y, mk[d].z, mk[d].w};
        float wv[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int i = i0 + e;
            const float c = f4c(zc, e);
            float xm = e == 0 ? left : f4c(zc, e - 1);
            float xp = e == 3 ? right : f4c(zc, e + 1);
            if (i == 0) xm = 0.0f;
            if (i == nx - 1) xp = 0.0f;
            const float diag = 6.0f - ((float)((i == 0) + (i == nx - 1)) + fy) + fz;
            float ww = diag * c - (((((xm + xp) + f4c(ym[d], e)) + f4c(yp[d], e)) + f4c(col[d], e)) + f4c(col[d + 2], e));
            if (mm[e]) ww = 0.0f;
            wv[e] = ww;
            acc[2] += c * ww;
        }
        *reinterpret_cast<float4*>(w + c0 + k * pl) = make_float4(wv[0], wv[1], wv[2], wv[3]);
    }
    // z.r and z.q_prev after the stencil (fewer registers held across it)
#pragma unroll
    for (int d = 0; d < ZC; ++d) {
        const int k = k0 + d;
        if (!in || k >= nz) continue;
        const int c = c0 + k * pl;
        const float4 zc = col[d + 1], rv = ld4g(r, c);
        acc[0] += dot4(zc, rv);
        if (!first) acc[1] += dot4(zc, ld4g(q_prev, c));
    }
    double tot[3];
    if (grid_sums<3>(acc, part, ctr, tot) && threadIdx.x == 0 && threadIdx.y == 0) cg_scalars(tot, first, sc);
}

// p = z + beta p_prev written over w (in p_w), q = w + beta q_prev (in place),
// delta (+)= alpha p, r -= alpha q, ||r||^2 into sc[S_R2].  p_prev and q_prev
// are not read when first is set (beta = 0).
__global__ void __launch_bounds__(kFlatBlock) k_mx_step(const float* __restrict__ z,
                                                        const float* __restrict__ p_prev, float* __restrict__ p_w,
                                                        float* __restrict__ q, float* __restrict__ d,
                                                        float* __restrict__ r, int n, int first, double* part,
                                                        unsigned* ctr, double* sc) {
    pdl_wait();
    const float a = (float)sc[S_ALPHA];
    const float b = first ? 0.0f : (float)sc[S_BETA];
    const bool use_prev = b != 0.0f;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float acc[1] = {0.0f};
    FLAT4_LOOP(
        const float4 zz = ld4(z, v4); const float4 ww = ld4(p_w, v4); const float4 r0 = ld4(r, v4);
        const float4 pp = use_prev ? fma4(b, ld4(p_prev, v4), zz) : zz;
        const float4 qq = use_prev ? fma4(b, ld4(q, v4), ww) : ww;
        const float4 d0 = first ? zero4 : ld4(d, v4);
        const float4 rr = fma4(-a, qq, r0); st4(p_w, v4, pp); st4(q, v4, qq); st4(r, v4, rr);
        st4(d, v4, fma4(a, pp, d0)); acc[0] += dot4(rr, rr);,
        const float pp = use_prev ? fmaf(b, p_prev[c], z[c]) : z[c]; const float qq = use_prev ? fmaf(b, q[c], p_w[c]) : p_w[c];
        p_w[c] = pp; q[c] = qq; d[c] = first ? a * pp : fmaf(a, pp, d[c]); const float rr = fmaf(-a, qq, r[c]); r[c] = rr;
        acc[0] += rr * rr;)
    double tot[1];
    if (grid_sums<1>(acc, part, ctr, tot) && threadIdx.x == 0) sc[S_R2] = tot[0];
}

// phi += delta in the pair format.
__global__ void __launch_bounds__(kFlatBlock) k_mx_commit(float* __restrict__ hi, float* __restrict__ lo,
                                                          const float* __restrict__ d, int n) {
    FLAT4_LOOP(
        const float4 h = ld4(hi, v4); const float4 l = ld4(lo, v4); const float4 dd = ld4(d, v4);
        const float2 a = df_add_f(make_float2(h.x, l.x), dd.x); const float2 b = df_add_f(make_float2(h.y, l.y), dd.y);
        const float2 e = df_add_f(make_float2(h.z, l.z), dd.z); const float2 f = df_add_f(make_float2(h.w, l.w), dd.w);
        st4(hi, v4, make_float4(a.x, b.x, e.x, f.x)); st4(lo, v4, make_float4(a.y, b.y, e.y, f.y));,
        const float2 v = df_add_f(make_float2(hi[c], lo[c]), d[c]); hi[c] = v.x; lo[c] = v.y;)
}

// out = 2 cur - prev (linear extrapolation in time), or out = cur.
__device__ __forceinline__ float2 extrap1(float ch, float cl, float ph, float pl, int have_prev) {
    float2 v = make_float2(ch, cl);
    if (have_prev) v = df_sub(make_float2(2.0f * v.x, 2.0f * v.y), make_float2(ph, pl));
    return v;
}
__global__ void __launch_bounds__(kFlatBlock) k_mx_extrapolate(const float* __restrict__ ch,
                                                               const float* __restrict__ cl,
                                                               const float* __restrict__ ph,
                                                               const float* __restrict__ pl, float* __restrict__ oh,
                                                               float* __restrict__ ol, int n, int have_prev) {
    FLAT4_LOOP(
        const float4 a = ld4(ch, v4); const float4 b = ld4(cl, v4);
        const float4 c4 = have_prev ? ld4(ph, v4) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 d4 = have_prev ? ld4(pl, v4) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float2 x = extrap1(a.x, b.x, c4.x, d4.x, have_prev); const float2 y = extrap1(a.y, b.y, c4.y, d4.y, have_prev);
        const float2 zz = extrap1(a.z, b.z, c4.z, d4.z, have_prev); const float2 w = extrap1(a.w, b.w, c4.w, d4.w, have_prev);
        st4(oh, v4, make_float4(x.x, y.x, zz.x, w.x)); st4(ol, v4, make_float4(x.y, y.y, zz.y, w.y));,
        const float2 v = extrap1(ch[c], cl[c], have_prev ? ph[c] : 0.f, have_prev ? pl[c] : 0.f, have_prev);
        oh[c] = v.x; ol[c] = v.y;)
}

// E = -grad(phi + delta) at cell centres (ghost rules as k_grad); with
// out_hi set, also writes phi + delta there in the pair format.  delta may
// be null, and is ignored when the device-driven loop state L (optional)
// says no iteration ran since the last refinement.  E4 (if set) gets one
// 16-byte store per cell.  Registers capped for ten blocks per SM.
__global__ void __launch_bounds__(BX * BY, 10) k_mx_grad(const float* __restrict__ hi, const float* __restrict__ lo,
                                                     const float* __restrict__ dl, float* __restrict__ out_hi,
                                                     float* __restrict__ out_lo, int nx, int ny, int nz, float inv2h,
                                                     MxBoundary bc, float* __restrict__ Ex, float* __restrict__ Ey,
                                                     float* __restrict__ Ez, float* __restrict__ E4,
                                                     const MxLoop* __restrict__ L) {
    if (L && L->it == 0) dl = nullptr;
    auto PH = [&](int x) {
        const float2 v = make_float2(__ldg(hi + x), __ldg(lo + x));
        return dl ? df_add_f(v, __ldg(dl + x)) : v;
    };
    const int lane = threadIdx.x;
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k0 = blockIdx.z * ZC;
    const bool in = i < nx && j < ny;
    const int pl = nx * ny;
    const int c0 = in ? lin(i, j, 0, nx, ny) : 0;
    float2 col[ZC + 2], ym[ZC], yp[ZC], xe[ZC];
#pragma unroll
    for (int d = 0; d < ZC + 2; ++d) {
        const int k = k0 - 1 + d;
        col[d] = (in && k >= 0 && k < nz) ? PH(c0 + k * pl) : make_float2(0.0f, 0.0f);
    }
#pragma unroll
    for (int d = 0; d < ZC; ++d) {
        const int k = k0 + d;
        const bool ok = in && k < nz;
        const int c = c0 + (ok ? k : 0) * pl;
        ym[d] = ok && j > 0 ? PH(c - nx) : make_float2(0.0f, 0.0f);
        yp[d] = ok && j < ny - 1 ? PH(c + nx) : make_float2(0.0f, 0.0f);
        xe[d] = make_float2(0.0f, 0.0f);
        if (ok && lane == 0 && i > 0) xe[d] = PH(c - 1);
        if (ok && lane == BX - 1 && i < nx - 1) xe[d] = PH(c + 1);
    }
#pragma unroll
    for (int d = 0; d < ZC; ++d) {
        const int k = k0 + d;
        const float2 pc = col[d + 1];
        float2 xm = make_float2(__shfl_up_sync(kFull, pc.x, 1), __shfl_up_sync(kFull, pc.y, 1));
        float2 xp = make_float2(__shfl_down_sync(kFull, pc.x, 1), __shfl_down_sync(kFull, pc.y, 1));
        if (lane == 0) xm = xe[d];
        if (lane == BX - 1) xp = xe[d];
        if (!in || k >= nz) continue;
        if (i == 0) xm = pc;
        if (i == nx - 1) xp = pc;
        const float2 y0 = j > 0 ? ym[d] : pc, y1 = j < ny - 1 ? yp[d] : pc;
        // Dirichlet ghost 2 v - phi (2 v is exact in the pair format)
        const float2 zm = k > 0 ? col[d] : df_sub(make_float2(2.0f * bc.v_lo.x, 2.0f * bc.v_lo.y), pc);
        const float2 zp = k < nz - 1 ? col[d + 2] : df_sub(make_float2(2.0f * bc.v_hi.x, 2.0f * bc.v_hi.y), pc);
        const float ex = -df_diff(xp, xm) * inv2h, ey = -df_diff(y1, y0) * inv2h, ez = -df_diff(zp, zm) * inv2h;
        const int c = c0 + k * pl;
        if (Ex) { Ex[c] = ex; Ey[c] = ey; Ez[c] = ez; }
        if (E4) reinterpret_cast<float4*>(E4)[c] = make_float4(ex, ey, ez, 0.0f);
        if (out_hi) { out_hi[c] = pc.x; out_lo[c] = pc.y; }
    }
}

// ---------------------------------------------------------------- device-driven loop
// One decision of the mixed solve's loop, the same as the host loop takes
// it: record the residual norm when a refinement pass starts; stop when
// ||r|| / ||b|| <= rtol or the cycle limit is reached (flagged); branch 3
// (commit the correction and re-form the residual) when the float32
// residual has dropped by kRefineDrop; else the CG iteration branch for the
// current index (0 first, 1 even, 2 odd).  The trip bound is a safeguard:
// every refinement is followed by an iteration or a stop, so the loop ends
// within 2 max_cycles + 1 trips.
__global__ void k_mx_decide(const double* __restrict__ sc, MxLoop* L, double rtol, int max_cycles,
                            double light_ratio, cudaGraphConditionalHandle h_loop,
                            cudaGraphConditionalHandle h_branch) {
    const double bn = sc[S_B2] > 0.0 ? sqrt(sc[S_B2]) : 1.0;
    const double rn = sqrt(sc[S_R2]);
    if (L->it == 0) L->r_pass = rn;
    L->rel = rn / bn;
    unsigned branch = kMxBranches;  // no branch
    bool stop = false;
    if (rn / bn <= rtol) {
        stop = true;
    } else if (L->cyc >= max_cycles || L->trips > 2 * max_cycles + 2) {
        stop = true;
        L->timeout = 1;
    } else if (L->it > 0 && rn <= kRefineDrop * L->r_pass) {
        branch = 3;
        L->it = 0;
    } else {
        const bool light = light_ratio > 0.0 && L->it > 0 && rn / bn <= light_ratio * rtol;
        branch = L->it == 0 ? 0u : (light ? 4u : 1u) + (unsigned)(L->it & 1);
        ++L->it;
        ++L->cyc;
    }
    ++L->trips;
    if (branch < (unsigned)kMxBranches) ++L->n_branch[branch];
    cudaGraphSetConditional(h_branch, branch);
    if (stop) cudaGraphSetConditional(h_loop, 0u);
}

// State after the first min_c iterations, which the graph runs back to back
// (as the host loop does: no test between them): the residual norm of the
// pass start, and the counters of the loop.
__global__ void k_mx_prime(const double* __restrict__ sc, MxLoop* L, int min_c) {
    L->r_pass = sqrt(sc[S_R2]);
    L->it = min_c;
    L->cyc = min_c;
    L->n_branch[0] = min_c > 0 ? 1 : 0;
    L->n_branch[2] = min_c > 1 ? 1 : 0;
}

// After the untested first iterations: whether the loop must run at all
// (the stop tests of k_mx_decide; its own first trip repeats them).
__global__ void k_mx_check(const double* __restrict__ sc, MxLoop* L, double rtol, int max_cycles,
                           cudaGraphConditionalHandle h_more) {
    const double bn = sc[S_B2] > 0.0 ? sqrt(sc[S_B2]) : 1.0;
    const double rn = sqrt(sc[S_R2]);
    L->rel = rn / bn;
    bool more = true;
    if (rn / bn <= rtol) {
        more = false;
    } else if (L->cyc >= max_cycles) {
        more = false;
        L->timeout = 1;
    }
    cudaGraphSetConditional(h_more, more ? 1u : 0u);
}

// Results of a device-driven solve: cycles, relative residual, the
// cycle-limit flag, and the kernels its loop ran (kb: per branch).
__global__ void k_mx_report(const MxLoop* __restrict__ L, int* cycles, double* rel, unsigned* err, unsigned bit,
                            unsigned long long* kernels, MxBranchKernels kb) {
    *cycles = L->cyc;
    *rel = L->rel;
    if (L->timeout) *err |= bit;
    unsigned long long k = (unsigned long long)L->trips;
    for (int b = 0; b < kMxBranches; ++b) k += (unsigned long long)L->n_branch[b] * kb.k[b];
    *kernels += k;
}

// float64 <-> float pair, for callers that hold the potential in float64.
__global__ void k_mx_split(const double* __restrict__ p, float* __restrict__ hi, float* __restrict__ lo, int n) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) {
        const double x = p[c];
        const float h = (float)x;
        hi[c] = h;
        lo[c] = (float)(x - (double)h);
    }
}
__global__ void k_mx_join(const float* __restrict__ hi, const float* __restrict__ lo, double* __restrict__ p, int n) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) p[c] = (double)hi[c] + (double)lo[c];
}
