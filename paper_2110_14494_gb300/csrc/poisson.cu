// Geometric multigrid Poisson solve with an embedded electrode mask.
//
// Sec. 2.5 of the paper: the field comes from Poisson's equation, solved with
// geometric multigrid, with the applied potential imposed on the electrode
// and E = -grad(phi).  Here the electrode is a mask of cells held at their
// potential (instead of a level set), the grid is uniform and cell-centred,
// the z faces are Dirichlet plates and the x, y faces homogeneous Neumann.
//
// Scheme: flexible conjugate gradients in float64 on the unmasked unknowns,
// preconditioned by one float32 V(2,2)-cycle (red-black Gauss-Seidel, 8-cell
// average restriction, trilinear prolongation, electrode cells and coarse
// cells touching the electrode held at zero), until ||b - A phi|| / ||b|| <=
// rtol.  A is the 7-point stencil scaled by h^2: diagonal 6 - (#Neumann faces)
// + (#Dirichlet faces), -1 per unmasked neighbour; b = h^2 rho / eps0 + plate
// and electrode terms.  The CG scalars stay on the device; the host reads the
// residual norm once per iteration.  Kernels map one thread to one cell with a
// (32, 4, 1) block over (x, y) and the z index in blockIdx.z.
#include <math.h>

#include "common.cuh"
#include "graph_util.cuh"
#include "poisson.cuh"

namespace pic {

namespace {

constexpr int BX = 32, BY = 4;

// Kernels of the V-cycle and of the CG iteration are launched with
// programmatic dependent launch: their blocks may be scheduled while the
// previous kernel's last blocks still run, and each waits here for that grid
// (and its memory) before its first access.  Without the launch attribute
// the wait returns at once.
__device__ __forceinline__ void pdl_wait() { cudaGridDependencySynchronize(); }

template <class... P, class... A>
void launch_pdl(void (*k)(P...), dim3 g, dim3 b, size_t smem, cudaStream_t s, A... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = g;
    cfg.blockDim = b;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k, args...);
}

__device__ __forceinline__ int lin(int i, int j, int k, int nx, int ny) { return (k * ny + j) * nx + i; }

// Block sum of a double into one atomicAdd (all threads of the block call).
__device__ __forceinline__ void block_add(double v, double* dst) {
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    const int t = threadIdx.x + threadIdx.y * blockDim.x;
    const int lane = t & 31, w = t >> 5, nw = (blockDim.x * blockDim.y) >> 5;
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (t == 0) {
        double s = 0.0;
        for (int q = 0; q < nw; ++q) s += red[q];
        if (s != 0.0) atomicAdd(dst, s);
    }
    __syncthreads();  // red[] is reused by the next call in the same kernel
}

// Scalars of the flexible CG, in device memory.
enum { S_B2 = 0, S_R2, S_RHO, S_GAM, S_T1, S_T2, S_ALPHA, S_BETA, S_N };

// Stencil sum of the neighbours of interior cell c (x, y Neumann mirror and
// z Dirichlet are folded into the diagonal; masked neighbours contribute 0).
template <class V>
__device__ __forceinline__ V nb_sum(const V* e, const uint8_t* m, int i, int j, int k, int nx, int ny, int nz, int c,
                                    V& diag) {
    const int pl = nx * ny;
    V s = (V)0;
    diag = (V)6;
    if (i > 0) { if (!m[c - 1]) s += e[c - 1]; } else diag -= (V)1;
    if (i < nx - 1) { if (!m[c + 1]) s += e[c + 1]; } else diag -= (V)1;
    if (j > 0) { if (!m[c - nx]) s += e[c - nx]; } else diag -= (V)1;
    if (j < ny - 1) { if (!m[c + nx]) s += e[c + nx]; } else diag -= (V)1;
    if (k > 0) { if (!m[c - pl]) s += e[c - pl]; } else diag += (V)1;
    if (k < nz - 1) { if (!m[c + pl]) s += e[c + pl]; } else diag += (V)1;
    return s;
}

#define CELL3D                                                   \
    const int i = blockIdx.x * BX + threadIdx.x;                 \
    const int j = blockIdx.y * BY + threadIdx.y;                 \
    const int k = blockIdx.z;                                    \
    const bool in = i < nx && j < ny;                            \
    const int c = in ? lin(i, j, k, nx, ny) : 0;

// Reducing kernels run a bounded grid (z extent kZRed) and loop over z.
constexpr int kZRed = 8;
#define CELL3D_LOOP_BEGIN                                        \
    const int i = blockIdx.x * BX + threadIdx.x;                 \
    const int j = blockIdx.y * BY + threadIdx.y;                 \
    const bool in = i < nx && j < ny;                            \
    double acc = 0.0;                                            \
    for (int k = blockIdx.z; k < nz; k += gridDim.z) {           \
        const int c = in ? lin(i, j, k, nx, ny) : 0;
#define CELL3D_LOOP_END }

// b = h^2 rho / eps0 + plate terms + electrode neighbours; accumulates ||b||^2.
__global__ void k_rhs_norm(const double* __restrict__ rho, const uint8_t* __restrict__ mask, int nx, int ny, int nz,
                           double h2e, double v_lo, double v_hi, double v_mask, double* sc) {
    CELL3D_LOOP_BEGIN
    if (in && !mask[c]) {
        const int pl = nx * ny;
        double s = h2e * rho[c];
        if (k == 0) s += 2.0 * v_lo;
        if (k == nz - 1) s += 2.0 * v_hi;
        if (i > 0 && mask[c - 1]) s += v_mask;
        if (i < nx - 1 && mask[c + 1]) s += v_mask;
        if (j > 0 && mask[c - nx]) s += v_mask;
        if (j < ny - 1 && mask[c + nx]) s += v_mask;
        if (k > 0 && mask[c - pl]) s += v_mask;
        if (k < nz - 1 && mask[c + pl]) s += v_mask;
        acc += s * s;
    }
    CELL3D_LOOP_END
    block_add(acc, sc + S_B2);
}

// r = b - A phi with the true boundary values (float64) and its float32 copy
// for the preconditioner; accumulates ||r||^2; electrode cells get phi = v_mask.
__global__ void k_resid64(double* __restrict__ phi, const double* __restrict__ rho, const uint8_t* __restrict__ mask,
                          int nx, int ny, int nz, double h2e, double v_lo, double v_hi, double v_mask,
                          double* __restrict__ r, float* __restrict__ g0, double* sc) {
    CELL3D_LOOP_BEGIN
    if (in) {
        if (mask[c]) {
            phi[c] = v_mask;
            r[c] = 0.0;
            g0[c] = 0.0f;
        } else {
            const int pl = nx * ny;
            const double pc = phi[c];
            auto val = [&](int q, bool inside, double ghost) -> double {
                if (!inside) return ghost;
                if (mask[q]) return v_mask;
                return phi[q];
            };
            const double sum = val(c - 1, i > 0, pc) + val(c + 1, i < nx - 1, pc) + val(c - nx, j > 0, pc) +
                               val(c + nx, j < ny - 1, pc) + val(c - pl, k > 0, 2.0 * v_lo - pc) +
                               val(c + pl, k < nz - 1, 2.0 * v_hi - pc);
            const double rr = h2e * rho[c] + sum - 6.0 * pc;
            r[c] = rr;
            g0[c] = (float)rr;
            acc += rr * rr;
        }
    }
    CELL3D_LOOP_END
    block_add(acc, sc + S_R2);
}

// q = A p (homogeneous boundary values) and p.q.
__global__ void k_apply(const double* __restrict__ p, const uint8_t* __restrict__ mask, int nx, int ny, int nz,
                        double* __restrict__ q, double* sc) {
    CELL3D_LOOP_BEGIN
    if (in) {
        if (mask[c]) {
            q[c] = 0.0;
        } else {
            double diag;
            const double s = nb_sum(p, mask, i, j, k, nx, ny, nz, c, diag);
            const double v = diag * p[c] - s;
            q[c] = v;
            acc += p[c] * v;
        }
    }
    CELL3D_LOOP_END
    block_add(acc, sc + S_GAM);
}

__global__ void k_alpha(double* sc) {
    sc[S_ALPHA] = sc[S_RHO] / sc[S_GAM];
    sc[S_R2] = 0.0;
    sc[S_T1] = 0.0;
    sc[S_T2] = 0.0;
}

// phi += alpha p; r -= alpha q; float32 copy of r; ||r||^2.
__global__ void k_update_xr(double* __restrict__ phi, double* __restrict__ r, const double* __restrict__ p,
                            const double* __restrict__ q, float* __restrict__ g0, int n, double* sc) {
    const double a = sc[S_ALPHA];
    double acc = 0.0;
    const int stride = gridDim.x * blockDim.x * blockDim.y;
    for (int c = (blockIdx.x * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x; c < n; c += stride) {
        phi[c] += a * p[c];
        const double rr = r[c] - a * q[c];
        r[c] = rr;
        g0[c] = (float)rr;
        acc += rr * rr;
    }
    block_add(acc, sc + S_R2);
}

// t1 = z.r, t2 = z.q with z the preconditioned residual (float32).
__global__ void k_dot2(const float* __restrict__ z, const double* __restrict__ r, const double* __restrict__ q, int n,
                       double* sc, int with_q) {
    const int stride = gridDim.x * blockDim.x * blockDim.y;
    double a = 0.0, b = 0.0;
    for (int c = (blockIdx.x * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x; c < n; c += stride) {
        const double zz = (double)z[c];
        a += zz * r[c];
        if (with_q) b += zz * q[c];
    }
    block_add(a, sc + S_T1);
    if (with_q) block_add(b, sc + S_T2);
}

// Flexible CG direction: beta = -alpha (z.q) / rho (equivalently
// z.(r_new - r_old) / rho), rho <- z.r.
__global__ void k_beta(double* sc, int first) {
    sc[S_BETA] = first ? 0.0 : -sc[S_ALPHA] * sc[S_T2] / sc[S_RHO];
    sc[S_RHO] = sc[S_T1];
    sc[S_GAM] = 0.0;
}

__global__ void k_update_p(double* __restrict__ p, const float* __restrict__ z, int n, const double* sc) {
    const double b = sc[S_BETA];
    const int c = (blockIdx.x * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x;
    if (c < n) p[c] = b != 0.0 ? (double)z[c] + b * p[c] : (double)z[c];
}

// Neighbour sum of the correction e, which is zero on electrode cells at
// every level (they are never updated, and prolongation writes 0 there), so
// the masks of the neighbours need not be read: all six loads are issued
// together.  Domain faces add nothing to the sum and change the diagonal as
// in nb_sum; the additions run in the same order, so the result is the same.
__device__ __forceinline__ float nb_sum_e(const float* __restrict__ e, int i, int j, int k, int nx, int ny, int nz,
                                          int c, float& diag) {
    const int pl = nx * ny;
    const float xm = i > 0 ? e[c - 1] : 0.0f, xp = i < nx - 1 ? e[c + 1] : 0.0f;
    const float ym = j > 0 ? e[c - nx] : 0.0f, yp = j < ny - 1 ? e[c + nx] : 0.0f;
    const float zm = k > 0 ? e[c - pl] : 0.0f, zp = k < nz - 1 ? e[c + pl] : 0.0f;
    diag = 6.0f - (float)((i == 0) + (i == nx - 1) + (j == 0) + (j == ny - 1)) + (float)((k == 0) + (k == nz - 1));
    return ((((xm + xp) + ym) + yp) + zm) + zp;
}

__device__ __forceinline__ float inv_diag(float diag) { return diag == 6.0f ? (1.0f / 6.0f) : 1.0f / diag; }

// One colour of red-black Gauss-Seidel for A e = g (masked cells stay 0).
// Thread (ii, j) handles ZS planes k0 .. k0 + ZS - 1, at each the cell
// i = 2 ii + ((j + k + colour) & 1).  All loads of the ZS cells (the other
// colour, not written by this launch) are issued before the first store.
// Large levels take ZS = 4 (fewer, longer threads); small ones ZS = 1 (more
// parallelism).  With omega != 1 the update is over-relaxed:
// e + omega ((g + s) / diag - e).
template <int ZS>
__global__ void __launch_bounds__(BX * BY) k_smooth(float* __restrict__ e, const float* __restrict__ g,
                                                    const uint8_t* __restrict__ mask, int nx, int ny, int nz,
                                                    int color, float omega) {
    pdl_wait();
    const int j = blockIdx.y * BY + threadIdx.y, k0 = blockIdx.z * ZS, ii = blockIdx.x * BX + threadIdx.x;
    if (j >= ny) return;
    const bool relax = omega != 1.0f;
    float s[ZS], gv[ZS], dg[ZS], eo[ZS];
    uint8_t mv[ZS];
    int cc[ZS];
#pragma unroll
    for (int d = 0; d < ZS; ++d) {
        const int k = k0 + d;
        const int i = 2 * ii + ((j + k + color) & 1);
        const bool ok = i < nx && k < nz;
        cc[d] = ok ? lin(i, j, k, nx, ny) : -1;
        s[d] = ok ? nb_sum_e(e, i, j, k, nx, ny, nz, cc[d], dg[d]) : 0.0f;
        gv[d] = ok ? g[cc[d]] : 0.0f;
        mv[d] = ok ? mask[cc[d]] : 1;
        eo[d] = ok && relax ? e[cc[d]] : 0.0f;
    }
#pragma unroll
    for (int d = 0; d < ZS; ++d)
        if (cc[d] >= 0 && !mv[d]) {
            const float v = (gv[d] + s[d]) * inv_diag(dg[d]);
            e[cc[d]] = relax ? fmaf(omega, v - eo[d], eo[d]) : v;
        }
}

__device__ __forceinline__ float diag_at(int i, int j, int k, int nx, int ny, int nz) {
    return 6.0f - (float)((i == 0) + (i == nx - 1) + (j == 0) + (j == ny - 1)) + (float)((k == 0) + (k == nz - 1));
}

// The first full red-black sweep of a V-cycle level, from e = 0, in one
// pass that needs no e: colour 0 cells get g * inv_diag (their neighbours
// are still 0), colour 1 cells get (g + sum of those colour-0 values at
// their neighbours) * inv_diag.  The same operations in the same order as a
// zero fill followed by two smooth_half launches, so the values are
// identical.  Thread (ii, j, k) takes the x pair (2 ii, 2 ii + 1) of row
// (j, k); the colour-0 value of the adjacent pair comes from the next or
// previous lane.  Electrode cells get 0.  With omega != 1 both values are
// scaled by omega (over-relaxation from e = 0).
__device__ __forceinline__ float first_red(const float* __restrict__ g, const uint8_t* __restrict__ mask, int i, int j,
                                           int k, int nx, int ny, int nz, float omega) {
    const int c = lin(i, j, k, nx, ny);
    const float zero = 0.0f;
    const float s = ((((zero + zero) + zero) + zero) + zero) + zero;
    const float v = (g[c] + s) * inv_diag(diag_at(i, j, k, nx, ny, nz));
    return mask[c] ? 0.0f : (omega != 1.0f ? omega * v : v);
}
__global__ void __launch_bounds__(BX * BY) k_sweep_first(float* __restrict__ e, const float* __restrict__ g,
                                                         const uint8_t* __restrict__ mask, int nx, int ny, int nz,
                                                         float omega) {
    pdl_wait();
    const int ii = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
    const int lane = threadIdx.x;
    const int par = (j + k) & 1;       // x offset of the colour-0 cell in the pair
    const int i0 = 2 * ii + par;       // colour 0
    const int i1 = 2 * ii + (1 - par); // colour 1
    const bool in = j < ny && 2 * ii < nx;
    const bool ok0 = in && i0 < nx, ok1 = in && i1 < nx;
    // colour-0 value of this pair, shared with the neighbouring lanes
    const float r0 = ok0 ? first_red(g, mask, i0, j, k, nx, ny, nz, omega) : 0.0f;
    // the colour-1 cell's x neighbours: one is this pair's colour-0 cell, the
    // other the adjacent pair's (previous pair when i1 < i0, else next)
    const float prev = __shfl_up_sync(kFull, r0, 1), next = __shfl_down_sync(kFull, r0, 1);
    if (!in) return;
    if (ok0) e[lin(i0, j, k, nx, ny)] = r0;
    if (!ok1) return;
    const int c1 = lin(i1, j, k, nx, ny);
    if (mask[c1]) {
        e[c1] = 0.0f;
        return;
    }
    // x neighbours of i1: i1 - 1 and i1 + 1
    float xm, xp;
    if (par == 1) {  // i1 = 2 ii: left neighbour in the previous pair, right one is i0
        xm = i1 > 0 ? (lane > 0 ? prev : first_red(g, mask, i1 - 1, j, k, nx, ny, nz, omega)) : 0.0f;
        xp = i0 < nx ? r0 : 0.0f;
    } else {         // i1 = 2 ii + 1: left neighbour is i0, right one in the next pair
        xm = r0;
        xp = i1 < nx - 1 ? (lane < BX - 1 ? next : first_red(g, mask, i1 + 1, j, k, nx, ny, nz, omega)) : 0.0f;
    }
    const float ym = j > 0 ? first_red(g, mask, i1, j - 1, k, nx, ny, nz, omega) : 0.0f;
    const float yp = j < ny - 1 ? first_red(g, mask, i1, j + 1, k, nx, ny, nz, omega) : 0.0f;
    const float zm = k > 0 ? first_red(g, mask, i1, j, k - 1, nx, ny, nz, omega) : 0.0f;
    const float zp = k < nz - 1 ? first_red(g, mask, i1, j, k + 1, nx, ny, nz, omega) : 0.0f;
    const float s = ((((xm + xp) + ym) + yp) + zm) + zp;
    const float v = (g[c1] + s) * inv_diag(diag_at(i1, j, k, nx, ny, nz));
    e[c1] = omega != 1.0f ? omega * v : v;
}

// Coarse right-hand side: g_c = 4 * mean of the 8 fine residuals g - A e
// (h^2 scaling: the coarse cell is twice as wide).  After a black half-sweep
// the residual of every black cell is zero (its value was just solved for
// from red neighbours that have not changed since), so with black_zero set
// only the four red children are evaluated.
__global__ void k_resid_restrict(const float* __restrict__ e, const float* __restrict__ g,
                                 const uint8_t* __restrict__ mask, int nx, int ny, int nz, float* __restrict__ gc,
                                 const uint8_t* __restrict__ maskc, int black_zero) {
    pdl_wait();
    const int cx = nx / 2, cy = ny / 2;
    const int I = blockIdx.x * BX + threadIdx.x, J = blockIdx.y * BY + threadIdx.y, K = blockIdx.z;
    if (I >= cx || J >= cy) return;
    const int q = lin(I, J, K, cx, cy);
    if (maskc[q]) { gc[q] = 0.0f; return; }
    float acc = 0.0f;
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        const int i = 2 * I + (d & 1), j = 2 * J + ((d >> 1) & 1), k = 2 * K + (d >> 2);
        // children of a coarse cell: (i + j + k) has the parity of d's bit count
        if (black_zero && (__popc(d) & 1)) continue;
        const int c = lin(i, j, k, nx, ny);
        float diag;
        const float s = nb_sum_e(e, i, j, k, nx, ny, nz, c, diag);
        const float r = g[c] - (diag * e[c] - s);
        acc += mask[c] ? 0.0f : r;
    }
    gc[q] = 0.5f * acc;
}

// Coarse value with ghost rules (Neumann mirror x, y; Dirichlet -e in z).
__device__ __forceinline__ float cval(const float* ec, int I, int J, int K, int cx, int cy, int cz) {
    float sgn = 1.0f;
    I = I < 0 ? 0 : (I >= cx ? cx - 1 : I);
    J = J < 0 ? 0 : (J >= cy ? cy - 1 : J);
    if (K < 0) { K = 0; sgn = -sgn; }
    if (K >= cz) { K = cz - 1; sgn = -sgn; }
    return sgn * ec[lin(I, J, K, cx, cy)];
}

// e_f += trilinear interpolation of e_c (weights 3/4, 1/4 per axis).  One
// thread per coarse cell writes its eight children from the 3x3x3 coarse
// neighbourhood; all loads are issued before the arithmetic.
__global__ void k_prolong_add(const float* __restrict__ ec, float* __restrict__ ef, const uint8_t* __restrict__ mask,
                              int nx, int ny, int nz) {
    pdl_wait();
    const int cx = nx / 2, cy = ny / 2, cz = nz / 2;
    const int I = blockIdx.x * BX + threadIdx.x, J = blockIdx.y * BY + threadIdx.y, K = blockIdx.z;
    if (I >= cx || J >= cy) return;
    float v[3][3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int d = 0; d < 3; ++d) v[a][b][d] = cval(ec, I + d - 1, J + b - 1, K + a - 1, cx, cy, cz);
    float fe[8];
    uint8_t fm[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int c = lin(2 * I + (q & 1), 2 * J + ((q >> 1) & 1), 2 * K + (q >> 2), nx, ny);
        fe[q] = ef[c];
        fm[q] = mask[c];
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int di = q & 1, dj = (q >> 1) & 1, dk = q >> 2;
        // the near coarse neighbour along each axis: -1 for the low child, +1 for the high one
        const int si = di ? 2 : 0, sj = dj ? 2 : 0, sk = dk ? 2 : 0;
        float acc = 0.0f;
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int d = 0; d < 2; ++d) {
                    const float wgt = (a ? 0.25f : 0.75f) * (b ? 0.25f : 0.75f) * (d ? 0.25f : 0.75f);
                    acc += wgt * v[a ? sk : 1][b ? sj : 1][d ? si : 1];
                }
        const int c = lin(2 * I + di, 2 * J + dj, 2 * K + dk, nx, ny);
        ef[c] = fm[q] ? 0.0f : fe[q] + acc;
    }
}

// Coarse mask: a coarse cell is held at zero if at least min_children of
// its 8 children are (1: any child).
__global__ void k_restrict_mask(const uint8_t* __restrict__ m, int nx, int ny, int nz, uint8_t* __restrict__ mc,
                                int min_children) {
    const int cx = nx / 2, cy = ny / 2;
    const int I = blockIdx.x * BX + threadIdx.x, J = blockIdx.y * BY + threadIdx.y, K = blockIdx.z;
    if (I >= cx || J >= cy) return;
    int v = 0;
#pragma unroll
    for (int d = 0; d < 8; ++d) v += m[lin(2 * I + (d & 1), 2 * J + ((d >> 1) & 1), 2 * K + (d >> 2), nx, ny)] ? 1 : 0;
    mc[lin(I, J, K, cx, cy)] = v >= min_children ? 1 : 0;
}

__global__ void k_copy_mask(const uint8_t* __restrict__ m, uint8_t* __restrict__ out, int n) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) out[c] = m ? (m[c] ? 1 : 0) : 0;
}


// The small levels of the hierarchy (from level t down to the coarsest; the
// first of them has at most kTailCells cells) run as one block in shared
// memory: pre-smooth, restrict, ... coarse sweeps ... prolong, post-smooth,
// with barriers between the phases instead of kernel launches.  Threads map
// to cells through a fixed 3D decomposition (no integer division); levels of
// at most kWarpCells cells run on warp 0 alone with warp barriers.  The block
// reads g and the masks of level t from global memory and writes back e of
// level t.
constexpr int kTailCells = 8192;
constexpr int kWarpCells = 64;

struct TailLevels {
    float* e_first;          // global e of level `first`
    const float* g_first;    // global g of level `first`
    const uint8_t* m[12];    // global masks
    int nx[12], ny[12], nz[12], off[12];  // shared-memory offsets (cells)
    int first, last, warp_from, pre, post, coarse, total;
    float omega;             // over-relaxation of the pre- and post-smoothing sweeps
};

struct TailSmem {
    float* e;
    float* g;
    uint8_t* m;
    float* rdiag;  // [16]: inv_diag(d) for the integer diagonals d = 0..15
};
__host__ __device__ constexpr size_t tail_smem_bytes(int cells) { return (((size_t)cells * (2 * sizeof(float) + 1) + 15) & ~(size_t)15) + 16 * sizeof(float); }

// Thread decomposition of a phase: thread owns (tx + a sx, ty + b sy, tz + c sz).
struct Dec {
    int tx, ty, tz, sx, sy, sz;
    bool on;
};
__device__ __forceinline__ Dec dec_block() {
    const int t = threadIdx.x;
    return Dec{t & 7, (t >> 3) & 7, t >> 6, 8, 8, 16, true};
}
__device__ __forceinline__ Dec dec_warp() {
    const int t = threadIdx.x;
    return Dec{t & 1, (t >> 1) & 3, (t >> 3) & 3, 2, 4, 4, t < 32};
}
template <bool WARP> __device__ __forceinline__ void tail_sync() {
    if (WARP) __syncwarp(); else __syncthreads();
}

template <bool WARP>
__device__ void tail_half(const TailLevels& T, const TailSmem& S, int l, int color, const Dec& D, float omega) {
    const int nx = T.nx[l], ny = T.ny[l], nz = T.nz[l], hx = (nx + 1) / 2, o = T.off[l];
    float* e = S.e + o;
    const float* g = S.g + o;
    const uint8_t* m = S.m + o;
    if (D.on)
        for (int k = D.tz; k < nz; k += D.sz)
            for (int j = D.ty; j < ny; j += D.sy)
                for (int ii = D.tx; ii < hx; ii += D.sx) {
                    const int i = 2 * ii + ((j + k + color) & 1);
                    if (i >= nx) continue;
                    const int c = lin(i, j, k, nx, ny);
                    float diag;
                    const float s = nb_sum_e(e, i, j, k, nx, ny, nz, c, diag);
                    if (!m[c]) {
                        // the diagonal is an integer (2..8): its reciprocal from the table (the same values)
                        const float v = (g[c] + s) * S.rdiag[(int)diag];
                        e[c] = omega != 1.0f ? fmaf(omega, v - e[c], e[c]) : v;
                    }
                }
    tail_sync<WARP>();
}

// Residual of level l restricted into the right-hand side of level l + 1.
template <bool WARP> __device__ void tail_restrict(const TailLevels& T, const TailSmem& S, int l, const Dec& D) {
    const int nx = T.nx[l], ny = T.ny[l], nz = T.nz[l];
    const int cx = nx / 2, cy = ny / 2, cz = nz / 2;
    const float* e = S.e + T.off[l];
    const float* g = S.g + T.off[l];
    const uint8_t* m = S.m + T.off[l];
    float* gc = S.g + T.off[l + 1];
    const uint8_t* mc = S.m + T.off[l + 1];
    const bool black_zero = T.pre > 0;
    if (D.on)
        for (int K = D.tz; K < cz; K += D.sz)
            for (int J = D.ty; J < cy; J += D.sy)
                for (int I = D.tx; I < cx; I += D.sx) {
                    const int q = lin(I, J, K, cx, cy);
                    float acc = 0.0f;
                    if (!mc[q])
                        for (int d = 0; d < 8; ++d) {
                            if (black_zero && (__popc(d) & 1)) continue;
                            const int i = 2 * I + (d & 1), j = 2 * J + ((d >> 1) & 1), k = 2 * K + (d >> 2);
                            const int c = lin(i, j, k, nx, ny);
                            if (m[c]) continue;
                            float diag;
                            const float s = nb_sum_e(e, i, j, k, nx, ny, nz, c, diag);
                            acc += g[c] - (diag * e[c] - s);
                        }
                    gc[q] = 0.5f * acc;
                }
    tail_sync<WARP>();
}

// e_l += trilinear interpolation of e_{l+1}.
template <bool WARP> __device__ void tail_prolong(const TailLevels& T, const TailSmem& S, int l, const Dec& D) {
    const int nx = T.nx[l], ny = T.ny[l], nz = T.nz[l];
    const int cx = nx / 2, cy = ny / 2, cz = nz / 2;
    float* e = S.e + T.off[l];
    const float* ec = S.e + T.off[l + 1];
    const uint8_t* m = S.m + T.off[l];
    if (D.on)
        for (int k = D.tz; k < nz; k += D.sz)
            for (int j = D.ty; j < ny; j += D.sy)
                for (int i = D.tx; i < nx; i += D.sx) {
                    const int c = lin(i, j, k, nx, ny);
                    if (m[c]) continue;
                    const int I = i >> 1, J = j >> 1, K = k >> 1;
                    const int si = (i & 1) ? 1 : -1, sj = (j & 1) ? 1 : -1, sk = (k & 1) ? 1 : -1;
                    float acc = 0.0f;
                    for (int a = 0; a < 2; ++a)
                        for (int b = 0; b < 2; ++b)
                            for (int d = 0; d < 2; ++d) {
                                const float wgt = (a ? 0.25f : 0.75f) * (b ? 0.25f : 0.75f) * (d ? 0.25f : 0.75f);
                                acc += wgt * cval(ec, I + (d ? si : 0), J + (b ? sj : 0), K + (a ? sk : 0), cx, cy, cz);
                            }
                    e[c] += acc;
                }
    tail_sync<WARP>();
}

template <bool WARP> __device__ void tail_down(const TailLevels& T, const TailSmem& S, int l, const Dec& D) {
    for (int s = 0; s < T.pre; ++s) { tail_half<WARP>(T, S, l, 0, D, T.omega); tail_half<WARP>(T, S, l, 1, D, T.omega); }
    tail_restrict<WARP>(T, S, l, D);
}
template <bool WARP> __device__ void tail_up(const TailLevels& T, const TailSmem& S, int l, const Dec& D) {
    tail_prolong<WARP>(T, S, l, D);
    for (int s = 0; s < T.post; ++s) { tail_half<WARP>(T, S, l, 1, D, T.omega); tail_half<WARP>(T, S, l, 0, D, T.omega); }
}
template <bool WARP> __device__ void tail_coarse(const TailLevels& T, const TailSmem& S, const Dec& D) {
    for (int s = 0; s < T.coarse; ++s) {
        tail_half<WARP>(T, S, T.last, 0, D, 1.0f);
        tail_half<WARP>(T, S, T.last, 1, D, 1.0f);
    }
}

__global__ void __launch_bounds__(1024) k_tail_vcycle(const TailLevels T) {
    pdl_wait();
    extern __shared__ __align__(16) unsigned char tail_raw[];
    TailSmem S;
    S.e = reinterpret_cast<float*>(tail_raw);
    S.g = S.e + T.total;
    S.m = reinterpret_cast<uint8_t*>(S.g + T.total);
    S.rdiag = reinterpret_cast<float*>(tail_raw + (tail_smem_bytes(T.total) - 16 * sizeof(float)));
    if (threadIdx.x < 16) S.rdiag[threadIdx.x] = inv_diag((float)threadIdx.x);
    {
        // every global load (the first level's g, the masks of all levels as
        // one run of T.total bytes) issued before the first store: one round
        // trip (the first level has at most kTailCells cells, the masks
        // together fewer than 2 kTailCells)
        constexpr int kTailLoad = kTailCells / 1024;
        const int n0 = T.nx[T.first] * T.ny[T.first] * T.nz[T.first];
        float gv[kTailLoad];
        uint8_t mv[2 * kTailLoad];
#pragma unroll
        for (int u = 0; u < kTailLoad; ++u) {
            const int c = threadIdx.x + u * 1024;
            gv[u] = c < n0 ? T.g_first[c] : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < 2 * kTailLoad; ++u) {
            const int c = threadIdx.x + u * 1024;
            mv[u] = 0;
            if (c < T.total) {
                int l = T.first;
                while (l < T.last && c >= T.off[l + 1]) ++l;
                mv[u] = T.m[l][c - T.off[l]];
            }
        }
#pragma unroll
        for (int u = 0; u < 2 * kTailLoad; ++u) {
            const int c = threadIdx.x + u * 1024;
            if (c < T.total) S.m[c] = mv[u];
        }
#pragma unroll
        for (int u = 0; u < kTailLoad; ++u) {
            const int c = threadIdx.x + u * 1024;
            if (c < n0) S.g[T.off[T.first] + c] = gv[u];
        }
        // a hierarchy of one level may have more cells than the batches cover
        for (int c = threadIdx.x + kTailCells; c < n0; c += 1024) S.g[T.off[T.first] + c] = T.g_first[c];
        for (int c = threadIdx.x + 2 * kTailCells; c < T.total; c += 1024) {
            int l = T.first;
            while (l < T.last && c >= T.off[l + 1]) ++l;
            S.m[c] = T.m[l][c - T.off[l]];
        }
        for (int c = threadIdx.x; c < T.total; c += blockDim.x) S.e[c] = 0.0f;
    }
    __syncthreads();
    const Dec DB = dec_block(), DW = dec_warp();
    const int wl = T.warp_from;  // first level run by warp 0 alone (last + 1: none)
    for (int l = T.first; l < wl && l < T.last; ++l) tail_down<false>(T, S, l, DB);
    if (wl > T.last) {
        tail_coarse<false>(T, S, DB);
    } else if (threadIdx.x < 32) {
        for (int l = wl; l < T.last; ++l) tail_down<true>(T, S, l, DW);
        tail_coarse<true>(T, S, DW);
        for (int l = T.last - 1; l >= wl; --l) tail_up<true>(T, S, l, DW);
    }
    __syncthreads();
    for (int l = (wl > T.last ? T.last : wl) - 1; l >= T.first; --l) tail_up<false>(T, S, l, DB);
    const int n0 = T.nx[T.first] * T.ny[T.first] * T.nz[T.first];
    for (int c = threadIdx.x; c < n0; c += blockDim.x) T.e_first[c] = S.e[T.off[T.first] + c];
}

// E = -grad(phi) at cell centres with the stencil's ghost values; writes any
// of the float planes and a packed [n][4] copy in T.
template <class T>
__global__ void k_grad(const double* __restrict__ phi, int nx, int ny, int nz, double h, double v_lo, double v_hi,
                       float* Ex, float* Ey, float* Ez, T* E4) {
    CELL3D
    if (!in) return;
    const int pl = nx * ny;
    const double inv = 1.0 / (2.0 * h);
    const double pc = phi[c];
    const double xm = i > 0 ? phi[c - 1] : pc, xp = i < nx - 1 ? phi[c + 1] : pc;
    const double ym = j > 0 ? phi[c - nx] : pc, yp = j < ny - 1 ? phi[c + nx] : pc;
    const double zm = k > 0 ? phi[c - pl] : 2.0 * v_lo - pc, zp = k < nz - 1 ? phi[c + pl] : 2.0 * v_hi - pc;
    const double ex = -(xp - xm) * inv, ey = -(yp - ym) * inv, ez = -(zp - zm) * inv;
    if (Ex) { Ex[c] = (float)ex; Ey[c] = (float)ey; Ez[c] = (float)ez; }
    if (E4) { E4[4 * c] = (T)ex; E4[4 * c + 1] = (T)ey; E4[4 * c + 2] = (T)ez; E4[4 * c + 3] = (T)0; }
}

#include "poisson_mixed.cuh"

dim3 grid3(int nx, int ny, int nz) { return dim3((nx + BX - 1) / BX, (ny + BY - 1) / BY, nz); }
const dim3 kBlk(BX, BY, 1);
constexpr long long kSmoothDeep = 1ll << 20;  // levels with at least this many cells use 4 planes per thread
void smooth_half(float* e, const float* g, const uint8_t* m, int nx, int ny, int nz, int color, float omega,
                 cudaStream_t s) {
    const int zs = (long long)nx * ny * nz >= kSmoothDeep ? 4 : 1;
    const dim3 gr(((nx + 1) / 2 + BX - 1) / BX, (ny + BY - 1) / BY, (nz + zs - 1) / zs);
    if (zs == 4) launch_pdl(k_smooth<4>, gr, kBlk, 0, s, e, g, m, nx, ny, nz, color, omega);
    else launch_pdl(k_smooth<1>, gr, kBlk, 0, s, e, g, m, nx, ny, nz, color, omega);
}
dim3 grid_flat(long long n) { return dim3((unsigned)((n + BX * BY - 1) / (BX * BY))); }
dim3 grid_red(long long n) {
    long long b = (n + BX * BY - 1) / (BX * BY);
    return dim3((unsigned)(b < 1216 ? b : 1216));
}
dim3 grid3_red(int nx, int ny, int nz) { return dim3((nx + BX - 1) / BX, (ny + BY - 1) / BY, nz < kZRed ? nz : kZRed); }

}  // namespace

// ------------------------------------------------------------------ host side
static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

void MG::plan(int nx_, int ny_, int nz_) {
    levels = 0;
    int x = nx_, y = ny_, z = nz_;
    for (;;) {
        lx[levels] = x; ly[levels] = y; lz[levels] = z;
        ++levels;
        if (levels >= kMaxLevels) break;
        if ((x % 2) || (y % 2) || (z % 2)) break;
        if (x < 4 || y < 4 || z < 4) break;
        x /= 2; y /= 2; z /= 2;
    }
}

bool MG::supported(int nx_, int ny_, int nz_) {
    if (nx_ < 2 || ny_ < 2 || nz_ < 2 || nz_ > 65535) return false;
    if ((long long)nx_ * ny_ * nz_ > 0x7fffffffLL) return false;
    MG m;
    m.plan(nx_, ny_, nz_);
    const int L = m.levels - 1;
    return (long long)m.lx[L] * m.ly[L] * m.lz[L] * 9 <= 200 * 1024;
}

size_t MG::bytes(int nx_, int ny_, int nz_, bool mixed_, bool pair_copy) {
    MG m;
    return m.carve(nullptr, nx_, ny_, nz_, mixed_, pair_copy);
}

// Lays the buffers out from base (base null: sizes only); returns the bytes.
size_t MG::carve(void* base, int nx_, int ny_, int nz_, bool mixed_, bool pair_copy) {
    plan(nx_, ny_, nz_);
    mixed = mixed_;
    uintptr_t p = (uintptr_t)base;
    const uintptr_t p0 = p;
    auto take = [&](size_t nb) {
        void* r = (void*)p;
        p += align256(nb);
        return r;
    };
    norms = (double*)take(S_N * 8);
    const size_t n0 = (size_t)nx_ * ny_ * nz_;
    if (mixed_) {
        d32 = (float*)take(n0 * 4);
        p32[0] = (float*)take(n0 * 4);
        p32[1] = (float*)take(n0 * 4);
        q32 = (float*)take(n0 * 4);
        // hi then lo, each 256-byte aligned (the pair kernels use 16-byte loads)
        phi_pair = pair_copy ? (float*)take(2 * align256(n0 * 4)) : nullptr;
        ctr = (unsigned*)take(8 * sizeof(unsigned));
        loop = (MxLoop*)take(sizeof(MxLoop));
        const size_t b3 = (size_t)((nx_ + BX - 1) / BX) * ((ny_ + BY - 1) / BY) * ((nz_ + ZC - 1) / ZC);
        const size_t bf = (n0 + kFlatBlock * kFlatPer - 1) / (kFlatBlock * kFlatPer);
        part = (double*)take(3 * 8 * (b3 > bf ? b3 : bf));  // up to three partial sums per block
        r64 = p64 = q64 = nullptr;
    } else {
        loop = nullptr;
        r64 = (double*)take(n0 * 8);
        p64 = (double*)take(n0 * 8);
        q64 = (double*)take(n0 * 8);
    }
    for (int l = 0; l < levels; ++l) {
        const size_t n = (size_t)lx[l] * ly[l] * lz[l];
        e[l] = (float*)take(n * sizeof(float));
        g[l] = (float*)take(n * sizeof(float));
        m[l] = (uint8_t*)take(n);
    }
    return (size_t)(p - p0);
}

// First level handled by the single-block tail: at most kTailCells cells,
// and the tail's levels must fit in shared memory together.
int MG::tail_level() const {
    int t = 0;
    while (t < levels - 1 && (long long)lx[t] * ly[t] * lz[t] > kTailCells) ++t;
    while (t < levels - 1) {
        long long cells = 0;
        for (int l = t; l < levels; ++l) cells += (long long)lx[l] * ly[l] * lz[l];
        if (cells * 9 <= 200 * 1024) break;
        ++t;
    }
    return t;
}


cudaError_t MG::build_masks(const uint8_t* mask, cudaStream_t s) {
    const long long n0 = (long long)lx[0] * ly[0] * lz[0];
    launches += levels;
    k_copy_mask<<<(unsigned)((n0 + 255) / 256), 256, 0, s>>>(mask, m[0], (int)n0);
    for (int l = 1; l < levels; ++l)
        k_restrict_mask<<<grid3(lx[l], ly[l], lz[l]), kBlk, 0, s>>>(m[l - 1], lx[l - 1], ly[l - 1], lz[l - 1], m[l],
                                                                    mask_min_children);
    return cudaGetLastError();
}

// One V(pre, post)-cycle on A e0 = g0 (light: V(light_pre, light_post)); e0 is overwritten.  Levels above the
// tail run as separate kernels; the tail runs as one block.
void MG::vcycle(cudaStream_t s, bool light) {
    const int t = tail_level();
    const int pre = light ? light_pre : this->pre, post = light ? light_post : this->post;
    // per level: pre-smoothing (the first sweep from zero is one kernel), restriction, prolongation,
    // post-smoothing; then the tail
    launches += (long long)t * ((pre > 0 ? 2 * pre - 1 : 0) + 2 * post + 2) + 1;
    for (int l = 0; l < t; ++l) {
        const long long n = (long long)lx[l] * ly[l] * lz[l];
        if (pre > 0) {
            launch_pdl(k_sweep_first, dim3(((lx[l] + 1) / 2 + BX - 1) / BX, (ly[l] + BY - 1) / BY, lz[l]), kBlk, 0,
                       s, e[l], (const float*)g[l], (const uint8_t*)m[l], lx[l], ly[l], lz[l], omega);
        } else {
            cudaMemsetAsync(e[l], 0, n * sizeof(float), s);
        }
        for (int it = 1; it < pre; ++it) {
            smooth_half(e[l], g[l], m[l], lx[l], ly[l], lz[l], 0, omega, s);
            smooth_half(e[l], g[l], m[l], lx[l], ly[l], lz[l], 1, omega, s);
        }
        launch_pdl(k_resid_restrict, grid3(lx[l + 1], ly[l + 1], lz[l + 1]), kBlk, 0, s, (const float*)e[l],
                   (const float*)g[l], (const uint8_t*)m[l], lx[l], ly[l], lz[l], g[l + 1], (const uint8_t*)m[l + 1],
                   pre > 0 ? 1 : 0);
    }
    TailLevels T;
    int off = 0;
    for (int l = 0; l < levels; ++l) {
        T.m[l] = m[l];
        T.nx[l] = lx[l]; T.ny[l] = ly[l]; T.nz[l] = lz[l];
        T.off[l] = off;
        if (l >= t) off += lx[l] * ly[l] * lz[l];
    }
    T.e_first = e[t];
    T.g_first = g[t];
    T.first = t;
    T.last = levels - 1;
    T.warp_from = levels;
    for (int l = levels - 1; l >= t && (long long)lx[l] * ly[l] * lz[l] <= kWarpCells; --l) T.warp_from = l;
    T.pre = pre;
    T.post = post;
    T.coarse = coarse_sweeps;
    T.omega = omega;
    T.total = off;
    const size_t smem = tail_smem_bytes(off);
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_tail_vcycle, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    launch_pdl(k_tail_vcycle, dim3(1), dim3(1024), smem, s, T);
    for (int l = t - 1; l >= 0; --l) {
        launch_pdl(k_prolong_add, grid3(lx[l + 1], ly[l + 1], lz[l + 1]), kBlk, 0, s, (const float*)e[l + 1], e[l],
                   (const uint8_t*)m[l], lx[l], ly[l], lz[l]);
        for (int it = 0; it < post; ++it) {
            smooth_half(e[l], g[l], m[l], lx[l], ly[l], lz[l], 1, omega, s);
            smooth_half(e[l], g[l], m[l], lx[l], ly[l], lz[l], 0, omega, s);
        }
    }
}

// One flexible-CG iteration: z = M r, direction, q = A p, alpha, updates.
void MG::iteration(cudaStream_t s, double* phi, const uint8_t* mk, bool first) {
    const int nx = lx[0], ny = ly[0], nz = lz[0];
    const int n = nx * ny * nz;
    vcycle(s, false);
    k_dot2<<<grid_red(n), kBlk, 0, s>>>(e[0], r64, q64, n, norms, first ? 0 : 1);
    k_beta<<<1, 1, 0, s>>>(norms, first ? 1 : 0);
    k_update_p<<<grid_flat(n), kBlk, 0, s>>>(p64, e[0], n, norms);
    k_apply<<<grid3_red(nx, ny, nz), kBlk, 0, s>>>(p64, mk, nx, ny, nz, q64, norms);
    k_alpha<<<1, 1, 0, s>>>(norms);
    k_update_xr<<<grid_red(n), kBlk, 0, s>>>(phi, r64, p64, q64, g[0], n, norms);
    launches += 6;
}

void MG::release() {
    for (int q = 0; q < 2; ++q)
        if (g_iter[q]) { cudaGraphExecDestroy(g_iter[q]); g_iter[q] = nullptr; }
    for (int q = 0; q < 3; ++q)
        if (cap_body[q]) { cudaStreamDestroy(cap_body[q]); cap_body[q] = nullptr; }
    for (int q = 0; q < 5; ++q)
        if (g_mx[q]) { cudaGraphExecDestroy(g_mx[q]); g_mx[q] = nullptr; }
    if (cap_stream) { cudaStreamDestroy(cap_stream); cap_stream = nullptr; }
}

int MG::solve(const double* rho, const uint8_t* mask, double* phi, double h, double v_lo, double v_hi, double v_mask,
              double rtol, int max_cycles, int packed_prec, void* E4, float* Ex, float* Ey, float* Ez,
              cudaStream_t s, int* cycles_out, double* rel_out, double* host_norms) {
    const int nx = lx[0], ny = ly[0], nz = lz[0];
    const double h2e = h * h / kEps0;
    if (!persistent || !masks_ready) {
        if (build_masks(mask, s) != cudaSuccess) return PIC_ERR_CUDA;
        masks_ready = true;
    }
    const uint8_t* mk = m[0];
    // graphs are tied to the pointers they were captured with
    if (persistent && (g_key[0] != phi || g_key[1] != rho || g_key[2] != mask)) {
        for (int q = 0; q < 2; ++q)
            if (g_iter[q]) { cudaGraphExecDestroy(g_iter[q]); g_iter[q] = nullptr; }
        g_key[0] = phi; g_key[1] = rho; g_key[2] = mask;
    }
    cudaMemsetAsync(norms, 0, S_N * 8, s);
    k_rhs_norm<<<grid3_red(nx, ny, nz), kBlk, 0, s>>>(rho, mk, nx, ny, nz, h2e, v_lo, v_hi, v_mask, norms);
    k_resid64<<<grid3_red(nx, ny, nz), kBlk, 0, s>>>(phi, rho, mk, nx, ny, nz, h2e, v_lo, v_hi, v_mask, r64, g[0], norms);
    launches += 2;
    int cyc = 0, rc = PIC_OK;
    double bn = 1.0, rn = 0.0;
    for (;;) {
        if (cudaMemcpyAsync(host_norms, norms, 2 * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess) return PIC_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return PIC_ERR_CUDA;
        bn = host_norms[S_B2] > 0.0 ? sqrt(host_norms[S_B2]) : 1.0;
        rn = sqrt(host_norms[S_R2]);
        if (rn / bn <= rtol) break;
        if (cyc >= max_cycles) { rc = PIC_ERR_TIMEOUT; break; }
        // z = M r (float32 V-cycle on g0), then the CG direction
        const int gi = cyc == 0 ? 0 : 1;
        if (persistent) {
            if (!g_iter[gi]) {
                if (!cap_stream && cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking) != cudaSuccess)
                    return PIC_ERR_CUDA;
                cudaGraph_t gr = nullptr;
                const long long l0 = launches;
                if (cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
                    return PIC_ERR_CUDA;
                iteration(cap_stream, phi, mk, cyc == 0);
                if (cudaStreamEndCapture(cap_stream, &gr) != cudaSuccess) return PIC_ERR_CUDA;
                if (cudaGraphInstantiate(&g_iter[gi], gr, 0) != cudaSuccess) { cudaGraphDestroy(gr); return PIC_ERR_CUDA; }
                cudaGraphDestroy(gr);
                graph_kernels[gi] = launches - l0;
                launches = l0;
            }
            if (cudaGraphLaunch(g_iter[gi], s) != cudaSuccess) return PIC_ERR_CUDA;
            launches += graph_kernels[gi];
        } else {
            iteration(s, phi, mk, cyc == 0);
        }
        ++cyc;
    }
    if (cycles_out) *cycles_out = cyc;
    if (rel_out) *rel_out = rn / bn;
    if (Ex || E4) {
        ++launches;
        if (packed_prec == 64)
            k_grad<double><<<grid3(nx, ny, nz), kBlk, 0, s>>>(phi, nx, ny, nz, h, v_lo, v_hi, Ex, Ey, Ez, (double*)E4);
        else
            k_grad<float><<<grid3(nx, ny, nz), kBlk, 0, s>>>(phi, nx, ny, nz, h, v_lo, v_hi, Ex, Ey, Ez, (float*)E4);
    }
    if (cudaGetLastError() != cudaSuccess) return PIC_ERR_CUDA;
    return rc;
}


// ------------------------------------------------------------------ mixed precision
namespace {
dim3 grid_mx3(int nx, int ny, int nz) { return dim3((nx + BX - 1) / BX, (ny + BY - 1) / BY, (nz + ZC - 1) / ZC); }
// the float4 stencil kernels: four x cells per thread (nx % 4 == 0)
dim3 grid_mx3v(int nx, int ny, int nz) {
    return dim3((nx / 4 + BX - 1) / BX, (ny + BY - 1) / BY, (nz + ZC - 1) / ZC);
}
dim3 grid_mxf(long long n) {
    const long long b = (n / 4 + kFlatBlock * kFlatPer - 1) / (kFlatBlock * kFlatPer);
    return dim3((unsigned)(b > 0 ? b : 1));
}
float2 pair_of(double v) {
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
}
}  // namespace

// One flexible-CG iteration on the float32 correction (it: index within the
// current refinement pass; the direction vectors alternate between p32[0]
// and p32[1] so the new direction can be formed while the old one is read).
int MG::mixed_min_cycles(int max_cycles) const {
    int m = min_cycles < 2 ? min_cycles : 2;
    if (m < 0) m = 0;
    return m < max_cycles ? m : max_cycles;
}

void MG::iteration_mixed(cudaStream_t s, int it, bool light) {
    const int nx = lx[0], ny = ly[0], nz = lz[0], n = nx * ny * nz;
    const int cur = it & 1, first = it == 0 ? 1 : 0;
    vcycle(s, light);
    // w = A z goes to p32[cur] (the direction of two iterations ago, free
    // here), where the second kernel replaces it by the new direction
    if (nx % 4 == 0)
        launch_pdl(k_mx_apply4, grid_mx3v(nx, ny, nz), kBlk, 0, s, (const float*)e[0], (const float*)g[0],
                   (const float*)q32, p32[cur], (const uint8_t*)m[0], nx, ny, nz, first, part, ctr + 1, norms);
    else
        launch_pdl(k_mx_apply, grid_mx3(nx, ny, nz), kBlk, 0, s, (const float*)e[0], (const float*)g[0],
                   (const float*)q32, p32[cur], (const uint8_t*)m[0], nx, ny, nz, first, part, ctr + 1, norms);
    launch_pdl(k_mx_step, grid_mxf(n), dim3(kFlatBlock), 0, s, (const float*)e[0], (const float*)p32[cur ^ 1],
               p32[cur], q32, d32, g[0], n, first, part, ctr + 3, norms);
    launches += 2;
}

void MG::extrapolate_pair(const float* ch, const float* cl, const float* ph, const float* pl, float* oh, float* ol,
                          int n, bool have_prev, cudaStream_t s) {
    k_mx_extrapolate<<<grid_mxf(n), kFlatBlock, 0, s>>>(ch, cl, ph, pl, oh, ol, n, have_prev ? 1 : 0);
    ++launches;
}

int MG::solve_mixed(const void* rho, bool rho64, const uint8_t* mask, float* phi_hi, float* phi_lo, float* out_hi,
                    float* out_lo, bool fix_mask, double h, double v_lo, double v_hi, double v_mask, double rtol, int max_cycles,
                    float* E4, float* Ex, float* Ey, float* Ez, cudaStream_t s, int* cycles_out, double* rel_out,
                    double* host_norms) {
    if (!mixed) return PIC_ERR_STATE;
    const int nx = lx[0], ny = ly[0], nz = lz[0], n = nx * ny * nz;
    if (!persistent || !masks_ready) {
        if (build_masks(mask, s) != cudaSuccess) return PIC_ERR_CUDA;
        masks_ready = true;
    }
    const MxBoundary bc{pair_of(v_lo), pair_of(v_hi), pair_of(v_mask)};
    const double h2e = h * h / kEps0;
    const dim3 g3 = grid_mx3(nx, ny, nz), gf = grid_mxf(n);
    if (cudaMemsetAsync(ctr, 0, 8 * sizeof(unsigned), s) != cudaSuccess) return PIC_ERR_CUDA;
    if (fix_mask) {
        k_mx_fix_mask<<<(n + 255) / 256, 256, 0, s>>>(m[0], phi_hi, phi_lo, n, bc.v_mask);
        ++launches;
    }
    auto resid = [&]() {
        if (rho64)
            k_mx_resid<double><<<g3, kBlk, 0, s>>>((const double*)rho, h2e, m[0], phi_hi, phi_lo, nx, ny, nz, bc, g[0],
                                                   part, ctr, norms);
        else
            k_mx_resid<float><<<g3, kBlk, 0, s>>>((const float*)rho, 1.0, m[0], phi_hi, phi_lo, nx, ny, nz, bc, g[0],
                                                  part, ctr, norms);
        ++launches;
    };
    resid();
    int cyc = 0, it = 0, rc = PIC_OK;
    double bn = 1.0, rn = 0.0, r_pass = 0.0;
    const int min_c = mixed_min_cycles(max_cycles);
    for (;;) {
        // the first min_c iterations run without a test between them (no read-back)
        if (cyc == 0 || cyc >= min_c) {
            if (cudaMemcpyAsync(host_norms, norms, 2 * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess)
                return PIC_ERR_CUDA;
            if (cudaStreamSynchronize(s) != cudaSuccess) return PIC_ERR_CUDA;
            bn = host_norms[S_B2] > 0.0 ? sqrt(host_norms[S_B2]) : 1.0;
            rn = sqrt(host_norms[S_R2]);
        }
        if (it == 0) r_pass = rn;
        if (cyc >= min_c && rn / bn <= rtol) break;
        if (cyc >= max_cycles) { rc = PIC_ERR_TIMEOUT; break; }
        if (cyc >= min_c && it > 0 && rn <= kRefineDrop * r_pass) {
            // iterative refinement: fold the correction into phi, re-form r
            k_mx_commit<<<gf, kFlatBlock, 0, s>>>(phi_hi, phi_lo, d32, n);
            ++launches;
            resid();
            it = 0;
            continue;
        }
        // an iteration after the untested ones whose residual is already within light_ratio of the target
        // takes the lighter V-cycle (flexible CG admits a preconditioner that changes between iterations)
        const bool light = light_ratio > 0.0 && cyc >= min_c && it > 0 && rn / bn <= light_ratio * rtol;
        const int gi = it == 0 ? 0 : (light ? 3 : 1) + (it & 1);
        if (persistent) {
            if (!g_mx[gi]) {
                if (!cap_stream && cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking) != cudaSuccess)
                    return PIC_ERR_CUDA;
                cudaGraph_t gr = nullptr;
                const long long l0 = launches;
                if (cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
                    return PIC_ERR_CUDA;
                iteration_mixed(cap_stream, it, light);
                if (cudaStreamEndCapture(cap_stream, &gr) != cudaSuccess) return PIC_ERR_CUDA;
                if (cudaGraphInstantiate(&g_mx[gi], gr, 0) != cudaSuccess) { cudaGraphDestroy(gr); return PIC_ERR_CUDA; }
                cudaGraphDestroy(gr);
                graph_kernels_mx[gi] = launches - l0;
                launches = l0;
            }
            if (cudaGraphLaunch(g_mx[gi], s) != cudaSuccess) return PIC_ERR_CUDA;
            launches += graph_kernels_mx[gi];
        } else {
            iteration_mixed(s, it, light);
        }
        ++it;
        ++cyc;
    }
    if (cycles_out) *cycles_out = cyc;
    if (rel_out) *rel_out = rn / bn;
    const float* dd = it > 0 ? d32 : nullptr;
    const float inv2h = (float)(1.0 / (2.0 * h));
    if (out_hi) {
        k_mx_grad<<<g3, kBlk, 0, s>>>(phi_hi, phi_lo, dd, out_hi, out_lo, nx, ny, nz, inv2h, bc, Ex, Ey, Ez, E4,
                                      nullptr);
        ++launches;
    } else {
        if (dd) {
            k_mx_commit<<<gf, kFlatBlock, 0, s>>>(phi_hi, phi_lo, dd, n);
            ++launches;
        }
        if (Ex || E4) {
            k_mx_grad<<<g3, kBlk, 0, s>>>(phi_hi, phi_lo, nullptr, nullptr, nullptr, nx, ny, nz, inv2h, bc, Ex,
                                                 Ey, Ez, E4, nullptr);
            ++launches;
        }
    }
    if (cudaGetLastError() != cudaSuccess) return PIC_ERR_CUDA;
    return rc;
}

// ------------------------------------------------------------------ device-driven solve

int MG::prepare_capture() {
    for (int q = 0; q < 3; ++q)
        if (!cap_body[q] && cudaStreamCreateWithFlags(&cap_body[q], cudaStreamNonBlocking) != cudaSuccess)
            return PIC_ERR_CUDA;
    return PIC_OK;
}

int MG::capture_solve_mixed(cudaStream_t cs, const float* rho, float* phi_hi, float* phi_lo, float* out_hi,
                            float* out_lo, double h, double v_lo, double v_hi, double v_mask, double rtol,
                            int max_cycles, float* E4, int* cycles_dst, double* rel_dst, unsigned* err_dst,
                            unsigned err_bit, unsigned long long* kernels_dst, long long* fixed_kernels) {
    if (!mixed || !loop || !out_hi || !masks_ready) return PIC_ERR_STATE;
    const int nx = lx[0], ny = ly[0], nz = lz[0], n = nx * ny * nz;
    const MxBoundary bc{pair_of(v_lo), pair_of(v_hi), pair_of(v_mask)};
    const dim3 g3 = grid_mx3(nx, ny, nz), gf = grid_mxf(n);
    if (!cap_body[0] || !cap_body[1] || !cap_body[2]) return PIC_ERR_STATE;
    cudaGraph_t top = capturing_graph(cs);
    if (!top) return PIC_ERR_CUDA;
    cudaGraphConditionalHandle h_loop, h_branch;
    auto resid = [&](cudaStream_t q) {
        k_mx_resid<float><<<g3, kBlk, 0, q>>>(rho, 1.0, m[0], phi_hi, phi_lo, nx, ny, nz, bc, g[0], part, ctr, norms);
        ++launches;
    };
    cudaMemsetAsync(ctr, 0, 8 * sizeof(unsigned), cs);
    cudaMemsetAsync(loop, 0, sizeof(MxLoop), cs);
    resid(cs);
    // the first iterations (index 0, then 1) without tests, as in the host loop
    const int min_c = mixed_min_cycles(max_cycles);
    cudaGraph_t body = nullptr;
    if (min_c > 0) {
        k_mx_prime<<<1, 1, 0, cs>>>(norms, loop, min_c);
        for (int q = 0; q < min_c; ++q) iteration_mixed(cs, q);
        // the loop only when those did not reach the tolerance (an if node
        // is cheaper than a loop trip that only decides to stop)
        cudaGraphConditionalHandle h_more;
        if (cudaGraphConditionalHandleCreate(&h_more, top, 0u, cudaGraphCondAssignDefault) != cudaSuccess)
            return PIC_ERR_CUDA;
        k_mx_check<<<1, 1, 0, cs>>>(norms, loop, rtol, max_cycles, h_more);
        cudaGraph_t ifb = nullptr;
        if (add_conditional(cs, h_more, cudaGraphCondTypeIf, 1, &ifb) != cudaSuccess) return PIC_ERR_CUDA;
        if (cudaGraphConditionalHandleCreate(&h_loop, ifb, 1u, cudaGraphCondAssignDefault) != cudaSuccess)
            return PIC_ERR_CUDA;
        if (cudaStreamBeginCaptureToGraph(cap_body[2], ifb, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
            cudaSuccess)
            return PIC_ERR_CUDA;
        const cudaError_t e_w = add_conditional(cap_body[2], h_loop, cudaGraphCondTypeWhile, 1, &body);
        if (end_body_capture(cap_body[2]) != cudaSuccess || e_w != cudaSuccess) return PIC_ERR_CUDA;
    } else {
        if (cudaGraphConditionalHandleCreate(&h_loop, top, 1u, cudaGraphCondAssignDefault) != cudaSuccess)
            return PIC_ERR_CUDA;
        if (add_conditional(cs, h_loop, cudaGraphCondTypeWhile, 1, &body) != cudaSuccess) return PIC_ERR_CUDA;
    }
    if (cudaGraphConditionalHandleCreate(&h_branch, body, 4u, cudaGraphCondAssignDefault) != cudaSuccess)
        return PIC_ERR_CUDA;
    // loop body: the decision, then the switch over the branches
    if (cudaStreamBeginCaptureToGraph(cap_body[0], body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
        cudaSuccess)
        return PIC_ERR_CUDA;
    k_mx_decide<<<1, 1, 0, cap_body[0]>>>(norms, loop, rtol, max_cycles, light_ratio, h_loop, h_branch);
    cudaGraph_t br[kMxBranches] = {};
    const cudaError_t e_sw = add_conditional(cap_body[0], h_branch, cudaGraphCondTypeSwitch, kMxBranches, br);
    if (end_body_capture(cap_body[0]) != cudaSuccess || e_sw != cudaSuccess) return PIC_ERR_CUDA;
    // branches: iterations with index 0 (first), 2 (even) and 1 (odd), the refinement, then the light
    // iterations (even, odd)
    const int its[kMxBranches] = {0, 2, 1, -1, 2, 1};
    MxBranchKernels kb;
    for (int b = 0; b < kMxBranches; ++b) {
        if (cudaStreamBeginCaptureToGraph(cap_body[1], br[b], nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return PIC_ERR_CUDA;
        const long long l0 = launches;
        if (b == 3) {
            k_mx_commit<<<gf, kFlatBlock, 0, cap_body[1]>>>(phi_hi, phi_lo, d32, n);
            ++launches;
            resid(cap_body[1]);
        } else {
            iteration_mixed(cap_body[1], its[b], b > 3);
        }
        kb.k[b] = (int)(launches - l0);
        if (end_body_capture(cap_body[1]) != cudaSuccess) return PIC_ERR_CUDA;
    }
    const float inv2h = (float)(1.0 / (2.0 * h));
    k_mx_grad<<<g3, kBlk, 0, cs>>>(phi_hi, phi_lo, d32, out_hi, out_lo, nx, ny, nz, inv2h, bc, nullptr, nullptr,
                                   nullptr, E4, loop);
    k_mx_report<<<1, 1, 0, cs>>>(loop, cycles_dst, rel_dst, err_dst, err_bit, kernels_dst, kb);
    if (fixed_kernels) *fixed_kernels = 3 + (min_c > 0 ? 2 : 0);  // residual, gradient, report, prime, check
    return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ERR_CUDA;
}

}  // namespace pic

// ------------------------------------------------------------------ C ABI
using pic::MG;

namespace {
bool poisson_args_ok(const poisson_config* pc, const double* rho, const double* phi, const float* Ex, const float* Ey,
                     const float* Ez, double rtol, int max_cycles) {
    if (!pc || !rho || !phi || pc->nx < 2 || pc->ny < 2 || pc->nz < 2 || !(pc->dx > 0) || !(rtol > 0) ||
        max_cycles < 0)
        return false;
    if (pc->precision != 0 && pc->precision != 32 && pc->precision != 64) return false;
    if ((Ex == nullptr) != (Ey == nullptr) || (Ex == nullptr) != (Ez == nullptr)) return false;
    return MG::supported(pc->nx, pc->ny, pc->nz);
}

size_t poisson_bytes(const poisson_config* pc) { return MG::bytes(pc->nx, pc->ny, pc->nz, pc->precision == 32, true); }

// The solve behind both entry points, on a workspace of poisson_bytes(pc).
int poisson_run(const poisson_config* pc, const double* rho, const uint8_t* mask, double* phi, float* Ex, float* Ey,
                float* Ez, double rtol, int max_cycles, void* ws, poisson_stats* st, cudaStream_t s) {
    MG mg;
    const bool mixed = pc->precision == 32;
    mg.carve(ws, pc->nx, pc->ny, pc->nz, mixed, true);
    double hn[2];
    int cycles = 0;
    double rel = 0.0;
    int rc;
    if (mixed) {
        const int n = pc->nx * pc->ny * pc->nz;
        float* hi = mg.phi_pair;
        float* lo = mg.phi_pair + pic::align256((size_t)n * 4) / 4;
        pic::k_mx_split<<<(n + 255) / 256, 256, 0, s>>>(phi, hi, lo, n);
        rc = mg.solve_mixed(rho, true, mask, hi, lo, nullptr, nullptr, true, pc->dx, pc->v_lo, pc->v_hi, pc->v_mask, rtol,
                            max_cycles, nullptr, Ex, Ey, Ez, s, &cycles, &rel, hn);
        if (rc != PIC_ERR_CUDA) pic::k_mx_join<<<(n + 255) / 256, 256, 0, s>>>(hi, lo, phi, n);
        if (cudaGetLastError() != cudaSuccess) rc = PIC_ERR_CUDA;
    } else {
        rc = mg.solve(rho, mask, phi, pc->dx, pc->v_lo, pc->v_hi, pc->v_mask, rtol, max_cycles, 32, nullptr, Ex, Ey,
                      Ez, s, &cycles, &rel, hn);
    }
    if (st) { st->cycles = cycles; st->rel_res = rel; }
    return rc;
}
}  // namespace

extern "C" size_t poisson_workspace_bytes(const poisson_config* pc) {
    if (!pc || (pc->precision != 0 && pc->precision != 32 && pc->precision != 64) ||
        !MG::supported(pc->nx, pc->ny, pc->nz))
        return 0;
    return poisson_bytes(pc);
}

extern "C" int poisson_solve(const poisson_config* pc, const double* rho, const uint8_t* mask, double* phi, float* Ex,
                             float* Ey, float* Ez, double rtol, int max_cycles, void* ws, size_t ws_bytes,
                             poisson_stats* st, pic_stream_t stream) {
    if (!ws || !poisson_args_ok(pc, rho, phi, Ex, Ey, Ez, rtol, max_cycles)) return PIC_ERR_ARG;
    if (ws_bytes < poisson_bytes(pc) || ((uintptr_t)ws & 255)) return PIC_ERR_ARG;
    return poisson_run(pc, rho, mask, phi, Ex, Ey, Ez, rtol, max_cycles, ws, st, (cudaStream_t)stream);
}

// ------------------------------------------------------------------ no-allocation variant
// Some callers cannot allocate device memory for a workspace: plugins that a
// host application hands only input and output pointers (the application owns
// every allocation), code that runs under an allocator it may not bypass, and
// hard-real-time loops that must not touch the allocator once running.  For
// them the multigrid hierarchy lives in a fixed device array owned by this
// library.  The solve itself is unchanged: it is poisson_run, as behind
// poisson_solve, and like it reads the residual back on the host after each
// iteration.
//
// The array is file-scope device memory of kNoAllocScratchBytes (32 MiB), held
// by every GPU that loads the library until the process exits.  In host code
// its name is only a host-side stand-in, so the device address is looked up
// with cudaGetSymbolAddress once per device (with that device current) and
// cached.
constexpr size_t kNoAllocScratchBytes = 32u << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

#include <mutex>
static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[64];

static int noalloc_scratch(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return PIC_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return PIC_ERR_CUDA;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return PIC_OK;
}

extern "C" int poisson_solve_noalloc(const poisson_config* pc, const double* rho, const uint8_t* mask, double* phi,
                                     float* Ex, float* Ey, float* Ez, double rtol, int max_cycles, poisson_stats* st,
                                     pic_stream_t stream) {
    if (!poisson_args_ok(pc, rho, phi, Ex, Ey, Ez, rtol, max_cycles)) return PIC_ERR_ARG;
    if (poisson_bytes(pc) > kNoAllocScratchBytes) return PIC_ERR_CAPACITY;
    void* ws = nullptr;
    int rc = noalloc_scratch(&ws);
    if (rc) return rc;
    return poisson_run(pc, rho, mask, phi, Ex, Ey, Ez, rtol, max_cycles, ws, st, (cudaStream_t)stream);
}
