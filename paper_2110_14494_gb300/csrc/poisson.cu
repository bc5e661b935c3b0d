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
#include "poisson.cuh"

namespace pic {

namespace {

constexpr int BX = 32, BY = 4;

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

// One colour of red-black Gauss-Seidel for A e = g (masked cells stay 0).
// Thread (ii, j, k) handles cell i = 2 ii + ((j + k + colour) & 1).
__global__ void k_smooth(float* __restrict__ e, const float* __restrict__ g, const uint8_t* __restrict__ mask, int nx,
                         int ny, int nz, int color) {
    const int j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
    const int i = 2 * (blockIdx.x * BX + threadIdx.x) + ((j + k + color) & 1);
    if (i >= nx || j >= ny) return;
    const int c = lin(i, j, k, nx, ny);
    if (mask[c]) return;
    float diag;
    const float s = nb_sum(e, mask, i, j, k, nx, ny, nz, c, diag);
    e[c] = (g[c] + s) / diag;
}

// Coarse right-hand side: g_c = 4 * mean of the 8 fine residuals g - A e
// (h^2 scaling: the coarse cell is twice as wide).
__global__ void k_resid_restrict(const float* __restrict__ e, const float* __restrict__ g,
                                 const uint8_t* __restrict__ mask, int nx, int ny, int nz, float* __restrict__ gc,
                                 const uint8_t* __restrict__ maskc) {
    const int cx = nx / 2, cy = ny / 2;
    const int I = blockIdx.x * BX + threadIdx.x, J = blockIdx.y * BY + threadIdx.y, K = blockIdx.z;
    if (I >= cx || J >= cy) return;
    const int q = lin(I, J, K, cx, cy);
    if (maskc[q]) { gc[q] = 0.0f; return; }
    float acc = 0.0f;
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        const int i = 2 * I + (d & 1), j = 2 * J + ((d >> 1) & 1), k = 2 * K + (d >> 2);
        const int c = lin(i, j, k, nx, ny);
        if (mask[c]) continue;
        float diag;
        const float s = nb_sum(e, mask, i, j, k, nx, ny, nz, c, diag);
        acc += g[c] - (diag * e[c] - s);
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

// e_f += trilinear interpolation of e_c (weights 3/4, 1/4 per axis).
__global__ void k_prolong_add(const float* __restrict__ ec, float* __restrict__ ef, const uint8_t* __restrict__ mask,
                              int nx, int ny, int nz) {
    CELL3D
    if (!in) return;
    if (mask[c]) { ef[c] = 0.0f; return; }
    const int cx = nx / 2, cy = ny / 2, cz = nz / 2;
    const int I = i >> 1, J = j >> 1, K = k >> 1;
    const int si = (i & 1) ? 1 : -1, sj = (j & 1) ? 1 : -1, sk = (k & 1) ? 1 : -1;
    float acc = 0.0f;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int d = 0; d < 2; ++d) {
                const float wgt = (a ? 0.25f : 0.75f) * (b ? 0.25f : 0.75f) * (d ? 0.25f : 0.75f);
                acc += wgt * cval(ec, I + (d ? si : 0), J + (b ? sj : 0), K + (a ? sk : 0), cx, cy, cz);
            }
    ef[c] += acc;
}

// Coarse mask: a coarse cell is held at zero if any of its 8 children is.
__global__ void k_restrict_mask(const uint8_t* __restrict__ m, int nx, int ny, int nz, uint8_t* __restrict__ mc) {
    const int cx = nx / 2, cy = ny / 2;
    const int I = blockIdx.x * BX + threadIdx.x, J = blockIdx.y * BY + threadIdx.y, K = blockIdx.z;
    if (I >= cx || J >= cy) return;
    uint8_t v = 0;
#pragma unroll
    for (int d = 0; d < 8; ++d) v |= m[lin(2 * I + (d & 1), 2 * J + ((d >> 1) & 1), 2 * K + (d >> 2), nx, ny)];
    mc[lin(I, J, K, cx, cy)] = v ? 1 : 0;
}

__global__ void k_copy_mask(const uint8_t* __restrict__ m, uint8_t* __restrict__ out, int n) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) out[c] = m ? (m[c] ? 1 : 0) : 0;
}


// The small levels of the hierarchy (from level t down to the coarsest; the
// first of them has at most kTailCells cells) run as one block in shared
// memory: zero, pre-smooth, restrict, ... coarse sweeps ... prolong,
// post-smooth, with block barriers between the phases instead of kernel
// launches.  The block reads g and the masks of level t from global memory
// and writes back e of level t.
constexpr int kTailCells = 8192;

struct TailLevels {
    float* e_first;          // global e of level `first`
    const float* g_first;    // global g of level `first`
    const uint8_t* m[12];    // global masks
    int nx[12], ny[12], nz[12], off[12];  // shared-memory offsets (cells)
    int first, last, pre, post, coarse, total;
};

struct TailSmem {
    float* e;
    float* g;
    uint8_t* m;
};

__device__ void tail_smooth(const TailLevels& T, const TailSmem& S, int l, int color) {
    const int nx = T.nx[l], ny = T.ny[l], nz = T.nz[l], n = nx * ny * nz, o = T.off[l];
    float* e = S.e + o;
    const float* g = S.g + o;
    const uint8_t* m = S.m + o;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        const int i = c % nx, j = (c / nx) % ny, k = c / (nx * ny);
        if (((i + j + k) & 1) != color || m[c]) continue;
        float diag;
        const float s = nb_sum(e, m, i, j, k, nx, ny, nz, c, diag);
        e[c] = (g[c] + s) / diag;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(1024) k_tail_vcycle(const TailLevels T) {
    extern __shared__ __align__(16) unsigned char tail_raw[];
    TailSmem S;
    S.e = reinterpret_cast<float*>(tail_raw);
    S.g = S.e + T.total;
    S.m = reinterpret_cast<uint8_t*>(S.g + T.total);
    {
        const int n0 = T.nx[T.first] * T.ny[T.first] * T.nz[T.first];
        for (int c = threadIdx.x; c < n0; c += blockDim.x) S.g[T.off[T.first] + c] = T.g_first[c];
        for (int l = T.first; l <= T.last; ++l) {
            const int n = T.nx[l] * T.ny[l] * T.nz[l];
            for (int c = threadIdx.x; c < n; c += blockDim.x) S.m[T.off[l] + c] = T.m[l][c];
        }
    }
    __syncthreads();
    for (int l = T.first; l <= T.last; ++l) {
        const int n = T.nx[l] * T.ny[l] * T.nz[l];
        for (int c = threadIdx.x; c < n; c += blockDim.x) S.e[T.off[l] + c] = 0.0f;
        __syncthreads();
        if (l == T.last) {
            for (int s = 0; s < T.coarse; ++s) { tail_smooth(T, S, l, 0); tail_smooth(T, S, l, 1); }
            break;
        }
        for (int s = 0; s < T.pre; ++s) { tail_smooth(T, S, l, 0); tail_smooth(T, S, l, 1); }
        // residual restricted to level l + 1 (h^2 scaling: 4 x mean of 8)
        const int nx = T.nx[l], ny = T.ny[l], nz = T.nz[l];
        const int cx = nx / 2, cy = ny / 2, cz = nz / 2, ncz = cx * cy * cz;
        const float* e = S.e + T.off[l];
        const float* g = S.g + T.off[l];
        const uint8_t* m = S.m + T.off[l];
        for (int q = threadIdx.x; q < ncz; q += blockDim.x) {
            float* gc = S.g + T.off[l + 1];
            if (S.m[T.off[l + 1] + q]) { gc[q] = 0.0f; continue; }
            const int I = q % cx, J = (q / cx) % cy, K = q / (cx * cy);
            float acc = 0.0f;
            for (int d = 0; d < 8; ++d) {
                const int i = 2 * I + (d & 1), j = 2 * J + ((d >> 1) & 1), k = 2 * K + (d >> 2);
                const int c = lin(i, j, k, nx, ny);
                if (m[c]) continue;
                float diag;
                const float s = nb_sum(e, m, i, j, k, nx, ny, nz, c, diag);
                acc += g[c] - (diag * e[c] - s);
            }
            gc[q] = 0.5f * acc;
        }
        __syncthreads();
    }
    for (int l = T.last - 1; l >= T.first; --l) {
        const int nx = T.nx[l], ny = T.ny[l], nz = T.nz[l], n = nx * ny * nz;
        const int cx = nx / 2, cy = ny / 2, cz = nz / 2;
        float* e = S.e + T.off[l];
        const float* ec = S.e + T.off[l + 1];
        const uint8_t* m = S.m + T.off[l];
        for (int c = threadIdx.x; c < n; c += blockDim.x) {
            if (m[c]) { e[c] = 0.0f; continue; }
            const int i = c % nx, j = (c / nx) % ny, k = c / (nx * ny);
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
        __syncthreads();
        for (int s = 0; s < T.post; ++s) { tail_smooth(T, S, l, 1); tail_smooth(T, S, l, 0); }
    }
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

dim3 grid3(int nx, int ny, int nz) { return dim3((nx + BX - 1) / BX, (ny + BY - 1) / BY, nz); }
dim3 grid3_half(int nx, int ny, int nz) { return dim3((nx / 2 + BX - 1) / BX, (ny + BY - 1) / BY, nz); }
dim3 grid_flat(long long n) { return dim3((unsigned)((n + BX * BY - 1) / (BX * BY))); }
dim3 grid_red(long long n) {
    long long b = (n + BX * BY - 1) / (BX * BY);
    return dim3((unsigned)(b < 1216 ? b : 1216));
}
dim3 grid3_red(int nx, int ny, int nz) { return dim3((nx + BX - 1) / BX, (ny + BY - 1) / BY, nz < kZRed ? nz : kZRed); }
const dim3 kBlk(BX, BY, 1);

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

size_t MG::bytes(int nx_, int ny_, int nz_) {
    MG m;
    m.plan(nx_, ny_, nz_);
    size_t b = align256(S_N * 8);
    const size_t n0 = (size_t)nx_ * ny_ * nz_;
    b += 3 * align256(n0 * 8);  // r, p, q in float64
    for (int l = 0; l < m.levels; ++l) {
        const size_t n = (size_t)m.lx[l] * m.ly[l] * m.lz[l];
        b += 2 * align256(n * sizeof(float)) + align256(n);
    }
    return b;
}

void MG::carve(void* base, int nx_, int ny_, int nz_) {
    plan(nx_, ny_, nz_);
    char* p = (char*)base;
    norms = (double*)p;
    p += align256(S_N * 8);
    const size_t n0 = (size_t)nx_ * ny_ * nz_;
    r64 = (double*)p; p += align256(n0 * 8);
    p64 = (double*)p; p += align256(n0 * 8);
    q64 = (double*)p; p += align256(n0 * 8);
    for (int l = 0; l < levels; ++l) {
        const size_t n = (size_t)lx[l] * ly[l] * lz[l];
        e[l] = (float*)p; p += align256(n * sizeof(float));
        g[l] = (float*)p; p += align256(n * sizeof(float));
        m[l] = (uint8_t*)p; p += align256(n);
    }
}

cudaError_t MG::build_masks(const uint8_t* mask, cudaStream_t s) {
    const long long n0 = (long long)lx[0] * ly[0] * lz[0];
    launches += levels;
    k_copy_mask<<<(unsigned)((n0 + 255) / 256), 256, 0, s>>>(mask, m[0], (int)n0);
    for (int l = 1; l < levels; ++l)
        k_restrict_mask<<<grid3(lx[l], ly[l], lz[l]), kBlk, 0, s>>>(m[l - 1], lx[l - 1], ly[l - 1], lz[l - 1], m[l]);
    return cudaGetLastError();
}

// One V(pre, post)-cycle on A e0 = g0; e0 is overwritten.  Levels above the
// tail run as separate kernels; the tail runs as one block.
void MG::vcycle(cudaStream_t s) {
    int t = 0;
    while (t < levels - 1 && (long long)lx[t] * ly[t] * lz[t] > kTailCells) ++t;
    // the tail's shared memory must fit: keep full levels above it otherwise
    while (t < levels - 1) {
        long long cells = 0;
        for (int l = t; l < levels; ++l) cells += (long long)lx[l] * ly[l] * lz[l];
        if (cells * 9 <= 200 * 1024) break;
        ++t;
    }
    launches += (long long)t * (1 + 2 * pre + 2 * post + 1) + 1;
    for (int l = 0; l < t; ++l) {
        const long long n = (long long)lx[l] * ly[l] * lz[l];
        cudaMemsetAsync(e[l], 0, n * sizeof(float), s);
        for (int it = 0; it < pre; ++it) {
            k_smooth<<<grid3_half(lx[l], ly[l], lz[l]), kBlk, 0, s>>>(e[l], g[l], m[l], lx[l], ly[l], lz[l], 0);
            k_smooth<<<grid3_half(lx[l], ly[l], lz[l]), kBlk, 0, s>>>(e[l], g[l], m[l], lx[l], ly[l], lz[l], 1);
        }
        k_resid_restrict<<<grid3(lx[l + 1], ly[l + 1], lz[l + 1]), kBlk, 0, s>>>(e[l], g[l], m[l], lx[l], ly[l],
                                                                                 lz[l], g[l + 1], m[l + 1]);
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
    T.pre = pre;
    T.post = post;
    T.coarse = coarse_sweeps;
    T.total = off;
    const size_t smem = (size_t)off * (2 * sizeof(float) + 1);
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_tail_vcycle, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_tail_vcycle<<<1, 1024, smem, s>>>(T);
    for (int l = t - 1; l >= 0; --l) {
        k_prolong_add<<<grid3(lx[l], ly[l], lz[l]), kBlk, 0, s>>>(e[l + 1], e[l], m[l], lx[l], ly[l], lz[l]);
        for (int it = 0; it < post; ++it) {
            k_smooth<<<grid3_half(lx[l], ly[l], lz[l]), kBlk, 0, s>>>(e[l], g[l], m[l], lx[l], ly[l], lz[l], 1);
            k_smooth<<<grid3_half(lx[l], ly[l], lz[l]), kBlk, 0, s>>>(e[l], g[l], m[l], lx[l], ly[l], lz[l], 0);
        }
    }
}

// One flexible-CG iteration: z = M r, direction, q = A p, alpha, updates.
void MG::iteration(cudaStream_t s, double* phi, const uint8_t* mk, bool first) {
    const int nx = lx[0], ny = ly[0], nz = lz[0];
    const int n = nx * ny * nz;
    vcycle(s);
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

}  // namespace pic

// ------------------------------------------------------------------ C ABI
using pic::MG;

extern "C" size_t poisson_workspace_bytes(const poisson_config* pc) {
    if (!pc || !MG::supported(pc->nx, pc->ny, pc->nz)) return 0;
    return MG::bytes(pc->nx, pc->ny, pc->nz);
}

extern "C" int poisson_solve(const poisson_config* pc, const double* rho, const uint8_t* mask, double* phi, float* Ex,
                             float* Ey, float* Ez, double rtol, int max_cycles, void* ws, size_t ws_bytes,
                             poisson_stats* st, pic_stream_t stream) {
    if (!pc || !rho || !phi || !ws || pc->nx < 2 || pc->ny < 2 || pc->nz < 2 || !(pc->dx > 0) || !(rtol > 0) ||
        max_cycles < 0)
        return PIC_ERR_ARG;
    if (!MG::supported(pc->nx, pc->ny, pc->nz)) return PIC_ERR_ARG;
    if (ws_bytes < MG::bytes(pc->nx, pc->ny, pc->nz) || ((uintptr_t)ws & 255)) return PIC_ERR_ARG;
    if ((Ex == nullptr) != (Ey == nullptr) || (Ex == nullptr) != (Ez == nullptr)) return PIC_ERR_ARG;
    MG mg;
    mg.carve(ws, pc->nx, pc->ny, pc->nz);
    double hn[2];
    int cycles = 0;
    double rel = 0.0;
    int rc = mg.solve(rho, mask, phi, pc->dx, pc->v_lo, pc->v_hi, pc->v_mask, rtol, max_cycles, 32, nullptr, Ex, Ey, Ez,
                      (cudaStream_t)stream, &cycles, &rel, hn);
    if (st) { st->cycles = cycles; st->rel_res = rel; }
    return rc;
}

// ------------------------------------------------------------------ no-allocation variant
// Some callers cannot allocate device memory for a workspace: code running
// where cudaMalloc is not permitted or not wanted (inside a region being
// captured into a CUDA graph by a framework that forbids allocation, plugins
// handed only input and output pointers by a host application, or
// hard-real-time loops that must not touch the allocator).  For them the
// multigrid hierarchy lives in a fixed device array owned by this library.
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
    if (!pc || !rho || !phi || pc->nx < 2 || pc->ny < 2 || pc->nz < 2 || !(pc->dx > 0) || !(rtol > 0) ||
        max_cycles < 0)
        return PIC_ERR_ARG;
    if ((Ex == nullptr) != (Ey == nullptr) || (Ex == nullptr) != (Ez == nullptr)) return PIC_ERR_ARG;
    if (!MG::supported(pc->nx, pc->ny, pc->nz)) return PIC_ERR_ARG;
    if (MG::bytes(pc->nx, pc->ny, pc->nz) > kNoAllocScratchBytes) return PIC_ERR_CAPACITY;
    void* ws = nullptr;
    int rc = noalloc_scratch(&ws);
    if (rc) return rc;
    MG mg;
    mg.carve(ws, pc->nx, pc->ny, pc->nz);
    double hn[2];
    int cycles = 0;
    double rel = 0.0;
    rc = mg.solve(rho, mask, phi, pc->dx, pc->v_lo, pc->v_hi, pc->v_mask, rtol, max_cycles, 32, nullptr, Ex, Ey, Ez,
                  (cudaStream_t)stream, &cycles, &rel, hn);
    if (st) { st->cycles = cycles; st->rel_res = rel; }
    return rc;
}
