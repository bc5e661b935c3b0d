// Geometric multigrid Poisson solve with an embedded electrode mask.
//
// Sec. 2.5 of the paper: the field comes from Poisson's equation, solved with
// geometric multigrid, with the applied potential imposed on the electrode
// and E = -grad(phi).  Here the electrode is a mask of cells held at their
// potential (instead of a level set), the grid is uniform and cell-centred,
// the z faces are Dirichlet plates and the x, y faces homogeneous Neumann.
//
// Scheme: defect correction.  The residual r = b - A phi is formed in float64
// with the true boundary values; the error equation A e = r is solved
// approximately by one float32 V(2,2)-cycle (red-black Gauss-Seidel,
// 8-cell average restriction, trilinear prolongation, electrode cells and
// coarse cells touching the electrode held at e = 0); phi += e; repeat until
// ||r|| / ||b|| <= rtol.  A is the 7-point stencil scaled by h^2: diagonal
// 6 - (#Neumann faces) + (#Dirichlet faces), -1 per unmasked neighbour.
#include <math.h>

#include "common.cuh"
#include "poisson.cuh"

namespace pic {

namespace {

__device__ __forceinline__ long long lin(int i, int j, int k, int nx, int ny) {
    return ((long long)k * ny + j) * nx + i;
}

__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    return s;
}

// b = h^2 rho / eps0 + plate terms + electrode neighbours; accumulates ||b||^2.
__global__ void k_rhs_norm(const double* __restrict__ rho, const uint8_t* __restrict__ mask, int nx, int ny, int nz,
                           double h2e, double v_lo, double v_hi, double v_mask, double* norm2) {
    __shared__ double red[32];
    const long long n = (long long)nx * ny * nz;
    double acc = 0.0;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        if (mask && mask[c]) continue;
        const int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / ((long long)nx * ny));
        double s = h2e * rho[c];
        if (k == 0) s += 2.0 * v_lo;
        if (k == nz - 1) s += 2.0 * v_hi;
        if (mask) {
            if (i > 0 && mask[c - 1]) s += v_mask;
            if (i < nx - 1 && mask[c + 1]) s += v_mask;
            if (j > 0 && mask[c - nx]) s += v_mask;
            if (j < ny - 1 && mask[c + nx]) s += v_mask;
            if (k > 0 && mask[c - (long long)nx * ny]) s += v_mask;
            if (k < nz - 1 && mask[c + (long long)nx * ny]) s += v_mask;
        }
        acc += s * s;
    }
    const double t = block_sum(acc, red);
    if (threadIdx.x == 0 && t != 0.0) atomicAdd(norm2, t);
}

// r = b - A phi in float64 (true boundary values), written as the float32
// right-hand side of the error equation; accumulates ||r||^2.  Electrode
// cells are set to v_mask in phi.
__global__ void k_resid64(double* __restrict__ phi, const double* __restrict__ rho, const uint8_t* __restrict__ mask,
                          int nx, int ny, int nz, double h2e, double v_lo, double v_hi, double v_mask,
                          float* __restrict__ g0, double* norm2) {
    __shared__ double red[32];
    const long long n = (long long)nx * ny * nz, pl = (long long)nx * ny;
    double acc = 0.0;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        if (mask && mask[c]) { g0[c] = 0.0f; continue; }
        const int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / pl);
        const double pc = phi[c];
        // neighbour values with ghosts: Neumann mirror in x, y; Dirichlet in z
        auto val = [&](long long q, bool inside, double ghost) -> double {
            if (!inside) return ghost;
            if (mask && mask[q]) return v_mask;
            return phi[q];
        };
        const double sum = val(c - 1, i > 0, pc) + val(c + 1, i < nx - 1, pc) + val(c - nx, j > 0, pc) +
                           val(c + nx, j < ny - 1, pc) + val(c - pl, k > 0, 2.0 * v_lo - pc) +
                           val(c + pl, k < nz - 1, 2.0 * v_hi - pc);
        const double r = h2e * rho[c] + sum - 6.0 * pc;
        g0[c] = (float)r;
        acc += r * r;
    }
    const double t = block_sum(acc, red);
    if (threadIdx.x == 0 && t != 0.0) atomicAdd(norm2, t);
}

__global__ void k_set_mask_phi(double* phi, const uint8_t* mask, long long n, double v_mask) {
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        if (mask[c]) phi[c] = v_mask;
}

// One colour of red-black Gauss-Seidel for A e = g (homogeneous boundary
// values: Neumann mirror in x, y; Dirichlet -e in z; masked cells e = 0).
__global__ void k_smooth(float* __restrict__ e, const float* __restrict__ g, const uint8_t* __restrict__ mask, int nx,
                         int ny, int nz, int color) {
    const long long half = ((long long)nx * ny * nz + 1) / 2, pl = (long long)nx * ny;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < half; t += (long long)gridDim.x * blockDim.x) {
        // t-th cell of the given colour in x-fastest order
        const long long row = (t * 2) / nx;          // (k*ny + j) of the pair
        const int j = (int)(row % ny), k = (int)(row / ny);
        int i = (int)((t * 2) % nx);
        if (((i + j + k) & 1) != color) i += 1;
        if (i >= nx) continue;
        const long long c = lin(i, j, k, nx, ny);
        if (mask[c]) continue;
        float diag = 6.0f, s = g[c];
        if (i > 0) s += e[c - 1]; else diag -= 1.0f;
        if (i < nx - 1) s += e[c + 1]; else diag -= 1.0f;
        if (j > 0) s += e[c - nx]; else diag -= 1.0f;
        if (j < ny - 1) s += e[c + nx]; else diag -= 1.0f;
        if (k > 0) s += e[c - pl]; else diag += 1.0f;
        if (k < nz - 1) s += e[c + pl]; else diag += 1.0f;
        e[c] = s / diag;
    }
}

// Coarse right-hand side: g_c = 4 * mean of the 8 fine residuals g - A e.
__global__ void k_resid_restrict(const float* __restrict__ e, const float* __restrict__ g,
                                 const uint8_t* __restrict__ mask, int nx, int ny, int nz, float* __restrict__ gc,
                                 const uint8_t* __restrict__ maskc) {
    const int cx = nx / 2, cy = ny / 2, cz = nz / 2;
    const long long nc = (long long)cx * cy * cz, pl = (long long)nx * ny;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nc; q += (long long)gridDim.x * blockDim.x) {
        if (maskc[q]) { gc[q] = 0.0f; continue; }
        const int I = (int)(q % cx), J = (int)((q / cx) % cy), K = (int)(q / ((long long)cx * cy));
        float acc = 0.0f;
        for (int d = 0; d < 8; ++d) {
            const int i = 2 * I + (d & 1), j = 2 * J + ((d >> 1) & 1), k = 2 * K + (d >> 2);
            const long long c = lin(i, j, k, nx, ny);
            if (mask[c]) continue;
            const float ec = e[c];
            float diag = 6.0f, s = 0.0f;
            if (i > 0) s += e[c - 1]; else diag -= 1.0f;
            if (i < nx - 1) s += e[c + 1]; else diag -= 1.0f;
            if (j > 0) s += e[c - nx]; else diag -= 1.0f;
            if (j < ny - 1) s += e[c + nx]; else diag -= 1.0f;
            if (k > 0) s += e[c - pl]; else diag += 1.0f;
            if (k < nz - 1) s += e[c + pl]; else diag += 1.0f;
            acc += g[c] - (diag * ec - s);
        }
        gc[q] = 0.5f * acc;  // 4 * acc / 8
    }
}

// Coarse value with ghost rules (Neumann mirror x, y; Dirichlet -e in z).
__device__ __forceinline__ float cval(const float* ec, int I, int J, int K, int cx, int cy, int cz) {
    float sgn = 1.0f;
    if (I < 0) I = 0;
    if (I >= cx) I = cx - 1;
    if (J < 0) J = 0;
    if (J >= cy) J = cy - 1;
    if (K < 0) { K = 0; sgn = -sgn; }
    if (K >= cz) { K = cz - 1; sgn = -sgn; }
    return sgn * ec[lin(I, J, K, cx, cy)];
}

// e_f += trilinear interpolation of e_c (weights 3/4, 1/4 per axis).
__global__ void k_prolong_add(const float* __restrict__ ec, float* __restrict__ ef, const uint8_t* __restrict__ mask,
                              int nx, int ny, int nz) {
    const int cx = nx / 2, cy = ny / 2, cz = nz / 2;
    const long long n = (long long)nx * ny * nz;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        if (mask[c]) { ef[c] = 0.0f; continue; }
        const int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / ((long long)nx * ny));
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
}

// Coarse mask: a coarse cell is held at zero if any of its 8 children is.
__global__ void k_restrict_mask(const uint8_t* __restrict__ m, int nx, int ny, int nz, uint8_t* __restrict__ mc) {
    const int cx = nx / 2, cy = ny / 2, cz = nz / 2;
    const long long nc = (long long)cx * cy * cz;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nc; q += (long long)gridDim.x * blockDim.x) {
        const int I = (int)(q % cx), J = (int)((q / cx) % cy), K = (int)(q / ((long long)cx * cy));
        uint8_t v = 0;
        for (int d = 0; d < 8; ++d) v |= m[lin(2 * I + (d & 1), 2 * J + ((d >> 1) & 1), 2 * K + (d >> 2), nx, ny)];
        mc[q] = v ? 1 : 0;
    }
}

__global__ void k_copy_mask(const uint8_t* __restrict__ m, uint8_t* __restrict__ out, long long n) {
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        out[c] = m ? (m[c] ? 1 : 0) : 0;
}

// Coarsest level: many Gauss-Seidel sweeps inside one block.
__global__ void k_coarse_solve(float* __restrict__ e, const float* __restrict__ g, const uint8_t* __restrict__ mask,
                               int nx, int ny, int nz, int sweeps) {
    const long long n = (long long)nx * ny * nz, pl = (long long)nx * ny;
    for (long long c = threadIdx.x; c < n; c += blockDim.x) e[c] = 0.0f;
    __syncthreads();
    for (int s = 0; s < sweeps; ++s)
        for (int color = 0; color < 2; ++color) {
            for (long long c = threadIdx.x; c < n; c += blockDim.x) {
                const int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / pl);
                if (((i + j + k) & 1) != color || mask[c]) continue;
                float diag = 6.0f, sm = g[c];
                if (i > 0) sm += e[c - 1]; else diag -= 1.0f;
                if (i < nx - 1) sm += e[c + 1]; else diag -= 1.0f;
                if (j > 0) sm += e[c - nx]; else diag -= 1.0f;
                if (j < ny - 1) sm += e[c + nx]; else diag -= 1.0f;
                if (k > 0) sm += e[c - pl]; else diag += 1.0f;
                if (k < nz - 1) sm += e[c + pl]; else diag += 1.0f;
                e[c] = sm / diag;
            }
            __syncthreads();
        }
}

__global__ void k_zero_f(float* p, long long n) {
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        p[c] = 0.0f;
}

__global__ void k_update(double* __restrict__ phi, const float* __restrict__ e, const uint8_t* __restrict__ mask,
                         long long n) {
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        if (!mask[c]) phi[c] += (double)e[c];
}

// E = -grad(phi) at cell centres with the stencil's ghost values; writes any
// of the float planes and a packed [n][4] copy in T.
template <class T>
__global__ void k_grad(const double* __restrict__ phi, int nx, int ny, int nz, double h, double v_lo, double v_hi,
                       float* Ex, float* Ey, float* Ez, T* E4) {
    const long long n = (long long)nx * ny * nz, pl = (long long)nx * ny;
    const double inv = 1.0 / (2.0 * h);
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / pl);
        const double pc = phi[c];
        const double xm = i > 0 ? phi[c - 1] : pc, xp = i < nx - 1 ? phi[c + 1] : pc;
        const double ym = j > 0 ? phi[c - nx] : pc, yp = j < ny - 1 ? phi[c + nx] : pc;
        const double zm = k > 0 ? phi[c - pl] : 2.0 * v_lo - pc, zp = k < nz - 1 ? phi[c + pl] : 2.0 * v_hi - pc;
        const double ex = -(xp - xm) * inv, ey = -(yp - ym) * inv, ez = -(zp - zm) * inv;
        if (Ex) { Ex[c] = (float)ex; Ey[c] = (float)ey; Ez[c] = (float)ez; }
        if (E4) { E4[4 * c] = (T)ex; E4[4 * c + 1] = (T)ey; E4[4 * c + 2] = (T)ez; E4[4 * c + 3] = (T)0; }
    }
}

int grid_for(long long n) {
    long long b = (n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    return (int)b;
}

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

size_t MG::bytes(int nx_, int ny_, int nz_) {
    MG m;
    m.plan(nx_, ny_, nz_);
    size_t b = align256(64);  // norms
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
    p += align256(64);
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
    k_copy_mask<<<grid_for(n0), 256, 0, s>>>(mask, m[0], n0);
    for (int l = 1; l < levels; ++l)
        k_restrict_mask<<<grid_for((long long)lx[l] * ly[l] * lz[l]), 256, 0, s>>>(m[l - 1], lx[l - 1], ly[l - 1],
                                                                                     lz[l - 1], m[l]);
    return cudaGetLastError();
}

void MG::vcycle(cudaStream_t s) {
    launches += (long long)(levels - 1) * (2 + 2 * pre + 2 * post + 1) + 1;
    for (int l = 0; l < levels - 1; ++l) {
        const long long n = (long long)lx[l] * ly[l] * lz[l];
        const int gh = grid_for((n + 1) / 2);
        k_zero_f<<<grid_for(n), 256, 0, s>>>(e[l], n);
        for (int it = 0; it < pre; ++it) {
            k_smooth<<<gh, 256, 0, s>>>(e[l], g[l], m[l], lx[l], ly[l], lz[l], 0);
            k_smooth<<<gh, 256, 0, s>>>(e[l], g[l], m[l], lx[l], ly[l], lz[l], 1);
        }
        k_resid_restrict<<<grid_for(n / 8), 256, 0, s>>>(e[l], g[l], m[l], lx[l], ly[l], lz[l], g[l + 1], m[l + 1]);
    }
    const int L = levels - 1;
    k_coarse_solve<<<1, 256, 0, s>>>(e[L], g[L], m[L], lx[L], ly[L], lz[L], coarse_sweeps);
    for (int l = levels - 2; l >= 0; --l) {
        const long long n = (long long)lx[l] * ly[l] * lz[l];
        const int gh = grid_for((n + 1) / 2);
        k_prolong_add<<<grid_for(n), 256, 0, s>>>(e[l + 1], e[l], m[l], lx[l], ly[l], lz[l]);
        for (int it = 0; it < post; ++it) {
            k_smooth<<<gh, 256, 0, s>>>(e[l], g[l], m[l], lx[l], ly[l], lz[l], 1);
            k_smooth<<<gh, 256, 0, s>>>(e[l], g[l], m[l], lx[l], ly[l], lz[l], 0);
        }
    }
}

int MG::solve(const double* rho, const uint8_t* mask, double* phi, double h, double v_lo, double v_hi, double v_mask,
              double rtol, int max_cycles, int packed_prec, void* E4, float* Ex, float* Ey, float* Ez,
              cudaStream_t s, int* cycles_out, double* rel_out, double* host_norms) {
    const int nx = lx[0], ny = ly[0], nz = lz[0];
    const long long n = (long long)nx * ny * nz;
    const double h2e = h * h / kEps0;
    if (build_masks(mask, s) != cudaSuccess) return PIC_ERR_CUDA;
    if (mask) { k_set_mask_phi<<<grid_for(n), 256, 0, s>>>(phi, mask, n, v_mask); ++launches; }
    ++launches;
    cudaMemsetAsync(norms, 0, 16, s);
    k_rhs_norm<<<grid_for(n), 256, 0, s>>>(rho, mask, nx, ny, nz, h2e, v_lo, v_hi, v_mask, norms);
    double bn2 = 0.0, rn2 = 0.0;
    int cyc = 0, rc = PIC_OK;
    for (;;) {
        cudaMemsetAsync(norms + 1, 0, 8, s);
        k_resid64<<<grid_for(n), 256, 0, s>>>(phi, rho, mask, nx, ny, nz, h2e, v_lo, v_hi, v_mask, g[0], norms + 1);
        ++launches;
        if (cudaMemcpyAsync(host_norms, norms, 16, cudaMemcpyDeviceToHost, s) != cudaSuccess) return PIC_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return PIC_ERR_CUDA;
        bn2 = host_norms[0];
        rn2 = host_norms[1];
        const double bn = bn2 > 0.0 ? sqrt(bn2) : 1.0;
        if (sqrt(rn2) / bn <= rtol) break;
        if (cyc >= max_cycles) { rc = PIC_ERR_TIMEOUT; break; }
        vcycle(s);
        k_update<<<grid_for(n), 256, 0, s>>>(phi, e[0], m[0], n);
        ++launches;
        ++cyc;
    }
    if (cycles_out) *cycles_out = cyc;
    if (rel_out) *rel_out = sqrt(rn2) / (bn2 > 0.0 ? sqrt(bn2) : 1.0);
    if (Ex || E4) {
        ++launches;
        if (packed_prec == 64)
            k_grad<double><<<grid_for(n), 256, 0, s>>>(phi, nx, ny, nz, h, v_lo, v_hi, Ex, Ey, Ez, (double*)E4);
        else
            k_grad<float><<<grid_for(n), 256, 0, s>>>(phi, nx, ny, nz, h, v_lo, v_hi, Ex, Ey, Ez, (float*)E4);
    }
    if (cudaGetLastError() != cudaSuccess) return PIC_ERR_CUDA;
    return rc;
}

}  // namespace pic

// ------------------------------------------------------------------ C ABI
using pic::MG;

extern "C" size_t poisson_workspace_bytes(const poisson_config* pc) {
    if (!pc || pc->nx < 2 || pc->ny < 2 || pc->nz < 2) return 0;
    return MG::bytes(pc->nx, pc->ny, pc->nz);
}

extern "C" int poisson_solve(const poisson_config* pc, const double* rho, const uint8_t* mask, double* phi, float* Ex,
                             float* Ey, float* Ez, double rtol, int max_cycles, void* ws, size_t ws_bytes,
                             poisson_stats* st, pic_stream_t stream) {
    if (!pc || !rho || !phi || !ws || pc->nx < 2 || pc->ny < 2 || pc->nz < 2 || !(pc->dx > 0) || !(rtol > 0) ||
        max_cycles < 0)
        return PIC_ERR_ARG;
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
