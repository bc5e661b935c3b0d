// Axisymmetric Poisson solve (Sec. 2.5 in the paper's axisymmetric geometry,
// Sec. 2.1.2 for the ring cells): -(1/r) d/dr (r dphi/dr) - d2phi/dz2 = rho /
// eps0 on a cell-centred (r, z) mesh, cells i = 0..nr-1 at r_i = (i + 1/2) h
// from the axis, k = 0..nz-1 along z, square cells of side h.
//
// Each row is the flux balance of a ring cell divided by 2 pi h (symmetric,
// positive definite): with r in units of h the face coefficients are i
// (inner radial face, 0 on the axis), i + 1 (outer radial face) and i + 1/2
// (the two axial faces), and the right-hand side is (i + 1/2) h^2 rho / eps0.
// Boundaries: the outer cylinder homogeneous Neumann (no flux), the z faces
// Dirichlet plates v_lo, v_hi (ghost 2 v - phi), cells of the electrode mask
// held at v_mask.  E = -grad(phi) by central differences at cell centres
// (mirror at the axis and the outer cylinder).
//
// Solver: flexible CG in float64 preconditioned by one float64 V(2,2)-cycle
// of red-black Gauss-Seidel on the same operator re-discretised on every
// level (coarse cells twice as wide; a coarse cell is held at zero if any
// child is masked).  The coarse right-hand side is half the sum of the four
// children's residuals: residuals are fluxes divided by 2 pi h, and the
// coarse cell's fluxes are the sums of its children's, divided by 2 pi (2h).
#include <math.h>

#include "common.cuh"
#include "graph_util.cuh"
#include "poisson_axi.cuh"
#include "../../include/picmcc.h"

namespace pic {

namespace {

constexpr int AX = 32, AZ = 8;
const dim3 kABlk(AX, AZ, 1);
enum { A_B2 = 0, A_R2, A_RHO, A_GAM, A_T1, A_T2, A_ALPHA, A_BETA, A_N };

dim3 agrid(int nr, int nz) { return dim3((nr + AX - 1) / AX, (nz + AZ - 1) / AZ); }

__device__ __forceinline__ void ablock_add(double v, double* dst) {
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
    __syncthreads();
}

// Face coefficients of cell (i, k): inner, outer radial and axial.
struct Coef {
    double ci, co, cz;
};
__device__ __forceinline__ Coef coef(int i, int nr) {
    return Coef{(double)i, i + 1 < nr ? (double)(i + 1) : 0.0, (double)i + 0.5};
}
__device__ __forceinline__ double diag_of(const Coef& c, int k, int nz) {
    return c.ci + c.co + 2.0 * c.cz + (k == 0 ? c.cz : 0.0) + (k == nz - 1 ? c.cz : 0.0);
}
// Weighted neighbour sum of the correction e (zero on masked cells and in
// the homogeneous ghosts: Dirichlet ghost -e is in the diagonal).
__device__ __forceinline__ double nb_e(const double* e, int i, int k, int nr, int nz, const Coef& c) {
    const int q = k * nr + i;
    double s = 0.0;
    if (i > 0) s += c.ci * e[q - 1];
    if (i + 1 < nr) s += c.co * e[q + 1];
    if (k > 0) s += c.cz * e[q - nr];
    if (k + 1 < nz) s += c.cz * e[q + nr];
    return s;
}

#define ACELL                                          \
    const int i = blockIdx.x * AX + threadIdx.x;      \
    const int k = blockIdx.y * AZ + threadIdx.y;      \
    const bool in = i < nr && k < nz;                 \
    const int c = in ? k * nr + i : 0;

__global__ void k_axi_copy_mask(const uint8_t* m, uint8_t* out, int n) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) out[c] = m ? (m[c] ? 1 : 0) : 0;
}

__global__ void k_axi_restrict_mask(const uint8_t* __restrict__ m, int nr, int nz, uint8_t* __restrict__ mc) {
    const int cr = nr / 2, cz = nz / 2;
    const int I = blockIdx.x * AX + threadIdx.x, K = blockIdx.y * AZ + threadIdx.y;
    if (I >= cr || K >= cz) return;
    uint8_t v = 0;
    for (int d = 0; d < 4; ++d) v |= m[(2 * K + (d >> 1)) * nr + 2 * I + (d & 1)];
    mc[K * cr + I] = v ? 1 : 0;
}

// b and r = b - A phi with the boundary values; ||b||^2, ||r||^2; electrode
// cells get phi = v_mask, r = 0.
__global__ void k_axi_resid(double* __restrict__ phi, const double* __restrict__ rho, const uint8_t* __restrict__ m,
                            int nr, int nz, double h2e, double v_lo, double v_hi, double v_mask,
                            double* __restrict__ r, double* __restrict__ g0, double* sc) {
    ACELL
    double bb = 0.0, rr2 = 0.0;
    if (in) {
        if (m[c]) {
            phi[c] = v_mask;
            r[c] = 0.0;
            g0[c] = 0.0;
        } else {
            const Coef cf = coef(i, nr);
            const double pc = phi[c];
            double b = cf.cz * h2e * rho[c], s = b;
            auto face = [&](int q, double w) {
                if (m[q]) { b += w * v_mask; s += w * (v_mask - pc); }
                else s += w * (phi[q] - pc);
            };
            if (i > 0) face(c - 1, cf.ci);
            if (i + 1 < nr) face(c + 1, cf.co);
            if (k > 0) face(c - nr, cf.cz);
            else { b += 2.0 * cf.cz * v_lo; s += 2.0 * cf.cz * (v_lo - pc); }
            if (k + 1 < nz) face(c + nr, cf.cz);
            else { b += 2.0 * cf.cz * v_hi; s += 2.0 * cf.cz * (v_hi - pc); }
            r[c] = s;
            g0[c] = s;
            bb = b * b;
            rr2 = s * s;
        }
    }
    ablock_add(bb, sc + A_B2);
    ablock_add(rr2, sc + A_R2);
}

__global__ void k_axi_smooth(double* __restrict__ e, const double* __restrict__ g, const uint8_t* __restrict__ m,
                             int nr, int nz, int color) {
    ACELL
    if (!in || ((i + k) & 1) != color || m[c]) return;
    const Coef cf = coef(i, nr);
    e[c] = (g[c] + nb_e(e, i, k, nr, nz, cf)) / diag_of(cf, k, nz);
}

__global__ void k_axi_resid_restrict(const double* __restrict__ e, const double* __restrict__ g,
                                     const uint8_t* __restrict__ m, int nr, int nz, double* __restrict__ gc,
                                     const uint8_t* __restrict__ mc) {
    const int cr = nr / 2, cz = nz / 2;
    const int I = blockIdx.x * AX + threadIdx.x, K = blockIdx.y * AZ + threadIdx.y;
    if (I >= cr || K >= cz) return;
    const int qc = K * cr + I;
    if (mc[qc]) { gc[qc] = 0.0; return; }
    double acc = 0.0;
    for (int d = 0; d < 4; ++d) {
        const int i = 2 * I + (d & 1), k = 2 * K + (d >> 1), c = k * nr + i;
        if (m[c]) continue;
        const Coef cf = coef(i, nr);
        acc += g[c] - (diag_of(cf, k, nz) * e[c] - nb_e(e, i, k, nr, nz, cf));
    }
    gc[qc] = 0.5 * acc;
}

__device__ __forceinline__ double acval(const double* ec, int I, int K, int cr, int cz) {
    double sgn = 1.0;
    I = I < 0 ? 0 : (I >= cr ? cr - 1 : I);
    if (K < 0) { K = 0; sgn = -1.0; }
    if (K >= cz) { K = cz - 1; sgn = -1.0; }
    return sgn * ec[K * cr + I];
}

__global__ void k_axi_prolong_add(const double* __restrict__ ec, double* __restrict__ ef,
                                  const uint8_t* __restrict__ m, int nr, int nz) {
    ACELL
    if (!in) return;
    if (m[c]) { ef[c] = 0.0; return; }
    const int cr = nr / 2, cz = nz / 2, I = i >> 1, K = k >> 1;
    const int si = (i & 1) ? 1 : -1, sk = (k & 1) ? 1 : -1;
    double acc = 0.0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            const double w = (a ? 0.25 : 0.75) * (b ? 0.25 : 0.75);
            acc += w * acval(ec, I + (b ? si : 0), K + (a ? sk : 0), cr, cz);
        }
    ef[c] += acc;
}

// Coarsest level: zero start and `sweeps` red-black sweeps in one block.
__global__ void __launch_bounds__(1024) k_axi_coarse(double* e, const double* g, const uint8_t* m, int nr, int nz,
                                                     int sweeps) {
    const int n = nr * nz;
    for (int c = threadIdx.x; c < n; c += blockDim.x) e[c] = 0.0;
    __syncthreads();
    for (int s = 0; s < 2 * sweeps; ++s) {
        const int color = s & 1;
        for (int c = threadIdx.x; c < n; c += blockDim.x) {
            const int i = c % nr, k = c / nr;
            if (((i + k) & 1) != color || m[c]) continue;
            const Coef cf = coef(i, nr);
            e[c] = (g[c] + nb_e(e, i, k, nr, nz, cf)) / diag_of(cf, k, nz);
        }
        __syncthreads();
    }
}

// q = A p (homogeneous) and p.q.
__global__ void k_axi_apply(const double* __restrict__ p, const uint8_t* __restrict__ m, int nr, int nz,
                            double* __restrict__ q, double* sc) {
    ACELL
    double acc = 0.0;
    if (in) {
        if (m[c]) {
            q[c] = 0.0;
        } else {
            const Coef cf = coef(i, nr);
            const double v = diag_of(cf, k, nz) * p[c] - nb_e(p, i, k, nr, nz, cf);
            q[c] = v;
            acc = p[c] * v;
        }
    }
    ablock_add(acc, sc + A_GAM);
}

__global__ void k_axi_dot2(const double* __restrict__ z, const double* __restrict__ r, const double* __restrict__ q,
                           int n, double* sc, int with_q) {
    const int c = blockIdx.x * blockDim.x * blockDim.y + threadIdx.y * blockDim.x + threadIdx.x;
    double a = 0.0, b = 0.0;
    if (c < n) {
        a = z[c] * r[c];
        if (with_q) b = z[c] * q[c];
    }
    ablock_add(a, sc + A_T1);
    ablock_add(b, sc + A_T2);
}

__global__ void k_axi_beta(double* sc, int first) {
    sc[A_BETA] = first ? 0.0 : -sc[A_ALPHA] * sc[A_T2] / sc[A_RHO];
    sc[A_RHO] = sc[A_T1];
    sc[A_GAM] = 0.0;
}

__global__ void k_axi_update_p(double* __restrict__ p, const double* __restrict__ z, int n, const double* sc) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const double b = sc[A_BETA];
    if (c < n) p[c] = b != 0.0 ? z[c] + b * p[c] : z[c];
}

__global__ void k_axi_alpha(double* sc) {
    sc[A_ALPHA] = sc[A_GAM] > 0.0 ? sc[A_RHO] / sc[A_GAM] : 0.0;
    sc[A_R2] = 0.0;
    sc[A_T1] = 0.0;
    sc[A_T2] = 0.0;
}

__global__ void k_axi_update_xr(double* __restrict__ phi, double* __restrict__ r, const double* __restrict__ p,
                                const double* __restrict__ q, double* __restrict__ g0, int n, double* sc) {
    const int c = blockIdx.x * blockDim.x * blockDim.y + threadIdx.y * blockDim.x + threadIdx.x;
    const double a = sc[A_ALPHA];
    double acc = 0.0;
    if (c < n) {
        phi[c] += a * p[c];
        const double rr = r[c] - a * q[c];
        r[c] = rr;
        g0[c] = rr;
        acc = rr * rr;
    }
    ablock_add(acc, sc + A_R2);
}

template <class T>
__global__ void k_axi_grad(const double* __restrict__ phi, int nr, int nz, double h, double v_lo, double v_hi,
                           float* Er, float* Ez, T* E4) {
    ACELL
    if (!in) return;
    const double inv = 1.0 / (2.0 * h), pc = phi[c];
    const double rm = i > 0 ? phi[c - 1] : pc, rp = i + 1 < nr ? phi[c + 1] : pc;
    const double zm = k > 0 ? phi[c - nr] : 2.0 * v_lo - pc, zp = k + 1 < nz ? phi[c + nr] : 2.0 * v_hi - pc;
    const double er = -(rp - rm) * inv, ez = -(zp - zm) * inv;
    if (Er) { Er[c] = (float)er; Ez[c] = (float)ez; }
    if (E4) { E4[4 * c] = (T)er; E4[4 * c + 1] = (T)0; E4[4 * c + 2] = (T)ez; E4[4 * c + 3] = (T)0; }
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

void AxiMG::plan(int nr, int nz) {
    levels = 0;
    int a = nr, b = nz;
    for (;;) {
        lr[levels] = a;
        lz[levels] = b;
        ++levels;
        if (levels >= kMaxLevels || (a % 2) || (b % 2) || a < 4 || b < 4) break;
        a /= 2;
        b /= 2;
    }
}

bool AxiMG::supported(int nr, int nz) {
    if (nr < 2 || nz < 2 || (long long)nr * nz > 0x7fffffffLL) return false;
    AxiMG g;
    g.plan(nr, nz);
    return (long long)g.lr[g.levels - 1] * g.lz[g.levels - 1] <= 4096;
}

size_t AxiMG::bytes(int nr, int nz) {
    AxiMG g;
    return g.carve(nullptr, nr, nz);
}

size_t AxiMG::carve(void* base, int nr, int nz) {
    plan(nr, nz);
    uintptr_t pp = (uintptr_t)base;
    const uintptr_t p0 = pp;
    auto take = [&](size_t b) {
        void* o = (void*)pp;
        pp += al256(b);
        return o;
    };
    const size_t n0 = (size_t)nr * nz;
    norms = (double*)take(A_N * 8);
    loop = (AxiLoop*)take(sizeof(AxiLoop));
    r = (double*)take(n0 * 8);
    p = (double*)take(n0 * 8);
    q = (double*)take(n0 * 8);
    for (int l = 0; l < levels; ++l) {
        const size_t n = (size_t)lr[l] * lz[l];
        e[l] = (double*)take(n * 8);
        g[l] = (double*)take(n * 8);
        m[l] = (uint8_t*)take(n);
    }
    return (size_t)(pp - p0);
}

cudaError_t AxiMG::build_masks(const uint8_t* mask, cudaStream_t s) {
    const int n0 = lr[0] * lz[0];
    k_axi_copy_mask<<<(n0 + 255) / 256, 256, 0, s>>>(mask, m[0], n0);
    for (int l = 1; l < levels; ++l)
        k_axi_restrict_mask<<<agrid(lr[l], lz[l]), kABlk, 0, s>>>(m[l - 1], lr[l - 1], lz[l - 1], m[l]);
    launches += levels;
    return cudaGetLastError();
}

void AxiMG::vcycle(cudaStream_t s) {
    const int L = levels - 1;
    for (int l = 0; l < L; ++l) {
        cudaMemsetAsync(e[l], 0, (size_t)lr[l] * lz[l] * 8, s);
        for (int it = 0; it < pre; ++it)
            for (int col = 0; col < 2; ++col)
                k_axi_smooth<<<agrid(lr[l], lz[l]), kABlk, 0, s>>>(e[l], g[l], m[l], lr[l], lz[l], col);
        k_axi_resid_restrict<<<agrid(lr[l + 1], lz[l + 1]), kABlk, 0, s>>>(e[l], g[l], m[l], lr[l], lz[l], g[l + 1],
                                                                          m[l + 1]);
    }
    k_axi_coarse<<<1, 1024, 0, s>>>(e[L], g[L], m[L], lr[L], lz[L], coarse_sweeps);
    for (int l = L - 1; l >= 0; --l) {
        k_axi_prolong_add<<<agrid(lr[l], lz[l]), kABlk, 0, s>>>(e[l + 1], e[l], m[l], lr[l], lz[l]);
        for (int it = 0; it < post; ++it)
            for (int col = 1; col >= 0; --col)
                k_axi_smooth<<<agrid(lr[l], lz[l]), kABlk, 0, s>>>(e[l], g[l], m[l], lr[l], lz[l], col);
    }
    launches += (long long)L * (1 + 2 * pre + 2 * post + 1) + 1;
}

int AxiMG::solve(const double* rho, const uint8_t* mask, double* phi, double h, double v_lo, double v_hi,
                 double v_mask, double rtol, int max_cycles, int packed_prec, void* E4, float* Er, float* Ez,
                 cudaStream_t s, int* cycles_out, double* rel_out, double* host_norms) {
    const int nr = lr[0], nz = lz[0], n = nr * nz;
    if (!persistent || !masks_ready) {
        if (build_masks(mask, s) != cudaSuccess) return PIC_ERR_CUDA;
        masks_ready = true;
    }
    const double h2e = h * h / kEps0;
    cudaMemsetAsync(norms, 0, A_N * 8, s);
    k_axi_resid<<<agrid(nr, nz), kABlk, 0, s>>>(phi, rho, m[0], nr, nz, h2e, v_lo, v_hi, v_mask, r, g[0], norms);
    ++launches;
    int cyc = 0, rc = PIC_OK;
    double bn = 1.0, rn = 0.0;
    const int nb = (n + 255) / 256;
    const int min_c = min_cycles_for(max_cycles);
    for (;;) {
        // the first min_c iterations run without a test between them (no read-back)
        if (cyc >= min_c) {
            if (cudaMemcpyAsync(host_norms, norms, 2 * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess)
                return PIC_ERR_CUDA;
            if (cudaStreamSynchronize(s) != cudaSuccess) return PIC_ERR_CUDA;
            bn = host_norms[A_B2] > 0.0 ? sqrt(host_norms[A_B2]) : 1.0;
            rn = sqrt(host_norms[A_R2]);
            if (rn / bn <= rtol) break;
            if (cyc >= max_cycles) { rc = PIC_ERR_TIMEOUT; break; }
        }
        const int first = cyc == 0 ? 1 : 0;
        vcycle(s);
        k_axi_dot2<<<nb, dim3(256, 1, 1), 0, s>>>(e[0], r, q, n, norms, first ? 0 : 1);
        k_axi_beta<<<1, 1, 0, s>>>(norms, first);
        k_axi_update_p<<<nb, 256, 0, s>>>(p, e[0], n, norms);
        k_axi_apply<<<agrid(nr, nz), kABlk, 0, s>>>(p, m[0], nr, nz, q, norms);
        k_axi_alpha<<<1, 1, 0, s>>>(norms);
        k_axi_update_xr<<<nb, dim3(256, 1, 1), 0, s>>>(phi, r, p, q, g[0], n, norms);
        launches += 6;
        ++cyc;
    }
    if (cycles_out) *cycles_out = cyc;
    if (rel_out) *rel_out = rn / bn;
    if (E4 || Er) {
        if (packed_prec == 64)
            k_axi_grad<double><<<agrid(nr, nz), kABlk, 0, s>>>(phi, nr, nz, h, v_lo, v_hi, Er, Ez, (double*)E4);
        else
            k_axi_grad<float><<<agrid(nr, nz), kABlk, 0, s>>>(phi, nr, nz, h, v_lo, v_hi, Er, Ez, (float*)E4);
        ++launches;
    }
    return cudaGetLastError() == cudaSuccess ? rc : PIC_ERR_CUDA;
}

// One decision of the device-driven loop, as the host loop takes it: stop
// when ||r|| / ||b|| <= rtol or the cycle limit is reached (flagged), else
// branch 0 (first CG iteration) or 1 (later ones).  The trip bound is a
// safeguard: every trip either iterates or stops.
__global__ void k_axi_decide(const double* __restrict__ sc, AxiLoop* L, double rtol, int max_cycles,
                             cudaGraphConditionalHandle h_loop, cudaGraphConditionalHandle h_branch) {
    const double bn = sc[A_B2] > 0.0 ? sqrt(sc[A_B2]) : 1.0;
    const double rn = sqrt(sc[A_R2]);
    L->rel = rn / bn;
    unsigned branch = 2;  // no branch
    bool stop = false;
    if (rn / bn <= rtol) {
        stop = true;
    } else if (L->cyc >= max_cycles || L->trips > max_cycles + 1) {
        stop = true;
        L->timeout = 1;
    } else {
        branch = L->cyc == 0 ? 0u : 1u;
        ++L->cyc;
    }
    ++L->trips;
    if (branch < 2) ++L->n_branch[branch];
    cudaGraphSetConditional(h_branch, branch);
    if (stop) cudaGraphSetConditional(h_loop, 0u);
}

__global__ void k_axi_report(const AxiLoop* __restrict__ L, int* cycles, double* rel, unsigned* err, unsigned bit,
                             unsigned long long* kernels, int kb0, int kb1) {
    *cycles = L->cyc;
    *rel = L->rel;
    if (L->timeout) *err |= bit;
    *kernels += (unsigned long long)L->trips + (unsigned long long)L->n_branch[0] * kb0 +
                (unsigned long long)L->n_branch[1] * kb1;
}

int AxiMG::min_cycles_for(int max_cycles) const {
    int m = min_cycles < 2 ? min_cycles : 2;
    if (m < 0) m = 0;
    return m < max_cycles ? m : max_cycles;
}

// Counters after the first min_c iterations, run back to back as in the host loop.
__global__ void k_axi_prime(AxiLoop* L, int min_c) {
    L->cyc = min_c;
    L->n_branch[0] = min_c > 0 ? 1 : 0;
    L->n_branch[1] = min_c > 1 ? min_c - 1 : 0;
}

int AxiMG::prepare_capture() {
    for (int q = 0; q < 2; ++q)
        if (!cap_body[q] && cudaStreamCreateWithFlags(&cap_body[q], cudaStreamNonBlocking) != cudaSuccess)
            return PIC_ERR_CUDA;
    return PIC_OK;
}

void AxiMG::release() {
    for (int q = 0; q < 2; ++q)
        if (cap_body[q]) { cudaStreamDestroy(cap_body[q]); cap_body[q] = nullptr; }
}

int AxiMG::capture_solve(cudaStream_t cs, const double* rho, double* phi, double h, double v_lo, double v_hi,
                         double v_mask, double rtol, int max_cycles, int packed_prec, void* E4, int* cycles_dst,
                         double* rel_dst, unsigned* err_dst, unsigned err_bit, unsigned long long* kernels_dst,
                         long long* fixed_kernels) {
    if (!loop || !masks_ready || !cap_body[0] || !cap_body[1]) return PIC_ERR_STATE;
    const int nr = lr[0], nz = lz[0], n = nr * nz;
    const double h2e = h * h / kEps0;
    const int nb = (n + 255) / 256;
    cudaGraph_t top = capturing_graph(cs);
    if (!top) return PIC_ERR_CUDA;
    cudaGraphConditionalHandle h_loop, h_branch;
    if (cudaGraphConditionalHandleCreate(&h_loop, top, 1u, cudaGraphCondAssignDefault) != cudaSuccess)
        return PIC_ERR_CUDA;
    cudaMemsetAsync(norms, 0, A_N * 8, cs);
    cudaMemsetAsync(loop, 0, sizeof(AxiLoop), cs);
    k_axi_resid<<<agrid(nr, nz), kABlk, 0, cs>>>(phi, rho, m[0], nr, nz, h2e, v_lo, v_hi, v_mask, r, g[0], norms);
    auto iteration = [&](cudaStream_t q, int first) {
        vcycle(q);
        k_axi_dot2<<<nb, dim3(256, 1, 1), 0, q>>>(e[0], r, this->q, n, norms, first ? 0 : 1);
        k_axi_beta<<<1, 1, 0, q>>>(norms, first);
        k_axi_update_p<<<nb, 256, 0, q>>>(p, e[0], n, norms);
        k_axi_apply<<<agrid(nr, nz), kABlk, 0, q>>>(p, m[0], nr, nz, this->q, norms);
        k_axi_alpha<<<1, 1, 0, q>>>(norms);
        k_axi_update_xr<<<nb, dim3(256, 1, 1), 0, q>>>(phi, r, p, this->q, g[0], n, norms);
        launches += 6;
    };
    // the first iterations without tests, as in the host loop
    const int min_c = min_cycles_for(max_cycles);
    if (min_c > 0) {
        k_axi_prime<<<1, 1, 0, cs>>>(loop, min_c);
        for (int it = 0; it < min_c; ++it) iteration(cs, it == 0 ? 1 : 0);
    }
    cudaGraph_t body = nullptr;
    if (add_conditional(cs, h_loop, cudaGraphCondTypeWhile, 1, &body) != cudaSuccess) return PIC_ERR_CUDA;
    if (cudaGraphConditionalHandleCreate(&h_branch, body, 2u, cudaGraphCondAssignDefault) != cudaSuccess)
        return PIC_ERR_CUDA;
    if (cudaStreamBeginCaptureToGraph(cap_body[0], body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
        cudaSuccess)
        return PIC_ERR_CUDA;
    k_axi_decide<<<1, 1, 0, cap_body[0]>>>(norms, loop, rtol, max_cycles, h_loop, h_branch);
    cudaGraph_t br[2] = {nullptr, nullptr};
    const cudaError_t e_sw = add_conditional(cap_body[0], h_branch, cudaGraphCondTypeSwitch, 2, br);
    if (end_body_capture(cap_body[0]) != cudaSuccess || e_sw != cudaSuccess) return PIC_ERR_CUDA;
    int kb[2];
    for (int b = 0; b < 2; ++b) {
        if (cudaStreamBeginCaptureToGraph(cap_body[1], br[b], nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return PIC_ERR_CUDA;
        const long long l0 = launches;
        iteration(cap_body[1], b == 0 ? 1 : 0);
        kb[b] = (int)(launches - l0);
        if (end_body_capture(cap_body[1]) != cudaSuccess) return PIC_ERR_CUDA;
    }
    long long fixed = 2 + (min_c > 0 ? 1 : 0);  // residual, report, prime
    if (E4) {
        if (packed_prec == 64)
            k_axi_grad<double><<<agrid(nr, nz), kABlk, 0, cs>>>(phi, nr, nz, h, v_lo, v_hi, nullptr, nullptr,
                                                                 (double*)E4);
        else
            k_axi_grad<float><<<agrid(nr, nz), kABlk, 0, cs>>>(phi, nr, nz, h, v_lo, v_hi, nullptr, nullptr,
                                                                (float*)E4);
        ++fixed;
    }
    k_axi_report<<<1, 1, 0, cs>>>(loop, cycles_dst, rel_dst, err_dst, err_bit, kernels_dst, kb[0], kb[1]);
    if (fixed_kernels) *fixed_kernels = fixed;
    return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ERR_CUDA;
}

}  // namespace pic

using pic::AxiMG;

extern "C" size_t poisson_axi_workspace_bytes(int nr, int nz) {
    if (!AxiMG::supported(nr, nz)) return 0;
    return AxiMG::bytes(nr, nz);
}

extern "C" int poisson_axi_solve(int nr, int nz, double dx, double v_lo, double v_hi, double v_mask,
                                 const double* rho, const uint8_t* mask, double* phi, float* Er, float* Ez,
                                 double rtol, int max_cycles, void* ws, size_t ws_bytes, poisson_stats* st,
                                 pic_stream_t stream) {
    if (!rho || !phi || !ws || !(dx > 0) || !(rtol > 0) || max_cycles < 0 || !AxiMG::supported(nr, nz))
        return PIC_ERR_ARG;
    if ((Er == nullptr) != (Ez == nullptr)) return PIC_ERR_ARG;
    if (ws_bytes < AxiMG::bytes(nr, nz) || ((uintptr_t)ws & 255)) return PIC_ERR_ARG;
    AxiMG mg;
    mg.carve(ws, nr, nz);
    double hn[2];
    int cycles = 0;
    double rel = 0.0;
    const int rc = mg.solve(rho, mask, phi, dx, v_lo, v_hi, v_mask, rtol, max_cycles, 32, nullptr, Er, Ez,
                            (cudaStream_t)stream, &cycles, &rel, hn);
    if (st) { st->cycles = cycles; st->rel_res = rel; }
    return rc;
}
