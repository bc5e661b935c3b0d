// PIC-MCC context, workspace layout, initialisation, cell sort, weight update,
// step driver and the C ABI of include/picmcc.h.
//
// Compiled with --fmad=false: the seeding, sort keys and weight-update
// arithmetic round every operation separately.
#include <limits.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <utility>
#include <vector>

#include "common.cuh"
#include "graph_util.cuh"
#include "poisson.cuh"
#include "poisson_axi.cuh"
#include "push.cuh"
#include "swarm_batch.cuh"

namespace pic {

// A coupled solve's CG iteration after the first two takes a V(1,1)-cycle
// when the relative residual is already within this factor of the target.
constexpr double kLightRatio = 3.0;

// ================================================================== scan
// Exclusive prefix sum of n uint32 values into out[0..n]; out[n] = total.
constexpr int kScanTile = 2048;

__global__ void k_scan_tiles(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, long long n,
                             uint32_t* __restrict__ sums) {
    __shared__ uint32_t sh[kScanTile];
    __shared__ uint32_t wsum[8];
    const long long base = (long long)blockIdx.x * kScanTile;
    for (int t = threadIdx.x; t < kScanTile; t += blockDim.x) {
        const long long i = base + t;
        sh[t] = i < n ? in[i] : 0u;
    }
    __syncthreads();
    // each thread scans 8 consecutive values
    const int t0 = threadIdx.x * 8;
    uint32_t run = 0;
    for (int q = 0; q < 8; ++q) { const uint32_t v = sh[t0 + q]; sh[t0 + q] = run; run += v; }
    // warp-level exclusive scan of the per-thread totals
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t inc = run;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    uint32_t woff = 0;
    for (int q = 0; q < w; ++q) woff += wsum[q];
    const uint32_t off = woff + inc - run;
    for (int q = 0; q < 8; ++q) sh[t0 + q] += off;
    __syncthreads();
    for (int t = threadIdx.x; t < kScanTile; t += blockDim.x) {
        const long long i = base + t;
        if (i < n) out[i] = sh[t];
    }
    if (threadIdx.x == blockDim.x - 1) sums[blockIdx.x] = off + run;
}

// Single block: exclusive scan of the tile sums in place; sums[nb] = total.
__global__ void k_scan_sums(uint32_t* sums, int nb) {
    __shared__ uint32_t carry;
    __shared__ uint32_t wsum[8];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const uint32_t v = i < nb ? sums[i] : 0u;
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        uint32_t inc = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) wsum[w] = inc;
        __syncthreads();
        uint32_t woff = 0;
        for (int q = 0; q < w; ++q) woff += wsum[q];
        const uint32_t c = carry;
        if (i < nb) sums[i] = c + woff + inc - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = c + woff + inc;
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[nb] = carry;
}

__global__ void k_scan_add(uint32_t* __restrict__ out, long long n, const uint32_t* __restrict__ sums, int nb) {
    const uint32_t add = sums[blockIdx.x];
    const long long base = (long long)blockIdx.x * kScanTile;
    for (int t = threadIdx.x; t < kScanTile; t += blockDim.x) {
        const long long i = base + t;
        if (i < n) out[i] += add;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = sums[nb];
}

static int scan_blocks(long long n) { return (int)((n + kScanTile - 1) / kScanTile); }

static cudaError_t scan_exclusive(const uint32_t* in, uint32_t* out, long long n, uint32_t* sums, cudaStream_t s) {
    const int nb = scan_blocks(n > 0 ? n : 1);
    k_scan_tiles<<<nb, 256, 0, s>>>(in, out, n, sums);
    k_scan_sums<<<1, 256, 0, s>>>(sums, nb);
    k_scan_add<<<nb, 256, 0, s>>>(out, n, sums, nb);
    return cudaGetLastError();
}

static int grid_n(long long n, int cap_blocks = 0) {
    if (cap_blocks <= 0) cap_blocks = device_sms() * 16;
    long long b = (n + 255) / 256;
    if (b > cap_blocks) b = cap_blocks;
    return b < 1 ? 1 : (int)b;
}

// ================================================================== kernels
// Rate table (Sec. 2.1.1 / 2.1.5): nu_k(eps_j) = N_k sigma_k(eps_j) v(eps_j) with
// v = sqrt(2 e eps / m_e), evaluated in float64; row j holds the n_proc rates
// and, in column 7, their sum; nu_max = max_j of the sum.
template <class T>
__global__ void k_rate_table(const double* __restrict__ eps, const double* __restrict__ sigma,
                             const double* __restrict__ dens, int n_proc, int n_bins, T* __restrict__ tab,
                             double* __restrict__ tab64, unsigned long long* numax_bits) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_bins) return;
    const double v = sqrt(2.0 * kQ * eps[j] / kMe);
    double tot = 0.0;
    for (int k = 0; k < kTableStride; ++k) {
        double r = 0.0;
        if (k < n_proc) r = dens[k] * sigma[k * n_bins + j] * v;
        if (k < 7) { tab[j * kTableStride + k] = (T)r; tab64[j * kTableStride + k] = r; }
        tot += r;
    }
    tab[j * kTableStride + 7] = (T)tot;
    tab64[j * kTableStride + 7] = tot;
    atomicMax(numax_bits, (unsigned long long)__double_as_longlong(tot));
}

// Initial seeding (Sec. 2.3, Eq. 7 read with a negative exponent): per cell
// floor(n dV / w0) particles plus one with probability equal to the remainder.
__global__ void k_seed_count(Grid g, const uint8_t* __restrict__ mask, double n0, double R2, double cx, double cy,
                             double cz, double w0, Keys K, uint32_t* __restrict__ cnt) {
    const long long n = g.ncell();
    const double dV = g.dx * g.dx * g.dx;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        if (mask && mask[c]) { cnt[c] = 0; continue; }
        const int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / ((long long)g.nx * g.ny));
        const double xc = g.ox + ((double)i + 0.5) * g.dx;
        const double yc = g.oy + ((double)j + 0.5) * g.dx;
        const double zc = g.oz + ((double)k + 0.5) * g.dx;
        // axisymmetric: ring cell at radius xc around the axis, centre on the axis
        const double r2 = g.axi ? xc * xc + (zc - cz) * (zc - cz)
                                : (xc - cx) * (xc - cx) + (yc - cy) * (yc - cy) + (zc - cz) * (zc - cz);
        const double dVc = g.axi ? kPi * (double)(2 * i + 1) * g.dx * g.dx * g.dx : dV;
        // same operation order as the definition: n0 exp(-r2 / R^2) dV / w0
        const double expct = n0 * exp(-r2 / R2) * dVc / w0;
        const double fl = floor(expct);
        long long m = (long long)fl;
        const u32x4 o = philox(u32x4{(uint32_t)c, 0u, 0u, 0xB0000000u}, K.init0, K.init1);
        if (unif<double>(o.x) < expct - fl) ++m;
        if (m > 0x7fffffffLL) m = 0x7fffffffLL;
        cnt[c] = (uint32_t)m;
    }
}

template <class T>
__global__ void k_seed_write(Grid g, const uint32_t* __restrict__ cnt, const uint32_t* __restrict__ off, double w0,
                             uint64_t id0, Keys K, Soa<T> p, long long cap, DevState* st) {
    const long long n = g.ncell();
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const uint32_t m = cnt[c];
        if (!m) continue;
        const int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / ((long long)g.nx * g.ny));
        for (uint32_t q = 0; q < m; ++q) {
            const long long s = (long long)off[c] + q;
            if (s >= cap) { atomicOr(&st->err, kErrOutCapacity); return; }
            const u32x4 o = philox(u32x4{(uint32_t)c, q + 1u, 0u, 0xB0000000u}, K.init0, K.init1);
            if (g.axi) {
                // uniform in the ring: r^2 uniform in [i^2, (i+1)^2] dx^2, angle uniform
                const double r = g.dx * sqrt((double)i * i + unif<double>(o.x) * (double)(2 * i + 1));
                double sn, cs;
                sincospi(2.0 * unif<double>(o.y), &sn, &cs);
                p.r[PX][s] = (T)(r * cs);
                p.r[PY][s] = (T)(r * sn);
            } else {
                p.r[PX][s] = (T)(g.ox + ((double)i + unif<double>(o.x)) * g.dx);
                p.r[PY][s] = (T)(g.oy + ((double)j + unif<double>(o.y)) * g.dx);
            }
            p.r[PZ][s] = (T)(g.oz + ((double)k + unif<double>(o.z)) * g.dx);
            for (int d = VX; d <= AZ; ++d) p.r[d][s] = (T)0;
            p.r[PW][s] = (T)w0;
            p.id[s] = id0 + (uint64_t)s;
        }
    }
}

// Swarm start: Maxwellian components N(0, kT e / m_e) by Box-Muller on draw
// (id, step 0, k 0); all at the origin, weight 1, ids 0..n-1.
template <class T>
__global__ void k_seed_maxwell(long long n, double sig, Keys K, Soa<T> p) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const u32x4 o = draw_words(K, (uint64_t)i, 0u, 0u);
        const double u0 = unif<double>(o.x), u1 = unif<double>(o.y), u2 = unif<double>(o.z), u3 = unif<double>(o.w);
        const double r1 = sqrt(-2.0 * log(u0)), r2 = sqrt(-2.0 * log(u2));
        double s1, c1, s3, c3;
        sincospi(2.0 * u1, &s1, &c1);
        sincospi(2.0 * u3, &s3, &c3);
        p.r[VX][i] = (T)(sig * r1 * c1);
        p.r[VY][i] = (T)(sig * r1 * s1);
        p.r[VZ][i] = (T)(sig * r2 * c3);
        p.r[PX][i] = p.r[PY][i] = p.r[PZ][i] = (T)0;
        p.r[AX][i] = p.r[AY][i] = p.r[AZ][i] = (T)0;
        p.r[PW][i] = (T)1;
        p.id[i] = (uint64_t)i;
    }
}

template <class TI, class T>
__global__ void k_pack_field(const TI* __restrict__ Ex, const TI* __restrict__ Ey, const TI* __restrict__ Ez,
                             long long n, T* __restrict__ E4) {
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        E4[4 * c] = (T)Ex[c];
        E4[4 * c + 1] = (T)Ey[c];
        E4[4 * c + 2] = (T)Ez[c];
        E4[4 * c + 3] = (T)0;
    }
}

// n = q / (2^32 dV); rho = e (n_pos - n_neg - n_e).
__global__ void k_fixed_to_rho(const long long* __restrict__ qe, const long long* __restrict__ qp,
                               const long long* __restrict__ qn, long long n, double inv, double* __restrict__ rho,
                               int nr) {
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        // axisymmetric (nr > 0): ring volume pi (2i + 1) dx^3, inv = 1 / (2^32 pi dx^3)
        const double iv = nr > 0 ? inv / (double)(2 * (int)(c % nr) + 1) : inv;
        const double ne = (double)qe[c] * iv, np = (double)qp[c] * iv, nn = (double)qn[c] * iv;
        rho[c] = kQ * (np - nn - ne);
    }
}

// Right-hand side of the float32 solve: h^2 rho / eps0 in float, the three
// fixed-point charges combined in 64-bit integers first (exact) and
// converted once.
__global__ void k_fixed_to_hrho(const long long* __restrict__ qe, const long long* __restrict__ qp,
                                const long long* __restrict__ qn, long long n, float scale, float* __restrict__ hrho) {
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        hrho[c] = scale * __ll2float_rn(qp[c] - qn[c] - qe[c]);
}

// Next step's input count; cursors that ran past the capacity (an error
// already flagged) are clamped so no kernel reads beyond the buffers.
// Warm start of the coupled solve: phi <- 2 phi_n - phi_{n-1} (linear
// extrapolation in time), phi_prev <- phi_n.  With no history, only the copy.
__global__ void k_extrapolate(double* __restrict__ phi, double* __restrict__ prev, long long n, int have_prev) {
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const double p = phi[c];
        if (have_prev) phi[c] = 2.0 * p - prev[c];
        prev[c] = p;
    }
}

__global__ void k_end_step(DevState* st, long long* count_slot, long long cap) {
    st->n_updates += st->n_in;
    st->n_parents += st->n_in;
    st->n_spill = 0;
    st->n_in = st->n_out < (unsigned long long)cap ? st->n_out : (unsigned long long)cap;
    st->n_fetch = 0;
    st->n_fetch_c = 0;
    st->n_out = 0;
    st->n_child = 0;
    if (count_slot) *count_slot = (long long)st->n_in;
}

// End-of-step statistics for the time-step control (Sec. 2.1.4): the
// largest and total fixed-point electron deposit (for the dielectric
// relaxation time and the growth limit).  The speed histogram for the 90 %
// quantile of the CFL condition is formed by the kernels that store the
// electrons (the collision kernels' output flush and the photoelectron
// append).  Each thread takes kStatsUnroll cells per trip, one grid stride
// apart, with all their loads issued before any use.
constexpr int kStatsUnroll = 4;

__global__ void k_step_stats(const unsigned long long* __restrict__ qe, long long ncell, int nr, DevState* st) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long mx = LLONG_MIN, sm = 0;
    for (long long c0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; c0 < ncell; c0 += kStatsUnroll * stride) {
        long long q[kStatsUnroll];
#pragma unroll
        for (int u = 0; u < kStatsUnroll; ++u) {
            const long long c = c0 + u * stride;
            q[u] = c < ncell ? (long long)qe[c] : 0;
        }
#pragma unroll
        for (int u = 0; u < kStatsUnroll; ++u) {
            const long long c = c0 + u * stride;
            if (c < ncell) {
                // axisymmetric (nr > 0): the maximum of q / (2i + 1), proportional to the density
                const long long qd = nr > 0 ? q[u] / (2 * (long long)(c % nr) + 1) : q[u];
                mx = qd > mx ? qd : mx;
                sm += q[u];
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const long long om = __shfl_xor_sync(kFull, mx, o);
        mx = om > mx ? om : mx;
        sm += __shfl_xor_sync(kFull, sm, o);
    }
    // one atomic per block and quantity (every block's warps would otherwise
    // queue on the same two addresses)
    __shared__ long long wmx[32], wsm[32];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        wmx[w] = mx;
        wsm[w] = sm;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) {
            mx = wmx[q] > mx ? wmx[q] : mx;
            sm += wsm[q];
        }
        atomicMax(&st->qe_max, mx);
        atomicAdd(&st->qe_sum, (unsigned long long)sm);
    }
}

// Clears error bits (a speculative field solve that was undone).
__global__ void k_clear_err(DevState* st, unsigned bits) { st->err &= ~bits; }

// Head of the float32 field-solve graph: a speculative solve goes ahead only
// when the step that was just pushed needs neither a weight update (its
// count above gate_thr) nor further product generations, and raised no error:
// the test the host applies to the same values once it has read them.
__global__ void k_solve_gate(const DevState* st, cudaGraphConditionalHandle h, unsigned long long cap) {
    bool go = true;
    if (st->gate_spec) {
        const unsigned long long n = st->n_out < cap ? st->n_out : cap;
        go = st->err == 0 && st->n_spill == 0 && !(n > 0 && (double)(long long)n > st->gate_thr);
    }
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

__global__ void k_gate_set(DevState* st, int spec, double thr) {
    st->gate_spec = spec;
    st->gate_thr = thr;
}

// Before children generation g >= 1: the queue it will spill into starts empty.
__global__ void k_next_generation(DevState* st, int gen) {
    st->n_fetch_c = 0;
    if (gen & 1) st->n_child = 0;
    else st->n_spill = 0;
}

__global__ void k_set_count(DevState* st, unsigned long long n) {
    st->n_in = n;
    st->n_fetch = 0;
    st->n_fetch_c = 0;
    st->n_out = 0;
    st->n_child = 0;
    st->n_extra = 0;
}

// Cell index in the particle precision (the same decision as the electrode test).
template <class T>
__device__ __forceinline__ uint32_t cell_index(T x, T y, T z, T ox, T oy, T oz, T dx, int nx, int ny, int nz) {
    const int i = fold_idx((int)floor((x - ox) / dx), nx);
    const int j = fold_idx((int)floor((y - oy) / dx), ny);
    const int k = fold_idx((int)floor((z - oz) / dx), nz);
    return (uint32_t)(((long long)k * ny + j) * nx + i);
}

struct GridT {
    double ox, oy, oz, dx;
    int nx, ny, nz, axi;
};

// ---------------------------------------------------------------- cell sort
template <class T>
__global__ void k_cell_count(const Soa<T> p, const DevState* st, GridT g, uint32_t* __restrict__ cnt,
                             uint32_t* __restrict__ key, uint32_t* __restrict__ rank) {
    const long long n = (long long)st->n_in;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        T x = p.r[PX][i], y = p.r[PY][i];
        if (g.axi) {
            x = sqrt(x * x + y * y);
            y = (T)g.oy + (T)0.5 * (T)g.dx;
        }
        const uint32_t c = cell_index<T>(x, y, p.r[PZ][i], (T)g.ox, (T)g.oy, (T)g.oz, (T)g.dx, g.nx, g.ny, g.nz);
        key[i] = c;
        rank[i] = atomicAdd(&cnt[c], 1u);
    }
}

template <class T>
__global__ void k_scatter(const Soa<T> a, Soa<T> b, const DevState* st, const uint32_t* __restrict__ start,
                          const uint32_t* __restrict__ key, const uint32_t* __restrict__ rank) {
    const long long n = (long long)st->n_in;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long d = (long long)start[key[i]] + rank[i];
#pragma unroll
        for (int f = 0; f < 10; ++f) b.r[f][d] = a.r[f][i];
        b.id[d] = a.id[i];
    }
}

// ---------------------------------------------------------------- weight update
// Sec. 2.1.2, Eq. 3: desired weight omega = max(W_cell / N_ppc, w_min); the
// per-cell weight W is summed as integers rint(w 2^24) so it does not depend
// on the order of the particles.
constexpr double kS24 = 16777216.0;

__device__ __forceinline__ double omega_of(long long W, int n_ppc, double w_min) {
    return fmax((double)W / kS24 / (double)n_ppc, w_min);
}

// Exact float64 operations done with integer instructions (the float64 pipe
// of this part is narrow): the same results as the float64 conversions.
// float -> double (exact: rebias the exponent, widen the significand).
__device__ __forceinline__ double f2d_exact(float x) {
    const unsigned u = __float_as_uint(x);
    const unsigned e = (u >> 23) & 0xffu;
    if (e == 0u || e == 255u) return (double)x;  // zero, subnormal, inf, NaN: the conversion instruction
    const unsigned long long b = ((unsigned long long)(u >> 31) << 63) | ((unsigned long long)(e + 896u) << 52) |
                                 ((unsigned long long)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)b);
}
__device__ __forceinline__ double to_d(float x) { return f2d_exact(x); }
__device__ __forceinline__ double to_d(double x) { return x; }
// unif<double>(w) = (2 (w >> 9) + 1) 2^-24, built from its bits
__device__ __forceinline__ double unif_d_exact(uint32_t w) {
    const unsigned v = 2u * (w >> 9) + 1u;  // odd, below 2^24
    const int pb = 31 - __clz(v);           // leading bit
    const unsigned long long mant = ((unsigned long long)v << (52 - pb)) & 0xfffffffffffffull;
    return __longlong_as_double((long long)(((unsigned long long)(pb - 24 + 1023) << 52) | mant));
}
// rint(w 2^24) of a float weight, rounded to nearest even: the value of
// __double2ll_rn((double)w * 2^24) by integer arithmetic
__device__ __forceinline__ long long fix24(float w) {
    const unsigned u = __float_as_uint(w);
    const int e = (int)((u >> 23) & 0xffu);
    if (e == 0 || e == 255) return __double2ll_rn((double)w * kS24);
    const long long m = (long long)((u & 0x7fffffu) | 0x800000u);  // w = m 2^(e - 150)
    const int sh = e - 126;                                         // w 2^24 = m 2^sh
    long long r;
    if (sh >= 0) {
        r = m << sh;
    } else if (sh < -25) {
        r = 0;
    } else {
        const int k = -sh;
        const long long q = m >> k, rem = m & ((1ll << k) - 1), half = 1ll << (k - 1);
        r = q + ((rem > half || (rem == half && (q & 1))) ? 1 : 0);
    }
    return (u >> 31) ? -r : r;
}
__device__ __forceinline__ long long fix24(double w) { return __double2ll_rn(w * kS24); }
// x < lo and x > hi of a float against float64 thresholds, as float compares
// (the thresholds rounded up, respectively down, to float: exact equivalents)
__device__ __forceinline__ bool lt_d(float x, double lo) { return x < __double2float_ru(lo); }
__device__ __forceinline__ bool lt_d(double x, double lo) { return x < lo; }
__device__ __forceinline__ bool gt_d(float x, double hi) { return x > __double2float_rd(hi); }
__device__ __forceinline__ bool gt_d(double x, double hi) { return x > hi; }

// Predicted particle count after the merge and split, in 2^-24 units:
// sum over cells of W / omega.  A warp takes 32 consecutive cells (one load
// of their bounds per lane) and sums the weights of each occupied one with
// all its lanes; the fixed-point sums are exact, so their order is free.
// The occupied cells are listed in occ (any order) for the merge kernel.
template <class T>
__global__ void k_cell_weight(const Soa<T> p, const uint32_t* __restrict__ start, long long ncell, int n_ppc,
                              double w_min, uint32_t* __restrict__ occ_list, DevState* st) {
    const int lane = threadIdx.x & 31;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    long long acc = 0;
    for (long long c0 = gw * 32; c0 < ncell; c0 += nw * 32) {
        const long long cl = c0 + lane;
        const uint32_t a0 = cl < ncell ? start[cl] : 0u, a1 = cl < ncell ? start[cl + 1] : 0u;
        unsigned occ = __ballot_sync(kFull, a1 > a0);
        if (occ) {
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(&st->n_occ, (unsigned long long)__popc(occ));
            base = __shfl_sync(kFull, base, 0);
            if (a1 > a0) occ_list[base + __popc(occ & ((1u << lane) - 1u))] = (uint32_t)cl;
        }
        long long Wc = 0;  // this lane's cell, for the divisions done in parallel below
        while (occ) {
            const int b = __ffs(occ) - 1;
            occ &= occ - 1;
            const uint32_t s0 = __shfl_sync(kFull, a0, b), s1 = __shfl_sync(kFull, a1, b);
            long long W = 0;
            for (uint32_t t = s0 + lane; t < s1; t += 32) W += fix24(p.r[PW][t]);
            for (int o = 16; o > 0; o >>= 1) W += __shfl_xor_sync(kFull, W, o);
            if (lane == b) Wc = W;
        }
        if (a1 > a0) acc += __double2ll_rn((double)Wc / omega_of(Wc, n_ppc, w_min));
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
    if (lane == 0 && acc) atomicAdd((unsigned long long*)&st->pred_total, (unsigned long long)acc);
}

template <class T> __device__ __forceinline__ double speed2_key(const Soa<T>& p, long long i) {
    const T a = p.r[VX][i], b = p.r[VY][i], c = p.r[VZ][i];
    const T r = (a * a + b * b) + c * c;
    return to_d(r);
}

struct MergeScratch {
    double* key;
    uint64_t* id;
    uint32_t* idx;
    double* skey;
    uint64_t* sid;
    uint32_t* sidx;
};

constexpr int kSortMax = 8192;  // candidates sorted in (dynamic) shared memory (else ranked in global memory)
constexpr size_t kMergeSmem = (size_t)kSortMax * (8 + 8 + 4);

// One block per occupied cell.  Merge: candidates w < (2/3) omega ordered by
// (|v|^2, id) are paired (0,1), (2,3), ...; the pair's weights are summed and
// one member's state is kept with probability proportional to its weight
// (draw keyed by the smaller id, the step and the round); rounds repeat while
// two or more candidates remain.  Split: w > (3/2) omega is halved m times
// (m minimal with w / 2^m <= (3/2) omega) and 2^m - 1 identical copies are
// appended after the n sorted particles.  In shared memory the candidates are
// sorted once: the survivors of a round (one member of each pair of a sorted
// list, then the odd last one) are written back in their order, which is the
// order a new sort would give.
template <class T>
__global__ void __launch_bounds__(256) k_merge_split(Soa<T> p, long long n, const uint32_t* __restrict__ start,
                                                     long long ncell, int n_ppc, double w_min, double scale,
                                                     MergeScratch sc, Keys K, uint32_t step, long long cap,
                                                     const uint32_t* __restrict__ cells, DevState* st) {
    __shared__ int m_sh, m2_sh;
    __shared__ long long wsum_sh;
    __shared__ int wtot[8];
    extern __shared__ __align__(16) unsigned char merge_raw[];
    unsigned long long* sk = reinterpret_cast<unsigned long long*>(merge_raw);
    unsigned long long* sid = sk + kSortMax;
    uint32_t* six = reinterpret_cast<uint32_t*>(sid + kSortMax);
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    // every cell, or only the listed ones (cells the warp kernel left to this one)
    const long long nc = cells ? (long long)st->n_big : ncell;
    for (long long ci = blockIdx.x; ci < nc; ci += gridDim.x) {
        const long long c = cells ? (long long)cells[ci] : ci;
        const uint32_t s0 = start[c], s1 = start[c + 1];
        if (s0 == s1) continue;
        if (threadIdx.x == 0) { m_sh = 0; wsum_sh = 0; }
        __syncthreads();
        long long Wp = 0;
        for (uint32_t t = s0 + threadIdx.x; t < s1; t += blockDim.x) Wp += fix24(p.r[PW][t]);
        for (int o = 16; o > 0; o >>= 1) Wp += __shfl_xor_sync(kFull, Wp, o);
        if ((threadIdx.x & 31) == 0) atomicAdd((unsigned long long*)&wsum_sh, (unsigned long long)Wp);
        __syncthreads();
        const double om = omega_of(wsum_sh, n_ppc, w_min) * scale;
        const double lo = 2.0 * om / 3.0, hi = 1.5 * om;
        // candidates
        for (uint32_t t = s0 + threadIdx.x; t < s1; t += blockDim.x) {
            if (lt_d(p.r[PW][t], lo)) {
                const int q = atomicAdd(&m_sh, 1);
                sc.key[s0 + q] = speed2_key(p, t);
                sc.id[s0 + q] = p.id[t];
                sc.idx[s0 + q] = t;
            }
        }
        __syncthreads();
        int m = m_sh;
        if (m <= kSortMax) {
            // shared-memory bitonic sort of (|v|^2 bits, id), padded to a power of two
            for (int t = threadIdx.x; t < m; t += blockDim.x) {
                sk[t] = (unsigned long long)__double_as_longlong(sc.key[s0 + t]);
                sid[t] = sc.id[s0 + t];
                six[t] = sc.idx[s0 + t];
            }
            {
                int P = 1;
                while (P < m) P <<= 1;
                for (int t = m + threadIdx.x; t < P; t += blockDim.x) { sk[t] = ~0ull; sid[t] = ~0ull; six[t] = 0; }
                __syncthreads();
                for (int kk = 2; kk <= P; kk <<= 1)
                    for (int jj = kk >> 1; jj > 0; jj >>= 1) {
                        for (int t = threadIdx.x; t < P; t += blockDim.x) {
                            const int u = t ^ jj;
                            if (u > t) {
                                const bool up = (t & kk) == 0;
                                const bool gt = sk[t] > sk[u] || (sk[t] == sk[u] && sid[t] > sid[u]);
                                if (gt == up) {
                                    const unsigned long long a1 = sk[t], a2 = sid[t];
                                    const uint32_t a3 = six[t];
                                    sk[t] = sk[u]; sid[t] = sid[u]; six[t] = six[u];
                                    sk[u] = a1; sid[u] = a2; six[u] = a3;
                                }
                            }
                        }
                        __syncthreads();
                    }
            }
            for (uint32_t round = 0; m >= 2; ++round) {
                const bool odd = (m & 1) != 0;
                const unsigned long long lk = odd ? sk[m - 1] : 0ull, lid = odd ? sid[m - 1] : 0ull;
                const uint32_t lix = odd ? six[m - 1] : 0u;
                int m2 = 0;
                // pairs in chunks of 256 (one per thread): all of a chunk's pairs are
                // read before its survivors are written, in pair order, below them
                for (int q0 = 0; q0 < m / 2; q0 += 256) {
                    const int q = q0 + threadIdx.x;
                    bool ok = false;
                    unsigned long long rk = 0, rid = 0;
                    uint32_t rix = 0;
                    if (q < m / 2) {
                        const uint32_t ia = six[2 * q], ib = six[2 * q + 1];
                        const uint64_t da = sid[2 * q], db = sid[2 * q + 1];
                        const T wa = p.r[PW][ia], wb = p.r[PW][ib];
                        const uint64_t mid = da < db ? da : db;
                        const u32x4 o = draw_words(K, mid, step, 0xC0000000u | round);
                        const double u = unif_d_exact(o.x);
                        const double dwa = to_d(wa);
                        const bool keep_a = u * (dwa + to_d(wb)) < dwa;
                        const uint32_t keep = keep_a ? ia : ib, drop = keep_a ? ib : ia;
                        const T ws = wa + wb;
                        p.r[PW][keep] = ws;
                        p.r[PW][drop] = (T)0;
                        if (lt_d(ws, lo)) {
                            ok = true;
                            rk = keep_a ? sk[2 * q] : sk[2 * q + 1];
                            rid = keep_a ? da : db;
                            rix = keep;
                        }
                    }
                    const unsigned bal = __ballot_sync(kFull, ok);
                    if (lane == 0) wtot[wq] = __popc(bal);
                    __syncthreads();
                    int off = m2, tot = 0;
                    for (int x = 0; x < 8; ++x) {
                        if (x < wq) off += wtot[x];
                        tot += wtot[x];
                    }
                    if (ok) {
                        const int t = off + __popc(bal & ((1u << lane) - 1u));
                        sk[t] = rk; sid[t] = rid; six[t] = rix;
                    }
                    m2 += tot;
                    __syncthreads();
                }
                if (odd) {
                    if (threadIdx.x == 0) { sk[m2] = lk; sid[m2] = lid; six[m2] = lix; }
                    ++m2;
                }
                __syncthreads();
                if (m2 == m) break;
                m = m2;
            }
        } else {
        for (uint32_t round = 0; m >= 2; ++round) {
            // rank by counting: position of each candidate in (key, id) order
            for (int a = threadIdx.x; a < m; a += blockDim.x) {
                const double ka = sc.key[s0 + a];
                const uint64_t ia = sc.id[s0 + a];
                int r = 0;
                for (int b = 0; b < m; ++b) {
                    const double kb = sc.key[s0 + b];
                    r += (kb < ka) || (kb == ka && sc.id[s0 + b] < ia);
                }
                sc.skey[s0 + r] = ka;
                sc.sid[s0 + r] = ia;
                sc.sidx[s0 + r] = sc.idx[s0 + a];
            }
            if (threadIdx.x == 0) m2_sh = 0;
            __syncthreads();
            for (int q = threadIdx.x; q < m / 2; q += blockDim.x) {
                const uint32_t ia = sc.sidx[s0 + 2 * q], ib = sc.sidx[s0 + 2 * q + 1];
                const uint64_t da = sc.sid[s0 + 2 * q], db = sc.sid[s0 + 2 * q + 1];
                const T wa = p.r[PW][ia], wb = p.r[PW][ib];
                const uint64_t mid = da < db ? da : db;
                const u32x4 o = draw_words(K, mid, step, 0xC0000000u | round);
                const double u = unif<double>(o.x);
                const bool keep_a = u * ((double)wa + (double)wb) < (double)wa;
                const uint32_t keep = keep_a ? ia : ib, drop = keep_a ? ib : ia;
                const T ws = wa + wb;
                p.r[PW][keep] = ws;
                p.r[PW][drop] = (T)0;
                if ((double)ws < lo) {
                    const int s = atomicAdd(&m2_sh, 1);
                    sc.key[s0 + s] = keep_a ? sc.skey[s0 + 2 * q] : sc.skey[s0 + 2 * q + 1];
                    sc.id[s0 + s] = keep_a ? da : db;
                    sc.idx[s0 + s] = keep;
                }
            }
            if ((m & 1) && threadIdx.x == 0) {
                const int s = atomicAdd(&m2_sh, 1);
                sc.key[s0 + s] = sc.skey[s0 + m - 1];
                sc.id[s0 + s] = sc.sid[s0 + m - 1];
                sc.idx[s0 + s] = sc.sidx[s0 + m - 1];
            }
            __syncthreads();
            const int m2 = m2_sh;
            __syncthreads();
            if (m2 == m) break;
            m = m2;
        }
        }
        // split
        for (uint32_t t = s0 + threadIdx.x; t < s1; t += blockDim.x) {
            const T w = p.r[PW][t];
            if (!((double)w > hi)) continue;
            int mm = 0;
            double wc = (double)w;
            while (wc > hi && mm < 30) { wc *= 0.5; ++mm; }   // hi >= 1.5 w / N_ppc bounds mm far below 30
            const T wn = (T)ldexp((double)w, -mm);
            p.r[PW][t] = wn;
            const unsigned long long copies = (1ull << mm) - 1ull;
            const unsigned long long base = atomicAdd(&st->n_extra, copies);
            for (unsigned long long q = 0; q < copies; ++q) {
                const long long d = n + (long long)(base + q);
                if (d >= cap) { atomicOr(&st->err, kErrSplitCapacity); break; }
                for (int f = 0; f < 10; ++f) p.r[f][d] = p.r[f][t];
                p.r[PW][d] = wn;
                p.id[d] = derived_id(K, p.id[t], step, 0x40000000u | (uint32_t)(q + 1));
            }
        }
        __syncthreads();
    }
}

// The same merge and split with one warp per cell (eight cells per block at
// a time, warp barriers only), for cells with at most kWarpSort merge
// candidates: warps take the occupied cells listed by k_cell_weight one at a
// time from a shared cursor, gather a cell's candidates
// with a ballot into its shared arrays, sorts them once by the same bitonic
// network (warp-synchronous stages), and pairs and draws exactly as above,
// round after round; the survivors (kept in their sorted order) and the odd
// one form the next round's list, which the block kernel's sort would leave
// unchanged.  Cells with more candidates are listed for k_merge_split (their
// split is left to it too).
constexpr int kWarpSort = 256;
constexpr int kWarpPairs = kWarpSort / 2 / 32;

template <class T>
__global__ void __launch_bounds__(256) k_merge_split_warp(Soa<T> p, long long n, const uint32_t* __restrict__ start,
                                                          const uint32_t* __restrict__ occ_list, int n_ppc,
                                                          double w_min, double scale, Keys K, uint32_t step,
                                                          long long cap, uint32_t* big, DevState* st) {
    __shared__ unsigned long long wsk[8][kWarpSort], wsid[8][kWarpSort];
    __shared__ uint32_t wsix[8][kWarpSort];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    unsigned long long* sk = wsk[w];
    unsigned long long* sid = wsid[w];
    uint32_t* six = wsix[w];
    const unsigned long long n_occ = st->n_occ;
    // warps take the occupied cells one at a time from a shared cursor, so
    // dense cells (long merges) spread over the whole GPU
    for (;;) {
        unsigned long long it = 0;
        if (lane == 0) it = atomicAdd(&st->n_occ_fetch, 1ull);
        it = __shfl_sync(kFull, it, 0);
        if (it >= n_occ) break;
        const long long c = (long long)occ_list[it];
        const uint32_t s0 = start[c], s1 = start[c + 1];
        long long Wp = 0;
        for (uint32_t t = s0 + lane; t < s1; t += 32) Wp += fix24(p.r[PW][t]);
        for (int o = 16; o > 0; o >>= 1) Wp += __shfl_xor_sync(kFull, Wp, o);
        const double om = omega_of(Wp, n_ppc, w_min) * scale;
        const double lo = 2.0 * om / 3.0, hi = 1.5 * om;
        int m = 0;
        for (uint32_t b = s0; b < s1; b += 32) {
            const uint32_t t = b + lane;
            const bool cand = t < s1 && lt_d(p.r[PW][t], lo);
            const unsigned bal = __ballot_sync(kFull, cand);
            if (cand) {
                const int q = m + __popc(bal & lt);
                if (q < kWarpSort) {
                    sk[q] = (unsigned long long)__double_as_longlong(speed2_key(p, t));
                    sid[q] = p.id[t];
                    six[q] = t;
                }
            }
            m += __popc(bal);
        }
        if (m > kWarpSort) {
            if (lane == 0) big[atomicAdd(&st->n_big, 1ull)] = (uint32_t)c;
            continue;
        }
        __syncwarp();
        for (uint32_t round = 0; m >= 2; ++round) {
            if (round == 0) {
                // the survivors of later rounds stay in (key, id) order: pairs of a
                // sorted list keep one member each, and the odd last one is the largest
                int P = 1;
                while (P < m) P <<= 1;
                for (int t = m + lane; t < P; t += 32) { sk[t] = ~0ull; sid[t] = ~0ull; six[t] = 0; }
                __syncwarp();
                for (int kk = 2; kk <= P; kk <<= 1)
                    for (int jj = kk >> 1; jj > 0; jj >>= 1) {
                        for (int t = lane; t < P; t += 32) {
                            const int u = t ^ jj;
                            if (u > t) {
                                const bool up = (t & kk) == 0;
                                const bool gt = sk[t] > sk[u] || (sk[t] == sk[u] && sid[t] > sid[u]);
                                if (gt == up) {
                                    const unsigned long long x1 = sk[t], x2 = sid[t];
                                    const uint32_t x3 = six[t];
                                    sk[t] = sk[u]; sid[t] = sid[u]; six[t] = six[u];
                                    sk[u] = x1; sid[u] = x2; six[u] = x3;
                                }
                            }
                        }
                        __syncwarp();
                    }
            }
            // pair q = lane + 32 j; all pairs are read before any slot is rewritten
            unsigned long long rk[kWarpPairs], rid[kWarpPairs];
            uint32_t rix[kWarpPairs];
            bool rok[kWarpPairs];
#pragma unroll
            for (int j = 0; j < kWarpPairs; ++j) {
                const int q = lane + 32 * j;
                rok[j] = false;
                rk[j] = 0; rid[j] = 0; rix[j] = 0;
                if (q < m / 2) {
                    const uint32_t ia = six[2 * q], ib = six[2 * q + 1];
                    const uint64_t da = sid[2 * q], db = sid[2 * q + 1];
                    const T wa = p.r[PW][ia], wb = p.r[PW][ib];
                    const uint64_t mid = da < db ? da : db;
                    const u32x4 o = draw_words(K, mid, step, 0xC0000000u | round);
                    const double u = unif_d_exact(o.x);
                    const double dwa = to_d(wa);
                    const bool keep_a = u * (dwa + to_d(wb)) < dwa;
                    const uint32_t keep = keep_a ? ia : ib, drop = keep_a ? ib : ia;
                    const T ws = wa + wb;
                    p.r[PW][keep] = ws;
                    p.r[PW][drop] = (T)0;
                    if (lt_d(ws, lo)) {
                        rok[j] = true;
                        rk[j] = keep_a ? sk[2 * q] : sk[2 * q + 1];
                        rid[j] = keep_a ? da : db;
                        rix[j] = keep;
                    }
                }
            }
            const bool odd = (m & 1) != 0;
            const unsigned long long lk = odd ? sk[m - 1] : 0ull, lid = odd ? sid[m - 1] : 0ull;
            const uint32_t lix = odd ? six[m - 1] : 0u;
            __syncwarp();
            // order-preserving compaction of the survivors, then the odd one
            int m2 = 0;
#pragma unroll
            for (int j = 0; j < kWarpPairs; ++j) {
                const unsigned bal = __ballot_sync(kFull, rok[j]);
                if (rok[j]) {
                    const int t = m2 + __popc(bal & lt);
                    sk[t] = rk[j]; sid[t] = rid[j]; six[t] = rix[j];
                }
                m2 += __popc(bal);
            }
            if (odd) {
                if (lane == 0) { sk[m2] = lk; sid[m2] = lid; six[m2] = lix; }
                ++m2;
            }
            __syncwarp();
            if (m2 == m) break;
            m = m2;
        }
        // split
        for (uint32_t t = s0 + lane; t < s1; t += 32) {
            const T wt = p.r[PW][t];
            if (!gt_d(wt, hi)) continue;
            int mm = 0;
            double wc = (double)wt;
            while (wc > hi && mm < 30) { wc *= 0.5; ++mm; }   // hi >= 1.5 w / N_ppc bounds mm far below 30
            const T wn = (T)ldexp((double)wt, -mm);
            p.r[PW][t] = wn;
            const unsigned long long copies = (1ull << mm) - 1ull;
            const unsigned long long base = atomicAdd(&st->n_extra, copies);
            for (unsigned long long q = 0; q < copies; ++q) {
                const long long d = n + (long long)(base + q);
                if (d >= cap) { atomicOr(&st->err, kErrSplitCapacity); break; }
                for (int f = 0; f < 10; ++f) p.r[f][d] = p.r[f][t];
                p.r[PW][d] = wn;
                p.id[d] = derived_id(K, p.id[t], step, 0x40000000u | (uint32_t)(q + 1));
            }
        }
        __syncwarp();
    }
}

// Copies live particles (w > 0) of a into b with a warp-aggregated cursor.
template <class T>
__global__ void k_compact(const Soa<T> a, long long n, Soa<T> b, DevState* st) {
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarp = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long base = warp * 32; base < n; base += nwarp * 32) {
        const long long i = base + lane;
        const bool live = i < n && a.r[PW][i] > (T)0;
        const unsigned m = __ballot_sync(kFull, live);
        if (!m) continue;
        unsigned long long s0 = 0;
        const int leader = __ffs(m) - 1;
        if (lane == leader) s0 = atomicAdd(&st->n_out, (unsigned long long)__popc(m));
        s0 = __shfl_sync(kFull, s0, leader);
        if (live) {
            const long long d = (long long)(s0 + __popc(m & ((1u << lane) - 1u)));
#pragma unroll
            for (int f = 0; f < 10; ++f) b.r[f][d] = a.r[f][i];
            b.id[d] = a.id[i];
        }
    }
}

// ---------------------------------------------------------------- swarm moments
// Accumulators are zeroed by the host; nothing else here.

}  // namespace pic

// ====================================================================== context
using namespace pic;

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
    size_t total = 0;
    size_t buf[2], cq[2], table, table64, E4, E4b, qe, qp, qn, st, cnt, start, sums, key, rank, msc, gas, rho, phi,
        phi_prev, phi_x, phi_y, mg, photo, hostio;
};

static size_t real_size(int prec) { return prec == 64 ? 8 : 4; }

static long long photo_cap(const pic_config* c);

static Layout make_layout(const pic_config* c) {
    Layout L;
    const size_t R = real_size(c->precision);
    const size_t cap = (size_t)c->capacity;
    const size_t ncell = (size_t)c->nx * c->ny * c->nz;
    size_t o = 0;
    auto take = [&](size_t b) { size_t r = o; o += al256(b); return r; };
    for (int b = 0; b < 2; ++b) {
        L.buf[b] = o;
        for (int f = 0; f < 10; ++f) take(cap * R);
        take(cap * 8);
    }
    for (int qq = 0; qq < 2; ++qq) {
        L.cq[qq] = o;
        for (int f = 0; f < 11; ++f) take(cap * R);  // 10 fields + t_left
        take(cap * 8);
        take(cap * 4);                               // draw index of the ionization
    }
    const int nb = c->gas.n_bins > 0 ? c->gas.n_bins : 2;
    L.table = take((size_t)nb * kTableStride * R);
    L.table64 = take((size_t)nb * kTableStride * 8);
    L.E4 = take(ncell * 4 * R);
    // float32 Cartesian coupled contexts alternate between two packed fields
    // (the solve writes the one the current push does not read)
    const bool pair = c->coupled && c->precision == 32 && c->geometry == 0;
    L.E4b = pair ? take(ncell * 4 * R) : L.E4;
    L.qe = take(ncell * 8);
    L.qp = take(ncell * 8);
    L.qn = take(ncell * 8);
    L.st = take(sizeof(DevState) + 64);
    L.cnt = take((ncell + 1) * 4);
    L.start = take((ncell + 1) * 4);
    L.sums = take(((ncell + 1) / kScanTile + 2) * 4);
    L.key = take(cap * 4);
    L.rank = take(cap * 4);
    L.msc = o;
    take(cap * 8); take(cap * 8); take(cap * 4); take(cap * 8); take(cap * 8); take(cap * 4);
    L.gas = take(((size_t)(c->gas.n_proc > 0 ? c->gas.n_proc : 1) + 1) * nb * 8 + 64 * 8);
    L.rho = take(ncell * 8);
    // a potential slot holds ncell doubles, or a float pair: hi, then lo at
    // the next 256-byte boundary (the pair kernels use 16-byte accesses)
    const size_t slot = 2 * al256(ncell * 4);
    L.phi = take(slot);
    L.phi_prev = take(slot);
    L.phi_x = take(slot);
    L.phi_y = pair ? take(slot) : L.phi_x;
    L.mg = take(c->geometry == 1 ? AxiMG::bytes(c->nx, c->nz) : MG::bytes(c->nx, c->ny, c->nz, c->precision == 32, false));
    {
        const size_t np = (size_t)photo_cap(c);
        L.photo = o;
        for (int f = 0; f < 8; ++f) take(np * R);
        take(np * 8);
        take(np * 8);
        take(np * 4);
    }
    L.hostio = 0;
    L.total = o;
    return L;
}

struct pic_ctx {
    pic_config cfg;
    int prec;
    cudaStream_t s;
    char* ws;
    Layout L;
    Grid g;
    Keys K;
    const uint8_t* mask;
    int cur = 0;
    long long n_host = 0;       // live particles (valid after any synchronising call)
    long long n_last_wu = 0;    // count after the last weight update
    uint32_t step = 0;
    int a_valid = 0;
    int field_valid = 0;
    int field_uniform = 0;
    double E0[3] = {0, 0, 0};
    double nu_max = 0, l0 = 0, inv_dl = 0;
    int n_proc = 0, n_bins = 0;
    int kind[8];
    double thr[8], mratio[8];
    int grid_push = 0;
    MG mg;
    AxiMG amg;  // coupled solve of axisymmetric contexts
    std::string err;
    long long n_wu = 0, n_sorts = 0;
    int last_cycles = 0;
    double last_rel = 0;
    long long steps_done = 0;
    long long n_next = 0;     // particle count after the step being run (known once its children finished)
    double dt_cur = 0, dt_prev = 0, dt_next = 0;  // time steps (fixed unless adaptive_dt)
    double w_prev = 0, ne_max = 0, t_total = 0;
    long long n_solves = 0;   // coupled solves so far (the warm start extrapolates after two)
    long long launches = 0;   // kernels launched by pic_step (for the profile)
    unsigned long long dev_kernels_seen = 0;  // DevState::dev_kernels already counted in launches
    // Float32 coupled field solve as one graph per current-potential slot
    // (prologue, device-driven solve, report); used from the third solve on.
    cudaGraphExec_t fgraph[4] = {nullptr, nullptr, nullptr, nullptr};
    long long fgraph_kernels[4] = {0, 0, 0, 0};
    // Speculative field solve (float32 Cartesian coupled steps): the step's
    // device state is copied to pinned host memory and the solve is enqueued
    // before the host looks at it.
    DevState* hs = nullptr;
    cudaEvent_t ev_state = nullptr;
    // Host exchanges under the speculative solve: ev_parts is recorded once a
    // speculative step's particles are final, before its solve is enqueued;
    // parts_event says that no work touching the particle buffers has been
    // enqueued since, so pic_download and pic_upload may copy on xs (waiting
    // for ev_parts only) while the solve runs.
    cudaStream_t xs = nullptr;
    cudaEvent_t ev_parts = nullptr, ev_up = nullptr;
    bool parts_event = false;
    bool spec_off = false;       // pinned memory or the event could not be had
    bool spec_now = false;       // the solve being enqueued is speculative
    int gate_spec = 0;           // the gate's settings in DevState (zero at init)
    double gate_thr = 0.0;
    cudaStream_t fbody = nullptr;  // records the gated body of the field-solve graph
    cudaGraphExec_t agraph = nullptr;  // the same for axisymmetric contexts (one potential buffer)
    long long agraph_kernels = 0;
    cudaStream_t fcap = nullptr;
    bool fgraph_off = false;     // the graph could not be recorded: host-driven solves
    bool last_on_device = false; // the last solve reported through DevState
    // Per-phase timing: events recorded on the stream at the phase marks and
    // resolved later (at pic_profile, or once many are pending), so that
    // timing adds no host synchronisation to the steps.
    int prof = 0;
    pic_profile_times pt = {};
    struct Pending {
        cudaEvent_t a, b;
        double* ms;
        long long* n;
    };
    std::vector<cudaEvent_t> ev_free, ev_used;
    std::vector<Pending> pending;
    cudaEvent_t cur_ev[8] = {};
    void mark(int i) {
        if (!prof) return;
        cudaEvent_t e = nullptr;
        if (!ev_free.empty()) {
            e = ev_free.back();
            ev_free.pop_back();
        } else if (cudaEventCreate(&e) != cudaSuccess) {
            cur_ev[i] = nullptr;
            return;
        }
        ev_used.push_back(e);
        cur_ev[i] = e;
        cudaEventRecord(e, s);
    }
    void accumulate(int a, int b, double* ms, long long* n) {
        if (prof && cur_ev[a] && cur_ev[b]) pending.push_back(Pending{cur_ev[a], cur_ev[b], ms, n});
    }
    // Adds the pending phase times (waits for their events); call between steps.
    void resolve_times() {
        for (const Pending& q : pending) {
            float t = 0.f;
            if (cudaEventSynchronize(q.b) == cudaSuccess && cudaEventElapsedTime(&t, q.a, q.b) == cudaSuccess) {
                *q.ms += t;
                ++*q.n;
            }
        }
        pending.clear();
        ev_free.insert(ev_free.end(), ev_used.begin(), ev_used.end());
        ev_used.clear();
        for (int i = 0; i < 8; ++i) cur_ev[i] = nullptr;
    }
    ~pic_ctx() {
        for (cudaEvent_t e : ev_free) cudaEventDestroy(e);
        for (cudaEvent_t e : ev_used) cudaEventDestroy(e);
        for (int q = 0; q < 4; ++q)
            if (fgraph[q]) cudaGraphExecDestroy(fgraph[q]);
        if (hs) cudaFreeHost(hs);
        if (ev_state) cudaEventDestroy(ev_state);
        if (ev_parts) cudaEventDestroy(ev_parts);
        if (ev_up) cudaEventDestroy(ev_up);
        if (xs) cudaStreamDestroy(xs);
        if (fbody) cudaStreamDestroy(fbody);
        if (agraph) cudaGraphExecDestroy(agraph);
        if (fcap) cudaStreamDestroy(fcap);
        amg.release();
        mg.release();
    }

    template <class T> Soa<T> soa(int b) {
        Soa<T> s;
        char* p = ws + L.buf[b];
        const size_t cap = (size_t)cfg.capacity;
        for (int f = 0; f < 10; ++f) { s.r[f] = (T*)p; p += al256(cap * sizeof(T)); }
        s.id = (uint64_t*)p;
        return s;
    }
    template <class T> ChildQ<T> childq(int which) {
        ChildQ<T> q;
        char* p = ws + L.cq[which];
        const size_t cap = (size_t)cfg.capacity;
        for (int f = 0; f < 10; ++f) { q.p.r[f] = (T*)p; p += al256(cap * sizeof(T)); }
        q.t_left = (T*)p;
        p += al256(cap * sizeof(T));
        q.p.id = (uint64_t*)p;
        p += al256(cap * 8);
        q.k = (uint32_t*)p;
        return q;
    }
    DevState* st() { return (DevState*)(ws + L.st); }
    unsigned long long* qe() { return (unsigned long long*)(ws + L.qe); }
    unsigned long long* qp() { return (unsigned long long*)(ws + L.qp); }
    unsigned long long* qn() { return (unsigned long long*)(ws + L.qn); }
    double* rho() { return (double*)(ws + L.rho); }
    double* phi() { return (double*)(ws + L.phi); }
    // float32 contexts keep the potential as float pairs ([hi][lo], n each)
    // in four rotating slots: the current solution, the previous one, the
    // warm-start guess and the next solution.  A solve writes only the last
    // two, so until the slots rotate the solve can be undone by the host
    // alone.  Rotation (cur, prev, free, out) <- (out, cur, prev, free) keeps
    // cur and out of opposite parity: the push reads packed field cur & 1 and
    // the solve writes field out & 1.
    int ph_cur = 0, ph_prev = 1, ph_free = 2, ph_out = 3;
    float* ph_hi(int slot) {
        const size_t o = slot == 0 ? L.phi : (slot == 1 ? L.phi_prev : (slot == 2 ? L.phi_x : L.phi_y));
        return (float*)(ws + o);
    }
    char* E4p(int slot) { return ws + ((slot & 1) ? L.E4b : L.E4); }
    void rotate_slots() {
        const int o = ph_out;
        ph_out = ph_free;
        ph_free = ph_prev;
        ph_prev = ph_cur;
        ph_cur = o;
    }
    float* ph_lo(int slot) { return ph_hi(slot) + al256((size_t)g.ncell() * 4) / 4; }
    MergeScratch msc() {
        MergeScratch m;
        const size_t cap = (size_t)cfg.capacity;
        char* p = ws + L.msc;
        m.key = (double*)p; p += al256(cap * 8);
        m.id = (uint64_t*)p; p += al256(cap * 8);
        m.idx = (uint32_t*)p; p += al256(cap * 4);
        m.skey = (double*)p; p += al256(cap * 8);
        m.sid = (uint64_t*)p; p += al256(cap * 8);
        m.sidx = (uint32_t*)p;
        return m;
    }
    int fail(int code, const std::string& msg) {
        err = msg;
        return code;
    }
    int cuda_fail(cudaError_t e, const char* where) {
        err = std::string(where) + ": " + cudaGetErrorString(e);
        return PIC_ERR_CUDA;
    }
};

static const char* kStatusText[] = {"ok", "invalid argument", "CUDA error", "capacity exceeded",
                                    "fixed-point overflow", "iteration limit reached", "invalid state"};

extern "C" const char* pic_status_string(int status) {
    if (status > 0 || status < -6) return "unknown status";
    return kStatusText[-status];
}

extern "C" const char* pic_last_error(const pic_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

static int validate(const pic_config* c) {
    if (!c) return PIC_ERR_ARG;
    if (c->precision != 32 && c->precision != 64) return PIC_ERR_ARG;
    if (c->geometry != 0 && c->geometry != 1) return PIC_ERR_ARG;
    // axisymmetric: one y cell, the axis at x = y = 0
    if (c->geometry == 1 && (c->ny != 1 || c->origin[0] != 0.0 || c->origin[1] != 0.0)) return PIC_ERR_ARG;
    if (c->nx < 2 || (c->geometry == 0 && c->ny < 2) || c->nz < 2 || !(c->dx > 0) || c->capacity < 1)
        return PIC_ERR_ARG;
    if (c->weight_interval < 0) return PIC_ERR_ARG;
    if (c->nx > 2046 || c->ny > 2046 || c->nz > 2046) return PIC_ERR_ARG;
    if ((long long)c->nx * c->ny * c->nz > 0x7fffffffLL) return PIC_ERR_ARG;
    if (c->capacity > 0x7fffffffLL) return PIC_ERR_ARG;
    if (!(c->dt > 0)) return PIC_ERR_ARG;
    const pic_gas& g = c->gas;
    if (g.n_proc < 1 || g.n_proc > 7 || g.n_bins < 2 || g.n_bins > 4096) return PIC_ERR_ARG;
    if (!g.eps || !g.sigma || !g.kind || !g.threshold || !g.density || !g.mass) return PIC_ERR_ARG;
    if (!(g.eps[0] > 0) || !(g.eps[g.n_bins - 1] > g.eps[0])) return PIC_ERR_ARG;
    for (int k = 0; k < g.n_proc; ++k)
        if (g.kind[k] < 0 || g.kind[k] > 3) return PIC_ERR_ARG;
    if (c->coupled && (!(c->poisson_rtol > 0) || c->poisson_max_cycles < 1)) return PIC_ERR_ARG;
    if (c->coupled && c->geometry == 0 && !MG::supported(c->nx, c->ny, c->nz)) return PIC_ERR_ARG;
    if (c->coupled && c->geometry == 1 && !AxiMG::supported(c->nx, c->nz)) return PIC_ERR_ARG;
    if (c->adaptive_dt && (!(c->cfl > 0) || c->mobility < 0 || !(c->max_growth > 1.0))) return PIC_ERR_ARG;
    if (c->photo_xi < 0) return PIC_ERR_ARG;
    if (c->photo_xi > 0) {
        if (!(c->photo_pq > 0) || !(c->pressure > 0) || !(c->p_o2 > 0) || !(c->chi_min > 0) ||
            !(c->chi_max > c->chi_min))
            return PIC_ERR_ARG;
        // one photon per ionization at most
        if (c->photo_xi * c->photo_pq / (c->pressure + c->photo_pq) > 1.0) return PIC_ERR_ARG;
    }
    return PIC_OK;
}

// Photoelectron queue slots (photons absorbed in the gas, appended after each
// step or product generation).
static long long photo_cap(const pic_config* c) {
    if (!(c->photo_xi > 0)) return 0;
    const long long q = c->capacity / 8;
    return q > 4096 ? q : 4096;
}

extern "C" size_t pic_workspace_bytes(const pic_config* cfg) {
    if (validate(cfg) != PIC_OK) return 0;
    return make_layout(cfg).total;
}

// Builds the rate table on the device and reads nu_max back.
static int build_table(pic_ctx* c) {
    const pic_gas& g = c->cfg.gas;
    const int nb = g.n_bins, np = g.n_proc;
    double* d = (double*)(c->ws + c->L.gas);
    std::vector<double> host((size_t)nb * (np + 1) + np + 8);
    memcpy(host.data(), g.eps, nb * 8);
    memcpy(host.data() + nb, g.sigma, (size_t)np * nb * 8);
    memcpy(host.data() + (size_t)nb * (np + 1), g.density, np * 8);
    cudaError_t e = cudaMemcpyAsync(d, host.data(), host.size() * 8, cudaMemcpyHostToDevice, c->s);
    if (e != cudaSuccess) return c->cuda_fail(e, "table upload");
    unsigned long long* nmx = (unsigned long long*)(d + (size_t)nb * (np + 1) + np);
    cudaMemsetAsync(nmx, 0, 8, c->s);
    if (c->prec == 32)
        k_rate_table<float><<<(nb + 127) / 128, 128, 0, c->s>>>(d, d + nb, d + (size_t)nb * (np + 1), np, nb,
                                                                (float*)(c->ws + c->L.table),
                                                                (double*)(c->ws + c->L.table64), nmx);
    else
        k_rate_table<double><<<(nb + 127) / 128, 128, 0, c->s>>>(d, d + nb, d + (size_t)nb * (np + 1), np, nb,
                                                                 (double*)(c->ws + c->L.table),
                                                                 (double*)(c->ws + c->L.table64), nmx);
    unsigned long long bits = 0;
    e = cudaMemcpyAsync(&bits, nmx, 8, cudaMemcpyDeviceToHost, c->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->s);
    if (e != cudaSuccess) return c->cuda_fail(e, "rate table");
    memcpy(&c->nu_max, &bits, 8);
    if (!(c->nu_max > 0)) return c->fail(PIC_ERR_ARG, "all collision rates are zero");
    c->n_proc = np;
    c->n_bins = nb;
    c->l0 = log(g.eps[0]);
    c->inv_dl = (double)(nb - 1) / (log(g.eps[nb - 1]) - c->l0);
    for (int k = 0; k < 8; ++k) {
        c->kind[k] = k < np ? g.kind[k] : 0;
        c->thr[k] = k < np ? g.threshold[k] : 0.0;
        c->mratio[k] = (k < np && g.mass[k] > 0) ? kMe / g.mass[k] : 0.0;
    }
    return PIC_OK;
}

extern "C" int pic_init(const pic_config* cfg, void* d_ws, size_t ws_bytes, const uint8_t* d_mask,
                        pic_stream_t stream, pic_ctx** out) {
    if (!out) return PIC_ERR_ARG;
    *out = nullptr;
    int rc = validate(cfg);
    if (rc) return rc;
    Layout L = make_layout(cfg);
    if (!d_ws || ws_bytes < L.total || ((uintptr_t)d_ws & 255)) return PIC_ERR_ARG;
    pic_ctx* c = new pic_ctx();
    c->cfg = *cfg;
    c->prec = cfg->precision;
    c->s = (cudaStream_t)stream;
    c->ws = (char*)d_ws;
    c->L = L;
    c->g = Grid{cfg->nx, cfg->ny, cfg->nz, cfg->dx, cfg->origin[0], cfg->origin[1], cfg->origin[2],
                cfg->geometry == 1 ? 1 : 0};
    c->K = make_keys(cfg->seed);
    c->mask = d_mask;
    c->dt_cur = c->dt_prev = c->dt_next = cfg->dt;
    cudaError_t e = cudaMemsetAsync(c->ws + L.st, 0, sizeof(DevState), c->s);
    const size_t ncell = (size_t)c->g.ncell();
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ws + L.qe, 0, ncell * 8, c->s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ws + L.qp, 0, ncell * 8, c->s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ws + L.qn, 0, ncell * 8, c->s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ws + L.phi, 0, ncell * 8, c->s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ws + L.phi_prev, 0, ncell * 8, c->s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ws + L.phi_x, 0, ncell * 8, c->s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ws + L.phi_y, 0, ncell * 8, c->s);
    if (e != cudaSuccess) { rc = c->cuda_fail(e, "pic_init"); delete c; return rc; }
    rc = build_table(c);
    if (rc) { delete c; return rc; }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int bps = c->prec == 32 ? PushLaunch<float>::blocks_per_sm(MODE_PIC, c->n_bins)
                                  : PushLaunch<double>::blocks_per_sm(MODE_PIC, c->n_bins);
    c->grid_push = sms * bps;
    if (cfg->coupled) {
        if (c->g.axi) {
            c->amg.carve(c->ws + L.mg, cfg->nx, cfg->nz);
            c->amg.persistent = true;
        } else {
            c->mg.carve(c->ws + L.mg, cfg->nx, cfg->ny, cfg->nz, c->prec == 32, false);
            c->mg.persistent = true;
            c->mg.min_cycles = 2;
            c->mg.light_ratio = kLightRatio;
        }
    }
    *out = c;
    return PIC_OK;
}

extern "C" void pic_destroy(pic_ctx* ctx) { delete ctx; }

template <class T> static PushArgs<T> make_args(pic_ctx* c, int mode) {
    PushArgs<T> A;
    memset(&A, 0, sizeof(A));
    A.in = c->soa<T>(c->cur);
    A.out = c->soa<T>(1 - c->cur);
    A.cq = c->childq<T>(0);
    A.cq2 = c->childq<T>(1);
    A.gen = 0;
    A.st = c->st();
    A.table = (const T*)(c->ws + c->L.table);
    A.n_bins = c->n_bins;
    A.n_proc = c->n_proc;
    for (int k = 0; k < 8; ++k) { A.kind[k] = c->kind[k]; A.thr[k] = (T)c->thr[k]; A.mratio[k] = (T)c->mratio[k]; }
    A.l0 = (T)c->l0;
    A.inv_dl = (T)c->inv_dl;
    A.eps_lo = (T)c->cfg.gas.eps[0];
    A.eps_hi = (T)c->cfg.gas.eps[c->n_bins - 1];
    A.nu_max = (T)c->nu_max;
    A.tau_scale = (T)(-0.69314718055994530942 / c->nu_max);
    A.inv_dl2 = (T)(0.69314718055994530942 * c->inv_dl);
    A.l0t = (T)(c->l0 * c->inv_dl);
    A.dt = (T)c->dt_cur;
    A.dt_kick = (T)c->dt_prev;
    A.K = c->K;
    A.step = c->step;
    A.first = c->a_valid ? 0 : 1;
    A.kick_on_load = 0;
    A.cap_out = c->cfg.capacity;
    A.cap_child = c->cfg.capacity;
    A.nx = c->g.nx; A.ny = c->g.ny; A.nz = c->g.nz;
    A.ox = (T)c->g.ox; A.oy = (T)c->g.oy; A.oz = (T)c->g.oz; A.dxr = (T)c->g.dx;
    A.hx = (T)(c->g.ox + (double)c->g.nx * c->g.dx);
    A.hy = (T)(c->g.oy + (double)c->g.ny * c->g.dx);
    A.hz = (T)(c->g.oz + (double)c->g.nz * c->g.dx);
    A.E4 = c->field_uniform ? nullptr : (const T*)c->E4p(c->ph_cur);
    for (int d = 0; d < 3; ++d) A.E0[d] = (T)c->E0[d];
    A.mask = c->mask;
    A.q_e = c->qe();
    A.vhist = mode == MODE_PIC && c->cfg.adaptive_dt ? c->st()->vhist : nullptr;
    A.q_pos = c->qp();
    A.q_neg = c->qn();
    A.boundary = c->cfg.boundary;
    A.axi = c->g.axi;
    if (mode == MODE_PIC && c->cfg.photo_xi > 0) {
        const pic_config& f = c->cfg;
        const double a = f.chi_min * f.p_o2, b = f.chi_max * f.p_o2;
        A.photo_prob = (T)(f.photo_xi * f.photo_pq / (f.pressure + f.photo_pq));
        A.chi_a = (T)a;
        A.chi_log = (T)log(b / a);
        const long long np = photo_cap(&f);
        const size_t R = sizeof(T);
        char* p = c->ws + c->L.photo;
        T** arr[8] = {&A.pe_x, &A.pe_y, &A.pe_z, &A.pe_w, &A.ph_x, &A.ph_y, &A.ph_z, &A.ph_w};
        for (int q = 0; q < 8; ++q) { *arr[q] = (T*)p; p += al256(np * R); }
        A.pe_id = (uint64_t*)p; p += al256(np * 8);
        A.ph_id = (uint64_t*)p; p += al256(np * 8);
        A.pe_k = (uint32_t*)p;
        A.cap_photo = np;
    }
    return A;
}

static int read_state(pic_ctx* c, DevState* h) {
    cudaError_t e = cudaMemcpyAsync(h, c->st(), sizeof(DevState), cudaMemcpyDeviceToHost, c->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->s);
    if (e != cudaSuccess) return c->cuda_fail(e, "state read-back");
    c->n_host = (long long)h->n_in;
    return PIC_OK;
}

static int check_err(pic_ctx* c, const DevState& h) {
    if (!h.err) return PIC_OK;
    cudaMemsetAsync(&c->st()->err, 0, sizeof(unsigned), c->s);
    char msg[192];
    snprintf(msg, sizeof msg, "device error flags 0x%x (1 output full, 2 child queue full, 4 fixed-point overflow, "
             "8 descendant stack, 16 split output full, 32 photoelectron queue full, 64 poisson cycle limit)", h.err);
    if (h.err & kErrOverflow) return c->fail(PIC_ERR_OVERFLOW, msg);
    if (h.err == kErrPoissonLimit) return c->fail(PIC_ERR_TIMEOUT, "poisson solve: cycle limit reached");
    return c->fail(PIC_ERR_CAPACITY, msg);
}

template <class T> static void deposit_current(pic_ctx* c, unsigned long long* q) {
    PushLaunch<T>::deposit(c->soa<T>(c->cur), c->st(), c->g, q, grid_n(c->cfg.capacity), c->s);
}

extern "C" int pic_seed_gaussian(pic_ctx* c, double n0, double radius, const double center[3], double w0,
                                 long long* n_out) {
    if (c) c->parts_event = false;  // work on the particle buffers may follow
    if (!c || !center || !(n0 >= 0) || !(radius > 0) || !(w0 > 0)) return PIC_ERR_ARG;
    if (c->g.axi && (center[0] != 0.0 || center[1] != 0.0))
        return c->fail(PIC_ERR_ARG, "axisymmetric seed: the centre must be on the axis");
    const long long ncell = c->g.ncell();
    uint32_t* cnt = (uint32_t*)(c->ws + c->L.cnt);
    uint32_t* off = (uint32_t*)(c->ws + c->L.start);
    k_seed_count<<<grid_n(ncell), 256, 0, c->s>>>(c->g, c->mask, n0, radius * radius, center[0], center[1],
                                                   center[2], w0, c->K, cnt);
    scan_exclusive(cnt, off, ncell, (uint32_t*)(c->ws + c->L.sums), c->s);
    uint32_t total = 0;
    cudaError_t e = cudaMemcpyAsync(&total, off + ncell, 4, cudaMemcpyDeviceToHost, c->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->s);
    if (e != cudaSuccess) return c->cuda_fail(e, "seed count");
    if ((long long)total > c->cfg.capacity) return c->fail(PIC_ERR_CAPACITY, "seed exceeds capacity");
    c->cur = 0;
    if (c->prec == 32)
        k_seed_write<float><<<grid_n(ncell), 256, 0, c->s>>>(c->g, cnt, off, w0, 0, c->K, c->soa<float>(0),
                                                             c->cfg.capacity, c->st());
    else
        k_seed_write<double><<<grid_n(ncell), 256, 0, c->s>>>(c->g, cnt, off, w0, 0, c->K, c->soa<double>(0),
                                                              c->cfg.capacity, c->st());
    k_set_count<<<1, 1, 0, c->s>>>(c->st(), total);
    cudaMemsetAsync(c->qp(), 0, ncell * 8, c->s);
    cudaMemsetAsync(c->qn(), 0, ncell * 8, c->s);
    if (c->prec == 32) deposit_current<float>(c, c->qp());
    else deposit_current<double>(c, c->qp());
    c->n_host = total;
    c->n_last_wu = total;
    c->a_valid = 0;
    if (n_out) *n_out = total;
    e = cudaGetLastError();
    return e == cudaSuccess ? PIC_OK : c->cuda_fail(e, "seed");
}

template <class T> static int set_particles(pic_ctx* c, long long n, const pic_particles_host* p) {
    std::vector<T> tmp((size_t)n);
    Soa<T> d = c->soa<T>(0);
    const double* src[10] = {p->x, p->y, p->z, p->vx, p->vy, p->vz, p->ax, p->ay, p->az, p->w};
    for (int f = 0; f < 10; ++f) {
        for (long long i = 0; i < n; ++i) tmp[i] = src[f] ? (T)src[f][i] : (T)0;
        cudaError_t e = cudaMemcpyAsync(d.r[f], tmp.data(), n * sizeof(T), cudaMemcpyHostToDevice, c->s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->s);
        if (e != cudaSuccess) return c->cuda_fail(e, "set particles");
    }
    cudaError_t e = cudaMemcpyAsync(d.id, p->id, n * 8, cudaMemcpyHostToDevice, c->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->s);
    if (e != cudaSuccess) return c->cuda_fail(e, "set particles");
    return PIC_OK;
}

extern "C" int pic_set_particles(pic_ctx* c, long long n, const pic_particles_host* p, int accel_valid) {
    if (c) c->parts_event = false;  // work on the particle buffers may follow
    if (!c || n < 0 || (n > 0 && (!p || !p->x || !p->y || !p->z || !p->w || !p->id))) return PIC_ERR_ARG;
    if (n > c->cfg.capacity) return c->fail(PIC_ERR_CAPACITY, "more particles than capacity");
    c->cur = 0;
    int rc = PIC_OK;
    if (n > 0) rc = c->prec == 32 ? set_particles<float>(c, n, p) : set_particles<double>(c, n, p);
    if (rc) return rc;
    k_set_count<<<1, 1, 0, c->s>>>(c->st(), (unsigned long long)n);
    c->n_host = n;
    c->n_last_wu = n;
    c->a_valid = accel_valid ? 1 : 0;
    return PIC_OK;
}

template <class T> static int get_particles(pic_ctx* c, pic_particles_host* p, long long cap, long long* n_out) {
    DevState h;
    int rc = read_state(c, &h);
    if (rc) return rc;
    const long long n = (long long)h.n_in;
    Soa<T> d = c->soa<T>(c->cur);
    std::vector<T> w((size_t)n);
    cudaError_t e = cudaMemcpy(w.data(), d.r[PW], n * sizeof(T), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return c->cuda_fail(e, "get particles");
    long long live = 0;
    for (long long i = 0; i < n; ++i) live += w[i] > (T)0;
    if (n_out) *n_out = live;
    if (!p) return PIC_OK;
    if (live > cap) return c->fail(PIC_ERR_CAPACITY, "host arrays too small");
    double* dst[10] = {p->x, p->y, p->z, p->vx, p->vy, p->vz, p->ax, p->ay, p->az, p->w};
    std::vector<T> tmp((size_t)n);
    for (int f = 0; f < 10; ++f) {
        if (!dst[f]) continue;
        e = cudaMemcpy(tmp.data(), d.r[f], n * sizeof(T), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return c->cuda_fail(e, "get particles");
        long long j = 0;
        for (long long i = 0; i < n; ++i)
            if (w[i] > (T)0) dst[f][j++] = (double)tmp[i];
    }
    if (p->id) {
        std::vector<uint64_t> ids((size_t)n);
        e = cudaMemcpy(ids.data(), d.id, n * 8, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return c->cuda_fail(e, "get particles");
        long long j = 0;
        for (long long i = 0; i < n; ++i)
            if (w[i] > (T)0) p->id[j++] = ids[i];
    }
    return PIC_OK;
}

extern "C" int pic_get_particles(pic_ctx* c, pic_particles_host* p, long long cap, long long* n_out) {
    if (c) c->parts_event = false;  // work on the particle buffers may follow
    if (!c) return PIC_ERR_ARG;
    return c->prec == 32 ? get_particles<float>(c, p, cap, n_out) : get_particles<double>(c, p, cap, n_out);
}

extern "C" int pic_count(pic_ctx* c, long long* n) {
    if (c) c->parts_event = false;  // work on the particle buffers may follow
    if (!c || !n) return PIC_ERR_ARG;
    DevState h;
    int rc = read_state(c, &h);
    *n = c->n_host;
    return rc;
}

// The field grids (float or double planes) packed into the context's [n][4]
// layout in its own precision.
template <class TI>
static int set_field(pic_ctx* c, const TI* Ex, const TI* Ey, const TI* Ez, const double E_uniform[3]) {
    if (!c) return PIC_ERR_ARG;
    if (Ex == nullptr) {
        if (!E_uniform) return PIC_ERR_ARG;
        c->field_uniform = 1;
        for (int d = 0; d < 3; ++d) c->E0[d] = E_uniform[d];
    } else {
        if (!Ey || !Ez) return PIC_ERR_ARG;
        c->field_uniform = 0;
        const long long n = c->g.ncell();
        if (c->prec == 32)
            k_pack_field<TI, float><<<grid_n(n), 256, 0, c->s>>>(Ex, Ey, Ez, n, (float*)c->E4p(c->ph_cur));
        else
            k_pack_field<TI, double><<<grid_n(n), 256, 0, c->s>>>(Ex, Ey, Ez, n, (double*)c->E4p(c->ph_cur));
    }
    c->field_valid = 1;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PIC_OK : c->cuda_fail(e, "set field");
}

extern "C" int pic_set_field(pic_ctx* c, const float* Ex, const float* Ey, const float* Ez, const double E_uniform[3]) {
    if (c) c->parts_event = false;  // work on the particle buffers may follow
    return set_field<float>(c, Ex, Ey, Ez, E_uniform);
}

extern "C" int pic_set_field_f64(pic_ctx* c, const double* Ex, const double* Ey, const double* Ez,
                                 const double E_uniform[3]) {
    if (c) c->parts_event = false;  // work on the particle buffers may follow
    return set_field<double>(c, Ex, Ey, Ez, E_uniform);
}

// Unpacks the packed field [n][4] (context precision) into float64 planes.
template <class T>
__global__ void k_unpack_field(const T* __restrict__ E4, long long n, double* __restrict__ Ex, double* __restrict__ Ey,
                               double* __restrict__ Ez) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        if (Ex) Ex[c] = (double)E4[4 * c];
        if (Ey) Ey[c] = (double)E4[4 * c + 1];
        if (Ez) Ez[c] = (double)E4[4 * c + 2];
    }
}

extern "C" int pic_get_field(pic_ctx* c, double* Ex, double* Ey, double* Ez) {
    if (c) c->parts_event = false;  // work on the particle buffers may follow
    if (!c) return PIC_ERR_ARG;
    if (!c->field_valid || c->field_uniform)
        return c->fail(PIC_ERR_STATE, "no field grid: set one, or step a coupled context (or call pic_step with 0 steps)");
    const long long n = c->g.ncell();
    if (c->prec == 32)
        k_unpack_field<float><<<grid_n(n), 256, 0, c->s>>>((const float*)c->E4p(c->ph_cur), n, Ex, Ey, Ez);
    else
        k_unpack_field<double><<<grid_n(n), 256, 0, c->s>>>((const double*)c->E4p(c->ph_cur), n, Ex, Ey, Ez);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PIC_OK : c->cuda_fail(e, "get field");
}

extern "C" int pic_get_deposit(pic_ctx* c, int64_t* q_e, int64_t* q_pos, int64_t* q_neg) {
    if (c) c->parts_event = false;  // work on the particle buffers may follow
    if (!c) return PIC_ERR_ARG;
    const size_t n = (size_t)c->g.ncell();
    cudaError_t e = cudaSuccess;
    if (q_e) e = cudaMemcpyAsync(q_e, c->qe(), n * 8, cudaMemcpyDeviceToDevice, c->s);
    if (e == cudaSuccess && q_pos) e = cudaMemcpyAsync(q_pos, c->qp(), n * 8, cudaMemcpyDeviceToDevice, c->s);
    if (e == cudaSuccess && q_neg) e = cudaMemcpyAsync(q_neg, c->qn(), n * 8, cudaMemcpyDeviceToDevice, c->s);
    return e == cudaSuccess ? PIC_OK : c->cuda_fail(e, "deposit copy");
}

static void fixed_to_rho(pic_ctx* c, double* rho) {
    const long long n = c->g.ncell();
    // cell volume dx^3, or pi dx^3 times (2i + 1) for the ring cells of an axisymmetric grid
    const double dV = c->g.dx * c->g.dx * c->g.dx * (c->g.axi ? kPi : 1.0);
    k_fixed_to_rho<<<grid_n(n), 256, 0, c->s>>>((const long long*)c->qe(), (const long long*)c->qp(),
                                                 (const long long*)c->qn(), n, 1.0 / (4294967296.0 * dV), rho,
                                                 c->g.axi ? c->g.nx : 0);
}

// The steady-state float32 field solve as one graph launch: h^2 rho / eps0
// from the fixed-point grids, the extrapolated warm start, and the
// device-driven mixed solve, which reports its cycles, residual and any
// cycle-limit flag into DevState (checked at the next state read-back).
// The graph for the current potential slot is recorded on first use.
// Returns PIC_ERR_STATE when the graph cannot be recorded.
static int solve_field_pair_graph(pic_ctx* c) {
    const long long n = c->g.ncell();
    const int slot = c->ph_cur;
    if (!c->fgraph[slot]) {
        if ((!c->fcap && cudaStreamCreateWithFlags(&c->fcap, cudaStreamNonBlocking) != cudaSuccess) ||
            (!c->fbody && cudaStreamCreateWithFlags(&c->fbody, cudaStreamNonBlocking) != cudaSuccess) ||
            c->mg.prepare_capture() != PIC_OK) {
            cudaGetLastError();
            return PIC_ERR_STATE;
        }
        if (cudaStreamBeginCapture(c->fcap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            return PIC_ERR_STATE;
        }
        // gate kernel, then the solve as the body of an if node
        DevState* st = c->st();
        long long fixed = 0;
        int rc = PIC_ERR_STATE;
        const cudaGraph_t top = capturing_graph(c->fcap);
        cudaGraphConditionalHandle h_go = 0;
        cudaGraph_t body = nullptr;
        if (top && cudaGraphConditionalHandleCreate(&h_go, top, 1u, cudaGraphCondAssignDefault) == cudaSuccess) {
            k_solve_gate<<<1, 1, 0, c->fcap>>>(st, h_go, (unsigned long long)c->cfg.capacity);
            if (add_conditional(c->fcap, h_go, cudaGraphCondTypeIf, 1, &body) == cudaSuccess &&
                cudaStreamBeginCaptureToGraph(c->fbody, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
                    cudaSuccess) {
                const double dV = c->g.dx * c->g.dx * c->g.dx;
                const double scale = kQ / (4294967296.0 * dV) * c->g.dx * c->g.dx / kEps0;
                k_fixed_to_hrho<<<grid_n(n), 256, 0, c->fbody>>>((const long long*)c->qe(), (const long long*)c->qp(),
                                                                  (const long long*)c->qn(), n, (float)scale,
                                                                  (float*)c->rho());
                c->mg.extrapolate_pair(c->ph_hi(c->ph_cur), c->ph_lo(c->ph_cur), c->ph_hi(c->ph_prev),
                                       c->ph_lo(c->ph_prev), c->ph_hi(c->ph_free), c->ph_lo(c->ph_free), (int)n, true,
                                       c->fbody);
                rc = c->mg.capture_solve_mixed(
                    c->fbody, (const float*)c->rho(), c->ph_hi(c->ph_free), c->ph_lo(c->ph_free), c->ph_hi(c->ph_out),
                    c->ph_lo(c->ph_out), c->g.dx, c->cfg.v_lo, c->cfg.v_hi, c->cfg.v_mask, c->cfg.poisson_rtol,
                    c->cfg.poisson_max_cycles, (float*)c->E4p(c->ph_out), &st->poisson_cycles, &st->poisson_rel,
                    &st->err, kErrPoissonLimit, &st->dev_kernels, &fixed);
                if (end_body_capture(c->fbody) != cudaSuccess) rc = PIC_ERR_STATE;
            }
        }
        cudaGraph_t gr = nullptr;
        const cudaError_t e = cudaStreamEndCapture(c->fcap, &gr);
        cudaGraphExec_t gx = nullptr;
        if (rc != PIC_OK || e != cudaSuccess || !gr || cudaGraphInstantiate(&gx, gr, 0) != cudaSuccess) {
            if (gr) cudaGraphDestroy(gr);
            cudaGetLastError();
            return PIC_ERR_STATE;
        }
        cudaGraphDestroy(gr);
        c->fgraph[slot] = gx;
        c->fgraph_kernels[slot] = fixed + 3;
    }
    // the gate's settings follow the solve's kind (they change rarely)
    const int spec = c->spec_now ? 1 : 0;
    const double thr = c->cfg.growth_trigger > 0 ? c->cfg.growth_trigger * (double)c->n_last_wu : HUGE_VAL;
    if (spec != c->gate_spec || (spec && thr != c->gate_thr)) {
        k_gate_set<<<1, 1, 0, c->s>>>(c->st(), spec, spec ? thr : c->gate_thr);
        c->launches += 1;
        c->gate_spec = spec;
        if (spec) c->gate_thr = thr;
    }
    const cudaError_t e = cudaGraphLaunch(c->fgraph[slot], c->s);
    if (e != cudaSuccess) return c->cuda_fail(e, "field solve graph");
    c->n_solves++;
    c->rotate_slots();
    c->launches += c->fgraph_kernels[slot];
    c->last_on_device = true;
    c->field_valid = 1;
    c->field_uniform = 0;
    return PIC_OK;
}

// Coupled field: rho from the fixed-point grids, multigrid Poisson (warm
// started from the previous potential), packed E for the next gather.
static int solve_field_pair(pic_ctx* c) {
    if (c->n_solves >= 2 && !c->fgraph_off) {
        const int rc = solve_field_pair_graph(c);
        if (rc != PIC_ERR_STATE) return rc;
        c->fgraph_off = true;
    }
    c->last_on_device = false;
    const long long n = c->g.ncell();
    const double dV = c->g.dx * c->g.dx * c->g.dx;
    const double scale = kQ / (4294967296.0 * dV) * c->g.dx * c->g.dx / kEps0;
    k_fixed_to_hrho<<<grid_n(n), 256, 0, c->s>>>((const long long*)c->qe(), (const long long*)c->qp(),
                                                  (const long long*)c->qn(), n, (float)scale, (float*)c->rho());
    ++c->launches;
    const long long l0 = c->mg.launches;
    // guess in the free slot, solution in the out slot
    c->mg.extrapolate_pair(c->ph_hi(c->ph_cur), c->ph_lo(c->ph_cur), c->ph_hi(c->ph_prev), c->ph_lo(c->ph_prev),
                           c->ph_hi(c->ph_free), c->ph_lo(c->ph_free), (int)n, c->n_solves >= 2, c->s);
    c->n_solves++;
    double hn[2];
    int rc = c->mg.solve_mixed(c->rho(), false, c->mask, c->ph_hi(c->ph_free), c->ph_lo(c->ph_free),
                               c->ph_hi(c->ph_out), c->ph_lo(c->ph_out), c->n_solves <= 2, c->g.dx,
                               c->cfg.v_lo, c->cfg.v_hi,
                               c->cfg.v_mask, c->cfg.poisson_rtol, c->cfg.poisson_max_cycles,
                               (float*)c->E4p(c->ph_out), nullptr, nullptr, nullptr, c->s, &c->last_cycles,
                               &c->last_rel, hn);
    if (rc == PIC_ERR_CUDA) return c->fail(rc, "poisson solve: CUDA error");
    if (rc == PIC_ERR_TIMEOUT) return c->fail(rc, "poisson solve: cycle limit reached");
    if (rc) return c->fail(rc, "poisson solve");
    c->rotate_slots();
    c->launches += c->mg.launches - l0;
    c->field_valid = 1;
    c->field_uniform = 0;
    return PIC_OK;
}

// The steady-state axisymmetric field solve as one graph launch: ring-cell
// charge density, extrapolated warm start and the device-driven (r, z) solve
// reporting into DevState.  Returns PIC_ERR_STATE when the graph cannot be
// recorded.
static int solve_field_axi_graph(pic_ctx* c) {
    const long long n = c->g.ncell();
    if (!c->agraph) {
        if ((!c->fcap && cudaStreamCreateWithFlags(&c->fcap, cudaStreamNonBlocking) != cudaSuccess) ||
            c->amg.prepare_capture() != PIC_OK) {
            cudaGetLastError();
            return PIC_ERR_STATE;
        }
        if (cudaStreamBeginCapture(c->fcap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            return PIC_ERR_STATE;
        }
        const double dV = c->g.dx * c->g.dx * c->g.dx * kPi;
        k_fixed_to_rho<<<grid_n(n), 256, 0, c->fcap>>>((const long long*)c->qe(), (const long long*)c->qp(),
                                                        (const long long*)c->qn(), n, 1.0 / (4294967296.0 * dV),
                                                        c->rho(), c->g.nx);
        k_extrapolate<<<grid_n(n), 256, 0, c->fcap>>>(c->phi(), (double*)(c->ws + c->L.phi_prev), n, 1);
        DevState* st = c->st();
        long long fixed = 0;
        const int rc = c->amg.capture_solve(c->fcap, c->rho(), c->phi(), c->g.dx, c->cfg.v_lo, c->cfg.v_hi,
                                            c->cfg.v_mask, c->cfg.poisson_rtol, c->cfg.poisson_max_cycles, c->prec,
                                            c->ws + c->L.E4, &st->poisson_cycles, &st->poisson_rel, &st->err,
                                            kErrPoissonLimit, &st->dev_kernels, &fixed);
        cudaGraph_t gr = nullptr;
        const cudaError_t e = cudaStreamEndCapture(c->fcap, &gr);
        cudaGraphExec_t gx = nullptr;
        if (rc != PIC_OK || e != cudaSuccess || !gr || cudaGraphInstantiate(&gx, gr, 0) != cudaSuccess) {
            if (gr) cudaGraphDestroy(gr);
            cudaGetLastError();
            return PIC_ERR_STATE;
        }
        cudaGraphDestroy(gr);
        c->agraph = gx;
        c->agraph_kernels = fixed + 2;
    }
    const cudaError_t e = cudaGraphLaunch(c->agraph, c->s);
    if (e != cudaSuccess) return c->cuda_fail(e, "axisymmetric field solve graph");
    c->n_solves++;
    c->launches += c->agraph_kernels;
    c->last_on_device = true;
    c->field_valid = 1;
    c->field_uniform = 0;
    return PIC_OK;
}

// Axisymmetric coupled field: rho in the ring cells, the (r, z) solve warm
// started from the extrapolated potential (float64 in both precisions),
// packed (E_r, 0, E_z).
static int solve_field_axi(pic_ctx* c) {
    if (c->n_solves >= 2 && !c->fgraph_off) {
        const int rc = solve_field_axi_graph(c);
        if (rc != PIC_ERR_STATE) return rc;
        c->fgraph_off = true;
    }
    c->last_on_device = false;
    fixed_to_rho(c, c->rho());
    k_extrapolate<<<grid_n(c->g.ncell()), 256, 0, c->s>>>(c->phi(), (double*)(c->ws + c->L.phi_prev), c->g.ncell(),
                                                           c->n_solves >= 2 ? 1 : 0);
    c->n_solves++;
    c->launches += 2;
    const long long l0 = c->amg.launches;
    double hn[2];
    int rc = c->amg.solve(c->rho(), c->mask, c->phi(), c->g.dx, c->cfg.v_lo, c->cfg.v_hi, c->cfg.v_mask,
                          c->cfg.poisson_rtol, c->cfg.poisson_max_cycles, c->prec, c->ws + c->L.E4, nullptr,
                          nullptr, c->s, &c->last_cycles, &c->last_rel, hn);
    if (rc == PIC_ERR_CUDA) return c->fail(rc, "axisymmetric poisson solve: CUDA error");
    if (rc == PIC_ERR_TIMEOUT) return c->fail(rc, "axisymmetric poisson solve: cycle limit reached");
    c->launches += c->amg.launches - l0;
    c->field_valid = 1;
    c->field_uniform = 0;
    return PIC_OK;
}

static int solve_field(pic_ctx* c) {
    if (c->g.axi) return solve_field_axi(c);
    if (c->prec == 32) return solve_field_pair(c);
    fixed_to_rho(c, c->rho());
    k_extrapolate<<<grid_n(c->g.ncell()), 256, 0, c->s>>>(c->phi(), (double*)(c->ws + c->L.phi_prev), c->g.ncell(),
                                                           c->n_solves >= 2 ? 1 : 0);
    c->n_solves++;
    c->launches += 2;
    const long long l0 = c->mg.launches;
    double hn[2];
    int rc = c->mg.solve(c->rho(), c->mask, c->phi(), c->g.dx, c->cfg.v_lo, c->cfg.v_hi, c->cfg.v_mask,
                         c->cfg.poisson_rtol, c->cfg.poisson_max_cycles, c->prec, c->ws + c->L.E4, nullptr, nullptr,
                         nullptr, c->s, &c->last_cycles, &c->last_rel, hn);
    if (rc == PIC_ERR_CUDA) return c->fail(rc, "poisson solve: CUDA error");
    if (rc == PIC_ERR_TIMEOUT) return c->fail(rc, "poisson solve: cycle limit reached");
    c->launches += c->mg.launches - l0;
    c->field_valid = 1;
    c->field_uniform = 0;
    return PIC_OK;
}

template <class T> static int sort_by_cell(pic_ctx* c) {
    c->parts_event = false;
    const long long ncell = c->g.ncell();
    uint32_t* cnt = (uint32_t*)(c->ws + c->L.cnt);
    uint32_t* start = (uint32_t*)(c->ws + c->L.start);
    cudaMemsetAsync(cnt, 0, (ncell + 1) * 4, c->s);
    GridT g{c->g.ox, c->g.oy, c->g.oz, c->g.dx, c->g.nx, c->g.ny, c->g.nz, c->g.axi};
    const int grid = grid_n(c->cfg.capacity);
    k_cell_count<T><<<grid, 256, 0, c->s>>>(c->soa<T>(c->cur), c->st(), g, cnt, (uint32_t*)(c->ws + c->L.key),
                                             (uint32_t*)(c->ws + c->L.rank));
    scan_exclusive(cnt, start, ncell, (uint32_t*)(c->ws + c->L.sums), c->s);
    k_scatter<T><<<grid, 256, 0, c->s>>>(c->soa<T>(c->cur), c->soa<T>(1 - c->cur), c->st(), start,
                                          (const uint32_t*)(c->ws + c->L.key), (const uint32_t*)(c->ws + c->L.rank));
    c->cur = 1 - c->cur;
    c->n_sorts++;
    c->launches += 5;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PIC_OK : c->cuda_fail(e, "sort");
}

// Weight update (Sec. 2.1.2): sort by cell, per-cell merge and split, compaction.
template <class T> static int weight_update(pic_ctx* c) {
    c->parts_event = false;
    int rc = sort_by_cell<T>(c);
    if (rc) return rc;
    const long long ncell = c->g.ncell();
    const uint32_t* start = (const uint32_t*)(c->ws + c->L.start);
    DevState h;
    cudaMemsetAsync(&c->st()->pred_total, 0, 8, c->s);
    cudaMemsetAsync(&c->st()->n_extra, 0, 8, c->s);
    cudaMemsetAsync(&c->st()->n_big, 0, 3 * 8, c->s);  // n_big, n_occ, n_occ_fetch
    // the occupied cells are listed in the count array (free once the starts are formed)
    uint32_t* occ_list = (uint32_t*)(c->ws + c->L.cnt);
    k_cell_weight<T><<<grid_n(ncell), 256, 0, c->s>>>(c->soa<T>(c->cur), start, ncell, c->cfg.n_ppc, c->cfg.w_min,
                                                       occ_list, c->st());
    rc = read_state(c, &h);
    if (rc) return rc;
    const long long n = c->n_host;
    double scale = 1.0;
    const long long capp = c->cfg.particle_cap;
    if (capp > 0 && h.pred_total > capp * 16777216LL) scale = (double)h.pred_total / ((double)capp * 16777216.0);
    // cells with up to kWarpSort merge candidates take one warp each; the
    // others are listed (in the key array, free after the sort) for one block each
    uint32_t* big = (uint32_t*)(c->ws + c->L.key);
    k_merge_split_warp<T><<<device_sms() * 4, 256, 0, c->s>>>(c->soa<T>(c->cur), n, start, occ_list, c->cfg.n_ppc,
                                                      c->cfg.w_min, scale, c->K, c->step, c->cfg.capacity, big,
                                                      c->st());
    cudaFuncSetAttribute(k_merge_split<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMergeSmem);
    k_merge_split<T><<<device_sms() * 2, 256, kMergeSmem, c->s>>>(c->soa<T>(c->cur), n, start, ncell, c->cfg.n_ppc,
                                                          c->cfg.w_min, scale, c->msc(), c->K, c->step,
                                                          c->cfg.capacity, big, c->st());
    rc = read_state(c, &h);
    if (rc) return rc;
    const long long ntot = n + (long long)h.n_extra;
    cudaMemsetAsync(&c->st()->n_out, 0, 8, c->s);
    k_compact<T><<<grid_n(ntot), 256, 0, c->s>>>(c->soa<T>(c->cur), ntot < c->cfg.capacity ? ntot : c->cfg.capacity,
                                                  c->soa<T>(1 - c->cur), c->st());
    k_end_step<<<1, 1, 0, c->s>>>(c->st(), nullptr, c->cfg.capacity);
    c->cur = 1 - c->cur;
    rc = read_state(c, &h);
    if (rc) return rc;
    c->n_last_wu = c->n_host;
    c->n_wu++;
    c->launches += 5;
    return check_err(c, h);
}

extern "C" int pic_weight_update(pic_ctx* c) {
    if (c) c->parts_event = false;  // work on the particle buffers may follow
    if (!c) return PIC_ERR_ARG;
    return c->prec == 32 ? weight_update<float>(c) : weight_update<double>(c);
}

// Time-step control (Sec. 2.1.4): dt_next = min(dt_max, CFL, dielectric
// relaxation, growth limit).  CFL: dt v_90 <= cfl dx with v_90 the upper edge
// of the speed-histogram bin holding the 90 % quantile; dielectric relaxation:
// eps0 / (e n_e,max mu_e); growth: if the electrons (total deposited weight)
// grew by g > max_growth in the last step, dt is scaled by ln(max_growth)/ln g.
// dt may at most double from one step to the next.
static void next_dt(pic_ctx* c, const DevState& h) {
    const double dV = c->g.dx * c->g.dx * c->g.dx;
    long long tot = 0;
    for (int b = 0; b < kVBins; ++b) tot += h.vhist[b];
    double v90 = 0.0;
    long long acc = 0;
    for (int b = 0; b < kVBins; ++b) {
        acc += h.vhist[b];
        if (tot > 0 && acc >= (long long)ceil(0.9 * (double)tot)) {
            v90 = exp2(10.0 + (double)(b + 1) / kVBinsPerOctave);
            break;
        }
    }
    const double ne_max = (double)h.qe_max / (4294967296.0 * dV * (c->g.axi ? kPi : 1.0));
    const double w_now = (double)(long long)h.qe_sum / 4294967296.0;
    double dt = c->cfg.dt;
    if (v90 > 0.0) dt = fmin(dt, c->cfg.cfl * c->g.dx / v90);
    if (ne_max > 0.0 && c->cfg.mobility > 0.0) dt = fmin(dt, kEps0 / (kQ * ne_max * c->cfg.mobility));
    if (c->w_prev > 0.0 && w_now > c->cfg.max_growth * c->w_prev && c->cfg.max_growth > 1.0)
        dt = fmin(dt, c->dt_cur * log(c->cfg.max_growth) / log(w_now / c->w_prev));
    dt = fmin(dt, 2.0 * c->dt_cur);
    c->ne_max = ne_max;
    c->w_prev = w_now;
    c->dt_next = dt;
}

// The photoelectrons of the generations so far join the output, and the
// time-step statistics of the particles are formed (adaptive dt).
template <class T> static int generation_tail(pic_ctx* c, PushArgs<T>& A, int mode) {
    if (A.cap_photo > 0) {
        cudaError_t e = PushLaunch<T>::photo_append(A, device_sms() * 2, c->s);
        if (e != cudaSuccess) return c->cuda_fail(e, "photoelectrons");
        c->launches += 3;
    }
    if (c->cfg.adaptive_dt && mode == MODE_PIC) {
        DevState* st = c->st();
        cudaMemsetAsync(&st->qe_max, 0, sizeof(long long) + sizeof(unsigned long long), c->s);
        k_step_stats<<<device_sms() * 4, 256, 0, c->s>>>(c->qe(), c->g.ncell(), c->g.axi ? c->g.nx : 0, st);
        c->launches += 1;
    }
    return PIC_OK;
}

// Further children generations while descendants spilled out of the lane
// stacks (deep ionization cascades within one step).  Reads the device state
// once (synchronising), or starts from h0, the state already read after
// generation_tail of generation 1; afterwards c->n_next holds the particle
// count the step will leave.
template <class T> static int extra_generations(pic_ctx* c, PushArgs<T>& A, int mode, bool stats,
                                                const DevState* h0 = nullptr) {
    for (int gen = 1;; ++gen) {
        DevState h;
        if (gen == 1 && h0) {
            h = *h0;
        } else {
            int rc = generation_tail<T>(c, A, mode);
            if (rc == PIC_OK) rc = read_state(c, &h);
            if (rc) return rc;
        }
        // error flags raised so far (this step's kernels, or the previous step's field solve)
        const int rc = check_err(c, h);
        if (rc) return rc;
        const unsigned long long pending = (gen & 1) ? h.n_spill : h.n_child;
        c->n_next = (long long)(h.n_out < (unsigned long long)c->cfg.capacity ? h.n_out : c->cfg.capacity);
        if (!pending) {
            if (c->cfg.adaptive_dt && mode == MODE_PIC) next_dt(c, h);
            break;
        }
        if (gen > 256) return c->fail(PIC_ERR_CAPACITY, "ionization cascade deeper than 256 generations");
        k_next_generation<<<1, 1, 0, c->s>>>(c->st(), gen);
        A.gen = gen;
        cudaError_t e = PushLaunch<T>::children(A, mode, stats, c->grid_push, c->s);
        if (e != cudaSuccess) return c->cuda_fail(e, "children");
        c->launches += 2;
    }
    return PIC_OK;
}

// Speculative field solve.  In float32 Cartesian coupled contexts whose
// solve runs as a graph, the solve for the next step is enqueued right after
// the step's statistics, before the host has read the step's counts (copied
// to pinned memory behind an event), so the GPU does not wait for the host's
// decisions.  Two outcomes change the charge the solve must see: a weight
// update (merged and split particles are deposited again) and further
// product generations.  When the counts call for either, the solve is
// undone: it wrote only the guess and out potential slots and the packed
// field the push does not read, so restoring the host's slot indices (and
// the cycle-limit flag it may have raised) puts the context back as it was,
// and the step goes on as without speculation.  Steps with a scheduled
// weight update do not speculate.
static bool can_speculate(pic_ctx* c) {
    if (!c->cfg.coupled || c->prec != 32 || c->g.axi || c->fgraph_off || c->spec_off || c->n_solves < 2)
        return false;
    if (c->cfg.weight_interval > 0 && (c->step % (uint32_t)c->cfg.weight_interval) == 0) return false;
    if (!c->hs && cudaHostAlloc((void**)&c->hs, sizeof(DevState), cudaHostAllocDefault) != cudaSuccess) c->hs = nullptr;
    if (c->hs && !c->ev_state && cudaEventCreateWithFlags(&c->ev_state, cudaEventDisableTiming) != cudaSuccess)
        c->ev_state = nullptr;
    if (!c->ev_parts && cudaEventCreateWithFlags(&c->ev_parts, cudaEventDisableTiming) != cudaSuccess) {
        c->ev_parts = nullptr;  // host exchanges then wait for the solve
        cudaGetLastError();
    }
    if (!c->hs || !c->ev_state) {
        cudaGetLastError();
        c->spec_off = true;
        return false;
    }
    return true;
}

template <class T> static int speculative_tail(pic_ctx* c, PushArgs<T>& A, bool stats, bool* solved) {
    int rc = generation_tail<T>(c, A, MODE_PIC);
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(c->hs, c->st(), sizeof(DevState), cudaMemcpyDeviceToHost, c->s);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_state, c->s);
    if (e != cudaSuccess) return c->cuda_fail(e, "state read-back");
    // the particles are final here unless the step is undone below
    const bool parts = c->ev_parts && cudaEventRecord(c->ev_parts, c->s) == cudaSuccess;
    const int slots[4] = {c->ph_cur, c->ph_prev, c->ph_free, c->ph_out};
    const long long n_solves = c->n_solves;
    const bool on_device = c->last_on_device;
    const int cycles = c->last_cycles;
    const double rel = c->last_rel;
    c->mark(5);
    c->spec_now = true;
    rc = solve_field(c);
    c->spec_now = false;
    if (rc) return rc;
    c->mark(6);
    c->accumulate(5, 6, &c->pt.ms_field, &c->pt.n_field);
    c->pt.n_speculative++;
    // a graph solve skips its body on the device when the host will undo it
    const bool gated = c->last_on_device;
    e = cudaEventSynchronize(c->ev_state);
    if (e != cudaSuccess) return c->cuda_fail(e, "state read-back");
    const DevState h = *c->hs;
    c->n_host = (long long)h.n_in;
    const long long n_next = (long long)(h.n_out < (unsigned long long)c->cfg.capacity ? h.n_out : c->cfg.capacity);
    const bool grown = c->cfg.growth_trigger > 0 && n_next > 0 &&
                       (double)n_next > c->cfg.growth_trigger * (double)c->n_last_wu;
    if (!h.err && !h.n_spill && !grown) {
        c->n_next = n_next;
        if (c->cfg.adaptive_dt) next_dt(c, h);
        *solved = true;
        c->parts_event = parts;
        return PIC_OK;
    }
    c->ph_cur = slots[0];
    c->ph_prev = slots[1];
    c->ph_free = slots[2];
    c->ph_out = slots[3];
    c->n_solves = n_solves;
    c->last_on_device = on_device;
    c->last_cycles = cycles;
    c->last_rel = rel;
    if (gated) {
        c->launches -= c->fgraph_kernels[slots[0]] - 1;  // only the gate ran
    } else {
        k_clear_err<<<1, 1, 0, c->s>>>(c->st(), kErrPoissonLimit);
        c->launches += 1;
    }
    c->pt.n_undone++;
    return extra_generations<T>(c, A, MODE_PIC, stats, &h);
}

template <class T> static int one_step(pic_ctx* c, bool stats, bool* solved) {
    *solved = false;
    c->parts_event = false;
    c->step++;
    PushArgs<T> A = make_args<T>(c, MODE_PIC);
    cudaMemsetAsync(c->qe(), 0, (size_t)c->g.ncell() * 8, c->s);
    // the step's speed histogram accumulates over every kernel that stores its electrons
    if (A.vhist) cudaMemsetAsync(A.vhist, 0, sizeof(c->st()->vhist), c->s);
    c->mark(0);
    c->launches += 3;
    // the gather and half-kick of Eq. 2 are done as the collision kernel loads each parent
    A.kick_on_load = 1;
    cudaError_t e = PushLaunch<T>::parents(A, MODE_PIC, stats, c->grid_push, c->s);
    c->mark(1);
    if (e == cudaSuccess) e = PushLaunch<T>::children(A, MODE_PIC, stats, c->grid_push, c->s);
    c->mark(2);
    if (e != cudaSuccess) return c->cuda_fail(e, "push");
    const int rc = can_speculate(c) ? speculative_tail<T>(c, A, stats, solved)
                                    : extra_generations<T>(c, A, MODE_PIC, stats);
    if (rc) return rc;
    k_end_step<<<1, 1, 0, c->s>>>(c->st(), nullptr, c->cfg.capacity);
    c->cur = 1 - c->cur;
    c->a_valid = 1;
    c->steps_done++;
    return PIC_OK;
}

extern "C" int pic_step(pic_ctx* c, int n_steps, pic_step_stats* stats) {
    if (!c || n_steps < 0) return PIC_ERR_ARG;
    if (!c->field_valid && !c->cfg.coupled) return c->fail(PIC_ERR_STATE, "no field: call pic_set_field first");
    const bool want = stats != nullptr;
    DevState h;
    int rc;
    if (want) {
        cudaMemsetAsync(&c->st()->n_events, 0, offsetof(DevState, pred_total) - offsetof(DevState, n_events),
                        c->s);
        rc = read_state(c, &h);
        if (rc) return rc;
        memset(stats, 0, sizeof(*stats));
        stats->n_start = c->n_host;
    }
    const long long wu0 = c->n_wu, so0 = c->n_sorts;
    if (c->cfg.coupled && !c->field_valid) {
        rc = solve_field(c);
        if (rc) return rc;
    }
    for (int it = 0; it < n_steps; ++it) {
        bool solved = false;  // the next step's field was solved within the step
        rc = c->prec == 32 ? one_step<float>(c, want, &solved) : one_step<double>(c, want, &solved);
        if (rc) return rc;
        c->t_total += c->dt_cur;
        c->dt_prev = c->dt_cur;
        if (c->cfg.adaptive_dt) c->dt_cur = c->dt_next;
        c->accumulate(0, 1, &c->pt.ms_push, &c->pt.n_push);
        c->accumulate(1, 2, &c->pt.ms_children, &c->pt.n_children);
        c->n_host = c->n_next;  // the step's count, read back after its collisions
        bool sorted = false;
        c->mark(3);
        if (!solved && (c->cfg.growth_trigger > 0 || c->cfg.weight_interval > 0)) {
            const bool grown = c->cfg.growth_trigger > 0 &&
                               (double)c->n_host > c->cfg.growth_trigger * (double)c->n_last_wu;
            const bool every = c->cfg.weight_interval > 0 && (c->step % (uint32_t)c->cfg.weight_interval) == 0;
            if ((grown || every) && c->n_host > 0) {
                rc = pic_weight_update(c);
                if (rc) return rc;
                sorted = true;
            }
        }
        if (!sorted && c->cfg.sort_interval > 0 && (c->step % (uint32_t)c->cfg.sort_interval) == 0) {
            rc = c->prec == 32 ? sort_by_cell<float>(c) : sort_by_cell<double>(c);
            if (rc) return rc;
        }
        if (sorted) {  // merged particles moved: redeposit the electrons
            cudaMemsetAsync(c->qe(), 0, (size_t)c->g.ncell() * 8, c->s);
            if (c->prec == 32) deposit_current<float>(c, c->qe());
            else deposit_current<double>(c, c->qe());
            c->launches += 1;
        }
        c->mark(4);
        c->accumulate(3, 4, &c->pt.ms_reorder, &c->pt.n_reorder);
        if (c->cfg.coupled && !solved) {
            c->mark(5);
            rc = solve_field(c);
            if (rc) return rc;
            c->mark(6);
            c->accumulate(5, 6, &c->pt.ms_field, &c->pt.n_field);
        }
        if (c->pending.size() >= 4096) c->resolve_times();
    }
    // Every step read the device state after its collisions and checked the
    // error flags; without statistics the call returns without waiting for
    // the last field solve, whose flags the next read reports.
    if (!want && n_steps > 0) return PIC_OK;
    rc = read_state(c, &h);
    if (rc) return rc;
    const int erc = check_err(c, h);
    if (want) {
        stats->n_end = c->n_host;
        stats->n_events = (long long)h.n_events;
        stats->n_null = (long long)h.n_null;
        for (int k = 0; k < PIC_MAX_PROC; ++k) stats->n_coll[k] = (long long)h.n_coll[k];
        stats->n_children = (long long)h.n_children;
        stats->n_attached = (long long)h.n_attached;
        stats->n_absorbed = (long long)h.n_absorbed;
        stats->n_clamped = (long long)h.n_clamped;
        stats->n_processed = (long long)h.n_processed;
        stats->w_ion = h.w_ion;
        stats->w_att = h.w_att;
        stats->w_absorbed = h.w_absorbed;
        stats->n_weight_updates = c->n_wu - wu0;
        stats->n_sorts = c->n_sorts - so0;
        if (c->last_on_device) {
            c->last_cycles = h.poisson_cycles;
            c->last_rel = h.poisson_rel;
        }
        stats->poisson_cycles = c->last_cycles;
        stats->poisson_rel_res = c->last_rel;
        stats->dt_last = c->dt_prev;
        stats->t_total = c->t_total;
        stats->ne_max = c->ne_max;
        stats->n_photo = (long long)h.n_photons;
    }
    return erc;
}

extern "C" int pic_deposit(pic_ctx* c, int64_t* q_e, int64_t* q_pos, int64_t* q_neg, double* rho) {
    if (c) c->parts_event = false;  // work on the particle buffers may follow
    if (!c) return PIC_ERR_ARG;
    const size_t n = (size_t)c->g.ncell();
    cudaMemsetAsync(c->qe(), 0, n * 8, c->s);
    if (c->prec == 32) deposit_current<float>(c, c->qe());
    else deposit_current<double>(c, c->qe());
    cudaError_t e = cudaSuccess;
    if (q_e) e = cudaMemcpyAsync(q_e, c->qe(), n * 8, cudaMemcpyDeviceToDevice, c->s);
    if (e == cudaSuccess && q_pos) e = cudaMemcpyAsync(q_pos, c->qp(), n * 8, cudaMemcpyDeviceToDevice, c->s);
    if (e == cudaSuccess && q_neg) e = cudaMemcpyAsync(q_neg, c->qn(), n * 8, cudaMemcpyDeviceToDevice, c->s);
    if (e != cudaSuccess) return c->cuda_fail(e, "deposit copy");
    if (rho) fixed_to_rho(c, rho);
    DevState h;
    int rc = read_state(c, &h);
    if (rc) return rc;
    return check_err(c, h);
}

// ---------------------------------------------------------------- checkpoint
// The blob holds the potential in float64; float32 contexts convert from and
// to their float pairs on the host (hi + lo is exact in float64).
static cudaError_t save_phi(pic_ctx* c, double* out) {
    const size_t n = (size_t)c->g.ncell();
    if (c->prec != 32 || c->g.axi) return cudaMemcpy(out, c->phi(), n * 8, cudaMemcpyDeviceToHost);
    std::vector<float> hl(2 * n);
    cudaError_t e = cudaMemcpy(hl.data(), c->ph_hi(c->ph_cur), n * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(hl.data() + n, c->ph_lo(c->ph_cur), n * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return e;
    for (size_t i = 0; i < n; ++i) out[i] = (double)hl[i] + (double)hl[n + i];
    return cudaSuccess;
}

static cudaError_t load_phi(pic_ctx* c, const double* in) {
    const size_t n = (size_t)c->g.ncell();
    if (c->prec != 32 || c->g.axi) return cudaMemcpy(c->phi(), in, n * 8, cudaMemcpyHostToDevice);
    std::vector<float> hl(2 * n);
    for (size_t i = 0; i < n; ++i) {
        hl[i] = (float)in[i];
        hl[n + i] = (float)(in[i] - (double)hl[i]);
    }
    cudaError_t e = cudaMemcpy(c->ph_hi(c->ph_cur), hl.data(), n * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->ph_lo(c->ph_cur), hl.data() + n, n * 4, cudaMemcpyHostToDevice);
    return e;
}

struct BlobHead {
    uint64_t magic;
    int32_t prec, a_valid;
    int64_t n, n_last_wu, ncell;
    uint32_t step, pad;
    int64_t n_wu, n_sorts;
    double dt_cur, dt_prev, w_prev, t_total;
};
static const uint64_t kMagic = 0x3230314D43435049ull;  // "IPCCM102"

extern "C" int pic_save(pic_ctx* c, void* blob, size_t* bytes) {
    if (c) c->parts_event = false;  // work on the particle buffers may follow
    if (!c || !bytes) return PIC_ERR_ARG;
    DevState h;
    int rc = read_state(c, &h);
    if (rc) return rc;
    const size_t R = real_size(c->prec), n = (size_t)c->n_host, ncell = (size_t)c->g.ncell();
    const size_t need = sizeof(BlobHead) + n * (10 * R + 8) + 3 * ncell * 8;
    if (!blob || *bytes < need) { *bytes = need; return blob ? PIC_ERR_CAPACITY : PIC_OK; }
    BlobHead hd{kMagic, c->prec, c->a_valid, (int64_t)n, c->n_last_wu, (int64_t)ncell, c->step, 0, c->n_wu, c->n_sorts,
                c->dt_cur, c->dt_prev, c->w_prev, c->t_total};
    char* p = (char*)blob;
    memcpy(p, &hd, sizeof hd);
    p += sizeof hd;
    char* base = c->ws + c->L.buf[c->cur];
    const size_t cap = (size_t)c->cfg.capacity;
    cudaError_t e = cudaSuccess;
    for (int f = 0; f < 10 && e == cudaSuccess; ++f) {
        e = cudaMemcpy(p, base + f * al256(cap * R), n * R, cudaMemcpyDeviceToHost);
        p += n * R;
    }
    if (e == cudaSuccess) e = cudaMemcpy(p, base + 10 * al256(cap * R), n * 8, cudaMemcpyDeviceToHost);
    p += n * 8;
    if (e == cudaSuccess) e = cudaMemcpy(p, c->qp(), ncell * 8, cudaMemcpyDeviceToHost);
    p += ncell * 8;
    if (e == cudaSuccess) e = cudaMemcpy(p, c->qn(), ncell * 8, cudaMemcpyDeviceToHost);
    p += ncell * 8;
    if (e == cudaSuccess) e = save_phi(c, (double*)p);
    if (e != cudaSuccess) return c->cuda_fail(e, "save");
    *bytes = need;
    return PIC_OK;
}

extern "C" int pic_load(pic_ctx* c, const void* blob, size_t bytes) {
    if (c) c->parts_event = false;  // work on the particle buffers may follow
    if (!c || !blob || bytes < sizeof(BlobHead)) return PIC_ERR_ARG;
    BlobHead hd;
    memcpy(&hd, blob, sizeof hd);
    const size_t R = real_size(c->prec), ncell = (size_t)c->g.ncell();
    if (hd.magic != kMagic || hd.prec != c->prec || (size_t)hd.ncell != ncell || hd.n < 0 ||
        hd.n > c->cfg.capacity)
        return c->fail(PIC_ERR_ARG, "blob does not match this context");
    const size_t n = (size_t)hd.n;
    if (bytes < sizeof(BlobHead) + n * (10 * R + 8) + 3 * ncell * 8) return PIC_ERR_ARG;
    const char* p = (const char*)blob + sizeof hd;
    c->cur = 0;
    char* base = c->ws + c->L.buf[0];
    const size_t cap = (size_t)c->cfg.capacity;
    cudaError_t e = cudaSuccess;
    for (int f = 0; f < 10 && e == cudaSuccess; ++f) {
        e = cudaMemcpy(base + f * al256(cap * R), p, n * R, cudaMemcpyHostToDevice);
        p += n * R;
    }
    if (e == cudaSuccess) e = cudaMemcpy(base + 10 * al256(cap * R), p, n * 8, cudaMemcpyHostToDevice);
    p += n * 8;
    if (e == cudaSuccess) e = cudaMemcpy(c->qp(), p, ncell * 8, cudaMemcpyHostToDevice);
    p += ncell * 8;
    if (e == cudaSuccess) e = cudaMemcpy(c->qn(), p, ncell * 8, cudaMemcpyHostToDevice);
    p += ncell * 8;
    if (e == cudaSuccess) e = load_phi(c, (const double*)p);
    if (e != cudaSuccess) return c->cuda_fail(e, "load");
    k_set_count<<<1, 1, 0, c->s>>>(c->st(), (unsigned long long)n);
    c->n_host = (long long)n;
    c->n_last_wu = hd.n_last_wu;
    c->step = hd.step;
    c->a_valid = hd.a_valid;
    c->n_wu = hd.n_wu;
    c->n_sorts = hd.n_sorts;
    c->dt_cur = hd.dt_cur;
    c->dt_prev = hd.dt_prev;
    c->w_prev = hd.w_prev;
    c->t_total = hd.t_total;
    if (c->cfg.coupled) {
        c->field_valid = 0;  // recomputed from the restored charge before the next step
        c->n_solves = 0;
    }
    return PIC_OK;
}

// ====================================================================== swarms
// Sec. 2.2.2: electrons traced in a uniform field give flux coefficients
// (averages over electrons) and bulk coefficients (motion and spread of the
// centre of mass).  Each swarm runs in turn over one shared set of buffers.
static pic_config swarm_pic_config(const swarm_config* sc) {
    pic_config c;
    memset(&c, 0, sizeof c);
    c.precision = sc->precision;
    c.nx = c.ny = c.nz = 2;
    c.dx = 1.0;
    c.capacity = sc->capacity;
    c.seed = sc->seed;
    c.dt = sc->dt;
    c.gas = sc->gas;
    return c;
}

static size_t swarm_extra(const swarm_config* sc) {
    return al256((size_t)sc->n_steps * kNMom * 8) + al256((size_t)sc->n_steps * 8);
}

struct BatchLayout {
    size_t total, ctx, ctx_bytes, buf[2], cq[2], csw[2], cnt_in, cnt_out, prefix, bd, Ez, mom, counts, zref, zhist;
    size_t tabs, numax, tau, dens, nmx, tab64;  // per-swarm rate tables
    long long segs, cap_child;
};

static BatchLayout batch_layout(const swarm_config* sc, int n) {
    BatchLayout L;
    pic_config pc = swarm_pic_config(sc);
    pc.capacity = 1;
    const size_t R = real_size(sc->precision);
    L.segs = (long long)n * sc->capacity;
    L.cap_child = L.segs / 2 > 4096 ? L.segs / 2 : 4096;
    size_t o = 0;
    auto take = [&](size_t b) { size_t r = o; o += al256(b); return r; };
    L.ctx_bytes = make_layout(&pc).total;
    L.ctx = take(L.ctx_bytes);
    for (int b = 0; b < 2; ++b) {
        L.buf[b] = o;
        for (int f = 0; f < 10; ++f) take((size_t)L.segs * R);
        take((size_t)L.segs * 8);
    }
    for (int q = 0; q < 2; ++q) {
        L.cq[q] = o;
        for (int f = 0; f < 11; ++f) take((size_t)L.cap_child * R);
        take((size_t)L.cap_child * 8);
        take((size_t)L.cap_child * 4);
        L.csw[q] = take((size_t)L.cap_child * 4);
    }
    L.cnt_in = take((size_t)n * 8);
    L.cnt_out = take((size_t)n * 8);
    L.prefix = take((size_t)(n + 1) * 8);
    L.bd = take(sizeof(BatchDev));
    L.Ez = take((size_t)n * 8);
    L.mom = take((size_t)n * sc->n_steps * kNMom * 8);
    L.counts = take((size_t)n * sc->n_steps * 8);
    L.zref = take((size_t)n * 8);
    L.zhist = take((size_t)n * sc->n_steps * 8);
    const int nb = sc->gas.n_bins, np = sc->gas.n_proc > 0 ? sc->gas.n_proc : 1;
    L.tabs = take((size_t)n * nb * kTableStride * R);
    L.numax = take((size_t)n * R);
    L.tau = take((size_t)n * R);
    L.dens = take((size_t)n * np * 8);
    L.nmx = take((size_t)n * 8);
    L.tab64 = take((size_t)nb * kTableStride * 8);
    L.total = o;
    return L;
}

// Target densities of the processes of a swarm with O2 fraction f: n_gas f
// for O2 targets, n_gas (1 - f) for the others (Sec. 2.3: the gas is N2 and
// O2); without fractions, the gas's own densities.
static void swarm_densities(const swarm_config* sc, const double* o2_frac, int s, double* out) {
    for (int k = 0; k < sc->gas.n_proc; ++k) {
        if (!o2_frac) { out[k] = sc->gas.density[k]; continue; }
        const double f = o2_frac[s];
        out[k] = sc->gas.species[k] == 1 ? sc->n_gas * f : sc->n_gas * (1.0 - f);
    }
}

extern "C" size_t swarm_workspace_bytes(const swarm_config* sc, int n_swarms) {
    if (!sc || n_swarms < 1 || sc->n_steps < 1) return 0;
    pic_config c = swarm_pic_config(sc);
    if (validate(&c) != PIC_OK) return 0;
    if (sc->batched) {
        if (n_swarms > kMaxSwarms) return 0;
        return batch_layout(sc, n_swarms).total;
    }
    return make_layout(&c).total + swarm_extra(sc);
}

// Swarm weight integrated over one step, per unit time.  Collisions alone
// change the weight inside a step, so it began the step at W_end - w_ion +
// w_att; over the step it is taken as exponential (a constant net rate), whose
// mean is the logarithmic mean W0 x / ln(1 + x) with x = W_end / W0 - 1.
static double step_weight_integral(const double* m) {
    const double w_end = m[0];
    const double w0 = w_end - m[14] + m[15];
    if (!(w0 > 0.0) || !(w_end > 0.0)) return 0.5 * (w0 + w_end);
    const double x = w_end / w0 - 1.0;
    if (fabs(x) < 1e-9) return 0.5 * (w0 + w_end);
    return w0 * x / log1p(x);
}

// Flux = time average of per-step electron averages; bulk = least-squares
// slopes of the centre of mass and of the spread; rate coefficients = time
// average of (event weight of the step) / (N x the step's integral of the
// swarm weight over time); errors from 10-block batch means.
static void swarm_coeffs(const double* mom, int r0, int r1, double dt, double n_gas, double* o) {
    const int n = r1 - r0;
    double wf = 0, dlf = 0, dtf = 0, me = 0, sion = 0, satt = 0, sw = 0;
    double st = 0, stt = 0, sz = 0, stz = 0, sl = 0, stl = 0, sr = 0, str = 0;
    for (int r = r0; r < r1; ++r) {
        const double* m = mom + (size_t)r * kNMom;
        const double W = m[0];
        const double mx = m[1] / W, my = m[2] / W, mz = m[3] / W;
        const double vx = m[7] / W, vy = m[8] / W, vz = m[9] / W;
        wf += vz;
        dlf += m[12] / W - mz * vz;
        dtf += 0.5 * ((m[10] / W - mx * vx) + (m[11] / W - my * vy));
        me += m[13] / W;
        const double Wt = step_weight_integral(m);
        sion += m[14] / Wt;
        satt += m[15] / Wt;
        sw += 1.0;
        const double t = (double)(r + 1) * dt;
        const double varz = m[6] / W - mz * mz;
        const double vart = (m[4] / W - mx * mx) + (m[5] / W - my * my);
        st += t; stt += t * t; sz += mz; stz += t * mz; sl += varz; stl += t * varz; sr += vart; str += t * vart;
    }
    const double den = n * stt - st * st;
    o[0] = wf / n;
    o[1] = (n * stz - st * sz) / den;
    o[2] = dlf / n;
    o[3] = dtf / n;
    o[4] = 0.5 * (n * stl - st * sl) / den;
    o[5] = 0.25 * (n * str - st * sr) / den;
    o[6] = me / n;
    o[7] = sion / (n_gas * dt * sw);
    o[8] = satt / (n_gas * dt * sw);
    o[9] = o[7] * n_gas / o[0];
    o[10] = o[8] * n_gas / o[0];
}

static void swarm_result_from(const double* mom, int n_steps, double sample_from, double dt, double n_gas,
                              swarm_result* res) {
    for (int q = 0; q < PIC_SWARM_NRES; ++q) res->v[q] = NAN;
    int i0 = (int)(sample_from * n_steps);
    if (i0 < 0) i0 = 0;
    const int nb = 10;
    if (n_steps - i0 < 2 * nb) return;
    swarm_coeffs(mom, i0, n_steps, dt, n_gas, res->v);
    const int len = (n_steps - i0) / nb;
    double blk[10][11];
    for (int b = 0; b < nb; ++b) swarm_coeffs(mom, i0 + b * len, i0 + (b + 1) * len, dt, n_gas, blk[b]);
    for (int q = 0; q < 11; ++q) {
        double mean = 0, var = 0;
        for (int b = 0; b < nb; ++b) mean += blk[b][q];
        mean /= nb;
        for (int b = 0; b < nb; ++b) var += (blk[b][q] - mean) * (blk[b][q] - mean);
        res->v[11 + q] = sqrt(var / (nb - 1)) / sqrt((double)nb);
    }
}

template <class T> static int swarm_one(pic_ctx* c, const swarm_config* sc, double EN, double* d_mom, long long* d_cnt,
                                        double* h_mom, long long* h_cnt, swarm_result* res) {
    const int ns = sc->n_steps;
    cudaMemsetAsync(d_mom, 0, (size_t)ns * kNMom * 8, c->s);
    cudaMemsetAsync(c->st(), 0, sizeof(DevState), c->s);
    c->cur = 0;
    const double sig = sqrt(sc->kT_eV * kQ / kMe);
    k_seed_maxwell<T><<<grid_n(sc->n0), 256, 0, c->s>>>(sc->n0, sig, c->K, c->soa<T>(0));
    k_set_count<<<1, 1, 0, c->s>>>(c->st(), (unsigned long long)sc->n0);
    const double E = EN * 1e-21 * sc->n_gas;
    c->field_uniform = 1;
    c->E0[0] = 0.0; c->E0[1] = 0.0; c->E0[2] = -E;
    c->step = 0;
    for (int s = 1; s <= ns; ++s) {
        c->step = (uint32_t)s;
        c->a_valid = 0;  // uniform field: no half-kick
        PushArgs<T> A = make_args<T>(c, MODE_SWARM);
        A.mom = d_mom + (size_t)(s - 1) * kNMom;
        A.n_lo = sc->n_lo;
        A.n_hi = sc->n_hi;
        A.mask = nullptr;
        A.q_e = A.q_pos = A.q_neg = nullptr;
        cudaError_t e = PushLaunch<T>::resample(A, grid_n(2 * sc->n_hi), c->s);
        if (e == cudaSuccess) e = PushLaunch<T>::field_kick(A, grid_n(2 * sc->n_hi), c->s);
        if (e == cudaSuccess) e = PushLaunch<T>::parents(A, MODE_SWARM, false, c->grid_push, c->s);
        if (e == cudaSuccess) e = PushLaunch<T>::children(A, MODE_SWARM, false, c->grid_push, c->s);
        if (e != cudaSuccess) return c->cuda_fail(e, "swarm push");
        int rc = extra_generations<T>(c, A, MODE_SWARM, false);
        if (rc) return rc;
        k_end_step<<<1, 1, 0, c->s>>>(c->st(), d_cnt + (s - 1), c->cfg.capacity);
        c->cur = 1 - c->cur;
    }
    cudaError_t e = cudaMemcpyAsync(h_mom, d_mom, (size_t)ns * kNMom * 8, cudaMemcpyDeviceToHost, c->s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_cnt, d_cnt, (size_t)ns * 8, cudaMemcpyDeviceToHost, c->s);
    DevState h;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, c->st(), sizeof h, cudaMemcpyDeviceToHost, c->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->s);
    if (e != cudaSuccess) return c->cuda_fail(e, "swarm read-back");
    if (h.err) return check_err(c, h);
    swarm_result_from(h_mom, ns, sc->sample_from, sc->dt, sc->n_gas, res);
    res->v[22] = (double)h_cnt[ns - 1];
    res->v[23] = h_mom[(size_t)(ns - 1) * kNMom];
    return PIC_OK;
}

// ------------------------------------------------------------------ batched swarms
template <class T> struct BatchRunner {
    pic_ctx* c = nullptr;
    BatchArgs<T> B;
    BatchLayout L;
    const swarm_config* sc;
    int n;
    cudaStream_t s;
    cudaStream_t cap = nullptr;
    std::string err;

    ~BatchRunner() {
        if (c) pic_destroy(c);
        if (cap) cudaStreamDestroy(cap);
    }

    // Rate table, nu_max and flight-time scale of every swarm's gas (its own
    // O2 fraction, or the gas as given), built on the device.
    int build_tables(char* ws, const double* o2) {
        const int nb = c->n_bins, np = c->n_proc;
        const double* d_gas = (const double*)(c->ws + c->L.gas);  // node energies, then cross sections
        std::vector<double> dens((size_t)n * np);
        for (int i = 0; i < n; ++i) swarm_densities(sc, o2, i, dens.data() + (size_t)i * np);
        double* d_dens = (double*)(ws + L.dens);
        unsigned long long* d_nmx = (unsigned long long*)(ws + L.nmx);
        T* tabs = (T*)(ws + L.tabs);
        cudaError_t e = cudaMemcpyAsync(d_dens, dens.data(), dens.size() * 8, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_nmx, 0, (size_t)n * 8, s);
        for (int i = 0; i < n && e == cudaSuccess; ++i) {
            k_rate_table<T><<<(nb + 127) / 128, 128, 0, s>>>(d_gas, d_gas + nb, d_dens + (size_t)i * np, np, nb,
                                                             tabs + (size_t)i * nb * kTableStride,
                                                             (double*)(ws + L.tab64), d_nmx + i);
            e = cudaGetLastError();
        }
        std::vector<unsigned long long> bits((size_t)n);
        if (e == cudaSuccess) e = cudaMemcpyAsync(bits.data(), d_nmx, (size_t)n * 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return PIC_ERR_CUDA;
        std::vector<T> numax((size_t)n), tau((size_t)n);
        for (int i = 0; i < n; ++i) {
            double v;
            memcpy(&v, &bits[i], 8);
            if (!(v > 0.0)) return PIC_ERR_ARG;
            numax[i] = (T)v;
            tau[i] = (T)(-0.69314718055994530942 / v);
        }
        e = cudaMemcpyAsync(ws + L.numax, numax.data(), (size_t)n * sizeof(T), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(ws + L.tau, tau.data(), (size_t)n * sizeof(T), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return PIC_ERR_CUDA;
        B.tab_s = tabs;
        B.tab_stride = (long long)nb * kTableStride;
        B.numax_s = (const T*)(ws + L.numax);
        B.tau_s = (const T*)(ws + L.tau);
        return PIC_OK;
    }

    int setup(const swarm_config* sc_, int n_, const double* EN, const double* o2, char* ws, cudaStream_t s_) {
        sc = sc_;
        n = n_;
        s = s_;
        L = batch_layout(sc, n);
        pic_config pc = swarm_pic_config(sc);
        pc.capacity = 1;
        int rc = pic_init(&pc, ws + L.ctx, L.ctx_bytes, nullptr, (pic_stream_t)s, &c);
        if (rc) return rc;
        memset(&B, 0, sizeof B);
        B.P = make_args<T>(c, MODE_SWARM);
        B.warp_chunk = sc->warp_chunk > 0 ? sc->warp_chunk : kWarpChunk;
        rc = build_tables(ws, o2);
        if (rc) return rc;
        const size_t R = sizeof(T);
        for (int b = 0; b < 2; ++b) {
            Soa<T>& q = b == 0 ? B.in : B.out;
            char* p = ws + L.buf[b];
            for (int f = 0; f < 10; ++f) { q.r[f] = (T*)p; p += al256((size_t)L.segs * R); }
            q.id = (uint64_t*)p;
        }
        for (int q = 0; q < 2; ++q) {
            char* p = ws + L.cq[q];
            for (int f = 0; f < 10; ++f) { B.cq[q].p.r[f] = (T*)p; p += al256((size_t)L.cap_child * R); }
            B.cq[q].t_left = (T*)p;
            p += al256((size_t)L.cap_child * R);
            B.cq[q].p.id = (uint64_t*)p;
            p += al256((size_t)L.cap_child * 8);
            B.cq[q].k = (uint32_t*)p;
            B.csw[q] = (uint32_t*)(ws + L.csw[q]);
        }
        B.cap_s = sc->capacity;
        B.n_swarms = n;
        B.cnt_in = (long long*)(ws + L.cnt_in);
        B.cnt_out = (unsigned long long*)(ws + L.cnt_out);
        B.prefix = (long long*)(ws + L.prefix);
        B.cap_child = L.cap_child;
        B.bd = (BatchDev*)(ws + L.bd);
        B.seed = sc->seed;
        B.Ez = (const double*)(ws + L.Ez);
        B.mom = (double*)(ws + L.mom);
        B.counts = (long long*)(ws + L.counts);
        B.zref = (double*)(ws + L.zref);
        B.zref_hist = (double*)(ws + L.zhist);
        B.n_steps = sc->n_steps;
        B.n_lo = sc->n_lo;
        B.n_hi = sc->n_hi;
        std::vector<double> ez((size_t)n);
        for (int i = 0; i < n; ++i) ez[i] = -EN[i] * 1e-21 * sc->n_gas;
        cudaError_t e = cudaMemcpyAsync(ws + L.Ez, ez.data(), (size_t)n * 8, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        return e == cudaSuccess ? PIC_OK : PIC_ERR_CUDA;
    }

    cudaError_t init_state() {
        cudaMemsetAsync(B.mom, 0, (size_t)n * sc->n_steps * kNMom * 8, s);
        cudaMemsetAsync(B.counts, 0, (size_t)n * sc->n_steps * 8, s);
        return BatchLaunch<T>::init(B, sc->n0, sqrt(sc->kT_eV * kQ / kMe), s);
    }

    // All `steps` steps in one persistent cooperative kernel, recorded in a
    // CUDA graph (launched directly if the recording fails).  bps is capped
    // at the blocks that can be resident together.
    int run_persistent(int steps, int block, int bps) {
        const int maxb = BatchLaunch<T>::persistent_blocks_per_sm(block);
        if (maxb < 1) return PIC_ERR_CUDA;
        const int grid = device_sms() * (bps < maxb ? bps : maxb);
        if (!cap && cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return PIC_ERR_CUDA;
        cudaGraph_t g = nullptr;
        cudaGraphExec_t x = nullptr;
        bool graphed = false;
        if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            const cudaError_t el = BatchLaunch<T>::run_persistent(B, steps, block, grid, cap);
            const cudaError_t ee = cudaStreamEndCapture(cap, &g);
            graphed = el == cudaSuccess && ee == cudaSuccess && g && cudaGraphInstantiate(&x, g, 0) == cudaSuccess;
        }
        cudaGetLastError();
        cudaError_t e = graphed ? cudaGraphLaunch(x, s) : BatchLaunch<T>::run_persistent(B, steps, block, grid, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (x) cudaGraphExecDestroy(x);
        if (g) cudaGraphDestroy(g);
        return e == cudaSuccess ? PIC_OK : PIC_ERR_CUDA;
    }

    // Runs `steps` steps: kernels per step (mode 0), a two-step CUDA graph
    // replayed (1), or one persistent kernel (2).
    int run(int steps, int block, int bps, int mode) {
        if (mode == 2) return run_persistent(steps, block, bps);
        return run_steps(steps, block, device_sms() * bps, mode == 1);
    }

    int run_steps(int steps, int block, int grid, bool graph) {
        if (BatchLaunch<T>::prepare(block) != cudaSuccess) return PIC_ERR_CUDA;
        BatchArgs<T> Bo = B;
        std::swap(Bo.in, Bo.out);
        if (!graph) {
            for (int i = 0; i < steps; ++i)
                if (BatchLaunch<T>::step((i & 1) ? Bo : B, block, grid, s, nullptr) != cudaSuccess) return PIC_ERR_CUDA;
            return PIC_OK;
        }
        if (!cap && cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return PIC_ERR_CUDA;
        cudaGraph_t g2 = nullptr, g1 = nullptr;
        cudaGraphExec_t x2 = nullptr, x1 = nullptr;
        int rc = PIC_OK;
        if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return PIC_ERR_CUDA;
        BatchLaunch<T>::step(B, block, grid, cap, nullptr);
        BatchLaunch<T>::step(Bo, block, grid, cap, nullptr);
        if (cudaStreamEndCapture(cap, &g2) != cudaSuccess || cudaGraphInstantiate(&x2, g2, 0) != cudaSuccess)
            rc = PIC_ERR_CUDA;
        if (rc == PIC_OK && (steps & 1)) {
            if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = PIC_ERR_CUDA;
            else {
                BatchLaunch<T>::step(B, block, grid, cap, nullptr);
                if (cudaStreamEndCapture(cap, &g1) != cudaSuccess || cudaGraphInstantiate(&x1, g1, 0) != cudaSuccess)
                    rc = PIC_ERR_CUDA;
            }
        }
        for (int i = 0; rc == PIC_OK && i + 1 < steps; i += 2)
            if (cudaGraphLaunch(x2, s) != cudaSuccess) rc = PIC_ERR_CUDA;
        if (rc == PIC_OK && (steps & 1) && cudaGraphLaunch(x1, s) != cudaSuccess) rc = PIC_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) rc = PIC_ERR_CUDA;
        if (x2) cudaGraphExecDestroy(x2);
        if (x1) cudaGraphExecDestroy(x1);
        if (g2) cudaGraphDestroy(g2);
        if (g1) cudaGraphDestroy(g1);
        return rc;
    }

    // ms per step of a short trial run (after two warm-up steps) of one
    // launch shape; negative on a CUDA error.
    double trial_ms(int block, int bps, long long chunk, int mode, cudaEvent_t e0, cudaEvent_t e1) {
        const int trial = sc->n_steps < 10 ? sc->n_steps : 10;
        B.warp_chunk = chunk;
        if (init_state() != cudaSuccess) return -1.0;
        if (run(2, block, bps, mode)) return -1.0;
        cudaEventRecord(e0, s);
        if (run(trial, block, bps, mode)) return -1.0;
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) return -1.0;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms / trial;
    }

    // Launch-shape autotuner: block size x blocks per SM (graph replay,
    // ranges of 1024 items), then the warp item range, then the launch mode.
    int tune(int* best_block, int* best_bps, int* best_chunk, int* best_mode, double* best_ms) {
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        double best = 1e300;
        int bb = 128, bp = 1, bm = 1;
        long long bc = kWarpChunk;
        int rc = PIC_OK;
        for (int block : {64, 128, 256}) {
            if (BatchLaunch<T>::prepare(block) != cudaSuccess) continue;
            const int maxb = BatchLaunch<T>::max_blocks_per_sm(block);
            for (int bps : {1, 2, 3, 4, maxb}) {
                if (bps > maxb) continue;
                const double per = trial_ms(block, bps, kWarpChunk, 1, e0, e1);
                if (per < 0) { rc = PIC_ERR_CUDA; break; }
                if (per < best) { best = per; bb = block; bp = bps; }
            }
            if (rc) break;
        }
        for (long long chunk : {256ll, 512ll, 2048ll}) {
            if (rc) break;
            const double per = trial_ms(bb, bp, chunk, 1, e0, e1);
            if (per < 0) { rc = PIC_ERR_CUDA; break; }
            if (per < best) { best = per; bc = chunk; }
        }
        if (!rc) {
            const double per = trial_ms(bb, bp, bc, 2, e0, e1);
            if (per < 0) rc = PIC_ERR_CUDA;
            else if (per < best) { best = per; bm = 2; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        B.warp_chunk = bc;
        *best_block = bb;
        *best_bps = bp;
        *best_chunk = (int)bc;
        *best_mode = bm;
        *best_ms = best;
        return rc;
    }
};

template <class T>
static int run_batched(const swarm_config* sc, int n, const double* EN, const double* o2, char* ws, cudaStream_t s,
                       swarm_result* res, double* moments, long long* counts) {
    BatchRunner<T> R;
    int rc = R.setup(sc, n, EN, o2, ws, s);
    if (rc) return rc;
    int block = sc->block, bps = sc->blocks_per_sm, mode = sc->use_graph, chunk = sc->warp_chunk;
    if (block == 0 || bps == 0) {
        double ms;
        rc = R.tune(&block, &bps, &chunk, &mode, &ms);
        if (rc) return rc;
    }
    if (block != 64 && block != 128 && block != 256) return PIC_ERR_ARG;
    R.B.warp_chunk = chunk > 0 ? chunk : kWarpChunk;
    if (R.init_state() != cudaSuccess) return PIC_ERR_CUDA;
    rc = R.run(sc->n_steps, block, bps, mode);
    if (rc) return rc;
    const int ns = sc->n_steps;
    std::vector<double> hm((size_t)n * ns * kNMom), hz((size_t)n * ns);
    std::vector<long long> hc((size_t)n * ns);
    BatchDev hb;
    cudaError_t e = cudaMemcpyAsync(hm.data(), R.B.mom, hm.size() * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hz.data(), R.B.zref_hist, hz.size() * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hc.data(), R.B.counts, hc.size() * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hb, R.B.bd, sizeof hb, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return PIC_ERR_CUDA;
    if (hb.err & kErrBarrier) return PIC_ERR_TIMEOUT;
    if (hb.err) return PIC_ERR_CAPACITY;
    // z moments back to the origin: z = dz + r
    for (size_t r = 0; r < (size_t)n * ns; ++r) {
        double* m = hm.data() + r * kNMom;
        const double ref = hz[r];
        const double m0 = m[0], m3 = m[3], m9 = m[9];
        m[6] = m[6] + 2.0 * ref * m3 + ref * ref * m0;
        m[3] = m3 + ref * m0;
        m[12] = m[12] + ref * m9;
    }
    for (int i = 0; i < n; ++i) {
        const double* m = hm.data() + (size_t)i * ns * kNMom;
        swarm_result_from(m, ns, sc->sample_from, sc->dt, sc->n_gas, &res[i]);
        res[i].v[22] = (double)hc[(size_t)i * ns + ns - 1];
        res[i].v[23] = m[(size_t)(ns - 1) * kNMom];
    }
    if (moments) memcpy(moments, hm.data(), hm.size() * 8);
    if (counts) memcpy(counts, hc.data(), hc.size() * 8);
    return PIC_OK;
}

static int swarm_check(const swarm_config* sc, int n_swarms, const double* EN_Td, const double* o2, void* d_ws,
                       size_t ws_bytes) {
    if (!sc || n_swarms < 1 || !EN_Td || !d_ws || ((uintptr_t)d_ws & 255)) return PIC_ERR_ARG;
    if (sc->n0 < 1 || sc->n0 > sc->capacity || sc->n_steps < 1 || !(sc->n_gas > 0) || !(sc->kT_eV >= 0) ||
        sc->n_lo < 0 || sc->n_hi < sc->n_lo || sc->capacity < 2 * sc->n_hi)
        return PIC_ERR_ARG;
    if (sc->batched && (sc->use_graph < 0 || sc->use_graph > 2 || sc->warp_chunk < 0 || sc->warp_chunk > 8192 ||
                        (sc->warp_chunk % 32) != 0))
        return PIC_ERR_ARG;
    if (o2) {
        if (!sc->gas.species) return PIC_ERR_ARG;
        for (int i = 0; i < n_swarms; ++i)
            if (!(o2[i] >= 0.0 && o2[i] <= 1.0)) return PIC_ERR_ARG;
    }
    const size_t need = swarm_workspace_bytes(sc, n_swarms);
    if (need == 0 || ws_bytes < need) return PIC_ERR_ARG;
    return PIC_OK;
}

extern "C" int swarm_autotune(const swarm_config* sc, int n_swarms, const double* EN_Td, const double* o2_frac,
                              void* d_ws, size_t ws_bytes, int* block, int* blocks_per_sm, int* warp_chunk,
                              int* use_graph, double* ms_per_step, pic_stream_t stream) {
    if (!sc || !sc->batched || !block || !blocks_per_sm || !warp_chunk || !use_graph || !ms_per_step)
        return PIC_ERR_ARG;
    int rc = swarm_check(sc, n_swarms, EN_Td, o2_frac, d_ws, ws_bytes);
    if (rc) return rc;
    if (sc->precision == 32) {
        BatchRunner<float> R;
        rc = R.setup(sc, n_swarms, EN_Td, o2_frac, (char*)d_ws, (cudaStream_t)stream);
        if (!rc) rc = R.tune(block, blocks_per_sm, warp_chunk, use_graph, ms_per_step);
    } else {
        BatchRunner<double> R;
        rc = R.setup(sc, n_swarms, EN_Td, o2_frac, (char*)d_ws, (cudaStream_t)stream);
        if (!rc) rc = R.tune(block, blocks_per_sm, warp_chunk, use_graph, ms_per_step);
    }
    return rc;
}

extern "C" int swarm_run(const swarm_config* sc, int n_swarms, const double* EN_Td, const double* o2_frac,
                         void* d_ws, size_t ws_bytes, swarm_result* results, double* moments, long long* counts,
                         pic_stream_t stream) {
    if (!results) return PIC_ERR_ARG;
    int rcc = swarm_check(sc, n_swarms, EN_Td, o2_frac, d_ws, ws_bytes);
    if (rcc) return rcc;
    if (sc->batched)
        return sc->precision == 32
                   ? run_batched<float>(sc, n_swarms, EN_Td, o2_frac, (char*)d_ws, (cudaStream_t)stream, results,
                                        moments, counts)
                   : run_batched<double>(sc, n_swarms, EN_Td, o2_frac, (char*)d_ws, (cudaStream_t)stream, results,
                                         moments, counts);
    const size_t need = swarm_workspace_bytes(sc, n_swarms);
    pic_config pc = swarm_pic_config(sc);
    Layout L = make_layout(&pc);
    double* d_mom = (double*)((char*)d_ws + L.total);
    long long* d_cnt = (long long*)((char*)d_ws + L.total + al256((size_t)sc->n_steps * kNMom * 8));
    std::vector<double> hm((size_t)sc->n_steps * kNMom);
    std::vector<long long> hc((size_t)sc->n_steps);
    std::vector<double> dens((size_t)(sc->gas.n_proc > 0 ? sc->gas.n_proc : 1));
    for (int s = 0; s < n_swarms; ++s) {
        pc.seed = sc->seed + (unsigned long long)s;
        swarm_densities(sc, o2_frac, s, dens.data());
        pc.gas.density = dens.data();
        pic_ctx* c = nullptr;
        int rc = pic_init(&pc, d_ws, L.total, nullptr, stream, &c);
        if (rc) return rc;
        rc = sc->precision == 32 ? swarm_one<float>(c, sc, EN_Td[s], d_mom, d_cnt, hm.data(), hc.data(), &results[s])
                                 : swarm_one<double>(c, sc, EN_Td[s], d_mom, d_cnt, hm.data(), hc.data(), &results[s]);
        pic_destroy(c);
        if (rc) return rc;
        if (moments) memcpy(moments + (size_t)s * sc->n_steps * kNMom, hm.data(), hm.size() * 8);
        if (counts) memcpy(counts + (size_t)s * sc->n_steps, hc.data(), hc.size() * 8);
    }
    return PIC_OK;
}

extern "C" int pic_progress(pic_ctx* c, long long* updates, long long* parents, long long* steps) {
    if (!c) return PIC_ERR_ARG;
    DevState h;
    int rc = read_state(c, &h);
    if (rc) return rc;
    if (updates) *updates = (long long)h.n_updates;
    if (parents) *parents = (long long)h.n_parents;
    if (steps) *steps = c->steps_done;
    return PIC_OK;
}

extern "C" int pic_set_poisson(pic_ctx* c, double rtol, int max_cycles, int device_loop) {
    if (c) c->parts_event = false;  // work on the particle buffers may follow
    if (!c || !(rtol > 0.0) || max_cycles < 1) return PIC_ERR_ARG;
    // recorded graphs hold the old settings
    for (int q = 0; q < 4; ++q)
        if (c->fgraph[q]) {
            cudaGraphExecDestroy(c->fgraph[q]);
            c->fgraph[q] = nullptr;
        }
    if (c->agraph) {
        cudaGraphExecDestroy(c->agraph);
        c->agraph = nullptr;
    }
    c->cfg.poisson_rtol = rtol;
    c->cfg.poisson_max_cycles = max_cycles;
    c->fgraph_off = device_loop == 0;
    return PIC_OK;
}

extern "C" int pic_set_multigrid(pic_ctx* c, int pre_sweeps, int post_sweeps) {
    if (c) c->parts_event = false;  // work on the particle buffers may follow
    if (!c || pre_sweeps < 1 || pre_sweeps > 4 || post_sweeps < 1 || post_sweeps > 4) return PIC_ERR_ARG;
    if (c->g.axi) return c->fail(PIC_ERR_STATE, "the axisymmetric solve keeps its V(2,2)-cycle");
    // recorded graphs hold the old cycle
    for (int q = 0; q < 4; ++q)
        if (c->fgraph[q]) {
            cudaGraphExecDestroy(c->fgraph[q]);
            c->fgraph[q] = nullptr;
        }
    c->mg.release();
    c->mg.pre = pre_sweeps;
    c->mg.post = post_sweeps;
    return PIC_OK;
}

extern "C" int pic_profile(pic_ctx* c, int enable, pic_profile_times* out) {
    if (c) c->parts_event = false;  // work on the particle buffers may follow
    if (!c) return PIC_ERR_ARG;
    DevState h;
    const int rc = read_state(c, &h);
    if (rc) return rc;
    // kernels run inside device-side loops are counted on the device
    if (h.dev_kernels >= c->dev_kernels_seen) c->launches += (long long)(h.dev_kernels - c->dev_kernels_seen);
    c->dev_kernels_seen = h.dev_kernels;
    c->resolve_times();
    c->pt.n_launches = c->launches;
    if (out) *out = c->pt;
    memset(&c->pt, 0, sizeof c->pt);
    c->launches = 0;
    c->prof = enable ? 1 : 0;
    return PIC_OK;
}

// Host arrays 0..9 laid out at one constant pitch of at least `row` bytes
// (one host block): returns the pitch, else 0.
static size_t host_pitch(const void* const* arrays, size_t row) {
    const char* a0 = static_cast<const char*>(arrays[0]);
    if (!a0 || !arrays[1]) return 0;
    const ptrdiff_t d = static_cast<const char*>(arrays[1]) - a0;
    if (d < (ptrdiff_t)row) return 0;
    for (int f = 2; f < 10; ++f)
        if (!arrays[f] || static_cast<const char*>(arrays[f]) - a0 != (ptrdiff_t)f * d) return 0;
    return (size_t)d;
}

// The copy stream of the host exchanges that overlap a speculative solve
// (false: exchange on the context's stream).
static bool exchange_stream(pic_ctx* c) {
    if (!c->parts_event || !c->ev_parts) return false;
    if (!c->xs && cudaStreamCreateWithFlags(&c->xs, cudaStreamNonBlocking) != cudaSuccess) c->xs = nullptr;
    if (c->xs && !c->ev_up && cudaEventCreateWithFlags(&c->ev_up, cudaEventDisableTiming) != cudaSuccess)
        c->ev_up = nullptr;
    if (!c->xs || !c->ev_up) {
        cudaGetLastError();
        return false;
    }
    return cudaStreamWaitEvent(c->xs, c->ev_parts, 0) == cudaSuccess;
}

extern "C" int pic_upload(pic_ctx* c, long long n, const void* const* arrays, int accel_valid) {
    if (!c || n < 0 || (n > 0 && !arrays)) return PIC_ERR_ARG;
    if (n > c->cfg.capacity) return c->fail(PIC_ERR_CAPACITY, "more particles than capacity");
    for (int f = 0; f < 11 && n > 0; ++f)
        if (!arrays[f]) return PIC_ERR_ARG;
    // Right after a speculative step nothing enqueued since its particles
    // were final touches a particle buffer (only its field solve may still
    // run), so the copies go on the exchange stream, behind those particles
    // only, and the context's stream waits for them.
    const bool ovl = exchange_stream(c);
    c->parts_event = false;
    if (ovl) c->pt.n_overlapped++;
    cudaStream_t us = ovl ? c->xs : c->s;
    c->cur = 0;
    const size_t R = real_size(c->prec), cap = (size_t)c->cfg.capacity;
    char* base = c->ws + c->L.buf[0];
    // the ten real arrays in one pitched copy when the host keeps them in one block
    const size_t hp = n > 0 ? host_pitch(arrays, (size_t)n * R) : 0;
    if (hp) {
        cudaError_t e = cudaMemcpy2DAsync(base, al256(cap * R), arrays[0], hp, (size_t)n * R, 10,
                                          cudaMemcpyHostToDevice, us);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(base + 10 * al256(cap * R), arrays[10], (size_t)n * 8, cudaMemcpyHostToDevice, us);
        if (e != cudaSuccess) return c->cuda_fail(e, "upload");
    }
    for (int f = 0; f < 11 && n > 0 && !hp; ++f) {
        cudaError_t e = cudaMemcpyAsync(base + f * al256(cap * R), arrays[f], n * (f < 10 ? R : 8),
                                        cudaMemcpyHostToDevice, us);
        if (e != cudaSuccess) return c->cuda_fail(e, "upload");
    }
    if (ovl) {
        cudaError_t e = cudaEventRecord(c->ev_up, c->xs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->s, c->ev_up, 0);
        if (e != cudaSuccess) return c->cuda_fail(e, "upload");
    }
    k_set_count<<<1, 1, 0, c->s>>>(c->st(), (unsigned long long)n);
    c->n_host = n;
    c->n_last_wu = n;
    c->a_valid = accel_valid ? 1 : 0;
    return PIC_OK;
}

// Copies n particles of the current buffer to the host arrays on stream ds (no wait).
static cudaError_t download_async(pic_ctx* c, void* const* arrays, long long n, cudaStream_t ds) {
    const size_t R = real_size(c->prec), capd = (size_t)c->cfg.capacity;
    char* base = c->ws + c->L.buf[c->cur];
    const size_t hp = n > 0 ? host_pitch(arrays, (size_t)n * R) : 0;
    if (hp) {  // the ten real arrays in one pitched copy (one host block)
        cudaError_t e = cudaMemcpy2DAsync(arrays[0], hp, base, al256(capd * R), (size_t)n * R, 10,
                                          cudaMemcpyDeviceToHost, ds);
        if (e == cudaSuccess && arrays[10])
            e = cudaMemcpyAsync(arrays[10], base + 10 * al256(capd * R), (size_t)n * 8, cudaMemcpyDeviceToHost, ds);
        return e;
    }
    for (int f = 0; f < 11 && n > 0; ++f) {
        if (!arrays[f]) continue;
        cudaError_t e = cudaMemcpyAsync(arrays[f], base + f * al256(capd * R), n * (f < 10 ? R : 8),
                                        cudaMemcpyDeviceToHost, ds);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

extern "C" int pic_download(pic_ctx* c, void* const* arrays, long long cap, long long* n_out) {
    if (!c || !arrays) return PIC_ERR_ARG;
    long long n = c->n_host;
    const bool fits = n <= cap;
    // Right after a speculative step: its particles and count are final
    // (the count was read back before the host let the solve stand), so the
    // copy waits for them only and overlaps the solve.
    if (fits && exchange_stream(c)) {
        c->pt.n_overlapped++;
        cudaError_t e = download_async(c, arrays, n, c->xs);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->xs);
        if (e != cudaSuccess) return c->cuda_fail(e, "download");
        if (n_out) *n_out = n;
        return PIC_OK;
    }
    // The host count is known after every call that changes it; the device
    // state and the particles are copied together and checked after one wait.
    DevState h;
    cudaError_t e = cudaMemcpyAsync(&h, c->st(), sizeof(DevState), cudaMemcpyDeviceToHost, c->s);
    if (e == cudaSuccess && fits) e = download_async(c, arrays, n, c->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->s);
    if (e != cudaSuccess) return c->cuda_fail(e, "download");
    if ((long long)h.n_in != n) {  // not expected: copy again with the device count
        n = (long long)h.n_in;
        c->n_host = n;
        if (n <= cap) {
            e = download_async(c, arrays, n, c->s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->s);
            if (e != cudaSuccess) return c->cuda_fail(e, "download");
        }
    }
    if (n_out) *n_out = n;
    if (n > cap) return c->fail(PIC_ERR_CAPACITY, "host arrays too small");
    return PIC_OK;
}
