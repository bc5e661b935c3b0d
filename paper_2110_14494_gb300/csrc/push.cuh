// Electron push + null-collision Monte Carlo + fixed-point deposit kernels.
//
// Sec. 2.1.1 of the paper: electrons are advanced with velocity Verlet
// (Eqs. 1-2, a = -(e/m_e) E) and collide with the gas by the null-collision
// method at the constant trial rate nu_max, using rates tabulated from cross
// sections.  Sec. 2.1.3: the field is interpolated to the particle and the
// particle mapped to the grid with trilinear (cloud-in-cell) weights.
//
// One thread owns one electron for the whole step: gather, half-kick, the
// chain of free flights and collisions, reflection at the domain faces,
// electrode absorption, append of the survivor to the other buffer with a
// warp-aggregated cursor, and its deposit.  Ionization products are queued
// with their remaining time and finished by k_children in the same step.
// Instantiated for T = float and T = double in separate translation units.
#pragma once
#include <type_traits>

#include "common.cuh"

namespace pic {

enum { MODE_PIC = 0, MODE_SWARM = 1 };
enum { RES_NONE = 0, RES_THIN = 1, RES_DUP = 2 };

template <class T> struct PushArgs {
    Soa<T> in, out;
    ChildQ<T> cq, cq2;         // product queues: parents fill cq; children generation g reads
                               // (g even ? cq : cq2) and spills into the other one
    int gen;
    DevState* st;
    const T* table;            // [n_bins][8]: nu_0..nu_{n_proc-1}, zeros, total
    int n_bins, n_proc;
    int kind[8];
    T thr[8];                  // eV
    T mratio[8];               // m_e / M (0 = infinite mass)
    T l0, inv_dl;              // ln(eps_0), (n_bins-1) / (ln eps_last - ln eps_0), in T
    T eps_lo, eps_hi;          // eV
    T nu_max;
    T tau_scale;               // -ln 2 / nu_max: single-precision flight times from base-2 logarithms
    T inv_dl2, l0t;            // ln 2 * inv_dl and l0 * inv_dl: table coordinate from a base-2 logarithm
    T dt;                      // duration of this step
    T dt_kick;                 // duration of the previous step (the half-kick completes its Eq. 2)
    Keys K;
    uint32_t step;
    int first;                 // previous acceleration unknown: no half-kick
    int kick_on_load;          // parents get the gather and half-kick when the collision kernel loads them
    long long cap_out, cap_child;
    // grid (PIC mode)
    int nx, ny, nz;
    T ox, oy, oz, dxr, hx, hy, hz;  // origin, cell size, upper faces
    const T* E4;               // [ncell][4] packed cell-centred field or nullptr (uniform)
    T E0[3];
    const uint8_t* mask;
    unsigned long long *q_e, *q_pos, *q_neg;
    unsigned int* vhist;  // speed histogram of the stored electrons (adaptive time step), or null
    int boundary;
    int axi;                   // axisymmetric grid (see grid_pt)
    // photoionization (Sec. 2.4): emission probability per ionization, the
    // absorption coefficient range [chi_a, chi_a e^chi_log] (1/m), and the
    // queue of photoelectrons appended after the step
    T photo_prob, chi_a, chi_log;
    T *pe_x, *pe_y, *pe_z, *pe_w;   // emitted photons: origin and weight
    uint64_t* pe_id;                // emitting electron and draw index
    uint32_t* pe_k;
    T *ph_x, *ph_y, *ph_z, *ph_w;   // photoelectrons
    uint64_t* ph_id;
    long long cap_photo;
    // swarm mode
    double* mom;               // [kNMom] accumulators of this step
    long long n_lo, n_hi;
};

// Per-process constants, staged in shared memory after the rate table so the
// process index can address them without a local-memory copy of the
// kernel parameters.
template <class T> struct ProcSmem {
    T thr[8];
    T mratio[8];
    int kind[8];
};

// ------------------------------------------------------------------ arithmetic
// Double precision follows the oracle's operation order (no FMA contraction in
// that translation unit); single precision uses precomputed factors.
template <class T> struct Arith;
template <> struct Arith<double> {
    static __device__ __forceinline__ double energy(double v2) { return 0.5 * kMe * v2 / kQ; }
    static __device__ __forceinline__ double speed(double e) { return sqrt(2.0 * kQ * e / kMe); }
    static __device__ __forceinline__ double lg(double u) { return log(u); }
    static __device__ __forceinline__ double tau(double u0, double nu_max) { return -log(u0) / nu_max; }
    static __device__ __forceinline__ void sc2pi(double u, double* s, double* c) { sincospi(2.0 * u, s, c); }
};
template <> struct Arith<float> {
    static __device__ __forceinline__ float energy(float v2) { return (float)(0.5 * kMe / kQ) * v2; }
    static __device__ __forceinline__ float speed(float e) { return sqrtf((float)(2.0 * kQ / kMe) * e); }
    static __device__ __forceinline__ float lg(float u) { return logf(u); }
    static __device__ __forceinline__ float tau(float u0, float nu_max) { return -logf(u0) / nu_max; }
    static __device__ __forceinline__ void sc2pi(float u, float* s, float* c) { sincospif(2.0f * u, s, c); }
};

template <class T> __device__ __forceinline__ void iso_dir(T u2, T u3, T n[3]) {
    T ct = (T)1 - (T)2 * u2;
    T st = sqrt(dmax((T)0, (T)1 - ct * ct));
    T s, c;
    Arith<T>::sc2pi(u3, &s, &c);
    n[0] = st * c;
    n[1] = st * s;
    n[2] = ct;
}

template <class T> __device__ __forceinline__ void fly(T x[3], T v[3], const T a[3], T tau) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        x[d] = x[d] + tau * (v[d] + (T)0.5 * tau * a[d]);
        v[d] = v[d] + tau * a[d];
    }
}

// ---------------------------------------------------------------- per-thread stats
struct LStats {
    unsigned long long events, nulls, clamped, absorbed, attached, children, processed;
    unsigned long long coll[8];
    double w_ion, w_att, w_abs;
    __device__ void zero() {
        events = nulls = clamped = absorbed = attached = children = processed = 0;
        for (int k = 0; k < 8; ++k) coll[k] = 0;
        w_ion = w_att = w_abs = 0.0;
    }
};

template <class T> struct MomAcc {
    double m[kNMom];
    __device__ void zero() {
        for (int q = 0; q < kNMom; ++q) m[q] = 0.0;
    }
    __device__ void add(const T x[3], const T v[3], T wt) {
        double w = wt, X = x[0], Y = x[1], Z = x[2], U = v[0], V = v[1], W = v[2];
        m[0] += w; m[1] += w * X; m[2] += w * Y; m[3] += w * Z;
        m[4] += w * X * X; m[5] += w * Y * Y; m[6] += w * Z * Z;
        m[7] += w * U; m[8] += w * V; m[9] += w * W;
        m[10] += w * X * U; m[11] += w * Y * V; m[12] += w * Z * W;
        m[13] += w * (0.5 * kMe * (U * U + V * V + W * W) / kQ);
    }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}
__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Flushes per-thread statistics (all threads of the block must call).
template <class T>
__device__ void flush_stats(const PushArgs<T>& A, LStats& s, int n_proc) {
    unsigned long long e = warp_sum(s.events), nn = warp_sum(s.nulls), cl = warp_sum(s.clamped);
    unsigned long long ab = warp_sum(s.absorbed), at = warp_sum(s.attached), ch = warp_sum(s.children);
    unsigned long long pr = warp_sum(s.processed);
    double wi = warp_sum(s.w_ion), wa = warp_sum(s.w_att), wb = warp_sum(s.w_abs);
    unsigned long long co[8];
    for (int k = 0; k < 8; ++k) co[k] = warp_sum(s.coll[k]);
    if ((threadIdx.x & 31) == 0) {
        DevState* st = A.st;
        if (e) atomicAdd(&st->n_events, e);
        if (nn) atomicAdd(&st->n_null, nn);
        if (cl) atomicAdd(&st->n_clamped, cl);
        if (ab) atomicAdd(&st->n_absorbed, ab);
        if (at) atomicAdd(&st->n_attached, at);
        if (ch) atomicAdd(&st->n_children, ch);
        if (pr) atomicAdd(&st->n_processed, pr);
        for (int k = 0; k < n_proc && k < 8; ++k)
            if (co[k]) atomicAdd(&st->n_coll[k], co[k]);
        if (wi != 0.0) atomicAdd(&st->w_ion, wi);
        if (wa != 0.0) atomicAdd(&st->w_att, wa);
        if (wb != 0.0) atomicAdd(&st->w_absorbed, wb);
    }
}

template <class T>
__device__ void flush_moments(const PushArgs<T>& A, MomAcc<T>& M, double* red /* smem [kNMom][32] */) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int q = 0; q < kNMom; ++q) {
        double v = warp_sum(M.m[q]);
        if (lane == 0) red[q * 32 + wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < kNMom) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += red[threadIdx.x * 32 + w];
        if (s != 0.0) atomicAdd(&A.mom[threadIdx.x], s);
    }
}

// ------------------------------------------------------------------ gather
template <class T>
__device__ __forceinline__ void axis_w(T x, T o, T dx, int n, int& i0, int& i1, T& f) {
    T s = (x - o) / dx - (T)0.5;
    if (s < (T)0) s = (T)0;
    if (s > (T)(n - 1)) s = (T)(n - 1);
    int i = (int)floor(s);
    if (i > n - 2) i = n - 2;
    if (i < 0) i = 0;
    i0 = i;
    i1 = i + 1;
    f = s - (T)i;
}

template <class T> struct Ld4;
template <> struct Ld4<float> {
    static __device__ __forceinline__ void get(const float* p, float e[3]) {
        float4 v = __ldg(reinterpret_cast<const float4*>(p));
        e[0] = v.x; e[1] = v.y; e[2] = v.z;
    }
};
template <> struct Ld4<double> {
    static __device__ __forceinline__ void get(const double* p, double e[3]) {
        double2 a = __ldg(reinterpret_cast<const double2*>(p));
        double b = __ldg(p + 2);
        e[0] = a.x; e[1] = a.y; e[2] = b;
    }
};

// Point of the grid that a particle position maps to.  Cartesian grids: the
// position itself.  Axisymmetric grids (Sec. 2.1.1: particles move in 3D,
// the field and densities live on an (r, z) mesh): (r, centre of the single
// y cell, z) with r = sqrt(x^2 + y^2), so cell indices, deposits and masks of
// the Cartesian code address the ring cell (i_r, 0, k).
template <class T> __device__ __forceinline__ void grid_pt(const PushArgs<T>& A, const T x[3], T g[3]) {
    if (A.axi) {
        g[0] = sqrt(x[0] * x[0] + x[1] * x[1]);
        g[1] = A.oy + (T)0.5 * A.dxr;
        g[2] = x[2];
    } else {
        g[0] = x[0]; g[1] = x[1]; g[2] = x[2];
    }
}

// Axisymmetric gather: E_r and E_z bilinear in (r, z) at cell centres
// (packed as (E_r, 0, E_z)), projected on x and y: E = (E_r x / r, E_r y / r,
// E_z) (Sec. 2.1.1), zero radial part on the axis.
template <class T>
__device__ __forceinline__ void gather_axi(const PushArgs<T>& A, const T x[3], T E[3]) {
    const T r = sqrt(x[0] * x[0] + x[1] * x[1]);
    int ir[2], iz[2];
    T fr, fz;
    axis_w(r, A.ox, A.dxr, A.nx, ir[0], ir[1], fr);
    axis_w(x[2], A.oz, A.dxr, A.nz, iz[0], iz[1], fz);
    const T gr[2] = {(T)1 - fr, fr}, gz[2] = {(T)1 - fz, fz};
    T er = (T)0, ez = (T)0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int dz = c >> 1, dr = c & 1;
        const long long idx = (long long)iz[dz] * A.nx + ir[dr];
        T e[3];
        Ld4<T>::get(A.E4 + 4 * idx, e);
        const T g = gz[dz] * gr[dr];
        er += g * e[0];
        ez += g * e[2];
    }
    const T inv = r > (T)0 ? er / r : (T)0;
    E[0] = inv * x[0];
    E[1] = inv * x[1];
    E[2] = ez;
}

template <class T>
__device__ __forceinline__ void gather(const PushArgs<T>& A, const T x[3], T E[3]) {
    if (A.E4 == nullptr) { E[0] = A.E0[0]; E[1] = A.E0[1]; E[2] = A.E0[2]; return; }
    if (A.axi) { gather_axi(A, x, E); return; }
    int ix[2], iy[2], iz[2];
    T fx, fy, fz;
    axis_w(x[0], A.ox, A.dxr, A.nx, ix[0], ix[1], fx);
    axis_w(x[1], A.oy, A.dxr, A.ny, iy[0], iy[1], fy);
    axis_w(x[2], A.oz, A.dxr, A.nz, iz[0], iz[1], fz);
    const T gx[2] = {(T)1 - fx, fx}, gy[2] = {(T)1 - fy, fy}, gz[2] = {(T)1 - fz, fz};
    T acc[3] = {(T)0, (T)0, (T)0};
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int dz = c >> 2, dy = (c >> 1) & 1, dxx = c & 1;
        const long long idx = ((long long)iz[dz] * A.ny + iy[dy]) * A.nx + ix[dxx];
        T e[3];
        Ld4<T>::get(A.E4 + 4 * idx, e);
        const T g = (gz[dz] * gy[dy]) * gx[dxx];
#pragma unroll
        for (int d = 0; d < 3; ++d) acc[d] += g * e[d];
    }
    E[0] = acc[0]; E[1] = acc[1]; E[2] = acc[2];
}

// ------------------------------------------------------------------ deposit
// Fixed-point cloud-in-cell: S = 2^32 per unit weight; corners 0..6 rounded to
// nearest even, corner 7 the remainder, so each particle adds exactly
// rint(w S).  Products are separately rounded (explicit _rn intrinsics).
__device__ __forceinline__ long long rint_ll(float v) { return __float2ll_rn(v); }
__device__ __forceinline__ long long rint_ll(double v) { return __double2ll_rn(v); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float div_rn(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double div_rn(double a, double b) { return __ddiv_rn(a, b); }

template <class T>
__device__ __forceinline__ void deposit(const T x, const T y, const T z, const T w, T ox, T oy, T oz, T dx, int nx,
                                        int ny, int nz, unsigned long long* q, DevState* st) {
    const T sx = sub_rn(div_rn(sub_rn(x, ox), dx), (T)0.5);
    const T sy = sub_rn(div_rn(sub_rn(y, oy), dx), (T)0.5);
    const T sz = sub_rn(div_rn(sub_rn(z, oz), dx), (T)0.5);
    const T flx = floor(sx), fly = floor(sy), flz = floor(sz);
    const T fx = sub_rn(sx, flx), fy = sub_rn(sy, fly), fz = sub_rn(sz, flz);
    const int i0 = (int)flx, j0 = (int)fly, k0 = (int)flz;
    const T gx[2] = {sub_rn((T)1, fx), fx}, gy[2] = {sub_rn((T)1, fy), fy}, gz[2] = {sub_rn((T)1, fz), fz};
    const T wS = mul_rn(w, (T)4294967296.0);
    if (!(wS < (T)4.0e18)) { atomicOr(&st->err, kErrOverflow); return; }
    long long sum = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int dz = c >> 2, dy = (c >> 1) & 1, dxx = c & 1;
        long long qc;
        if (c < 7) {
            qc = rint_ll(mul_rn(mul_rn(mul_rn(wS, gz[dz]), gy[dy]), gx[dxx]));
            sum += qc;
        } else {
            qc = rint_ll(wS) - sum;
        }
        const int ii = fold_idx(i0 + dxx, nx), jj = fold_idx(j0 + dy, ny), kk = fold_idx(k0 + dz, nz);
        if (qc != 0) atomicAdd(q + (((long long)kk * ny + jj) * nx + ii), (unsigned long long)qc);
    }
}

// Deposit of weight w at particle position x (through grid_pt).
template <class T>
__device__ __forceinline__ void deposit_at(const PushArgs<T>& A, T x0, T x1, T x2, T w, unsigned long long* q) {
    const T x[3] = {x0, x1, x2};
    T g[3];
    grid_pt(A, x, g);
    deposit(g[0], g[1], g[2], w, A.ox, A.oy, A.oz, A.dxr, A.nx, A.ny, A.nz, q, A.st);
}

// ------------------------------------------------------------------ rates
// Arithmetic of one candidate collision.  Double precision follows the
// oracle's operations.  Single precision takes the hardware base-2 logarithm
// (absolute error near 1e-7) and multiplies by precomputed constants instead
// of dividing: a flight time then carries an absolute error near 1e-7 / nu_max
// (far below a cell crossing), a table coordinate one near 1e-5 of a bin, and
// the scattering cosine a reciprocal square root.
// The collision rates a candidate event is tested against: the table
// ([n_bins][8]: the rates, zeros, their total), its maximum total nu_max and
// -ln 2 / nu_max.  One gas for a PIC context; batched swarms of different
// compositions each have their own.
template <class T> struct Rates {
    const T* tab;
    T nu_max, tau_scale;
};

template <class T> struct EvArith;
template <> struct EvArith<double> {
    static __device__ __forceinline__ double flight(const Rates<double>& R, double u0) {
        return -log(u0) / R.nu_max;
    }
    static __device__ __forceinline__ double coord(const PushArgs<double>& A, double e) {
        return (log(e) - A.l0) * A.inv_dl;
    }
    static __device__ __forceinline__ double cosine(double dot, double v2) {
        const double sp = sqrt(v2);
        return sp > 0.0 ? dot / sp : 0.0;
    }
};
template <> struct EvArith<float> {
    static __device__ __forceinline__ float flight(const Rates<float>& R, float u0) {
        return __log2f(u0) * R.tau_scale;
    }
    static __device__ __forceinline__ float coord(const PushArgs<float>& A, float e) {
        return fmaf(__log2f(e), A.inv_dl2, -A.l0t);
    }
    static __device__ __forceinline__ float cosine(float dot, float v2) { return v2 > 0.0f ? dot * rsqrtf(v2) : 0.0f; }
};

// Index and fraction in the table, linear in ln(eps), clamped at both ends.
template <class T>
__device__ __forceinline__ void table_pos(const PushArgs<T>& A, T e, int& j, T& f, LStats& ls) {
    if (e <= A.eps_lo) {
        j = 0; f = (T)0;
        if (e < A.eps_lo) ++ls.clamped;
    } else if (e >= A.eps_hi) {
        j = A.n_bins - 2; f = (T)1;
        if (e > A.eps_hi) ++ls.clamped;
    } else {
        T t = EvArith<T>::coord(A, e);
        int jj = (int)floor(t);
        if (jj > A.n_bins - 2) jj = A.n_bins - 2;
        if (jj < 0) jj = 0;
        j = jj;
        f = t - (T)jj;
    }
}

// Chooses the process for a candidate collision: the smallest k with
// u1 nu_max < sum_{i<=k} nu_i(eps); -1 = null collision.
template <class T, bool FAST>
__device__ __forceinline__ int select_process(const PushArgs<T>& A, const Rates<T>& R, T e, T u1, LStats& ls) {
    int j;
    T f;
    table_pos(A, e, j, f, ls);
    const T* r0 = R.tab + j * kTableStride;
    const T* r1 = r0 + kTableStride;
    const T target = u1 * R.nu_max;
    if (FAST) {
        const T t0 = __ldg(r0 + 7), t1 = __ldg(r1 + 7);
        const T tot = t0 + f * (t1 - t0);
        if (target >= tot) return -1;
    }
    // the first k with target < sum_{i<=k} nu_i: every process is visited by
    // every lane (the same sums in the same order), so the lanes of a warp
    // stay together whichever process they pick
    T cum = (T)0;
    int sel = -1;
#pragma unroll
    for (int k = 0; k < kTableStride - 1; ++k) {
        if (k < A.n_proc) {
            const T a = __ldg(r0 + k), b = __ldg(r1 + k);
            cum += a + f * (b - a);
            sel = (sel < 0 && target < cum) ? k : sel;
        }
    }
    return sel;
}

// ------------------------------------------------------------------ flight
// The product of an ionization by draw k of electron `pid`: id from the
// derived-id stream, isotropic direction from its own draw k = 0, speed sp.
template <class T>
__device__ __forceinline__ uint64_t make_child(const Keys& K, uint32_t step, uint64_t pid, uint32_t k, T sp, T vc[3]) {
    const uint64_t cid = derived_id(K, pid, step, 0x80000000u | k);
    const u32x4 rb = draw_words(K, cid, step, 0u);
    T nb[3];
    iso_dir(unif<T>(rb.z), unif<T>(rb.w), nb);
    vc[0] = sp * nb[0]; vc[1] = sp * nb[1]; vc[2] = sp * nb[2];
    return cid;
}

// Products of products (rare) are built at once and wait on the lane's stack.
template <class T> struct StackSink {
    static constexpr int kDepth = 8;
    T x[kDepth][3], v[kDepth][3], w[kDepth], t[kDepth];
    uint64_t id[kDepth];
    int n = 0;
};

// One electron in flight on a lane: start position x, displacement d within
// the step (x + d is the position; single precision keeps the resolution of
// the short flights that way), velocity, acceleration, weight, remaining time
// and the index k of its next draw.
template <class T> struct Lane {
    T x[3], d[3], v[3], a[3];
    T w, t_left;
    uint64_t id;
    uint32_t k;
};

enum { EV_CONTINUE = 0, EV_DONE = 1, EV_ATTACHED = 2, EV_IONIZED = 3 };

// Electrode mask of the cell containing x (cell index by correctly rounded
// (x - origin) / dx, folded into the grid).
template <class T> __device__ __forceinline__ bool masked_at(const PushArgs<T>& A, const T xp[3]) {
    T x[3];
    grid_pt(A, xp, x);
    const int i = fold_idx((int)floor(div_rn(sub_rn(x[0], A.ox), A.dxr)), A.nx);
    const int j = fold_idx((int)floor(div_rn(sub_rn(x[1], A.oy), A.dxr)), A.ny);
    const int k = fold_idx((int)floor(div_rn(sub_rn(x[2], A.oz), A.dxr)), A.nz);
    return A.mask[((long long)k * A.ny + j) * A.nx + i] != 0;
}

// Photon of an ionization event (Sec. 2.4, discrete Monte Carlo model), in
// two parts.  In the collision loop only the emission test: draw (id, step,
// 0xD0000000 | k) of the event's draw index k, u0 < photo_prob emits one
// photon of the electron's weight; an emitted photon's origin (position,
// weight, id, k) goes to a queue.  After each launch k_photo_resolve draws
// its path: the absorption coefficient chi log-uniform on [a, b] (u1) and an
// exponential path with rate chi (u2).  This mixture has exactly Zheleznyak's
// absorption density: f(r) = (e^-ar - e^-br) / (r ln(b/a)) = integral over
// chi in [a, b] of [1 / (chi ln(b/a))] chi e^(-chi r).  Direction: cos(theta)
// = 1 - 2 u3 and azimuth 2 pi u0' of draw (id, step, 0xE0000000 | k).  A
// photon absorbed inside the domain and outside the electrode records a
// positive ion there and queues a photoelectron (id derived with tag
// 0xD0000000 | k).
template <class T>
__device__ __forceinline__ void photo_test(const PushArgs<T>& A, const Keys& K, uint32_t step, uint64_t id,
                                           uint32_t k, const T x[3], T w) {
    const u32x4 r = draw_words(K, id, step, 0xD0000000u | k);
    if (!(unif<T>(r.x) < A.photo_prob)) return;
    const unsigned long long slot = atomicAdd(&A.st->n_photo_src, 1ull);
    if ((long long)slot >= A.cap_photo) {
        atomicOr(&A.st->err, kErrPhotoCapacity);
        return;
    }
    A.pe_x[slot] = x[0];
    A.pe_y[slot] = x[1];
    A.pe_z[slot] = x[2];
    A.pe_w[slot] = w;
    A.pe_id[slot] = id;
    A.pe_k[slot] = k;
}

// One candidate collision of the null-collision method (Sec. 2.1.1): flight
// time tau = -ln(u0) / nu_max; if it ends the step, fly to the end; else fly
// tau, pick the process with u1 nu_max against the cumulative rates at the
// electron's energy (none = null collision) and scatter isotropically with
// u2, u3.  Ionization returns EV_IONIZED with the product's speed in sp (the
// caller queues the product, which flies the remaining time, and its
// positive-ion event); attachment returns EV_ATTACHED (the caller records the
// negative-ion event at the electron's position) and ends the electron.
template <class T, int MODE, bool FAST, bool STATS>
__device__ __forceinline__ int event(const PushArgs<T>& A, const Rates<T>& R, const Keys& K, uint32_t step,
                                     const ProcSmem<T>* ps, Lane<T>& L, LStats& ls, T& sp) {
    const u32x4 r = draw_words(K, L.id, step, L.k);
    ++L.k;
    const T tau = EvArith<T>::flight(R, unif<T>(r.x));
    if (tau >= L.t_left) { fly(L.d, L.v, L.a, L.t_left); return EV_DONE; }
    fly(L.d, L.v, L.a, tau);
    L.t_left -= tau;
    ++ls.events;
    T* v = L.v;
    const T v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    const T e = Arith<T>::energy(v2);
    const int p = select_process<T, FAST>(A, R, e, unif<T>(r.y), ls);
    if (p < 0) { ++ls.nulls; return EV_CONTINUE; }
    if (STATS) ++ls.coll[p & 7];
    const int kind = ps->kind[p];
    if (kind == PIC_PROC_ATTACHMENT) {
        if (MODE == MODE_SWARM || STATS) ls.w_att += (double)L.w;
        ++ls.attached;
        return EV_ATTACHED;
    }
    T n[3];
    iso_dir(unif<T>(r.z), unif<T>(r.w), n);
    // energy after the collision: elastic recoil with cos(chi) = n_old . n_new,
    // excitation loss, or half of what ionization leaves (all three formed,
    // one kept: no branch on the process kind)
    const T cchi = EvArith<T>::cosine(v[0] * n[0] + v[1] * n[1] + v[2] * n[2], v2);
    const T e_el = dmax(e * ((T)1 - (T)2 * ps->mratio[p] * ((T)1 - cchi)), (T)0);
    const T e_in = dmax(e - ps->thr[p], (T)0);
    const T e2 = kind == PIC_PROC_ELASTIC ? e_el : (kind == PIC_PROC_EXCITATION ? e_in : (T)0.5 * e_in);
    const T sp2 = Arith<T>::speed(e2);
    v[0] = sp2 * n[0]; v[1] = sp2 * n[1]; v[2] = sp2 * n[2];
    if (kind == PIC_PROC_IONIZATION) {
        sp = sp2;
        if (MODE == MODE_SWARM || STATS) ls.w_ion += (double)L.w;
        return EV_IONIZED;
    }
    return EV_CONTINUE;
}

// Domain faces (specular reflection or absorption) and electrode cells.
template <class T>
__device__ __forceinline__ bool boundaries(const PushArgs<T>& A, T x[3], T v[3], T w, LStats& ls) {
    const T lo[3] = {A.ox, A.oy, A.oz}, hi[3] = {A.hx, A.hy, A.hz};
    bool out = false;
    if (A.axi) {
        // the cylinder r = R of an axisymmetric grid: outflow, or specular
        // reflection (r -> 2R - r, radial velocity reversed)
        const T R = A.hx;
        T r = sqrt(x[0] * x[0] + x[1] * x[1]);
        if (A.boundary == 1) {
            if (r > R) out = true;
        } else {
            for (int it = 0; it < 8 && r > R; ++it) {
                const T rn = (T)2 * R - r, s = rn / r;
                const T ux = x[0] / r, uy = x[1] / r;
                const T vr = v[0] * ux + v[1] * uy;
                x[0] *= s;
                x[1] *= s;
                v[0] -= (T)2 * vr * ux;
                v[1] -= (T)2 * vr * uy;
                r = fabs(rn);
            }
        }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (A.axi && d < 2) continue;
        if (A.boundary == 1) {
            if (x[d] < lo[d] || x[d] > hi[d]) out = true;
            continue;
        }
        for (int it = 0; it < 8 && (x[d] < lo[d] || x[d] > hi[d]); ++it) {
            if (x[d] < lo[d]) x[d] = (T)2 * lo[d] - x[d];
            else x[d] = (T)2 * hi[d] - x[d];
            v[d] = -v[d];
        }
        if (x[d] < lo[d]) x[d] = lo[d];
        if (x[d] > hi[d]) x[d] = hi[d];
    }
    if (!out && A.mask && masked_at(A, x)) out = true;
    if (out) { ++ls.absorbed; ls.w_abs += (double)w; }
    return !out;
}

template <class T>
__device__ __forceinline__ void store(const Soa<T>& o, unsigned long long s, const T x[3], const T v[3], const T a[3],
                                      T w, uint64_t id) {
    o.r[PX][s] = x[0]; o.r[PY][s] = x[1]; o.r[PZ][s] = x[2];
    o.r[VX][s] = v[0]; o.r[VY][s] = v[1]; o.r[VZ][s] = v[2];
    o.r[AX][s] = a[0]; o.r[AY][s] = a[1]; o.r[AZ][s] = a[2];
    o.r[PW][s] = w; o.id[s] = id;
}

// ------------------------------------------------------------------ field kick
// Sec. 2.1.1, Eq. 2: a_new = -(e/m_e) E(x) from the trilinear gather; the
// half-kick v += dt/2 (a_new - a_old) completes the previous step's velocity
// update (skipped when a_old is unknown); a_old <- a_new.  A streaming pass in
// place over the input buffer, so the collision kernel starts electrons
// without a dependent gather.
template <class T>
__global__ void __launch_bounds__(256) k_field_kick(const PushArgs<T> A) {
    const long long n = (long long)A.st->n_in;
    const T qm = (T)(kQ / kMe);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const T x[3] = {A.in.r[PX][i], A.in.r[PY][i], A.in.r[PZ][i]};
        T E[3];
        gather(A, x, E);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const T an = -qm * E[d];
            if (!A.first) A.in.r[VX + d][i] = A.in.r[VX + d][i] + (T)0.5 * A.dt_kick * (an - A.in.r[AX + d][i]);
            A.in.r[AX + d][i] = an;
        }
    }
}

// The same half-kick for one loaded electron (f = x y z vx vy vz ax ay az w),
// done by the collision kernel as it stages its parents.
template <class T> __device__ __forceinline__ void half_kick(const PushArgs<T>& A, T f[10]) {
    const T qm = (T)(kQ / kMe);
    T E[3];
    gather(A, f, E);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const T an = -qm * E[d];
        if (!A.first) f[VX + d] = f[VX + d] + (T)0.5 * A.dt_kick * (an - f[AX + d]);
        f[AX + d] = an;
    }
}

// Path of every photon emitted in the launch before (see photo_test): the
// absorbed ones inside the gas deposit their ion and queue a photoelectron.
template <class T>
__global__ void __launch_bounds__(256) k_photo_resolve(const PushArgs<T> A) {
    const unsigned long long nq = A.st->n_photo_src;
    const long long n = (long long)nq < A.cap_photo ? (long long)nq : A.cap_photo;
    const uint32_t step = A.step;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const uint64_t id = A.pe_id[i];
        const uint32_t k = A.pe_k[i];
        const T w = A.pe_w[i];
        const u32x4 r = draw_words(A.K, id, step, 0xD0000000u | k);
        const T chi = A.chi_a * exp(unif<T>(r.y) * A.chi_log);
        const T dist = -log(unif<T>(r.z)) / chi;
        const u32x4 r2 = draw_words(A.K, id, step, 0xE0000000u | k);
        T n3[3];
        iso_dir(unif<T>(r.w), unif<T>(r2.x), n3);
        const T xp[3] = {A.pe_x[i] + dist * n3[0], A.pe_y[i] + dist * n3[1], A.pe_z[i] + dist * n3[2]};
            const T lo[3] = {A.ox, A.oy, A.oz}, hi[3] = {A.hx, A.hy, A.hz};
        bool in = true;
        for (int d = A.axi ? 2 : 0; d < 3; ++d)
            if (!(xp[d] >= lo[d] && xp[d] <= hi[d])) in = false;
        if (A.axi && !(sqrt(xp[0] * xp[0] + xp[1] * xp[1]) <= A.hx)) in = false;
        if (!in || (A.mask && masked_at(A, xp))) continue;
        if (A.q_pos) deposit_at(A, xp[0], xp[1], xp[2], w, A.q_pos);
        const unsigned long long slot = atomicAdd(&A.st->n_photo, 1ull);
        if ((long long)slot >= A.cap_photo) {
            atomicOr(&A.st->err, kErrPhotoCapacity);
            continue;
        }
        A.ph_x[slot] = xp[0];
        A.ph_y[slot] = xp[1];
        A.ph_z[slot] = xp[2];
        A.ph_w[slot] = w;
        A.ph_id[slot] = derived_id(A.K, id, step, 0xD0000000u | k);
    }
}

// Photoelectrons queued by k_photo_resolve join the output buffer at rest, with
// the acceleration of the field at their position (so the next step's
// half-kick adds nothing they did not experience), and their charge is
// deposited with the electrons of the step.
template <class T>
__global__ void __launch_bounds__(256) k_photo_append(const PushArgs<T> A) {
    const unsigned long long nq = A.st->n_photo;
    const long long n = (long long)nq < A.cap_photo ? (long long)nq : A.cap_photo;
    const T qm = (T)(kQ / kMe);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const T x[3] = {A.ph_x[i], A.ph_y[i], A.ph_z[i]};
        const T w = A.ph_w[i];
        T E[3];
        gather(A, x, E);
        const T v[3] = {(T)0, (T)0, (T)0};
        const T a[3] = {-qm * E[0], -qm * E[1], -qm * E[2]};
        const unsigned long long slot = atomicAdd(&A.st->n_out, 1ull);
        if ((long long)slot >= A.cap_out) {
            atomicOr(&A.st->err, kErrOutCapacity);
            continue;
        }
        store(A.out, slot, x, v, a, w, A.ph_id[i]);
        if (A.q_e) deposit_at(A, x[0], x[1], x[2], w, A.q_e);
        if (A.vhist && w > (T)0) atomicAdd(&A.vhist[0], 1u);  // at rest: the lowest speed bin
    }
}

// Closes the photoelectron queue of the launch before.
static __global__ void k_photo_done(DevState* st, long long cap) {
    const unsigned long long n = st->n_photo;
    st->n_photons += n < (unsigned long long)cap ? n : (unsigned long long)cap;
    st->n_photo = 0;
    st->n_photo_src = 0;
}

// Swarm resampling in place (decided from the count after the previous step):
// above n_hi each electron survives with probability 1/2 (draw keyed by id,
// step and 0xA0000000), the others get weight 0; below n_lo every electron
// gets a copy with a derived id, appended after the last one.  Weights are
// not rescaled: the coefficients are ratios of moments of the same step.
template <class T>
__global__ void k_resample(const PushArgs<T> A) {
    const long long n = (long long)A.st->n_in;
    const bool thin = n > A.n_hi, dup = n > 0 && n < A.n_lo;
    if (!thin && !dup) return;
    if (dup && 2 * n > A.cap_out) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&A.st->err, kErrOutCapacity);
        return;
    }
    const Soa<T>& p = A.in;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (thin) {
            const u32x4 r = draw_words(A.K, p.id[i], A.step, 0xA0000000u);
            if (!(unif<T>(r.x) < (T)0.5)) p.r[PW][i] = (T)0;
        } else {
            const long long j = n + i;
            for (int f = 0; f < 10; ++f) p.r[f][j] = p.r[f][i];
            p.id[j] = derived_id(A.K, p.id[i], A.step, 0xA0000000u);
        }
    }
    if (dup && blockIdx.x == 0 && threadIdx.x == 0) A.st->n_extra = (unsigned long long)(2 * n);
}

static __global__ void k_resample_commit(DevState* st) {
    if (st->n_extra) {
        st->n_in = st->n_extra;
        st->n_extra = 0;
    }
}

// ------------------------------------------------------------------ collisions
// Lanes refill from per-warp shared-memory stages.  Every lane owns one
// electron at a time and advances it by up to two candidate collisions per
// loop iteration; a lane whose electron has finished the step takes the next
// electron from the warp's input stage at once, so the warp stays converged
// while electrons need different numbers of events.  All per-electron memory
// work is done by the whole warp, 32 electrons at a time: the input stage is
// filled with one coalesced load of 32 consecutive work items, finished
// electrons wait in the output stage until 32 are there and are then
// reflected at the faces, tested against the electrode, appended with one
// cursor increment, stored and deposited by 32 lanes together.  An
// ionization product is built at once (derived id, direction from its own
// draw, positive-ion event of its birth) and pushed on the lane's stack;
// the lane finishes its stack before it takes the next work item, flying
// each product for the remaining time with the acceleration of the electron
// the stack started from.  A product that finds the stack full waits, as a
// compact entry, in the queue of the next (children) launch.
//
// CHILD = false: work item = one electron of the input buffer (already kicked
// by k_field_kick), flying dt.  CHILD = true: work item = one queued
// ionization product, built when it is staged.
constexpr int kRow = 11;    // padded row of a stage entry: x y z vx vy vz ax ay az w t
constexpr int kOut = 64;    // output stage capacity (flushed at 32)
constexpr int kCh = 64;     // product stage capacity of the batched swarm kernel (flushed at 32)
constexpr int kPQ = 40;     // warp queue of ionization products (built 32 at a time)
constexpr int kPQRow = 9;   // x y z, product speed, ax ay az of the ionizing electron, w, remaining time
constexpr int kAtt = 32;    // warp buffer of attachment events awaiting their deposit

template <class T> struct Stage {
    T in[32 * kRow];
    T out[kOut * kRow];
    uint64_t in_id[32], out_id[kOut];
    T pq[kPQ * kPQRow];
    uint64_t pq_id[kPQ];    // the ionizing electron
    uint32_t pq_k[kPQ];     // index of its draw that ionized
    T att[kAtt * 4];        // x y z w of negative-ion events
};

template <class T> constexpr size_t collide_smem() {
    return ((sizeof(ProcSmem<T>) + 15) & ~(size_t)15) + 4 * sizeof(Stage<T>);
}

// Writes staged finished electrons [0, cnt) (lane l takes entry l): faces,
// electrode, output append, deposit or moments; then moves entries cnt..n-1 down.
template <class T, int MODE>
__device__ __forceinline__ void flush_out(const PushArgs<T>& A, Stage<T>* sg, int& n, int cnt, LStats& ls,
                                          MomAcc<T>& M) {
    const int lane = threadIdx.x & 31;
    __syncwarp();
    bool live = lane < cnt;
    T x[3], v[3], a[3], w = (T)0;
    uint64_t id = 0;
    if (live) {
        const T* r = sg->out + lane * kRow;
        x[0] = r[0]; x[1] = r[1]; x[2] = r[2];
        v[0] = r[3]; v[1] = r[4]; v[2] = r[5];
        a[0] = r[6]; a[1] = r[7]; a[2] = r[8];
        w = r[9];
        id = sg->out_id[lane];
        if (MODE == MODE_PIC) live = boundaries(A, x, v, w, ls);
    }
    const unsigned m = __ballot_sync(kFull, live);
    if (m) {
        unsigned long long s0 = 0;
        if (lane == 0) s0 = atomicAdd(&A.st->n_out, (unsigned long long)__popc(m));
        s0 = __shfl_sync(kFull, s0, 0);
        bool stored = false;
        if (live) {
            const unsigned long long slot = s0 + __popc(m & ((1u << lane) - 1u));
            if ((long long)slot < A.cap_out) {
                store(A.out, slot, x, v, a, w, id);
                stored = true;
                if (MODE == MODE_PIC) {
                    if (A.q_e) deposit_at(A, x[0], x[1], x[2], w, A.q_e);
                } else {
                    M.add(x, v, w);
                }
            } else {
                atomicOr(&A.st->err, kErrOutCapacity);
            }
        }
        if (MODE == MODE_PIC && A.vhist) {
            // the speed histogram of the time-step control (Sec. 2.1.4) over the stored electrons; lanes
            // with the same bin add once
            const int b = stored && w > (T)0 ? speed_bin((float)v[0], (float)v[1], (float)v[2]) : -1;
            const unsigned grp = __match_any_sync(kFull, b);
            if (b >= 0 && __ffs(grp) - 1 == lane) atomicAdd(&A.vhist[b], (unsigned)__popc(grp));
        }
    }
    __syncwarp();
    const int rest = n - cnt;
    if (lane < rest) {
        for (int f = 0; f < 10; ++f) sg->out[lane * kRow + f] = sg->out[(cnt + lane) * kRow + f];
        sg->out_id[lane] = sg->out_id[cnt + lane];
    }
    __syncwarp();
    n = rest;
}

// An ionization product as a work item of the input stage: derived id and
// direction from its own draw (make_child), its positive-ion event and, with
// photoionization, the photon test of the ionizing event (Sec. 2.4).  e: the
// compact entry (x y z, speed, a, w, remaining time) of electron pid's draw k.
template <class T, int MODE>
__device__ __forceinline__ void build_product(const PushArgs<T>& A, const T* e, uint64_t pid, uint32_t k, T* row,
                                              uint64_t* rid) {
    T vc[3];
    *rid = make_child(A.K, A.step, pid, k, e[3], vc);
    if (MODE == MODE_PIC) {
        if (A.q_pos) deposit_at(A, e[0], e[1], e[2], e[7], A.q_pos);
        if (A.photo_prob > (T)0) photo_test(A, A.K, A.step, pid, k, e, e[7]);
    }
    row[0] = e[0]; row[1] = e[1]; row[2] = e[2];
    row[3] = vc[0]; row[4] = vc[1]; row[5] = vc[2];
    row[6] = e[4]; row[7] = e[5]; row[8] = e[6];
    row[9] = e[7];
    row[10] = e[8];
}

// Deposits the buffered negative-ion events [0, n) of the warp, one per lane.
template <class T>
__device__ __forceinline__ void flush_att(const PushArgs<T>& A, Stage<T>* sg, int& n) {
    const int lane = threadIdx.x & 31;
    __syncwarp();
    if (lane < n) {
        const T* a = sg->att + lane * 4;
        deposit_at(A, a[0], a[1], a[2], a[3], A.q_neg);
    }
    __syncwarp();
    n = 0;
}

template <class T, int MODE, bool FAST, bool STATS, bool CHILD>
__device__ __forceinline__ void collide_loop(const PushArgs<T>& A, const ProcSmem<T>* ps, Stage<T>* sg) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    long long n_items;
    unsigned long long* cursor;
    const ChildQ<T>& src = (A.gen & 1) ? A.cq2 : A.cq;
    // products the warp queue cannot take: the parents' go to the queue of the
    // first children launch, a children launch's to the other queue
    const ChildQ<T>& dst = CHILD ? ((A.gen & 1) ? A.cq : A.cq2) : A.cq;
    unsigned long long* dst_cnt = CHILD ? ((A.gen & 1) ? &A.st->n_child : &A.st->n_spill) : &A.st->n_child;
    if (CHILD) {
        n_items = (long long)((A.gen & 1) ? A.st->n_spill : A.st->n_child);
        if (n_items > A.cap_child) n_items = A.cap_child;
        if (n_items == 0) return;  // the warp queues took every product
        cursor = &A.st->n_fetch_c;
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&A.st->n_updates, (unsigned long long)n_items);
    } else {
        n_items = (long long)A.st->n_in;
        cursor = &A.st->n_fetch;
    }
    LStats ls;
    ls.zero();
    MomAcc<T> M;
    if (MODE == MODE_SWARM) M.zero();
    const Rates<T> rates{A.table, A.nu_max, A.tau_scale};
    Lane<T> L;
    bool active = false, dry = false;
    // warp-uniform counters: input stage head and size, output stage size,
    // queued products, buffered negative-ion events
    int in_head = 0, in_count = 0, n_out = 0, n_pq = 0, n_att = 0;
    unsigned built = 0;  // products this lane built from the warp queue (counted as updates)
    for (;;) {
        // 1. idle lanes take staged work items
        const bool want = !active;
        const unsigned need = __ballot_sync(kFull, want);
        const int avail = in_count - in_head;
        if (need && avail > 0) {
            const int rank = __popc(need & lt);
            if (want && rank < avail) {
                const int e = in_head + rank;
                const T* r = sg->in + e * kRow;
                for (int d = 0; d < 3; ++d) { L.x[d] = r[d]; L.v[d] = r[3 + d]; L.a[d] = r[6 + d]; L.d[d] = (T)0; }
                L.w = r[9];
                L.t_left = r[10];
                L.id = sg->in_id[e];
                L.k = 1;
                active = L.w > (T)0;
                if (active) ++ls.processed;
            }
            const int took = __popc(need) < avail ? __popc(need) : avail;
            in_head += took;
        }
        // 2. refill the input stage once it is drained: 32 queued products when
        //    there are that many (the rest once the input has run dry), else 32
        //    work items of the input; every lane prepares one entry
        if (in_head >= in_count && (!dry || n_pq > 0)) {
            int cnt = 0;
            __syncwarp();
            if (n_pq >= 32 || (dry && n_pq > 0)) {
                cnt = n_pq < 32 ? n_pq : 32;
                if (lane < cnt) {
                    const int j = n_pq - cnt + lane;
                    build_product<T, MODE>(A, sg->pq + j * kPQRow, sg->pq_id[j], sg->pq_k[j], sg->in + lane * kRow,
                                           &sg->in_id[lane]);
                    ++built;
                }
                n_pq -= cnt;
            } else {
                unsigned long long b = 0;
                if (lane == 0) b = atomicAdd(cursor, 32ull);
                b = __shfl_sync(kFull, b, 0);
                if ((long long)b >= n_items) {
                    dry = true;
                } else {
                    const long long left = n_items - (long long)b;
                    cnt = left < 32 ? (int)left : 32;
                    if (lane < cnt) {
                        const long long it = (long long)b + lane;
                        T* r = sg->in + lane * kRow;
                        if (CHILD) {
                            const Soa<T>& q = src.p;
                            const T e[kPQRow] = {q.r[PX][it], q.r[PY][it], q.r[PZ][it], q.r[VX][it], q.r[AX][it],
                                                 q.r[AY][it], q.r[AZ][it], q.r[PW][it], src.t_left[it]};
                            build_product<T, MODE>(A, e, q.id[it], src.k[it], r, &sg->in_id[lane]);
                        } else {
                            T f[10];
                            for (int q = 0; q < 10; ++q) f[q] = A.in.r[q][it];
                            if (MODE == MODE_PIC && A.kick_on_load) half_kick(A, f);
                            for (int q = 0; q < 10; ++q) r[q] = f[q];
                            r[10] = A.dt;
                            sg->in_id[lane] = A.in.id[it];
                        }
                    }
                }
            }
            in_head = 0;
            in_count = cnt;
            __syncwarp();
        }
        // 3. termination
        if (!__any_sync(kFull, active)) {
            if (dry && in_head >= in_count && n_pq == 0) break;
            continue;
        }
        // 4. up to two candidate collisions: the second only when the first
        //    needs nothing from the warp (a null, elastic or excitation
        //    collision), which halves the warp bookkeeping per draw (three
        //    per trip measured slower: more lanes idle behind the others)
        int r = EV_CONTINUE;
        T sp = (T)0;
        if (active) {
            r = event<T, MODE, FAST, STATS>(A, rates, A.K, A.step, ps, L, ls, sp);
            if (r == EV_CONTINUE) r = event<T, MODE, FAST, STATS>(A, rates, A.K, A.step, ps, L, ls, sp);
        }
        const bool done = r == EV_DONE, ion = r == EV_IONIZED, att = r == EV_ATTACHED;
        if (done || att) active = false;
        // 5. ionization products wait in the warp queue as compact entries (the
        //    queue of the next launch when it is full)
        const unsigned im = __ballot_sync(kFull, ion);
        if (im) {
            if (ion) {
                const int slot = n_pq + __popc(im & lt);
                const T e[kPQRow] = {L.x[0] + L.d[0], L.x[1] + L.d[1], L.x[2] + L.d[2], sp,
                                     L.a[0], L.a[1], L.a[2], L.w, L.t_left};
                if (slot < kPQ) {
                    T* q = sg->pq + slot * kPQRow;
                    for (int f = 0; f < kPQRow; ++f) q[f] = e[f];
                    sg->pq_id[slot] = L.id;
                    sg->pq_k[slot] = L.k - 1;
                    ++ls.children;
                } else {
                    const unsigned long long q = atomicAdd(dst_cnt, 1ull);
                    if ((long long)q < A.cap_child) {
                        const Soa<T>& d = dst.p;
                        d.r[PX][q] = e[0]; d.r[PY][q] = e[1]; d.r[PZ][q] = e[2];
                        d.r[VX][q] = sp;
                        d.r[AX][q] = e[4]; d.r[AY][q] = e[5]; d.r[AZ][q] = e[6];
                        d.r[PW][q] = L.w;
                        d.id[q] = L.id;
                        dst.t_left[q] = L.t_left;
                        dst.k[q] = L.k - 1;
                        ++ls.children;
                    } else {
                        atomicOr(&A.st->err, kErrChildCapacity);
                    }
                }
            }
            n_pq += __popc(im);
            if (n_pq > kPQ) n_pq = kPQ;
        }
        // 6. negative-ion events wait for a deposit by 32 lanes at once
        if (MODE == MODE_PIC) {
            const unsigned am = __ballot_sync(kFull, att);
            if (am && A.q_neg) {
                if (n_att + __popc(am) > kAtt) flush_att(A, sg, n_att);
                if (att) {
                    T* q = sg->att + (n_att + __popc(am & lt)) * 4;
                    q[0] = L.x[0] + L.d[0]; q[1] = L.x[1] + L.d[1]; q[2] = L.x[2] + L.d[2]; q[3] = L.w;
                }
                n_att += __popc(am);
            }
        }
        // 7. finished electrons
        const unsigned dm = __ballot_sync(kFull, done);
        if (dm) {
            if (done) {
                const int e = n_out + __popc(dm & lt);
                T* q = sg->out + e * kRow;
                q[0] = L.x[0] + L.d[0]; q[1] = L.x[1] + L.d[1]; q[2] = L.x[2] + L.d[2];
                q[3] = L.v[0]; q[4] = L.v[1]; q[5] = L.v[2];
                q[6] = L.a[0]; q[7] = L.a[1]; q[8] = L.a[2];
                q[9] = L.w;
                sg->out_id[e] = L.id;
            }
            n_out += __popc(dm);
            if (n_out >= 32) flush_out<T, MODE>(A, sg, n_out, 32, ls, M);
        }
    }
    if (n_out > 0) flush_out<T, MODE>(A, sg, n_out, n_out, ls, M);
    if (MODE == MODE_PIC && n_att > 0) flush_att(A, sg, n_att);
    {
        unsigned pw = built;
        for (int o = 16; o > 0; o >>= 1) pw += __shfl_xor_sync(kFull, pw, o);
        if (lane == 0 && pw) atomicAdd(&A.st->n_updates, (unsigned long long)pw);
    }
    if (STATS) flush_stats(A, ls, A.n_proc);
    if (MODE == MODE_SWARM) {
        M.m[14] += ls.w_ion;
        M.m[15] += ls.w_att;
        __syncthreads();
        flush_moments(A, M, reinterpret_cast<double*>(sg - (threadIdx.x >> 5)));  // block-wide scratch
    }
}

template <class T> __device__ __forceinline__ ProcSmem<T>* stage_proc(unsigned char* raw, const PushArgs<T>& A) {
    ProcSmem<T>* ps = reinterpret_cast<ProcSmem<T>*>(raw);
    if (threadIdx.x < 8) {
        ps->thr[threadIdx.x] = A.thr[threadIdx.x];
        ps->mratio[threadIdx.x] = A.mratio[threadIdx.x];
        ps->kind[threadIdx.x] = A.kind[threadIdx.x];
    }
    __syncthreads();
    return ps;
}

template <class T> __device__ __forceinline__ Stage<T>* warp_stage(unsigned char* raw) {
    return reinterpret_cast<Stage<T>*>(raw + ((sizeof(ProcSmem<T>) + 15) & ~(size_t)15)) + (threadIdx.x >> 5);
}

constexpr int kCollideThreads = 128;
// Resident blocks per SM the collision kernels are compiled for: seven (28
// warps, 72 registers) in single precision, four in double precision.
template <class T> constexpr int collide_min_blocks() { return sizeof(T) == 4 ? 7 : 4; }

template <class T, int MODE, bool FAST, bool STATS>
__global__ void __launch_bounds__(kCollideThreads, collide_min_blocks<T>()) k_push(const PushArgs<T> A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const ProcSmem<T>* ps = stage_proc(smem_raw, A);
    collide_loop<T, MODE, FAST, STATS, false>(A, ps, warp_stage<T>(smem_raw));
}

template <class T, int MODE, bool FAST, bool STATS>
__global__ void __launch_bounds__(kCollideThreads, collide_min_blocks<T>()) k_children(const PushArgs<T> A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const ProcSmem<T>* ps = stage_proc(smem_raw, A);
    collide_loop<T, MODE, FAST, STATS, true>(A, ps, warp_stage<T>(smem_raw));
}

// Deposit of the current particle set (no push).
template <class T>
__global__ void __launch_bounds__(256) k_deposit(const Soa<T> p, const DevState* st, T ox, T oy, T oz, T dx, int nx,
                                                 int ny, int nz, int axi, unsigned long long* q, DevState* stw) {
    const unsigned long long n = st->n_in;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (long long)n; i += stride) {
        const T w = p.r[PW][i];
        if (!(w > (T)0)) continue;
        const T x = p.r[PX][i], y = p.r[PY][i];
        if (axi) deposit(sqrt(x * x + y * y), oy + (T)0.5 * dx, p.r[PZ][i], w, ox, oy, oz, dx, nx, ny, nz, q, stw);
        else deposit(x, y, p.r[PZ][i], w, ox, oy, oz, dx, nx, ny, nz, q, stw);
    }
}

// Host-side launchers (defined in push_f32.cu / push_f64.cu).
template <class T> struct PushLaunch {
    static cudaError_t parents(const PushArgs<T>& A, int mode, bool stats, int grid, cudaStream_t s);
    static cudaError_t children(const PushArgs<T>& A, int mode, bool stats, int grid, cudaStream_t s);
    static cudaError_t deposit(const Soa<T>& p, DevState* st, const Grid& g, unsigned long long* q, int grid,
                               cudaStream_t s);
    static cudaError_t field_kick(const PushArgs<T>& A, int grid, cudaStream_t s);
    static cudaError_t resample(const PushArgs<T>& A, int grid, cudaStream_t s);
    static cudaError_t photo_append(const PushArgs<T>& A, int grid, cudaStream_t s);
    static size_t smem_bytes(int n_bins);
    static int blocks_per_sm(int mode, int n_bins);
};

}  // namespace pic
