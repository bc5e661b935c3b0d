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
#include "common.cuh"

namespace pic {

enum { MODE_PIC = 0, MODE_SWARM = 1 };
enum { RES_NONE = 0, RES_THIN = 1, RES_DUP = 2 };

template <class T> struct PushArgs {
    Soa<T> in, out;
    ChildQ<T> cq;
    DevState* st;
    const T* table;            // [n_bins][8]: nu_0..nu_{n_proc-1}, zeros, total
    int n_bins, n_proc;
    int kind[8];
    T thr[8];                  // eV
    T mratio[8];               // m_e / M (0 = infinite mass)
    double l0, inv_dl;         // ln(eps_0), (n_bins-1) / (ln eps_last - ln eps_0)
    T eps_lo, eps_hi;          // eV
    T nu_max;
    T dt;
    Keys K;
    uint32_t step;
    int first;                 // previous acceleration unknown: no half-kick
    long long cap_out, cap_child;
    // grid (PIC mode)
    int nx, ny, nz;
    T ox, oy, oz, dxr, hx, hy, hz;  // origin, cell size, upper faces
    const T* E4;               // [ncell][4] packed cell-centred field or nullptr (uniform)
    T E0[3];
    const uint8_t* mask;
    unsigned long long *q_e, *q_pos, *q_neg;
    int boundary;
    // swarm mode
    double* mom;               // [kNMom] accumulators of this step
    long long n_lo, n_hi;
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

template <class T>
__device__ __forceinline__ void gather(const PushArgs<T>& A, const T x[3], T E[3]) {
    if (A.E4 == nullptr) { E[0] = A.E0[0]; E[1] = A.E0[1]; E[2] = A.E0[2]; return; }
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

// ------------------------------------------------------------------ rates
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
        T t = (Arith<T>::lg(e) - (T)A.l0) * (T)A.inv_dl;
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
__device__ __forceinline__ int select_process(const PushArgs<T>& A, const T* tab, T e, T u1, LStats& ls) {
    int j;
    T f;
    table_pos(A, e, j, f, ls);
    const T* r0 = tab + j * kTableStride;
    const T* r1 = r0 + kTableStride;
    const T target = u1 * A.nu_max;
    if (FAST) {
        const T tot = r0[7] + f * (r1[7] - r0[7]);
        if (target >= tot) return -1;
    }
    T cum = (T)0;
    for (int k = 0; k < A.n_proc; ++k) {
        cum += r0[k] + f * (r1[k] - r0[k]);
        if (target < cum) return k;
    }
    return -1;
}

// ------------------------------------------------------------------ flight
// Child sink policies: append to the global queue (parents) or to a small
// per-thread stack (children finishing their step).
template <class T> struct StackSink {
    static constexpr int kDepth = 8;
    T x[kDepth][3], v[kDepth][3], w[kDepth], t[kDepth];
    uint64_t id[kDepth];
    int n = 0;
    __device__ bool push(const PushArgs<T>& A, const T xx[3], const T vv[3], const T a[3], T ww, uint64_t cid, T tl) {
        (void)A; (void)a;
        if (n >= kDepth) return false;
        for (int d = 0; d < 3; ++d) { x[n][d] = xx[d]; v[n][d] = vv[d]; }
        w[n] = ww; id[n] = cid; t[n] = tl;
        ++n;
        return true;
    }
};
template <class T> struct QueueSink {
    __device__ bool push(const PushArgs<T>& A, const T xx[3], const T vv[3], const T a[3], T ww, uint64_t cid, T tl) {
        unsigned long long s = atomicAdd(&A.st->n_child, 1ull);
        if ((long long)s >= A.cap_child) return false;
        const Soa<T>& q = A.cq.p;
        q.r[PX][s] = xx[0]; q.r[PY][s] = xx[1]; q.r[PZ][s] = xx[2];
        q.r[VX][s] = vv[0]; q.r[VY][s] = vv[1]; q.r[VZ][s] = vv[2];
        q.r[AX][s] = a[0]; q.r[AY][s] = a[1]; q.r[AZ][s] = a[2];
        q.r[PW][s] = ww; q.id[s] = cid; A.cq.t_left[s] = tl;
        return true;
    }
};

// Advances one electron over t_left; returns false if it attached.  The
// displacement within the step is accumulated separately from the position
// (x = x_start + displacement), so single precision keeps the resolution of
// the small flights instead of rounding to the absolute coordinate each time.
template <class T, int MODE, bool FAST, class Sink>
__device__ bool advance(const PushArgs<T>& A, const T* tab, T x[3], T v[3], const T a[3], T w, uint64_t id, T t_left,
                        LStats& ls, Sink& sink) {
    T dsp[3] = {(T)0, (T)0, (T)0};
    bool alive = true;
    for (uint32_t k = 1;; ++k) {
        const u32x4 r = draw_words(A.K, id, A.step, k);
        const T tau = Arith<T>::tau(unif<T>(r.x), A.nu_max);
        if (tau >= t_left) { fly(dsp, v, a, t_left); break; }
        fly(dsp, v, a, tau);
        t_left -= tau;
        ++ls.events;
        const T v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        const T e = Arith<T>::energy(v2);
        const int p = select_process<T, FAST>(A, tab, e, unif<T>(r.y), ls);
        if (p < 0) { ++ls.nulls; continue; }
        ++ls.coll[p & 7];
        T n[3];
        iso_dir(unif<T>(r.z), unif<T>(r.w), n);
        const int kind = A.kind[p];
        if (kind == PIC_PROC_ELASTIC) {
            const T sp = sqrt(v2);
            T cchi = (T)0;
            if (sp > (T)0) cchi = (v[0] * n[0] + v[1] * n[1] + v[2] * n[2]) / sp;
            const T e2 = e * ((T)1 - (T)2 * A.mratio[p] * ((T)1 - cchi));
            const T sp2 = Arith<T>::speed(dmax(e2, (T)0));
            v[0] = sp2 * n[0]; v[1] = sp2 * n[1]; v[2] = sp2 * n[2];
        } else if (kind == PIC_PROC_EXCITATION) {
            const T sp2 = Arith<T>::speed(dmax(e - A.thr[p], (T)0));
            v[0] = sp2 * n[0]; v[1] = sp2 * n[1]; v[2] = sp2 * n[2];
        } else if (kind == PIC_PROC_IONIZATION) {
            const T er = dmax(e - A.thr[p], (T)0);
            const T sp2 = Arith<T>::speed((T)0.5 * er);
            v[0] = sp2 * n[0]; v[1] = sp2 * n[1]; v[2] = sp2 * n[2];
            const uint64_t cid = derived_id(A.K, id, A.step, 0x80000000u | k);
            const u32x4 rb = draw_words(A.K, cid, A.step, 0u);
            T nb[3];
            iso_dir(unif<T>(rb.z), unif<T>(rb.w), nb);
            const T vc[3] = {sp2 * nb[0], sp2 * nb[1], sp2 * nb[2]};
            const T xc[3] = {x[0] + dsp[0], x[1] + dsp[1], x[2] + dsp[2]};
            if (!sink.push(A, xc, vc, a, w, cid, t_left)) atomicOr(&A.st->err, kErrChildCapacity | kErrStack);
            else ++ls.children;
            ls.w_ion += (double)w;
            if (MODE == MODE_PIC && A.q_pos)
                deposit(xc[0], xc[1], xc[2], w, A.ox, A.oy, A.oz, A.dxr, A.nx, A.ny, A.nz, A.q_pos, A.st);
        } else {  // attachment
            ls.w_att += (double)w;
            ++ls.attached;
            if (MODE == MODE_PIC && A.q_neg)
                deposit(x[0] + dsp[0], x[1] + dsp[1], x[2] + dsp[2], w, A.ox, A.oy, A.oz, A.dxr, A.nx, A.ny, A.nz,
                        A.q_neg, A.st);
            alive = false;
            break;
        }
    }
    x[0] += dsp[0];
    x[1] += dsp[1];
    x[2] += dsp[2];
    return alive;
}

// Domain faces (specular reflection or absorption) and electrode cells.
template <class T>
__device__ __forceinline__ bool boundaries(const PushArgs<T>& A, T x[3], T v[3], T w, LStats& ls) {
    const T lo[3] = {A.ox, A.oy, A.oz}, hi[3] = {A.hx, A.hy, A.hz};
    bool out = false;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
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
    if (!out && A.mask) {
        int i = fold_idx((int)floor(div_rn(sub_rn(x[0], A.ox), A.dxr)), A.nx);
        int j = fold_idx((int)floor(div_rn(sub_rn(x[1], A.oy), A.dxr)), A.ny);
        int k = fold_idx((int)floor(div_rn(sub_rn(x[2], A.oz), A.dxr)), A.nz);
        if (A.mask[((long long)k * A.ny + j) * A.nx + i]) out = true;
    }
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

template <class T> __device__ __forceinline__ void load_table(const PushArgs<T>& A, T* tab) {
    const int n = A.n_bins * kTableStride;
    for (int i = threadIdx.x; i < n; i += blockDim.x) tab[i] = A.table[i];
    __syncthreads();
}

// Survivor bookkeeping common to parents and children.
template <class T, int MODE>
__device__ __forceinline__ void emit(const PushArgs<T>& A, unsigned long long slot, const T x[3], const T v[3],
                                     const T a[3], T w, uint64_t id, MomAcc<T>& M) {
    if ((long long)slot >= A.cap_out) { atomicOr(&A.st->err, kErrOutCapacity); return; }
    store(A.out, slot, x, v, a, w, id);
    if (MODE == MODE_PIC) {
        if (A.q_e) deposit(x[0], x[1], x[2], w, A.ox, A.oy, A.oz, A.dxr, A.nx, A.ny, A.nz, A.q_e, A.st);
    } else {
        M.add(x, v, w);
    }
}

// ------------------------------------------------------------------ parents
template <class T, int MODE, bool FAST, bool STATS>
__global__ void __launch_bounds__(256) k_push(const PushArgs<T> A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* tab = reinterpret_cast<T*>(smem_raw);
    load_table(A, tab);
    const unsigned long long n = A.st->n_in;
    int res = RES_NONE;
    if (MODE == MODE_SWARM) {
        if ((long long)n > A.n_hi) res = RES_THIN;
        else if (n > 0 && (long long)n < A.n_lo) res = RES_DUP;
    }
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarp = ((long long)gridDim.x * blockDim.x) >> 5;
    const T qm = (T)(kQ / kMe);
    LStats ls;
    ls.zero();
    MomAcc<T> M;
    if (MODE == MODE_SWARM) M.zero();
    QueueSink<T> sink;
    for (long long base = warp * 32; base < (long long)n; base += nwarp * 32) {
        const long long i = base + lane;
        const bool valid = i < (long long)n;
        T x0[3], v0[3], a0[3], w0 = (T)0;
        uint64_t id0 = 0;
        if (valid) {
            x0[0] = A.in.r[PX][i]; x0[1] = A.in.r[PY][i]; x0[2] = A.in.r[PZ][i];
            v0[0] = A.in.r[VX][i]; v0[1] = A.in.r[VY][i]; v0[2] = A.in.r[VZ][i];
            a0[0] = A.in.r[AX][i]; a0[1] = A.in.r[AY][i]; a0[2] = A.in.r[AZ][i];
            w0 = A.in.r[PW][i];
            id0 = A.in.id[i];
        }
        const int reps = (res == RES_DUP) ? 2 : 1;
        for (int rep = 0; rep < reps; ++rep) {
            bool alive = valid && w0 > (T)0;
            T x[3] = {x0[0], x0[1], x0[2]}, v[3] = {v0[0], v0[1], v0[2]}, a[3] = {a0[0], a0[1], a0[2]};
            T w = w0;
            uint64_t id = id0;
            if (alive && res == RES_DUP) {
                w = (T)0.5 * w0;
                if (rep == 1) id = derived_id(A.K, id0, A.step, 0xA0000000u);
            }
            if (alive && res == RES_THIN) {
                const u32x4 r = draw_words(A.K, id0, A.step, 0xA0000000u);
                if (unif<T>(r.x) < (T)0.5) w = (T)2 * w0;
                else alive = false;
            }
            if (alive) {
                ++ls.processed;
                T E[3];
                gather(A, x, E);
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const T an = -qm * E[d];
                    if (!A.first) v[d] = v[d] + (T)0.5 * A.dt * (an - a[d]);
                    a[d] = an;
                }
                alive = advance<T, MODE, FAST>(A, tab, x, v, a, w, id, A.dt, ls, sink);
                if (alive && MODE == MODE_PIC) alive = boundaries(A, x, v, w, ls);
            }
            const unsigned m = __ballot_sync(kFull, alive);
            if (m == 0) continue;
            unsigned long long slot0 = 0;
            const int leader = __ffs(m) - 1;
            if (lane == leader) slot0 = atomicAdd(&A.st->n_out, (unsigned long long)__popc(m));
            slot0 = __shfl_sync(kFull, slot0, leader);
            if (alive) emit<T, MODE>(A, slot0 + __popc(m & lt_mask), x, v, a, w, id, M);
        }
    }
    if (STATS) flush_stats(A, ls, A.n_proc);
    if (MODE == MODE_SWARM) {
        M.m[14] += ls.w_ion;
        M.m[15] += ls.w_att;
        __syncthreads();
        flush_moments(A, M, reinterpret_cast<double*>(smem_raw));
    }
}

// ------------------------------------------------------------------ children
template <class T, int MODE, bool FAST, bool STATS>
__global__ void __launch_bounds__(256) k_children(const PushArgs<T> A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* tab = reinterpret_cast<T*>(smem_raw);
    load_table(A, tab);
    unsigned long long n = A.st->n_child;
    if ((long long)n > A.cap_child) n = (unsigned long long)A.cap_child;
    LStats ls;
    ls.zero();
    MomAcc<T> M;
    if (MODE == MODE_SWARM) M.zero();
    StackSink<T> stk;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (long long)n; i += stride) {
        const Soa<T>& q = A.cq.p;
        T x[3] = {q.r[PX][i], q.r[PY][i], q.r[PZ][i]};
        T v[3] = {q.r[VX][i], q.r[VY][i], q.r[VZ][i]};
        const T a[3] = {q.r[AX][i], q.r[AY][i], q.r[AZ][i]};
        T w = q.r[PW][i];
        uint64_t id = q.id[i];
        T tl = A.cq.t_left[i];
        stk.n = 0;
        for (;;) {
            ++ls.processed;
            bool alive = advance<T, MODE, FAST>(A, tab, x, v, a, w, id, tl, ls, stk);
            if (alive && MODE == MODE_PIC) alive = boundaries(A, x, v, w, ls);
            if (alive) {
                const unsigned long long s = atomicAdd(&A.st->n_out, 1ull);
                emit<T, MODE>(A, s, x, v, a, w, id, M);
            }
            if (stk.n == 0) break;
            --stk.n;
            const int t = stk.n;
            x[0] = stk.x[t][0]; x[1] = stk.x[t][1]; x[2] = stk.x[t][2];
            v[0] = stk.v[t][0]; v[1] = stk.v[t][1]; v[2] = stk.v[t][2];
            w = stk.w[t]; id = stk.id[t]; tl = stk.t[t];
        }
    }
    if (STATS) flush_stats(A, ls, A.n_proc);
    if (MODE == MODE_SWARM) {
        M.m[14] += ls.w_ion;
        M.m[15] += ls.w_att;
        __syncthreads();
        flush_moments(A, M, reinterpret_cast<double*>(smem_raw));
    }
}

// Deposit of the current particle set (no push).
template <class T>
__global__ void __launch_bounds__(256) k_deposit(const Soa<T> p, const DevState* st, T ox, T oy, T oz, T dx, int nx,
                                                 int ny, int nz, unsigned long long* q, DevState* stw) {
    const unsigned long long n = st->n_in;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (long long)n; i += stride) {
        const T w = p.r[PW][i];
        if (w > (T)0) deposit(p.r[PX][i], p.r[PY][i], p.r[PZ][i], w, ox, oy, oz, dx, nx, ny, nz, q, stw);
    }
}

// Host-side launchers (defined in push_f32.cu / push_f64.cu).
template <class T> struct PushLaunch {
    static cudaError_t parents(const PushArgs<T>& A, int mode, bool stats, int grid, cudaStream_t s);
    static cudaError_t children(const PushArgs<T>& A, int mode, bool stats, int grid, cudaStream_t s);
    static cudaError_t deposit(const Soa<T>& p, DevState* st, const Grid& g, unsigned long long* q, int grid,
                               cudaStream_t s);
    static size_t smem_bytes(int n_bins);
    static int blocks_per_sm(int mode, int n_bins);
};

}  // namespace pic
