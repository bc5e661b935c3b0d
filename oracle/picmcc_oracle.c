/*
 * picmcc_oracle.c -- plain, slow, FP64 CPU restatement of the PIC-MCC electron
 * step of Wang, Sun & Teunissen (arXiv 2110.14494), Sec. 2.1.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle the CUDA library is
 * checked against.  Only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark may load it; the product path never does.  It shares no
 * code, header, table or constant with the CUDA library.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared -o liboracle.so picmcc_oracle.c -lm
 * (-ffp-contract=off: no fused multiply-add, so every product and sum is a
 * separately rounded IEEE operation, as written).
 *
 * Pins (closed forms and invariants each function is tested against) are
 * listed next to each function.  Functions with no such pin say
 * "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* CODATA 2018 */
#define Q_E 1.602176634e-19
#define M_ELEC 9.1093837015e-31
#define EPS_0 8.8541878128e-12
#define TWO_PI 6.283185307179586476925286766559
#define M_PI_ORC 3.14159265358979323846264338327950

#define ORC_MAX_PROC 16
#define ORC_NMOM 16
#define ORC_NRES 24

enum { K_ELASTIC = 0, K_EXCITATION = 1, K_IONIZATION = 2, K_ATTACHMENT = 3 };

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, written from Salmon, Moraes, Dror & Shaw, "Parallel random  */
/* numbers: as easy as 1, 2, 3" (SC'11): ten rounds of two 32x32->64-bit     */
/* multiplications with a Weyl-sequence key schedule.                        */
/* Pin: cross-implementation agreement (CUDA) + uniformity statistics.       */
/* ------------------------------------------------------------------------ */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* A 32-bit word to a uniform number in (0,1): the top 23 bits, centred in
 * their bin, ((w >> 9) + 1/2) 2^-23.  The value has at most 24 significant
 * bits, so it is exact in binary32 and binary64 alike, and never 0 or 1. */
static double unif(uint32_t w) { return ((double)(w >> 9) + 0.5) * (1.0 / 8388608.0); }

/* Stream keys.  The MCC stream is keyed by the seed itself; derived ids and the
 * initial seeding use the seed xor-ed with fixed words. */
static void key_mcc(uint64_t seed, uint32_t k[2]) { k[0] = (uint32_t)seed; k[1] = (uint32_t)(seed >> 32); }
static void key_ids(uint64_t seed, uint32_t k[2]) { k[0] = (uint32_t)seed ^ 0x5A5A5A5Au; k[1] = (uint32_t)(seed >> 32) ^ 0xC3C3C3C3u; }
static void key_init(uint64_t seed, uint32_t k[2]) { k[0] = (uint32_t)seed ^ 0x1B873593u; k[1] = (uint32_t)(seed >> 32) ^ 0xCC9E2D51u; }

static void draw(uint64_t seed, uint64_t id, uint32_t step, uint32_t k, double u[4])
{
    uint32_t c[4] = {(uint32_t)id, (uint32_t)(id >> 32), step, k}, key[2], o[4];
    key_mcc(seed, key);
    orc_philox(c, key, o);
    for (int i = 0; i < 4; ++i) u[i] = unif(o[i]);
}

static uint64_t derived_id(uint64_t seed, uint64_t id, uint32_t step, uint32_t tag)
{
    uint32_t c[4] = {(uint32_t)id, (uint32_t)(id >> 32), step, tag}, key[2], o[4];
    key_ids(seed, key);
    orc_philox(c, key, o);
    return (uint64_t)o[0] | ((uint64_t)o[1] << 32);
}

/* ------------------------------------------------------------------------ */
/* Data passed in from Python (ctypes mirrors these layouts).               */
/* ------------------------------------------------------------------------ */
typedef struct orc_setup {
    int n_proc, n_bins;
    const double *eps;        /* [n_bins] node energies, eV, uniform in ln(eps) */
    const double *nu;         /* [n_proc][n_bins] collision rates, 1/s (orc_rate_table) */
    double nu_max;            /* 1/s */
    const int *kind;          /* [n_proc] K_* */
    const double *threshold;  /* [n_proc] eV */
    const double *mass;       /* [n_proc] target mass, kg; 0 = infinitely heavy */
    double dt;                /* s */
    uint64_t seed;
    int prec;                 /* 32 or 64: precision of deposit quantisation and cell decisions */
    int nx, ny, nz;           /* nx == 0: swarm (no grid, no boundaries, uniform field) */
    double dx, ox, oy, oz;
    const uint8_t *mask;      /* [nz][ny][nx] electrode cells or NULL */
    const float *Ex, *Ey, *Ez;/* [nz][ny][nx] cell-centred field (V/m) or NULL = uniform E0 */
    double E0[3];
    int boundary;             /* 0 = specular reflection, 1 = absorb at domain faces */
    /* photoionization (Sec. 2.4): photon emission probability per ionization
     * xi p_q / (p + p_q) (0 = off) and the absorption coefficient range
     * [chi_a, chi_b] = [chi_min, chi_max] p_O2, 1/m */
    double photo_prob, chi_a, chi_b;
    /* axisymmetric geometry (Sec. 2.1.1-2.1.2): particles move in 3D, the
     * field, densities and mask live on the (r, z) mesh of nx radial cells
     * from the axis x = y = 0 (ny = 1); the field arrays hold E_r (Ex) and
     * E_z (Ez) */
    int axi;
    /* the same field in float64 (used instead of Ex, Ey, Ez when set) */
    const double *Ex64, *Ey64, *Ez64;
    /* length of the velocity-Verlet half-kick that completes Eq. 2 for the
     * previous step: that step's dt, which differs from dt when the time step
     * changes between steps (Sec. 2.1.4); 0 = dt */
    double dt_kick;
} orc_setup;

typedef struct orc_parts {
    long long n, cap;
    double *x, *y, *z, *vx, *vy, *vz, *ax, *ay, *az, *w;
    uint64_t *id;
} orc_parts;

typedef struct orc_stats {
    long long n_start, n_children, n_end, n_attached, n_absorbed, n_null, n_clamped, n_events, n_photo;
    long long n_coll[ORC_MAX_PROC];
    double w_ion, w_att, w_absorbed;
} orc_stats;

/* ------------------------------------------------------------------------ */
/* Rate table, Sec. 2.1.1 / 2.1.5: nu_k(eps_j) = N_k sigma_k(eps_j) v(eps_j),  */
/* v = sqrt(2 e eps / m_e); nu_max = max_j sum_k nu_k(eps_j).                  */
/* Pin: constant sigma*v gives constant nu; hand-evaluated node values.      */
/* ------------------------------------------------------------------------ */
int orc_rate_table(int n_proc, int n_bins, const double *eps, const double *sigma,
                   const double *density, double *nu, double *nu_max)
{
    if (n_proc < 1 || n_proc > ORC_MAX_PROC || n_bins < 2) return -1;
    double mx = 0.0;
    for (int j = 0; j < n_bins; ++j) {
        double v = sqrt(2.0 * Q_E * eps[j] / M_ELEC);
        double tot = 0.0;
        for (int k = 0; k < n_proc; ++k) {
            double r = density[k] * sigma[k * n_bins + j] * v;
            nu[k * n_bins + j] = r;
            tot += r;
        }
        if (tot > mx) mx = tot;
    }
    *nu_max = mx;
    return 0;
}

/* Rates at energy e, linear in ln(eps) between nodes, clamped to the table. */
static void rates_at(const orc_setup *s, double e, double *out, long long *clamped)
{
    int n = s->n_bins, j;
    double f;
    if (e <= s->eps[0]) {
        j = 0; f = 0.0;
        if (e < s->eps[0]) ++*clamped;
    } else if (e >= s->eps[n - 1]) {
        j = n - 2; f = 1.0;
        if (e > s->eps[n - 1]) ++*clamped;
    } else {
        double l0 = log(s->eps[0]);
        double inv = (double)(n - 1) / (log(s->eps[n - 1]) - l0);
        double t = (log(e) - l0) * inv;
        j = (int)floor(t);
        if (j > n - 2) j = n - 2;
        if (j < 0) j = 0;
        f = t - (double)j;
    }
    for (int k = 0; k < s->n_proc; ++k) {
        double a = s->nu[k * n + j], b = s->nu[k * n + j + 1];
        out[k] = a + f * (b - a);
    }
}

/* ------------------------------------------------------------------------ */
/* Cell-centred trilinear interpolation of E at x (Sec. 2.1.3).               */
/* s = (x - origin)/dx - 1/2, clamped to [0, n-1] per axis.                   */
/* Pin: a linear field is reproduced exactly inside the grid.               */
/* ------------------------------------------------------------------------ */
/* field value d at cell idx, from whichever precision was given */
static double field_at(const orc_setup *s, int d, long long idx)
{
    if (s->Ex64) return (d == 0 ? s->Ex64 : (d == 1 ? s->Ey64 : s->Ez64))[idx];
    return (double)(d == 0 ? s->Ex : (d == 1 ? s->Ey : s->Ez))[idx];
}

static void axis_interp(double x, double o, double dx, int n, int *i0, int *i1, double *f)
{
    double s = (x - o) / dx - 0.5;
    if (s < 0.0) s = 0.0;
    if (s > (double)(n - 1)) s = (double)(n - 1);
    int i = (int)floor(s);
    if (i > n - 2) i = n - 2;
    if (i < 0) i = 0;
    *i0 = i;
    *i1 = (n > 1) ? i + 1 : i;
    *f = (n > 1) ? s - (double)i : 0.0;
}

/* Axisymmetric field at a 3D position: E_r and E_z bilinear in (r, z) at the
 * cell centres, the radial part projected: (E_r x/r, E_r y/r, E_z), and 0 on
 * the axis (Sec. 2.1.1). */
static void gather_axi(const orc_setup *s, double x, double y, double z, double E[3])
{
    double r = sqrt(x * x + y * y);
    int ir[2], iz[2];
    double fr, fz;
    axis_interp(r, s->ox, s->dx, s->nx, &ir[0], &ir[1], &fr);
    axis_interp(z, s->oz, s->dx, s->nz, &iz[0], &iz[1], &fz);
    double gr[2] = {1.0 - fr, fr}, gz[2] = {1.0 - fz, fz};
    double er = 0.0, ez = 0.0;
    for (int c = 0; c < 4; ++c) {
        int dz = c >> 1, dr = c & 1;
        long long idx = (long long)iz[dz] * s->nx + ir[dr];
        er += (gz[dz] * gr[dr]) * field_at(s, 0, idx);
        ez += (gz[dz] * gr[dr]) * field_at(s, 2, idx);
    }
    double inv = r > 0.0 ? er / r : 0.0;
    E[0] = inv * x;
    E[1] = inv * y;
    E[2] = ez;
}

static void gather(const orc_setup *s, double x, double y, double z, double E[3])
{
    if (s->Ex == NULL && s->Ex64 == NULL) { E[0] = s->E0[0]; E[1] = s->E0[1]; E[2] = s->E0[2]; return; }
    if (s->axi) { gather_axi(s, x, y, z, E); return; }
    int ix[2], iy[2], iz[2];
    double fx, fy, fz;
    axis_interp(x, s->ox, s->dx, s->nx, &ix[0], &ix[1], &fx);
    axis_interp(y, s->oy, s->dx, s->ny, &iy[0], &iy[1], &fy);
    axis_interp(z, s->oz, s->dx, s->nz, &iz[0], &iz[1], &fz);
    double gx[2] = {1.0 - fx, fx}, gy[2] = {1.0 - fy, fy}, gz[2] = {1.0 - fz, fz};
    for (int d = 0; d < 3; ++d) {
        double acc = 0.0;
        for (int c = 0; c < 8; ++c) {
            int dz = c >> 2, dy = (c >> 1) & 1, dxx = c & 1;
            long long idx = ((long long)iz[dz] * s->ny + iy[dy]) * s->nx + ix[dxx];
            acc += ((gz[dz] * gy[dy]) * gx[dxx]) * field_at(s, d, idx);
        }
        E[d] = acc;
    }
}

/* ------------------------------------------------------------------------ */
/* Fixed-point cell-centred CIC deposit (Sec. 2.1.3, "standard trilinear").   */
/* S = 2^32 per unit weight; corners 0..6 rounded to nearest (even), corner 7 */
/* takes the remainder so the cell sum is exactly llrint(w S).  Indices -1 and */
/* n fold back onto 0 and n-1.  prec = 32 evaluates everything in binary32.   */
/* Pin: sum over cells = sum llrint(w S); particle at a cell centre fills one */
/* cell; translation by whole cells shifts the grid.                         */
/* ------------------------------------------------------------------------ */
static int fold(int i, int n) { return i < 0 ? 0 : (i >= n ? n - 1 : i); }

/* The mesh point of a particle position: itself, or on an axisymmetric mesh
 * (r, centre of the single y cell, z) with r = sqrt(x^2 + y^2) evaluated in
 * the precision s->prec. */
static void grid_point(const orc_setup *s, double *x, double *y)
{
    if (!s->axi) return;
    if (s->prec == 32) {
        float xf = (float)*x, yf = (float)*y;
        *x = (double)sqrtf(xf * xf + yf * yf);
        *y = (double)((float)s->oy + 0.5f * (float)s->dx);
    } else {
        *x = sqrt(*x * *x + *y * *y);
        *y = s->oy + 0.5 * s->dx;
    }
}

static void deposit_one(const orc_setup *s, double x, double y, double z, double w, int64_t *q)
{
    int64_t qc[8];
    int i0, j0, k0;
    grid_point(s, &x, &y);
    if (s->prec == 32) {
        float xf = (float)x, yf = (float)y, zf = (float)z, wf = (float)w;
        float dxf = (float)s->dx;
        float sx = (xf - (float)s->ox) / dxf - 0.5f;
        float sy = (yf - (float)s->oy) / dxf - 0.5f;
        float sz = (zf - (float)s->oz) / dxf - 0.5f;
        float flx = floorf(sx), fly = floorf(sy), flz = floorf(sz);
        float fx = sx - flx, fy = sy - fly, fz = sz - flz;
        i0 = (int)flx; j0 = (int)fly; k0 = (int)flz;
        float gx[2] = {1.0f - fx, fx}, gy[2] = {1.0f - fy, fy}, gz[2] = {1.0f - fz, fz};
        float wS = wf * 4294967296.0f;
        int64_t sum = 0;
        for (int c = 0; c < 7; ++c) {
            int dz = c >> 2, dy = (c >> 1) & 1, dxx = c & 1;
            float v = ((wS * gz[dz]) * gy[dy]) * gx[dxx];
            qc[c] = (int64_t)llrintf(v);
            sum += qc[c];
        }
        qc[7] = (int64_t)llrintf(wS) - sum;
    } else {
        double sx = (x - s->ox) / s->dx - 0.5;
        double sy = (y - s->oy) / s->dx - 0.5;
        double sz = (z - s->oz) / s->dx - 0.5;
        double flx = floor(sx), fly = floor(sy), flz = floor(sz);
        double fx = sx - flx, fy = sy - fly, fz = sz - flz;
        i0 = (int)flx; j0 = (int)fly; k0 = (int)flz;
        double gx[2] = {1.0 - fx, fx}, gy[2] = {1.0 - fy, fy}, gz[2] = {1.0 - fz, fz};
        double wS = w * 4294967296.0;
        int64_t sum = 0;
        for (int c = 0; c < 7; ++c) {
            int dz = c >> 2, dy = (c >> 1) & 1, dxx = c & 1;
            double v = ((wS * gz[dz]) * gy[dy]) * gx[dxx];
            qc[c] = (int64_t)llrint(v);
            sum += qc[c];
        }
        qc[7] = (int64_t)llrint(wS) - sum;
    }
    for (int c = 0; c < 8; ++c) {
        int dz = c >> 2, dy = (c >> 1) & 1, dxx = c & 1;
        int ii = fold(i0 + dxx, s->nx), jj = fold(j0 + dy, s->ny), kk = fold(k0 + dz, s->nz);
        q[((long long)kk * s->ny + jj) * s->nx + ii] += qc[c];
    }
}

void orc_deposit(const orc_setup *s, const orc_parts *p, int64_t *q)
{
    for (long long i = 0; i < p->n; ++i)
        if (p->w[i] > 0.0) deposit_one(s, p->x[i], p->y[i], p->z[i], p->w[i], q);
}

/* Cell index of a position (the integer decision is taken in s->prec). */
static long long cell_of(const orc_setup *s, double x, double y, double z)
{
    int ii, jj, kk;
    grid_point(s, &x, &y);
    if (s->prec == 32) {
        float dxf = (float)s->dx;
        ii = (int)floorf(((float)x - (float)s->ox) / dxf);
        jj = (int)floorf(((float)y - (float)s->oy) / dxf);
        kk = (int)floorf(((float)z - (float)s->oz) / dxf);
    } else {
        ii = (int)floor((x - s->ox) / s->dx);
        jj = (int)floor((y - s->oy) / s->dx);
        kk = (int)floor((z - s->oz) / s->dx);
    }
    ii = fold(ii, s->nx); jj = fold(jj, s->ny); kk = fold(kk, s->nz);
    return ((long long)kk * s->ny + jj) * s->nx + ii;
}

/* ------------------------------------------------------------------------ */
/* One electron over its remaining time (Sec. 2.1.1).                        */
/* Free flight at constant a (Eq. 1 on sub-intervals, v += a tau) between     */
/* candidate collisions drawn with the null-collision method at the constant */
/* rate nu_max.  Draw k gives u0 (flight time), u1 (process), u2, u3          */
/* (isotropic scattering direction).                                        */
/* ------------------------------------------------------------------------ */
typedef struct { double t_left; int alive; } flight_out;

static void fly(double *x, double *v, const double *a, double tau)
{
    for (int d = 0; d < 3; ++d) {
        x[d] = x[d] + tau * (v[d] + 0.5 * tau * a[d]);
        v[d] = v[d] + tau * a[d];
    }
}

static double energy_eV(const double *v)
{
    double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    return 0.5 * M_ELEC * v2 / Q_E;
}

static void iso_dir(double u2, double u3, double n[3])
{
    double ct = 1.0 - 2.0 * u2;
    double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    double ph = TWO_PI * u3;
    n[0] = st * cos(ph);
    n[1] = st * sin(ph);
    n[2] = ct;
}

static int append(orc_parts *p, const double *x, const double *v, const double *a, double w, uint64_t id)
{
    if (p->n >= p->cap) return -1;
    long long j = p->n++;
    p->x[j] = x[0]; p->y[j] = x[1]; p->z[j] = x[2];
    p->vx[j] = v[0]; p->vy[j] = v[1]; p->vz[j] = v[2];
    p->ax[j] = a[0]; p->ay[j] = a[1]; p->az[j] = a[2];
    p->w[j] = w; p->id[j] = id;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Photoionization, Sec. 2.4 (discrete Monte Carlo photons).  Per ionization  */
/* event (draw index k of the ionizing electron), draw (id, step,            */
/* 0xD0000000 | k): u0 < photo_prob emits one photon of the electron's       */
/* weight.  Absorption distance from Zheleznyak's function                   */
/*   f(r) = (exp(-a r) - exp(-b r)) / (r ln(b/a)),                            */
/* which equals the integral over chi in [a, b] of                            */
/*   [1 / (chi ln(b/a))] * chi exp(-chi r):                                    */
/* chi is drawn log-uniform on [a, b] (chi = a exp(u1 ln(b/a))) and then r     */
/* exponential with rate chi (r = -ln(u2) / chi).  Direction isotropic:       */
/* cos(theta) = 1 - 2 u3, azimuth 2 pi u0' of draw (id, step, 0xE0000000 | k). */
/* A photon absorbed inside the domain and outside the electrode records a   */
/* positive ion there and a photoelectron (id derived with tag 0xD0000000|k) */
/* that joins the electrons at rest after the step.                          */
/* Pins: the distance distribution against 1 - (E1(a r) - E1(b r))/ln(b/a)    */
/* (scipy's exponential integral), the emission fraction (also at the       */
/* paper's printed xi and p_q), isotropy, charge neutrality of each         */
/* photoionization.                                                          */
/* ------------------------------------------------------------------------ */
static void photon_draw(const orc_setup *s, uint64_t id, uint32_t step, uint32_t k, int *emit, double *r,
                        double n[3])
{
    double u[4], u2[4];
    draw(s->seed, id, step, 0xD0000000u | k, u);
    *emit = u[0] < s->photo_prob;
    if (!*emit) return;
    double chi = s->chi_a * exp(u[1] * log(s->chi_b / s->chi_a));
    *r = -log(u[2]) / chi;
    draw(s->seed, id, step, 0xE0000000u | k, u2);
    iso_dir(u[3], u2[0], n);
}

static void photo_emit(const orc_setup *s, const double *x, double w, uint64_t id, uint32_t step, uint32_t k,
                       orc_parts *ph, int64_t *q_pos)
{
    int emit;
    double r, n[3];
    photon_draw(s, id, step, k, &emit, &r, n);
    if (!emit) return;
    double xp[3] = {x[0] + r * n[0], x[1] + r * n[1], x[2] + r * n[2]};
    double lo[3] = {s->ox, s->oy, s->oz};
    int nn[3] = {s->nx, s->ny, s->nz};
    for (int d = s->axi ? 2 : 0; d < 3; ++d) {
        double h = lo[d] + (double)nn[d] * s->dx;
        if (!(xp[d] >= lo[d] && xp[d] <= h)) return;
    }
    if (s->axi && !(sqrt(xp[0] * xp[0] + xp[1] * xp[1]) <= (double)s->nx * s->dx)) return;
    if (s->mask && s->mask[cell_of(s, xp[0], xp[1], xp[2])]) return;
    if (q_pos) deposit_one(s, xp[0], xp[1], xp[2], w, q_pos);
    double zero[3] = {0.0, 0.0, 0.0};
    append(ph, xp, zero, zero, w, derived_id(s->seed, id, step, 0xD0000000u | k));
}

/* Test helper: n photon draws of electron `id` at step `step` with draw
 * indices 1..n; emitted[k], r[k] and dir[3k..3k+2] per draw. */
void orc_photon_draws(const orc_setup *s, uint64_t id, uint32_t step, int n, int *emitted, double *r, double *dir)
{
    for (int k = 0; k < n; ++k) {
        double rr = 0.0, nd[3] = {0.0, 0.0, 0.0};
        photon_draw(s, id, step, (uint32_t)(k + 1), &emitted[k], &rr, nd);
        r[k] = rr;
        dir[3 * k] = nd[0]; dir[3 * k + 1] = nd[1]; dir[3 * k + 2] = nd[2];
    }
}

/* Advances particle i by t_left, appending ionization products to p (their
 * remaining time goes to tl[]) and photoelectrons to ph.  Returns 0, or -3
 * when p or ph is full. */
static int advance(const orc_setup *s, orc_parts *p, long long i, double t_left, uint32_t step,
                   double *tl, int64_t *q_pos, int64_t *q_neg, orc_stats *st, orc_parts *ph)
{
    double x[3] = {p->x[i], p->y[i], p->z[i]};
    double v[3] = {p->vx[i], p->vy[i], p->vz[i]};
    double a[3] = {p->ax[i], p->ay[i], p->az[i]};
    double w = p->w[i];
    uint64_t id = p->id[i];
    double rates[ORC_MAX_PROC];
    int alive = 1, rc = 0;
    for (uint32_t k = 1;; ++k) {
        double u[4];
        draw(s->seed, id, step, k, u);
        double tau = -log(u[0]) / s->nu_max;
        if (tau >= t_left) { fly(x, v, a, t_left); break; }
        fly(x, v, a, tau);
        t_left -= tau;
        st->n_events++;
        double e = energy_eV(v);
        rates_at(s, e, rates, &st->n_clamped);
        double target = u[1] * s->nu_max, cum = 0.0;
        int proc = -1;
        for (int kk = 0; kk < s->n_proc; ++kk) {
            cum += rates[kk];
            if (target < cum) { proc = kk; break; }
        }
        if (proc < 0) { st->n_null++; continue; }
        st->n_coll[proc]++;
        double nn[3];
        iso_dir(u[2], u[3], nn);
        int kind = s->kind[proc];
        if (kind == K_ELASTIC) {
            double sp = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            double cchi = 0.0;
            if (sp > 0.0) cchi = (v[0] * nn[0] + v[1] * nn[1] + v[2] * nn[2]) / sp;
            double ratio = s->mass[proc] > 0.0 ? M_ELEC / s->mass[proc] : 0.0;
            double e2 = e * (1.0 - 2.0 * ratio * (1.0 - cchi));
            double sp2 = sqrt(2.0 * Q_E * fmax(e2, 0.0) / M_ELEC);
            for (int d = 0; d < 3; ++d) v[d] = sp2 * nn[d];
        } else if (kind == K_EXCITATION) {
            double e2 = fmax(e - s->threshold[proc], 0.0);
            double sp2 = sqrt(2.0 * Q_E * e2 / M_ELEC);
            for (int d = 0; d < 3; ++d) v[d] = sp2 * nn[d];
        } else if (kind == K_IONIZATION) {
            double er = fmax(e - s->threshold[proc], 0.0);
            double sp2 = sqrt(2.0 * Q_E * (0.5 * er) / M_ELEC);
            for (int d = 0; d < 3; ++d) v[d] = sp2 * nn[d];
            uint64_t cid = derived_id(s->seed, id, step, 0x80000000u | k);
            double ub[4], nb[3], vc[3];
            draw(s->seed, cid, step, 0u, ub);
            iso_dir(ub[2], ub[3], nb);
            for (int d = 0; d < 3; ++d) vc[d] = sp2 * nb[d];
            if (append(p, x, vc, a, w, cid) != 0) { rc = -3; }
            else { tl[p->n - 1] = t_left; st->n_children++; }
            st->w_ion += w;
            if (s->nx > 0 && q_pos) deposit_one(s, x[0], x[1], x[2], w, q_pos);
            if (s->nx > 0 && s->photo_prob > 0.0 && ph) photo_emit(s, x, w, id, step, k, ph, q_pos);
        } else { /* attachment */
            st->w_att += w;
            st->n_attached++;
            if (s->nx > 0 && q_neg) deposit_one(s, x[0], x[1], x[2], w, q_neg);
            alive = 0;
            break;
        }
    }
    p->x[i] = x[0]; p->y[i] = x[1]; p->z[i] = x[2];
    p->vx[i] = v[0]; p->vy[i] = v[1]; p->vz[i] = v[2];
    p->ax[i] = a[0]; p->ay[i] = a[1]; p->az[i] = a[2];
    if (!alive) p->w[i] = 0.0;
    return rc;
}

/* Domain faces (Sec. 2.3: homogeneous Neumann for the electron density is read
 * as specular reflection), then absorption by electrode cells. */
static void boundaries(const orc_setup *s, orc_parts *p, long long i, orc_stats *st)
{
    if (s->nx == 0 || p->w[i] <= 0.0) return;
    double *X[3] = {&p->x[i], &p->y[i], &p->z[i]};
    double *V[3] = {&p->vx[i], &p->vy[i], &p->vz[i]};
    double lo[3] = {s->ox, s->oy, s->oz};
    int n[3] = {s->nx, s->ny, s->nz};
    int out = 0;
    if (s->axi) {
        /* the cylinder r = R: outflow, or specular reflection r -> 2R - r with
         * the radial velocity reversed */
        double R = (double)s->nx * s->dx;
        double r = sqrt(p->x[i] * p->x[i] + p->y[i] * p->y[i]);
        if (s->boundary == 1) {
            if (r > R) out = 1;
        } else {
            for (int it = 0; it < 8 && r > R; ++it) {
                double rn = 2.0 * R - r, sc = rn / r;
                double ux = p->x[i] / r, uy = p->y[i] / r;
                double vr = p->vx[i] * ux + p->vy[i] * uy;
                p->x[i] *= sc;
                p->y[i] *= sc;
                p->vx[i] -= 2.0 * vr * ux;
                p->vy[i] -= 2.0 * vr * uy;
                r = fabs(rn);
            }
        }
    }
    for (int d = 0; d < 3; ++d) {
        if (s->axi && d < 2) continue;
        double l = lo[d], h = lo[d] + (double)n[d] * s->dx;
        if (s->boundary == 1) {
            if (*X[d] < l || *X[d] > h) out = 1;
            continue;
        }
        for (int it = 0; it < 8 && (*X[d] < l || *X[d] > h); ++it) {
            if (*X[d] < l) *X[d] = 2.0 * l - *X[d];
            else *X[d] = 2.0 * h - *X[d];
            *V[d] = -*V[d];
        }
        if (*X[d] < l) *X[d] = l;
        if (*X[d] > h) *X[d] = h;
    }
    if (!out && s->mask) {
        long long c = cell_of(s, p->x[i], p->y[i], p->z[i]);
        if (s->mask[c]) out = 1;
    }
    if (out) {
        st->n_absorbed++;
        st->w_absorbed += p->w[i];
        p->w[i] = 0.0;
    }
}

static void compact(orc_parts *p)
{
    long long j = 0;
    for (long long i = 0; i < p->n; ++i) {
        if (p->w[i] <= 0.0) continue;
        if (j != i) {
            p->x[j] = p->x[i]; p->y[j] = p->y[i]; p->z[j] = p->z[i];
            p->vx[j] = p->vx[i]; p->vy[j] = p->vy[i]; p->vz[j] = p->vz[i];
            p->ax[j] = p->ax[i]; p->ay[j] = p->ay[i]; p->az[j] = p->az[i];
            p->w[j] = p->w[i]; p->id[j] = p->id[i];
        }
        ++j;
    }
    p->n = j;
}

/* ------------------------------------------------------------------------ */
/* One PIC time step for all electrons (Sec. 2.1.1, Eqs. 1-2):               */
/*  a_new = -(e/m_e) E(x);  v += dt/2 (a_new - a_old) completes Eq. 2 of the  */
/*  previous step (first step: a_old = a_new);  then the collisional flight   */
/*  over dt with a = a_new.  Children born in the step finish the step with   */
/*  the parent's remaining time, generation after generation.  Survivors are */
/*  deposited into q_e (if given); ion events went to q_pos / q_neg.          */
/* Pins: ballistic motion (Eq. 1-2 exact for constant a), constant-nu drift   */
/* W = eE/(m nu), exp(nu t) growth, exp(-nu t) loss, energy balance.         */
/* ------------------------------------------------------------------------ */
int orc_step(const orc_setup *s, orc_parts *p, uint32_t step, int first, int64_t *q_e,
             int64_t *q_pos, int64_t *q_neg, orc_stats *st)
{
    memset(st, 0, sizeof(*st));
    long long n0 = p->n;
    st->n_start = n0;
    double *tl = (double *)calloc((size_t)(p->cap > 0 ? p->cap : 1), sizeof(double));
    if (!tl) return -2;
    /* photoelectrons of the step, kept apart until the step ends */
    orc_parts ph;
    memset(&ph, 0, sizeof ph);
    double *phb = NULL;
    if (s->photo_prob > 0.0 && s->nx > 0) {
        ph.cap = p->cap > 0 ? p->cap : 1;
        phb = (double *)calloc((size_t)ph.cap * 10, sizeof(double));
        ph.id = (uint64_t *)calloc((size_t)ph.cap, sizeof(uint64_t));
        if (!phb || !ph.id) { free(tl); free(phb); free(ph.id); return -2; }
        double **f[10] = {&ph.x, &ph.y, &ph.z, &ph.vx, &ph.vy, &ph.vz, &ph.ax, &ph.ay, &ph.az, &ph.w};
        for (int q = 0; q < 10; ++q) *f[q] = phb + (size_t)q * ph.cap;
    }
    int rc = 0;
    const double qm = Q_E / M_ELEC;
    const double kick = s->dt_kick > 0.0 ? s->dt_kick : s->dt;
    for (long long i = 0; i < n0; ++i) {
        if (p->w[i] <= 0.0) continue;
        double E[3];
        gather(s, p->x[i], p->y[i], p->z[i], E);
        double an[3] = {-qm * E[0], -qm * E[1], -qm * E[2]};
        double *ao[3] = {&p->ax[i], &p->ay[i], &p->az[i]};
        double *vv[3] = {&p->vx[i], &p->vy[i], &p->vz[i]};
        for (int d = 0; d < 3; ++d) {
            if (!first) *vv[d] = *vv[d] + 0.5 * kick * (an[d] - *ao[d]);
            *ao[d] = an[d];
        }
        int r = advance(s, p, i, s->dt, step, tl, q_pos, q_neg, st, phb ? &ph : NULL);
        if (r) rc = r;
    }
    for (long long i = n0; i < p->n; ++i) {
        int r = advance(s, p, i, tl[i], step, tl, q_pos, q_neg, st, phb ? &ph : NULL);
        if (r) rc = r;
    }
    for (long long i = 0; i < p->n; ++i) boundaries(s, p, i, st);
    compact(p);
    /* photoelectrons join at rest with the acceleration of the field at their
     * position (their first half-kick then adds nothing) */
    for (long long j = 0; j < ph.n; ++j) {
        double xp[3] = {ph.x[j], ph.y[j], ph.z[j]}, E[3], a[3], v0[3] = {0.0, 0.0, 0.0};
        gather(s, xp[0], xp[1], xp[2], E);
        for (int d = 0; d < 3; ++d) a[d] = -qm * E[d];
        if (append(p, xp, v0, a, ph.w[j], ph.id[j]) != 0) rc = -3;
        st->n_photo++;
    }
    free(phb);
    free(ph.id);
    if (q_e && s->nx > 0) orc_deposit(s, p, q_e);
    st->n_end = p->n;
    free(tl);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Fixed point -> densities and space charge (Sec. 2.5: rho feeds Poisson).  */
/* n = q / (2^32 dV); rho = e (n_pos - n_neg - n_e).                          */
/* ------------------------------------------------------------------------ */
void orc_fixed_to_rho(long long ncell, double dV, const int64_t *q_e, const int64_t *q_pos,
                      const int64_t *q_neg, double *rho)
{
    const double inv = 1.0 / (4294967296.0 * dV);
    for (long long c = 0; c < ncell; ++c) {
        double ne = (double)q_e[c] * inv, np = (double)q_pos[c] * inv, nn = (double)q_neg[c] * inv;
        rho[c] = Q_E * (np - nn - ne);
    }
}

/* ------------------------------------------------------------------------ */
/* Initial particles (Sec. 2.3, Eq. 7 with the sign of the exponent read as   */
/* negative): per cell floor(n dV / w0) particles plus one with probability  */
/* equal to the remainder, uniform in the cell, at rest, weight w0.  Cells    */
/* inside the electrode get none.  Cells are visited in x-fastest order and  */
/* ids count up from id0 in that order.                                      */
/* Pin: expected count = sum n dV / w0; positions inside their cells.         */
/* ------------------------------------------------------------------------ */
long long orc_seed_gaussian(const orc_setup *s, double n0, double radius, double cx, double cy,
                            double cz, double w0, uint64_t id0, orc_parts *p)
{
    uint32_t key[2];
    key_init(s->seed, key);
    const double dV = s->dx * s->dx * s->dx;
    const double zero[3] = {0.0, 0.0, 0.0};
    uint64_t nid = id0;
    for (int k = 0; k < s->nz; ++k)
        for (int j = 0; j < s->ny; ++j)
            for (int i = 0; i < s->nx; ++i) {
                long long c = ((long long)k * s->ny + j) * s->nx + i;
                if (s->mask && s->mask[c]) continue;
                double xc = s->ox + ((double)i + 0.5) * s->dx;
                double yc = s->oy + ((double)j + 0.5) * s->dx;
                double zc = s->oz + ((double)k + 0.5) * s->dx;
                /* axisymmetric: ring cell at radius xc, volume pi (2i + 1) dx^3, centre on the axis */
                double r2 = s->axi ? xc * xc + (zc - cz) * (zc - cz)
                                   : (xc - cx) * (xc - cx) + (yc - cy) * (yc - cy) + (zc - cz) * (zc - cz);
                double dVc = s->axi ? M_PI_ORC * (double)(2 * i + 1) * s->dx * s->dx * s->dx : dV;
                double expct = n0 * exp(-r2 / (radius * radius)) * dVc / w0;
                double fl = floor(expct);
                long long cnt = (long long)fl;
                uint32_t ctr[4] = {(uint32_t)c, 0u, 0u, 0xB0000000u}, o[4];
                orc_philox(ctr, key, o);
                if (unif(o[0]) < expct - fl) ++cnt;
                for (long long m = 0; m < cnt; ++m) {
                    uint32_t c2[4] = {(uint32_t)c, (uint32_t)(m + 1), 0u, 0xB0000000u};
                    orc_philox(c2, key, o);
                    double x[3] = {s->ox + ((double)i + unif(o[0])) * s->dx,
                                   s->oy + ((double)j + unif(o[1])) * s->dx,
                                   s->oz + ((double)k + unif(o[2])) * s->dx};
                    if (s->axi) {
                        /* uniform in the ring: r^2 uniform in [i^2, (i+1)^2] dx^2, angle uniform */
                        double r = s->dx * sqrt((double)i * i + unif(o[0]) * (double)(2 * i + 1));
                        x[0] = r * cos(TWO_PI * unif(o[1]));
                        x[1] = r * sin(TWO_PI * unif(o[1]));
                    }
                    if (append(p, x, zero, zero, w0, nid++) != 0) return -3;
                }
            }
    return (long long)(nid - id0);
}

/* Maxwellian start for swarms: components N(0, kT e / m_e) by Box-Muller on draw
 * (id, step 0, k 0); all particles at the origin with weight 1, ids 0..n-1. */
int orc_seed_maxwell(const orc_setup *s, long long n, double kT_eV, orc_parts *p)
{
    if (n > p->cap) return -3;
    double sig = sqrt(kT_eV * Q_E / M_ELEC);
    p->n = 0;
    const double zero[3] = {0.0, 0.0, 0.0};
    for (long long i = 0; i < n; ++i) {
        double u[4];
        draw(s->seed, (uint64_t)i, 0u, 0u, u);
        double r1 = sqrt(-2.0 * log(u[0])), r2 = sqrt(-2.0 * log(u[2]));
        double v[3] = {sig * r1 * cos(TWO_PI * u[1]), sig * r1 * sin(TWO_PI * u[1]),
                       sig * r2 * cos(TWO_PI * u[3])};
        append(p, zero, v, zero, 1.0, (uint64_t)i);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Super-particle weight update (Sec. 2.1.2, Eq. 3).                          */
/* Per cell: omega = max(W / N_ppc, w_min), W = sum of weights (summed as     */
/* integers llrint(w 2^24) so the total is order-free).  If the predicted    */
/* number of particles sum_c W_c/omega_c exceeds `cap`, every omega is scaled */
/* by the same factor.  Merge: particles with w < (2/3) omega, ordered by    */
/* (|v|^2, id), are paired (0,1), (2,3), ...; the pair's weights are summed */
/* and the state of one of them is kept, chosen with probability             */
/* proportional to its weight; rounds repeat while two or more candidates    */
/* remain.  Split: w > (3/2) omega is halved m times (m minimal with           */
/* w/2^m <= (3/2) omega), giving 2^m identical copies.                        */
/* Pins: total weight conserved; every particle ends in [(2/3) omega,         */
/* (3/2) omega] except at most one unpaired candidate per cell.              */
/* ------------------------------------------------------------------------ */
typedef struct { double key; uint64_t id; long long idx; } cand_t;
static int cand_cmp(const void *a, const void *b)
{
    const cand_t *x = (const cand_t *)a, *y = (const cand_t *)b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    if (x->id < y->id) return -1;
    if (x->id > y->id) return 1;
    return 0;
}

static double speed2(const orc_setup *s, const orc_parts *p, long long i)
{
    if (s->prec == 32) {
        float a = (float)p->vx[i], b = (float)p->vy[i], c = (float)p->vz[i];
        float r = (a * a + b * b) + c * c;
        return (double)r;
    }
    return (p->vx[i] * p->vx[i] + p->vy[i] * p->vy[i]) + p->vz[i] * p->vz[i];
}

typedef struct orc_ms_stats {
    long long n_before, n_after, n_merged_pairs, n_split_added, n_cells;
    double scale;
} orc_ms_stats;

static int cmp_ll(const void *a, const void *b)
{
    long long x = *(const long long *)a, y = *(const long long *)b;
    return (x > y) - (x < y);
}

int orc_merge_split(const orc_setup *s, orc_parts *p, uint32_t step, int n_ppc, double w_min,
                    long long cap, orc_ms_stats *ms)
{
    memset(ms, 0, sizeof(*ms));
    long long n = p->n;
    ms->n_before = n;
    if (n == 0) return 0;
    /* (cell << 32 | index) pairs sorted -> particles grouped by cell */
    long long *ci = (long long *)malloc(sizeof(long long) * (size_t)n);
    cand_t *cd = (cand_t *)malloc(sizeof(cand_t) * (size_t)n);
    if (!ci || !cd) { free(ci); free(cd); return -2; }
    long long ncell_tot = (long long)s->nx * s->ny * s->nz;
    for (long long i = 0; i < n; ++i) ci[i] = cell_of(s, p->x[i], p->y[i], p->z[i]) * (n + 1) + i;
    (void)ncell_tot;
    qsort(ci, (size_t)n, sizeof(long long), cmp_ll);
    /* pass 1: per-cell integer weight sums and the predicted count */
    int64_t pred_total = 0;
    const double S24 = 16777216.0;
    for (long long a = 0; a < n;) {
        long long c = ci[a] / (n + 1), b = a;
        int64_t W = 0;
        while (b < n && ci[b] / (n + 1) == c) { W += (int64_t)llrint(p->w[ci[b] % (n + 1)] * S24); ++b; }
        double om = fmax((double)W / S24 / (double)n_ppc, w_min);
        pred_total += (int64_t)llrint((double)W / om);
        ms->n_cells++;
        a = b;
    }
    double scale = 1.0;
    if (cap > 0 && pred_total > (int64_t)cap * (int64_t)16777216) scale = (double)pred_total / ((double)cap * S24);
    ms->scale = scale;
    long long n_orig = n;
    for (long long a = 0; a < n_orig;) {
        long long c = ci[a] / (n_orig + 1), b = a;
        int64_t W = 0;
        while (b < n_orig && ci[b] / (n_orig + 1) == c) { W += (int64_t)llrint(p->w[ci[b] % (n_orig + 1)] * S24); ++b; }
        double om = fmax((double)W / S24 / (double)n_ppc, w_min) * scale;
        double lo = 2.0 * om / 3.0, hi = 1.5 * om;
        /* merge rounds */
        int m = 0;
        for (long long t = a; t < b; ++t) {
            long long i = ci[t] % (n_orig + 1);
            if (p->w[i] < lo) { cd[m].idx = i; cd[m].id = p->id[i]; cd[m].key = speed2(s, p, i); ++m; }
        }
        for (uint32_t round = 0; m >= 2; ++round) {
            qsort(cd, (size_t)m, sizeof(cand_t), cand_cmp);
            int m2 = 0;
            for (int q = 0; q + 1 < m; q += 2) {
                long long ia = cd[q].idx, ib = cd[q + 1].idx;
                double wa = p->w[ia], wb = p->w[ib];
                uint64_t mid = cd[q].id < cd[q + 1].id ? cd[q].id : cd[q + 1].id;
                double u[4];
                draw(s->seed, mid, step, 0xC0000000u | round, u);
                long long keep = (u[0] * (wa + wb) < wa) ? ia : ib, drop = keep == ia ? ib : ia;
                double wsum = (s->prec == 32) ? (double)((float)wa + (float)wb) : wa + wb;
                p->w[keep] = wsum;
                p->w[drop] = 0.0;
                ms->n_merged_pairs++;
                if (wsum < lo) { cd[m2].idx = keep; cd[m2].id = p->id[keep]; cd[m2].key = speed2(s, p, keep); ++m2; }
            }
            if (m % 2 == 1) {  /* unpaired leftover stays a candidate */
                long long i = cd[m - 1].idx;
                cd[m2].idx = i; cd[m2].id = p->id[i]; cd[m2].key = speed2(s, p, i); ++m2;
            }
            if (m2 == m) break;
            m = m2;
        }
        /* split */
        for (long long t = a; t < b; ++t) {
            long long i = ci[t] % (n_orig + 1);
            double w = p->w[i];
            if (!(w > hi)) continue;
            int mm = 0;
            double wc = w;
            while (wc > hi) { wc *= 0.5; ++mm; }
            if (s->prec == 32) wc = (double)((float)w * (float)ldexp(1.0, -mm));
            p->w[i] = wc;
            long long copies = (1LL << mm) - 1;
            double x[3] = {p->x[i], p->y[i], p->z[i]}, v[3] = {p->vx[i], p->vy[i], p->vz[i]},
                   ac[3] = {p->ax[i], p->ay[i], p->az[i]};
            for (long long cc = 1; cc <= copies; ++cc) {
                uint64_t nid = derived_id(s->seed, p->id[i], step, 0x40000000u | (uint32_t)cc);
                if (append(p, x, v, ac, wc, nid) != 0) { free(ci); free(cd); return -3; }
                ms->n_split_added++;
            }
        }
        a = b;
    }
    free(ci); free(cd);
    compact(p);
    ms->n_after = p->n;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Poisson (Sec. 2.5): -lap(phi) = rho / eps0 (the paper's sign is read as    */
/* a typo), 7-point cell-centred stencil, Dirichlet phi = v_lo at z = 0 and   */
/* v_hi at z = L (ghost = 2 phi_b - phi), homogeneous Neumann on x and y,     */
/* electrode cells (mask != 0) held at v_mask.  Solved by Jacobi-            */
/* preconditioned conjugate gradients on the unmasked unknowns to            */
/* ||b - A phi|| / ||b|| <= rtol.  Deliberately not multigrid.               */
/* Pins: discrete eigenfunction manufactured solution; plates-only linear.   */
/* ------------------------------------------------------------------------ */
typedef struct { int nx, ny, nz; double h; const uint8_t *mask; } pgrid;

static double diag_of(const pgrid *g, int i, int j, int k)
{
    (void)i; (void)j;
    double d = 6.0;
    if (g->nx == 1) d -= 2.0; else { if (i == 0) d -= 1.0; if (i == g->nx - 1) d -= 1.0; }
    if (g->ny == 1) d -= 2.0; else { if (j == 0) d -= 1.0; if (j == g->ny - 1) d -= 1.0; }
    if (k == 0) d += 1.0;
    if (k == g->nz - 1) d += 1.0;
    return d;
}

/* y = A x on unmasked cells (masked cells contribute 0 and get y = 0). */
static void apply_A(const pgrid *g, const double *x, double *y)
{
    int nx = g->nx, ny = g->ny, nz = g->nz;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                long long c = ((long long)k * ny + j) * nx + i;
                if (g->mask && g->mask[c]) { y[c] = 0.0; continue; }
                double s = diag_of(g, i, j, k) * x[c];
                long long nb[6] = {-1, -1, -1, -1, -1, -1};
                if (i > 0) nb[0] = c - 1;
                if (i < nx - 1) nb[1] = c + 1;
                if (j > 0) nb[2] = c - nx;
                if (j < ny - 1) nb[3] = c + nx;
                if (k > 0) nb[4] = c - (long long)nx * ny;
                if (k < nz - 1) nb[5] = c + (long long)nx * ny;
                for (int q = 0; q < 6; ++q)
                    if (nb[q] >= 0 && !(g->mask && g->mask[nb[q]])) s -= x[nb[q]];
                y[c] = s;
            }
}

int orc_poisson_cg(int nx, int ny, int nz, double h, const double *rho, const uint8_t *mask,
                   double v_mask, double v_lo, double v_hi, double *phi, double rtol, int max_iter,
                   double *rel_res, int *iters)
{
    pgrid g = {nx, ny, nz, h, mask};
    long long n = (long long)nx * ny * nz;
    double *b = calloc((size_t)n, sizeof(double)), *r = calloc((size_t)n, sizeof(double));
    double *z = calloc((size_t)n, sizeof(double)), *pp = calloc((size_t)n, sizeof(double));
    double *Ap = calloc((size_t)n, sizeof(double)), *dg = calloc((size_t)n, sizeof(double));
    if (!b || !r || !z || !pp || !Ap || !dg) return -2;
    /* right-hand side: h^2 rho / eps0 + Dirichlet plate terms + electrode neighbours */
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                long long c = ((long long)k * ny + j) * nx + i;
                if (mask && mask[c]) { phi[c] = v_mask; continue; }
                double s = h * h * rho[c] / EPS_0;
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
                b[c] = s;
                dg[c] = diag_of(&g, i, j, k);
            }
    double *x = calloc((size_t)n, sizeof(double));
    for (long long c = 0; c < n; ++c) x[c] = (mask && mask[c]) ? 0.0 : phi[c];
    apply_A(&g, x, Ap);
    double bn = 0.0, rz = 0.0, rn = 0.0;
    for (long long c = 0; c < n; ++c) {
        if (mask && mask[c]) { r[c] = z[c] = pp[c] = 0.0; continue; }
        r[c] = b[c] - Ap[c];
        z[c] = r[c] / dg[c];
        pp[c] = z[c];
        bn += b[c] * b[c];
        rz += r[c] * z[c];
        rn += r[c] * r[c];
    }
    bn = sqrt(bn);
    if (bn == 0.0) bn = 1.0;
    int it = 0;
    while (sqrt(rn) / bn > rtol && it < max_iter) {
        apply_A(&g, pp, Ap);
        double pAp = 0.0;
        for (long long c = 0; c < n; ++c) pAp += pp[c] * Ap[c];
        double alpha = rz / pAp;
        double rz2 = 0.0;
        rn = 0.0;
        for (long long c = 0; c < n; ++c) {
            if (mask && mask[c]) continue;
            x[c] += alpha * pp[c];
            r[c] -= alpha * Ap[c];
            z[c] = r[c] / dg[c];
            rz2 += r[c] * z[c];
            rn += r[c] * r[c];
        }
        double beta = rz2 / rz;
        rz = rz2;
        for (long long c = 0; c < n; ++c) pp[c] = (mask && mask[c]) ? 0.0 : z[c] + beta * pp[c];
        ++it;
    }
    /* true residual */
    apply_A(&g, x, Ap);
    rn = 0.0;
    for (long long c = 0; c < n; ++c) {
        if (mask && mask[c]) continue;
        double d = b[c] - Ap[c];
        rn += d * d;
        phi[c] = x[c];
    }
    *rel_res = sqrt(rn) / bn;
    *iters = it;
    free(b); free(r); free(z); free(pp); free(Ap); free(dg); free(x);
    return 0;
}

/* E = -grad(phi) at cell centres by central differences, with the same ghost
 * values as the Poisson stencil (Neumann: mirror; Dirichlet: 2 phi_b - phi). */
/* ------------------------------------------------------------------------ */
/* Axisymmetric Poisson (Sec. 2.5 in the axisymmetric geometry of Sec. 2.1.2):  */
/* -(1/r) d/dr (r dphi/dr) - d2phi/dz2 = rho / eps0 on nr x nz square ring     */
/* cells of side h, cell i at r = (i + 1/2) h.  Integrating over the ring cell */
/* and dividing by 2 pi h gives a symmetric system: face coefficients r_face/h */
/* = i (inner, zero on the axis), i + 1 (outer), i + 1/2 (each axial face);    */
/* right-hand side (i + 1/2) h^2 rho / eps0.  Outer cylinder: no flux; z faces */
/* Dirichlet v_lo, v_hi (ghost 2v - phi); mask cells at v_mask.  Solved by CG  */
/* with a Jacobi preconditioner (deliberately not multigrid) to ||r||/||b|| <= */
/* rtol.  Pins: plates only gives phi linear in z; the discrete Gauss law (the */
/* boundary fluxes balance the charge); O(h^2) convergence to a Bessel-sine    */
/* manufactured solution.                                                     */
/* ------------------------------------------------------------------------ */
typedef struct { int nr, nz; const uint8_t *mask; } agrid;

static void axi_coef(int i, int nr, double *ci, double *co, double *cz)
{
    *ci = (double)i;
    *co = (i + 1 < nr) ? (double)(i + 1) : 0.0;
    *cz = (double)i + 0.5;
}

/* y = A x on the unmasked unknowns (homogeneous boundary values). */
static void axi_apply(const agrid *g, const double *x, double *y)
{
    for (int k = 0; k < g->nz; ++k)
        for (int i = 0; i < g->nr; ++i) {
            long long c = (long long)k * g->nr + i;
            if (g->mask && g->mask[c]) { y[c] = 0.0; continue; }
            double ci, co, cz;
            axi_coef(i, g->nr, &ci, &co, &cz);
            double diag = ci + co + 2.0 * cz + (k == 0 ? cz : 0.0) + (k == g->nz - 1 ? cz : 0.0);
            double v = diag * x[c];
            if (i > 0 && !(g->mask && g->mask[c - 1])) v -= ci * x[c - 1];
            if (i + 1 < g->nr && !(g->mask && g->mask[c + 1])) v -= co * x[c + 1];
            if (k > 0 && !(g->mask && g->mask[c - g->nr])) v -= cz * x[c - g->nr];
            if (k + 1 < g->nz && !(g->mask && g->mask[c + g->nr])) v -= cz * x[c + g->nr];
            y[c] = v;
        }
}

int orc_poisson_axi(int nr, int nz, double h, const double *rho, const uint8_t *mask, double v_mask,
                    double v_lo, double v_hi, double *phi, double rtol, int max_iter, double *rel_res,
                    int *iters)
{
    agrid g = {nr, nz, mask};
    long long n = (long long)nr * nz;
    double *b = calloc((size_t)n, sizeof(double)), *r = calloc((size_t)n, sizeof(double));
    double *z = calloc((size_t)n, sizeof(double)), *pp = calloc((size_t)n, sizeof(double));
    double *q = calloc((size_t)n, sizeof(double)), *dg = calloc((size_t)n, sizeof(double));
    if (!b || !r || !z || !pp || !q || !dg) return -2;
    double h2e = h * h / EPS_0;
    for (int k = 0; k < nz; ++k)
        for (int i = 0; i < nr; ++i) {
            long long c = (long long)k * nr + i;
            if (mask && mask[c]) { phi[c] = v_mask; continue; }
            double ci, co, cz;
            axi_coef(i, nr, &ci, &co, &cz);
            dg[c] = ci + co + 2.0 * cz + (k == 0 ? cz : 0.0) + (k == nz - 1 ? cz : 0.0);
            double bb = cz * h2e * rho[c];
            if (k == 0) bb += 2.0 * cz * v_lo;
            if (k == nz - 1) bb += 2.0 * cz * v_hi;
            if (mask) {
                if (i > 0 && mask[c - 1]) bb += ci * v_mask;
                if (i + 1 < nr && mask[c + 1]) bb += co * v_mask;
                if (k > 0 && mask[c - nr]) bb += cz * v_mask;
                if (k + 1 < nz && mask[c + nr]) bb += cz * v_mask;
            }
            b[c] = bb;
        }
    axi_apply(&g, phi, q);
    double bn = 0.0, rz = 0.0;
    for (long long c = 0; c < n; ++c) {
        if (mask && mask[c]) { r[c] = 0.0; z[c] = 0.0; pp[c] = 0.0; continue; }
        r[c] = b[c] - q[c];
        z[c] = r[c] / dg[c];
        pp[c] = z[c];
        rz += r[c] * z[c];
        bn += b[c] * b[c];
    }
    bn = sqrt(bn);
    if (bn == 0.0) bn = 1.0;
    int it = 0;
    double rn = 0.0;
    for (; it < max_iter; ++it) {
        rn = 0.0;
        for (long long c = 0; c < n; ++c) rn += r[c] * r[c];
        rn = sqrt(rn);
        if (rn / bn <= rtol) break;
        axi_apply(&g, pp, q);
        double pq = 0.0;
        for (long long c = 0; c < n; ++c) pq += pp[c] * q[c];
        double alpha = rz / pq;
        for (long long c = 0; c < n; ++c) {
            if (mask && mask[c]) continue;
            phi[c] += alpha * pp[c];
            r[c] -= alpha * q[c];
        }
        double rz2 = 0.0;
        for (long long c = 0; c < n; ++c) {
            if (mask && mask[c]) continue;
            z[c] = r[c] / dg[c];
            rz2 += r[c] * z[c];
        }
        double beta = rz2 / rz;
        rz = rz2;
        for (long long c = 0; c < n; ++c) pp[c] = (mask && mask[c]) ? 0.0 : z[c] + beta * pp[c];
    }
    *rel_res = rn / bn;
    *iters = it;
    free(b); free(r); free(z); free(pp); free(q); free(dg);
    return it < max_iter ? 0 : -5;
}

/* E_r, E_z at cell centres: central differences, mirror at the axis and the
 * outer cylinder, Dirichlet ghosts at the plates. */
void orc_grad_axi(int nr, int nz, double h, const double *phi, double v_lo, double v_hi, double *Er, double *Ez)
{
    for (int k = 0; k < nz; ++k)
        for (int i = 0; i < nr; ++i) {
            long long c = (long long)k * nr + i;
            double pc = phi[c];
            double rm = i > 0 ? phi[c - 1] : pc, rp = i + 1 < nr ? phi[c + 1] : pc;
            double zm = k > 0 ? phi[c - nr] : 2.0 * v_lo - pc, zp = k + 1 < nz ? phi[c + nr] : 2.0 * v_hi - pc;
            Er[c] = -(rp - rm) / (2.0 * h);
            Ez[c] = -(zp - zm) / (2.0 * h);
        }
}

/* Densities of ring cells: n = q / (2^32 pi (2i + 1) dx^3) (the volume 2 pi r dr dz
 * of Sec. 2.1.2 at r = (i + 1/2) dx); rho = e (n_pos - n_neg - n_e). */
void orc_fixed_to_rho_axi(int nr, int nz, double dx, const int64_t *q_e, const int64_t *q_pos,
                          const int64_t *q_neg, double *rho)
{
    for (int k = 0; k < nz; ++k)
        for (int i = 0; i < nr; ++i) {
            long long c = (long long)k * nr + i;
            double inv = 1.0 / (4294967296.0 * (M_PI_ORC * (double)(2 * i + 1) * dx * dx * dx));
            double ne = (double)q_e[c] * inv, np = (double)q_pos[c] * inv, nn = (double)q_neg[c] * inv;
            rho[c] = Q_E * (np - nn - ne);
        }
}

void orc_grad_phi(int nx, int ny, int nz, double h, const double *phi, double v_lo, double v_hi,
                  double *Ex, double *Ey, double *Ez)
{
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                long long c = ((long long)k * ny + j) * nx + i;
                double pc = phi[c];
                double xm = i > 0 ? phi[c - 1] : pc, xp = i < nx - 1 ? phi[c + 1] : pc;
                double ym = j > 0 ? phi[c - nx] : pc, yp = j < ny - 1 ? phi[c + nx] : pc;
                double zm = k > 0 ? phi[c - (long long)nx * ny] : 2.0 * v_lo - pc;
                double zp = k < nz - 1 ? phi[c + (long long)nx * ny] : 2.0 * v_hi - pc;
                Ex[c] = -(xp - xm) / (2.0 * h);
                Ey[c] = -(yp - ym) / (2.0 * h);
                Ez[c] = -(zp - zm) / (2.0 * h);
            }
}

/* ------------------------------------------------------------------------ */
/* Monte Carlo swarm in a uniform field (Sec. 2.2.2): electrons start        */
/* Maxwellian at the origin and are traced with the same mover and          */
/* collisions; weighted moments are taken at the end of every step.         */
/* Adaptive resampling at the start of a step: above n_hi each electron      */
/* survives with probability 1/2; below n_lo every electron is duplicated.   */
/* Weights are left as they are: every coefficient is built from ratios of   */
/* moments of the same step, so the swarm's overall weight scale (which     */
/* grows like e^{nu t} in an ionizing field) is implicit and never overflows. */
/* Moments per step (row of ORC_NMOM):                                       */
/*  0 sw, 1 swx, 2 swy, 3 swz, 4 swx2, 5 swy2, 6 swz2, 7 swvx, 8 swvy, 9 swvz, */
/*  10 swxvx, 11 swyvy, 12 swzvz, 13 sw eps, 14 ionization weight in step,   */
/*  15 attachment weight in step.                                            */
/* ------------------------------------------------------------------------ */
typedef struct orc_swarm_cfg {
    long long n0, n_lo, n_hi;
    int n_steps;
    double kT_eV;
} orc_swarm_cfg;

int orc_swarm_run(const orc_setup *s, const orc_swarm_cfg *c, orc_parts *p, double *mom,
                  long long *n_per_step)
{
    int rc = orc_seed_maxwell(s, c->n0, c->kT_eV, p);
    if (rc) return rc;
    orc_stats st;
    for (int step = 1; step <= c->n_steps; ++step) {
        /* resampling decision from the count at the end of the previous step */
        long long n = p->n;
        if (n > c->n_hi) {
            for (long long i = 0; i < n; ++i) {
                double u[4];
                draw(s->seed, p->id[i], (uint32_t)step, 0xA0000000u, u);
                if (!(u[0] < 0.5)) p->w[i] = 0.0;
            }
            compact(p);
        } else if (n > 0 && n < c->n_lo) {
            for (long long i = 0; i < n; ++i) {
                double x[3] = {p->x[i], p->y[i], p->z[i]}, v[3] = {p->vx[i], p->vy[i], p->vz[i]},
                       a[3] = {p->ax[i], p->ay[i], p->az[i]};
                uint64_t nid = derived_id(s->seed, p->id[i], (uint32_t)step, 0xA0000000u);
                if (append(p, x, v, a, p->w[i], nid) != 0) return -3;
            }
        }
        /* uniform field: a is constant, so the Verlet correction vanishes */
        rc = orc_step(s, p, (uint32_t)step, 1, NULL, NULL, NULL, &st);
        if (rc) return rc;
        double *m = mom + (size_t)(step - 1) * ORC_NMOM;
        for (int q = 0; q < ORC_NMOM; ++q) m[q] = 0.0;
        for (long long i = 0; i < p->n; ++i) {
            double w = p->w[i], x = p->x[i], y = p->y[i], z = p->z[i];
            double vx = p->vx[i], vy = p->vy[i], vz = p->vz[i];
            double v3[3] = {vx, vy, vz};
            m[0] += w; m[1] += w * x; m[2] += w * y; m[3] += w * z;
            m[4] += w * x * x; m[5] += w * y * y; m[6] += w * z * z;
            m[7] += w * vx; m[8] += w * vy; m[9] += w * vz;
            m[10] += w * x * vx; m[11] += w * y * vy; m[12] += w * z * vz;
            m[13] += w * energy_eV(v3);
        }
        m[14] = st.w_ion;
        m[15] = st.w_att;
        if (n_per_step) n_per_step[step - 1] = p->n;
    }
    return 0;
}

/* Flux and bulk coefficients from the moment rows (Sec. 2.2.2; flux = mean  */
/* of per-electron averages, bulk = rate of change of the centre of mass and */
/* of the spread, rate coefficients = mean over steps of the event weight of */
/* the step per N and per time integral of the swarm weight over the step).  */
/* Rows i0..n_steps-1 are used (earlier ones are relaxation).               */
/* out[0..10]  W_flux, W_bulk, DL_flux, DT_flux, DL_bulk, DT_bulk, <eps>,     */
/*             k_ion, k_att, alpha, eta                                       */
/* out[11..21] 1-sigma errors by 10-block batch means                        */
/* Pins: constant-nu closed forms (W = eE/(m nu), D_T = <vx^2>/nu, ...).       */
/* Time integral of the swarm weight over one step, divided by dt.  Within a */
/* step only collisions change the weight: it starts at W_end - (ionization */
/* weight) + (attachment weight) and ends at W_end.  The logarithmic mean of */
/* the two is exact when the weight grows or decays exponentially over the   */
/* step (a constant net rate); equal ends give the weight itself.            */
static double step_mean_weight(const double *m)
{
    double w1 = m[0], w0 = m[0] - m[14] + m[15];
    if (!(w0 > 0.0) || !(w1 > 0.0)) return 0.5 * (w0 + w1);
    if (fabs(w1 - w0) <= 1e-9 * w1) return 0.5 * (w0 + w1);
    return (w1 - w0) / log(w1 / w0);
}

static void coeffs_range(const double *mom, int r0, int r1, double dt, double n_gas, double *o)
{
    int n = r1 - r0;
    double wf = 0, dlf = 0, dtf = 0, me = 0, sion = 0, satt = 0, sw = 0;
    double st = 0, stt = 0, sz = 0, stz = 0, sl = 0, stl = 0, str = 0, sttr = 0;
    for (int r = r0; r < r1; ++r) {
        const double *m = mom + (size_t)r * ORC_NMOM;
        double W = m[0];
        double mx = m[1] / W, my = m[2] / W, mz = m[3] / W;
        double mvx = m[7] / W, mvy = m[8] / W, mvz = m[9] / W;
        wf += mvz;
        dlf += m[12] / W - mz * mvz;
        dtf += 0.5 * ((m[10] / W - mx * mvx) + (m[11] / W - my * mvy));
        me += m[13] / W;
        double wm = step_mean_weight(m);
        sion += m[14] / wm; satt += m[15] / wm; sw += 1.0;
        double t = (double)(r + 1) * dt;
        double varz = m[6] / W - mz * mz;
        double vart = (m[4] / W - mx * mx) + (m[5] / W - my * my);
        st += t; stt += t * t; sz += mz; stz += t * mz; sl += varz; stl += t * varz;
        str += vart; sttr += t * vart;
    }
    double den = (double)n * stt - st * st;
    o[0] = wf / n;
    o[1] = ((double)n * stz - st * sz) / den;
    o[2] = dlf / n;
    o[3] = dtf / n;
    o[4] = 0.5 * ((double)n * stl - st * sl) / den;
    o[5] = 0.25 * ((double)n * sttr - st * str) / den;
    o[6] = me / n;
    o[7] = sion / (n_gas * dt * sw);
    o[8] = satt / (n_gas * dt * sw);
    o[9] = o[7] * n_gas / o[0];
    o[10] = o[8] * n_gas / o[0];
}

int orc_swarm_coefficients(const double *mom, int n_steps, int i0, double dt, double n_gas, double *out)
{
    int nb = 10;
    if (n_steps - i0 < 2 * nb) return -1;
    coeffs_range(mom, i0, n_steps, dt, n_gas, out);
    double blk[10][11];
    int len = (n_steps - i0) / nb;
    for (int b = 0; b < nb; ++b) coeffs_range(mom, i0 + b * len, i0 + (b + 1) * len, dt, n_gas, blk[b]);
    for (int q = 0; q < 11; ++q) {
        double mean = 0, var = 0;
        for (int b = 0; b < nb; ++b) mean += blk[b][q];
        mean /= nb;
        for (int b = 0; b < nb; ++b) var += (blk[b][q] - mean) * (blk[b][q] - mean);
        out[11 + q] = sqrt(var / (nb - 1)) / sqrt((double)nb);
    }
    return 0;
}

/* Exported views of internal steps, for pin tests. */
void orc_gather_field(const orc_setup *s, long long n, const double *x, const double *y,
                      const double *z, double *E /* [n][3] */)
{
    for (long long i = 0; i < n; ++i) gather(s, x[i], y[i], z[i], E + 3 * i);
}

void orc_rates_at_energy(const orc_setup *s, long long n, const double *e, double *out /* [n][n_proc] */)
{
    long long cl = 0;
    for (long long i = 0; i < n; ++i) rates_at(s, e[i], out + i * s->n_proc, &cl);
}

void orc_draw(uint64_t seed, uint64_t id, uint32_t step, uint32_t k, double u[4]) { draw(seed, id, step, k, u); }

uint64_t orc_derived_id(uint64_t seed, uint64_t id, uint32_t step, uint32_t tag) { return derived_id(seed, id, step, tag); }
