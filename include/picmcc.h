/*
 * picmcc.h -- C ABI of the GB300 PIC-MCC electron library.
 *
 * The library implements the particle model of Wang, Sun & Teunissen,
 * "A comparison of particle and fluid models for positive streamer
 * discharges in air" (arXiv 2110.14494), Sec. 2.1: electrons are
 * super-particles advanced with the velocity-Verlet scheme (Eqs. 1-2) and
 * collide with the neutral gas by the null-collision Monte Carlo method
 * against rates tabulated from cross sections (Sec. 2.1.1, 2.1.5); they are
 * mapped to the grid and the field is interpolated back with trilinear
 * weights (Sec. 2.1.3); weights follow Eq. 3 with merge and split
 * (Sec. 2.1.2); the field comes from Poisson's equation with the electrode
 * held at its potential (Sec. 2.5); and a uniform-field swarm mode gives
 * flux and bulk transport data (Sec. 2.2.2).
 *
 * Conventions for every call:
 *  - Status codes: PIC_OK (0) or a negative PIC_ERR_*; no exception ever
 *    crosses the ABI.  pic_last_error() gives a message for a context.
 *  - Memory: the library never allocates device memory with the CUDA
 *    allocator.  The caller passes one device workspace of the size returned
 *    by the matching *_workspace_bytes() call (alignment 256 bytes) and owns
 *    it; all device-pointer arguments are caller-owned.  Host arrays are
 *    read during the call only.  What a context creates for itself and
 *    releases in pic_destroy: CUDA events, streams used to record CUDA
 *    graphs, the recorded graphs, and (float32 coupled contexts) one pinned
 *    host block holding a copy of its device counters.  poisson_solve_noalloc
 *    uses a fixed device array inside the library (see there).
 *  - Streams: work is enqueued on the stream given at init (or per call);
 *    calls return without waiting unless they return data to the host
 *    (statistics, particle read-back, swarm results), which synchronise that
 *    stream.  One host thread per context.
 *  - Grids are cell-centred, x fastest: index (k * ny + j) * nx + i, cell
 *    (i, j, k) centred at origin + (i + 1/2, j + 1/2, k + 1/2) dx.
 */
#ifndef PICMCC_H
#define PICMCC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *pic_stream_t; /* a cudaStream_t; NULL = legacy default stream */

enum {
    PIC_OK = 0,
    PIC_ERR_ARG = -1,      /* invalid argument or configuration */
    PIC_ERR_CUDA = -2,     /* a CUDA runtime call failed */
    PIC_ERR_CAPACITY = -3, /* a particle buffer or queue ran full; the step's result is incomplete */
    PIC_ERR_OVERFLOW = -4, /* a fixed-point value left its range */
    PIC_ERR_TIMEOUT = -5,  /* an iteration limit was reached before convergence */
    PIC_ERR_STATE = -6     /* call not valid in the context's current state */
};

enum { PIC_PROC_ELASTIC = 0, PIC_PROC_EXCITATION = 1, PIC_PROC_IONIZATION = 2, PIC_PROC_ATTACHMENT = 3 };

#define PIC_MAX_PROC 16
#define PIC_SWARM_NMOM 16
#define PIC_SWARM_NRES 24

/* Neutral gas as collision processes with tabulated cross sections
 * (Sec. 2.1.5).  All pointers are host arrays read at init. */
typedef struct pic_gas {
    int n_proc;              /* 1..PIC_MAX_PROC (7 used at most by the fast table) */
    int n_bins;              /* >= 2 nodes */
    const double *eps;       /* [n_bins] node energies in eV, uniform in ln(eps) */
    const double *sigma;     /* [n_proc][n_bins] cross sections, m^2 */
    const int *kind;         /* [n_proc] PIC_PROC_* */
    const double *threshold; /* [n_proc] energy loss / ionization energy, eV */
    const double *density;   /* [n_proc] number density of the target species, m^-3 */
    const double *mass;      /* [n_proc] target mass for elastic recoil, kg (0 = infinite) */
    const int *species;      /* [n_proc] target species, 0 = N2, 1 = O2 (NULL: untagged); swarm_run reads it
                                when it is given per-swarm O2 fractions */
} pic_gas;

typedef struct pic_config {
    int precision;            /* 32 or 64: arithmetic of the particle state and push */
    int nx, ny, nz;           /* grid cells (each >= 2, at most 2046; with coupled != 0 the grid must halve
                                 down to a coarsest multigrid level of at most ~22,000 cells, e.g. every
                                 dimension a multiple of 16 for grids up to 512) */
    double dx;                /* cell size, m */
    double origin[3];         /* lower corner, m */
    long long capacity;       /* particle slots per buffer (two buffers are kept) */
    unsigned long long seed;  /* key of all random streams */
    double dt;                /* time step, s */
    pic_gas gas;
    int n_ppc;                /* desired particles per cell, Eq. 3 (paper: 75) */
    double w_min;             /* minimum desired weight (paper: 1) */
    double growth_trigger;    /* weight update when N > trigger * N_last (paper: 1.25); <= 0 disables */
    long long particle_cap;   /* predicted count above which all desired weights are raised (0 = none) */
    int boundary;             /* 0: specular reflection at domain faces, 1: absorption */
    int sort_interval;        /* sort particles by cell every this many steps (0 = never) */
    /* coupled field solve inside pic_step (Sec. 2.5); coupled = 0 keeps the field set by pic_set_field */
    int coupled;
    double v_lo, v_hi;        /* plate potentials at z = origin and z = origin + nz dx, V */
    double v_mask;            /* electrode potential, V */
    double poisson_rtol;      /* relative residual target of the coupled solve (e.g. 1e-6) */
    int poisson_max_cycles;   /* V-cycle limit per solve */
    /* time-step control (Sec. 2.1.4); adaptive_dt = 0 keeps dt fixed */
    int adaptive_dt;          /* 1: dt_next = min(dt, CFL, dielectric relaxation, growth limit) */
    double cfl;               /* dt v_90 <= cfl dx, v_90 the 90 % quantile of the speeds (paper: 0.5) */
    double mobility;          /* electron mobility for dt_drt = eps0 / (e n_e,max mu_e), m^2/(V s) */
    double max_growth;        /* electrons may grow by at most this factor per step (paper: 1.2) */
    /* photoionization (Sec. 2.4): discrete Monte Carlo photons.  Each ionization
     * by an electron of weight w emits, with probability xi p_q / (p + p_q), one
     * photon of weight w in an isotropic direction; its absorption distance
     * follows Zheleznyak's function f(r) = (exp(-a r) - exp(-b r)) / (r ln(b/a)),
     * a = chi_min p_O2, b = chi_max p_O2.  A photon absorbed inside the domain
     * and outside the electrode creates an electron at rest and a positive ion
     * there (after the step).  photo_xi = 0 disables it; it needs a grid. */
    double photo_xi;          /* proportionality factor xi (paper: 0.075) */
    double photo_pq;          /* quenching pressure p_q, Pa (paper: 40 mbar = 4000 Pa) */
    double pressure;          /* gas pressure p, Pa */
    double p_o2;              /* O2 partial pressure, Pa */
    double chi_min, chi_max;  /* absorption coefficients per O2 pressure, 1/(m Pa) (Zheleznyak:
                                 0.035 and 2 per mm Torr = 0.2625 and 15.0 per m Pa) */
    /* geometry 1: axisymmetric (Sec. 2.1.1-2.1.2).  Electrons still move in 3D
     * (x, y, z); the field, densities and electrode live on an (r, z) mesh of
     * nx radial cells from the axis x = y = 0 (origin[0] = origin[1] = 0,
     * ny = 1).  The gathered field is projected, a = (a_r x/r, a_r y/r, a_z);
     * deposits go to ring cells of volume 2 pi r dr dz; the coupled solve is
     * the axisymmetric Poisson equation (see poisson_axi_solve); domain faces
     * are the cylinder r = nx dx and the z planes. */
    int geometry;             /* 0: 3D Cartesian, 1: axisymmetric */
    int weight_interval;      /* also update weights every this many steps (paper: 10 in axisymmetric runs;
                                 0 = only on growth) */
} pic_config;

/* Host-side particle arrays (float64, any n).  Positions m, velocities m/s,
 * accelerations m/s^2 (the a(t) of Eq. 2 carried between steps), weights. */
typedef struct pic_particles_host {
    double *x, *y, *z, *vx, *vy, *vz, *ax, *ay, *az, *w;
    uint64_t *id;
} pic_particles_host;

typedef struct pic_step_stats {
    long long n_start, n_end;          /* live particles before the first / after the last step */
    long long n_events;                /* candidate collisions that fell inside the step */
    long long n_null;                  /* of which null */
    long long n_coll[PIC_MAX_PROC];    /* real collisions per process */
    long long n_children, n_attached, n_absorbed, n_clamped;
    long long n_processed;             /* particle-updates (parents + children) */
    long long n_weight_updates;        /* merge/split passes run */
    long long n_sorts;
    double w_ion, w_att, w_absorbed;   /* weights of ionization / attachment / absorption events */
    int poisson_cycles;                /* V-cycles of the last coupled solve */
    double poisson_rel_res;
    double dt_last;                    /* time step of the last step, s */
    double t_total;                    /* simulated time since init, s */
    double ne_max;                     /* largest cell electron density after the last step, m^-3 */
    long long n_photo;                 /* photoelectrons created (photons absorbed in the gas) */
} pic_step_stats;

typedef struct pic_ctx pic_ctx;

/* Workspace size for pic_init (bytes); 0 when cfg is invalid (a size, the
 * precision, the gas tables, or a coupled grid the multigrid cannot halve). */
size_t pic_workspace_bytes(const pic_config *cfg);

/* Creates a context over caller memory.  d_mask: [nz][ny][nx] electrode
 * cells (non-zero = conductor) in device memory, or NULL; it must outlive the
 * context.  Builds the rate table (Sec. 2.1.1: nu_k = N_k sigma_k v) on the
 * device; the particle set starts empty and ion grids at zero. */
int pic_init(const pic_config *cfg, void *d_workspace, size_t workspace_bytes, const uint8_t *d_mask,
             pic_stream_t stream, pic_ctx **out);

/* Releases what the context created (see Memory above); the caller's
 * workspace and mask are not touched.  NULL is ignored.  Synchronise the
 * stream first if work of the context may still be running. */
void pic_destroy(pic_ctx *ctx);
/* Message of the last failed call on ctx (valid until the next call on
 * ctx); "null context" for NULL. */
const char *pic_last_error(const pic_ctx *ctx);
/* Static text of a status code. */
const char *pic_status_string(int status);

/* Gaussian neutral seed (Sec. 2.3, Eq. 7 with a negative exponent):
 * n(r) = n0 exp(-|r - center|^2 / radius^2).  Each cell outside the
 * electrode gets floor(n dV / w0) particles plus one with probability equal
 * to the remainder, uniform in the cell, at rest, weight w0; the positive-ion
 * grid receives the same deposit.  Replaces the particle set. */
int pic_seed_gaussian(pic_ctx *ctx, double n0, double radius, const double center[3], double w0,
                      long long *n_out);

/* Replaces the particle set with n host particles (float64 arrays of n
 * entries, converted to the context precision; ids must be unique).
 * x, y, z, w and id are required; any of vx..az may be NULL (zero).
 * accel_valid != 0: ax, ay, az hold each particle's a(t) of Eq. 2 and the
 * first step completes its velocity-Verlet half-kick; 0: the first step
 * starts from the gathered field without one.  Synchronises.  Errors:
 * PIC_ERR_ARG (a required array NULL, n < 0), PIC_ERR_CAPACITY
 * (n > capacity). */
int pic_set_particles(pic_ctx *ctx, long long n, const pic_particles_host *p, int accel_valid);

/* Copies the particles of positive weight, in buffer order, to float64 host
 * arrays of at least `cap` entries (NULL arrays are skipped) and writes their
 * number to n_out; with p == NULL only the number.  Synchronises.  Errors:
 * PIC_ERR_CAPACITY when there are more than cap (nothing copied). */
int pic_get_particles(pic_ctx *ctx, pic_particles_host *p, long long cap, long long *n_out);

/* Sets the cell-centred field (V/m) that the trilinear gather of Sec. 2.1.3
 * interpolates, from device arrays [nz][ny][nx] of float; with Ex == NULL
 * the field is uniform and equal to E_uniform (host, 3 values).  The arrays
 * are read by stream-ordered work: keep them unchanged until the stream has
 * passed this call.  Errors: PIC_ERR_ARG (Ey or Ez NULL with Ex set, or no
 * E_uniform without Ex). */
int pic_set_field(pic_ctx *ctx, const float *Ex, const float *Ey, const float *Ez, const double E_uniform[3]);

/* The same from float64 device arrays: a float64 context gathers from them
 * unrounded, a float32 context from their rounding to float. */
int pic_set_field_f64(pic_ctx *ctx, const double *Ex, const double *Ey, const double *Ez,
                      const double E_uniform[3]);

/* Advances all electrons n_steps times (Sec. 2.1): trilinear gather, Verlet
 * half-kick completing Eq. 2, collisional flight over dt with the
 * null-collision method, children finishing the step, reflection at the
 * domain faces, absorption by the electrode, fixed-point deposit of electrons
 * and of ion-producing events; on schedule the cell sort and the weight
 * update (Sec. 2.1.2); with cfg.coupled the space charge and Poisson solve
 * that give the next step's field.  stats (host, optional) accumulates over
 * the n_steps and synchronises the stream.  Each step reads the device
 * counters once after its collisions (and reports any error flag then);
 * without stats the call returns once the last step's field solve is
 * enqueued.  Float32 Cartesian coupled contexts enqueue that solve before
 * the read (the counters are copied to pinned host memory behind an event)
 * and undo it when the counts call for a weight update or further product
 * generations: the results are those of the unspeculated order, bit for bit.
 * A field solve's own error flag (cycle limit) is reported by the next call
 * that reads the counters. */
int pic_step(pic_ctx *ctx, int n_steps, pic_step_stats *stats);

/* Coupled solve settings of a live context (Sec. 2.5): the relative residual
 * target, the V-cycle limit per solve, and how float32 contexts drive their
 * iterations.  device_loop != 0 (the default): from the third solve on, each
 * solve is one CUDA graph whose conditional nodes run the CG loop on the
 * device, without host synchronisation; a solve that reaches max_cycles
 * raises a device flag that pic_step reports as PIC_ERR_TIMEOUT when it next
 * reads the device state (after the collisions of the next step, or before
 * returning when statistics are asked for).  device_loop == 0:
 * the host reads the residual after every iteration and fails at once.  Both
 * take the same decisions on the same values, so they give identical
 * results.  Float64 and axisymmetric contexts always drive from the host.
 * rtol must be positive and max_cycles at least 1; errors: PIC_ERR_ARG. */
int pic_set_poisson(pic_ctx *ctx, double rtol, int max_cycles, int device_loop);

/* Smoothing of the V-cycle that preconditions the Cartesian coupled solve
 * (Sec. 2.5): pre_sweeps red-black Gauss-Seidel sweeps before each
 * restriction and post_sweeps after each prolongation, on every level
 * (default 2 and 2).  Fewer sweeps make each CG iteration cheaper and may
 * need more iterations for the same rtol; the solution's tolerance is
 * unchanged.  Each in 1..4; errors: PIC_ERR_ARG, PIC_ERR_STATE for an
 * axisymmetric context (its solve keeps V(2,2)). */
int pic_set_multigrid(pic_ctx *ctx, int pre_sweeps, int post_sweeps);

/* Deposits the current electrons (Sec. 2.1.3, cell-centred trilinear
 * weights in 64-bit fixed point) and returns the fixed-point grids (units of
 * 2^-32 physical particles per cell, int64) and the space charge
 * rho = e (n_pos - n_neg - n_e) in C/m^3 of Sec. 2.5.  Any output may be
 * NULL; all are device arrays [nz][ny][nx].  Synchronises and reports device
 * error flags (PIC_ERR_OVERFLOW for a fixed-point overflow). */
int pic_deposit(pic_ctx *ctx, int64_t *q_e, int64_t *q_pos, int64_t *q_neg, double *rho);

/* Copies the fixed-point grids as the last step left them, without a new
 * deposit: q_e is the electron deposit the step's own kernels made at its end
 * (Sec. 2.1.3; made again after a weight update), which is the charge a
 * coupled solve used for the next field, and q_pos, q_neg are the ion grids.
 * Device arrays [nz][ny][nx] of int64 (units of 2^-32 particles), any may be
 * NULL.  Stream-ordered, does not synchronise.  Before the first step q_e
 * holds whatever the last pic_deposit (or nothing: zeros) left. */
int pic_get_deposit(pic_ctx *ctx, int64_t *q_e, int64_t *q_pos, int64_t *q_neg);

/* Copies the cell-centred field (V/m) that the next step's trilinear gather
 * (Sec. 2.1.3) reads into device float64 arrays [nz][ny][nx] (exact: the
 * field is held in the context precision): the one given to pic_set_field,
 * or in a coupled context the one solved from the charge of the last step
 * (Sec. 2.5); pic_step with 0 steps makes a coupled context solve its first
 * field.  Axisymmetric contexts give E_r, 0, E_z on [nz][1][nx].  Any output
 * may be NULL.  Stream-ordered, does not synchronise.  Errors:
 * PIC_ERR_STATE when the context has no field grid (none set yet, or a
 * uniform field). */
int pic_get_field(pic_ctx *ctx, double *Ex, double *Ey, double *Ez);

/* Runs the super-particle weight update now (Sec. 2.1.2, Eq. 3): cell sort,
 * merge and split, compaction; reads the predicted count back
 * (synchronises).  Errors: PIC_ERR_CAPACITY when splitting would exceed the
 * capacity. */
int pic_weight_update(pic_ctx *ctx);

/* Number of particles in the current set, zero-weight slots awaiting
 * compaction included (synchronises). */
int pic_count(pic_ctx *ctx, long long *n);

/* Cumulative particle-updates (parents plus queued children advanced), of
 * which parents, and steps since init (synchronises).  Any output may be NULL. */
int pic_progress(pic_ctx *ctx, long long *particle_updates, long long *parent_updates, long long *steps);

/* Per-phase device times, measured with CUDA events on the context stream. */
typedef struct pic_profile_times {
    double ms_push, ms_children, ms_field, ms_reorder; /* accumulated milliseconds */
    long long n_push, n_children, n_field, n_reorder;  /* timed launches / phases */
    long long n_launches;                              /* kernels pic_step launched since the last clear */
    /* float32 Cartesian coupled steps enqueue the next field solve before the
     * host reads the step's counts; a step that then needs a weight update or
     * further product generations undoes that solve and solves again */
    long long n_speculative, n_undone;                 /* such solves, and those undone */
    long long n_overlapped;                            /* pic_upload / pic_download calls that ran
                                                          under such a solve (see pic_download) */
} pic_profile_times;

/* enable != 0 starts timing (cleared); out (optional) receives the
 * accumulated times since the last clear, after which they are cleared.
 * Synchronises (the phase events are resolved). */
int pic_profile(pic_ctx *ctx, int enable, pic_profile_times *out);

/* Native-precision particle exchange with host memory (use pinned memory for
 * asynchronous copies): arrays[0..9] = x, y, z, vx, vy, vz, ax, ay, az, w in
 * the context precision (float or double), arrays[10] = uint64 ids.
 * pic_upload replaces the particle set with n particles (accel_valid as
 * for pic_set_particles; errors PIC_ERR_ARG for a null array, PIC_ERR_CAPACITY
 * for n > capacity); the host arrays are read by stream-ordered copies, so
 * keep them unchanged until the stream has passed the call.  pic_download
 * writes the current set (including any not-yet-compacted zero-weight slots,
 * which callers skip) and its size, and synchronises; PIC_ERR_CAPACITY (with
 * *n_out set, nothing copied) when the set is larger than cap.  When
 * arrays[0..9] lie at one constant pitch (one host block, rows at least n
 * elements apart) they move in one pitched copy, else in ten; the ids
 * always in one more.  Right after a pic_step whose last step's field solve
 * was enqueued speculatively (float32 Cartesian coupled contexts), with no
 * other call on the context in between, both run their copies on a
 * context-owned copy stream that waits only for that step's particles, so
 * they overlap the solve still running: pic_download then returns once the
 * particles are on the host, and pic_upload makes the context's stream wait
 * for its copies.  Results are the same either way. */
int pic_upload(pic_ctx *ctx, long long n, const void *const *arrays, int accel_valid);
int pic_download(pic_ctx *ctx, void *const *arrays, long long cap, long long *n_out);

/* Checkpoint (no passage of the paper): the particle set, ion grids,
 * potential, step counter, time-step state and flags into a host blob;
 * *bytes in: blob capacity (or 0 to query), out: size; PIC_ERR_CAPACITY when
 * the blob is too small.  pic_load restores a blob into a context created
 * with the same precision and grid (PIC_ERR_ARG otherwise); a coupled
 * context solves for its field again before the next step.  Both
 * synchronise. */
int pic_save(pic_ctx *ctx, void *host_blob, size_t *bytes);
int pic_load(pic_ctx *ctx, const void *host_blob, size_t bytes);

/* ------------------------------------------------------------------ Poisson */
/* -lap(phi) = rho / eps0 (Sec. 2.5; the sign printed there is read as a
 * typo) on the cell-centred grid: Dirichlet phi = v_lo at the z = origin
 * face and v_hi at the top face (ghost 2 phi_b - phi), homogeneous Neumann on
 * the x and y faces, cells with mask != 0 held at v_mask.  Flexible CG
 * preconditioned by a float32 geometric-multigrid V(2,2)-cycle until the
 * CG residual satisfies ||b - A phi|| / ||b|| <= rtol; the Krylov part runs
 * in float64 or, with precision 32, in float32 on a correction to a
 * float-pair potential (see poisson_config).  E = -grad(phi) by central
 * differences at cell centres (float32).  Coupled PIC contexts use the
 * float64 variant with precision 64 and the float-pair one with 32. */
typedef struct poisson_config {
    int nx, ny, nz;           /* as for pic_config with coupled != 0; unsupported sizes give PIC_ERR_ARG */
    double dx;
    double v_lo, v_hi, v_mask;
    int precision;            /* 0 or 64: CG in float64; 32: the potential as a pair of floats (about
                                 48 bits) with the correction found by CG in float32 and iterative
                                 refinement: no float64 arithmetic in the iterations.  Both use the
                                 float32 V-cycle preconditioner.  The pair residual bounds the reachable
                                 rtol near 1e-9 relative for 32. */
} poisson_config;

typedef struct poisson_stats {
    int cycles;
    double rel_res;
} poisson_stats;

/* Workspace size for poisson_solve; 0 for unsupported sizes. */
size_t poisson_workspace_bytes(const poisson_config *pc);

/* rho, mask, phi, Ex, Ey, Ez: device arrays [nz][ny][nx]; phi is the
 * initial guess on entry and the solution on return; mask may be NULL;
 * E outputs may be NULL.  Returns PIC_ERR_TIMEOUT if max_cycles ran out. */
int poisson_solve(const poisson_config *pc, const double *rho, const uint8_t *mask, double *phi,
                  float *Ex, float *Ey, float *Ez, double rtol, int max_cycles, void *d_workspace,
                  size_t workspace_bytes, poisson_stats *stats, pic_stream_t stream);

/* Axisymmetric variant (the paper's axisymmetric geometry, Sec. 2.1.1-2.1.2
 * and 2.5): -(1/r) d/dr (r dphi/dr) - d2phi/dz2 = rho / eps0 on nr x nz square
 * cells of side dx, cell i centred at r = (i + 1/2) dx from the axis; the
 * outer cylinder r = nr dx homogeneous Neumann, z faces Dirichlet v_lo / v_hi,
 * mask cells at v_mask.  Each row is the ring cell's flux balance divided by
 * 2 pi dx (symmetric); flexible CG in float64 with a float64 multigrid
 * V-cycle preconditioner until the CG residual satisfies ||b - A phi|| /
 * ||b|| <= rtol.  rho, phi: device float64 [nz][nr]; mask: device uint8
 * [nz][nr] or NULL; Er, Ez: optional device float32 [nz][nr] (both or
 * neither).  Sizes must halve to a coarsest level of at most 4096 cells.
 * Errors as poisson_solve. */
size_t poisson_axi_workspace_bytes(int nr, int nz);
int poisson_axi_solve(int nr, int nz, double dx, double v_lo, double v_hi, double v_mask, const double *rho,
                      const uint8_t *mask, double *phi, float *Er, float *Ez, double rtol, int max_cycles,
                      void *d_workspace, size_t workspace_bytes, poisson_stats *stats, pic_stream_t stream);

/* Same solve as poisson_solve, for callers that cannot allocate device
 * memory (no workspace argument): plugins handed only input and output
 * pointers by a host application that owns every allocation, and loops that
 * must not touch an allocator once running.  The paper has no counterpart:
 * this is a deployment convenience.  The multigrid scratch is a fixed 32 MiB device
 * array inside the library (held on every GPU that loads it until the
 * process exits), enough for grids of up to about 0.95 million cells (96^3
 * fits, 100^3 does not, at either precision); larger grids return
 * PIC_ERR_CAPACITY and touch nothing.  The first call on
 * a device looks up that array's device address (cudaGetSymbolAddress) with
 * the device current and keeps it for later calls on that device.  Every
 * call shares the one array: calls that can overlap
 * on the GPU (other streams, other host threads) race and must be
 * serialised by the caller.  Nothing is allocated; arguments and results are
 * as for poisson_solve. */
int poisson_solve_noalloc(const poisson_config *pc, const double *rho, const uint8_t *mask, double *phi,
                          float *Ex, float *Ey, float *Ez, double rtol, int max_cycles, poisson_stats *stats,
                          pic_stream_t stream);

/* -------------------------------------------------------------------- swarm */
/* Monte Carlo swarms in uniform fields (Sec. 2.2.2).  Each swarm starts
 * n0 electrons at the origin with Maxwellian velocities at temperature kT,
 * field E = -(E/N) N z-hat, and is advanced n_steps with the same collisions.
 * Weighted moments are accumulated at the end of every step; adaptive
 * resampling keeps counts in [n_lo, n_hi]: above n_hi each electron survives
 * with probability 1/2, below n_lo every electron is duplicated, and neither
 * changes any weight (every coefficient is a ratio of sums taken at one step,
 * in which a common weight factor cancels).
 * Results per swarm (swarm_result.v):
 *   0 W_flux  1 W_bulk  2 DL_flux  3 DT_flux  4 DL_bulk  5 DT_bulk
 *   6 <eps> (eV)  7 k_ion  8 k_att (m^3/s)  9 alpha  10 eta (1/m)
 *   11..21 one-sigma errors of 0..10 (10-block batch means)
 *   22 final particle count  23 final total weight
 * Moments per step (16): sw, swx, swy, swz, swx^2, swy^2, swz^2, swvx, swvy,
 *   swvz, swxvx, swyvy, swzvz, sw eps, ionization weight, attachment weight. */
typedef struct swarm_config {
    int precision;           /* 32 or 64 */
    pic_gas gas;
    double n_gas;            /* total gas density N for E/N and the rate coefficients, m^-3 */
    long long n0, n_lo, n_hi;
    long long capacity;      /* particle slots per swarm and buffer (>= 2 n_hi) */
    int n_steps;
    double dt;
    double kT_eV;
    unsigned long long seed; /* swarm s uses seed + s */
    double sample_from;      /* fraction of steps discarded before sampling (0.25) */
    /* batched mode: all swarms advance together over per-swarm segments of
     * shared buffers; warps take item ranges of any swarm from one cursor */
    int batched;             /* 0: swarms one after another; 1: batched */
    int block;               /* batched: threads per block (64, 128 or 256); 0 = autotune */
    int blocks_per_sm;       /* batched: resident blocks per SM; 0 = autotune */
    int use_graph;           /* batched: how the steps are launched.  0: kernels per step (resampling, prefix
                                sums, parents, three product generations, counts); 1: that step recorded once
                                in a CUDA graph and replayed; 2: one persistent kernel for every step (grid-wide
                                barriers between the phases, as many product generations as a step needs),
                                a cooperative launch recorded in a CUDA graph.  With block == 0 the autotuner
                                picks 1 or 2 too. */
    int warp_chunk;          /* batched: largest item range a warp takes at once (multiple of 32, 32..8192;
                                0 = 1024, or the autotuned value when block == 0) */
} swarm_config;

typedef struct swarm_result {
    double v[PIC_SWARM_NRES];
} swarm_result;

/* Workspace size for swarm_run and swarm_autotune; 0 for invalid input. */
size_t swarm_workspace_bytes(const swarm_config *sc, int n_swarms);

/* Batched mode only: times short trial runs of the batched step and returns
 * the fastest launch shape and its ms per step: block sizes {64, 128, 256} x
 * blocks per SM {1, 2, 3, 4, max}, then the warp item range {256, 512, 1024,
 * 2048} and the launch mode {1, 2} (see use_graph) for the best pair.  Uses
 * the same workspace and arguments as swarm_run; the trial state is
 * discarded.  Outputs may not be NULL. */
int swarm_autotune(const swarm_config *sc, int n_swarms, const double *EN_Td, const double *o2_frac,
                   void *d_workspace, size_t workspace_bytes, int *block, int *blocks_per_sm, int *warp_chunk,
                   int *use_graph, double *ms_per_step, pic_stream_t stream);

/* EN_Td: host [n_swarms]; o2_frac: host [n_swarms] O2 fractions of the gas of
 * each swarm (Sec. 2.3 uses 0.2), or NULL for the gas as given: with it, the
 * target density of process k of swarm s is n_gas (1 - o2_frac[s]) for N2
 * targets and n_gas o2_frac[s] for O2 targets (gas.species must be set;
 * PIC_ERR_ARG otherwise), and each swarm gets its own rate table and nu_max.
 * results: host [n_swarms]; moments (optional): host [n_swarms][n_steps][16];
 * counts (optional): host [n_swarms][n_steps].  Errors: PIC_ERR_CAPACITY when
 * a buffer or product queue ran full, PIC_ERR_TIMEOUT when a grid-wide
 * barrier of the persistent kernel gave up waiting (the launch ended early). */
int swarm_run(const swarm_config *sc, int n_swarms, const double *EN_Td, const double *o2_frac,
              void *d_workspace, size_t workspace_bytes, swarm_result *results, double *moments,
              long long *counts, pic_stream_t stream);

/* ---------------------------------------------------------------- surrogate */
/* Transport-data surrogate: the flux transport data that the local-field
 * fluid model reads (Sec. 2.2.4: mobility, diffusion, ionization and
 * attachment coefficients and mean energy versus the field, computed there by
 * Monte Carlo swarms) represented by a network 2 -> 128 -> 128 -> 6 with tanh
 * hidden units and a linear output, fitted to swarm_run results.  Inputs and
 * targets are standardized by the caller (two inputs: log10 E/N and the O2
 * fraction; six targets: the logarithms of mu N, D_L N, D_T N, alpha / N,
 * eta / N and the mean energy).  The 128 x 128 layer runs on the tensor cores
 * in BF16 with FP32 accumulation, everything else in FP32.
 *
 * params: device float32 [MLP_NPARAMS] in the order W1[128][2], b1[128],
 * W2[128][128], b2[128], W3[6][128], b3[6] (W[o][i] multiplies input i of
 * unit o).  x: device float32 [n][2]; y, t: device float32 [n][6].
 * Workspaces are caller-allocated, 256-byte aligned, sized by
 * mlp_workspace_bytes(n) (n = 0: forward only).  Calls are stream-ordered
 * and asynchronous.  Errors: PIC_ERR_ARG for null or misaligned pointers,
 * a short workspace or a training n that is not a multiple of 64 (of 256
 * above 256); PIC_ERR_CUDA if a launch fails. */
#define MLP_NI 2
#define MLP_NH 128
#define MLP_NO 6
#define MLP_NPARAMS 17670

size_t mlp_workspace_bytes(int n_max);

/* y = network(x) for n points (any n >= 0), on the tcgen05 tensor cores
 * with the accumulators in tensor memory (h1 and h2 rounded to BF16). */
int mlp_forward(const float *params, const float *x, float *y, long long n, void *d_workspace,
                size_t workspace_bytes, pic_stream_t stream);

/* Folds the caller's standardizations into the parameters (Sec. 2.2.4 data:
 * the network maps standardized inputs to standardized targets): out holds
 * the parameters of the same network taking raw inputs x and giving raw
 * targets, W1'[o][i] = W1[o][i] / x_scale[i], b1'[o] = b1[o] - sum_i W1[o][i]
 * x_mean[i] / x_scale[i], W3'[o][j] = W3[o][j] y_scale[o], b3'[o] = b3[o]
 * y_scale[o] + y_mean[o] (W2, b2 copied), in float64 arithmetic rounded to
 * float once.  params, out: device float32 [MLP_NPARAMS], distinct; the
 * means and scales: host arrays.  Errors: PIC_ERR_ARG (null or aliased
 * pointers, a zero or non-finite scale, a non-finite mean). */
int mlp_fold_standardization(const float *params, const double x_mean[2], const double x_scale[2],
                             const double y_mean[6], const double y_scale[6], float *out, pic_stream_t stream);

/* The network's raw inputs for transport-data queries: x[i] = (log10 EN_Td[i],
 * f_o2[i]) as float32 (the logarithm of EN_Td rounded to float, in float32
 * arithmetic).  EN_Td (Td), f_o2: device float64 [n]; x: device
 * float32 [n][2].  Errors: PIC_ERR_ARG (n < 0, null pointers with n > 0). */
int mlp_features(const double *EN_Td, const double *f_o2, float *x, long long n, pic_stream_t stream);

/* The same with the kernel chosen: variant 0 = tcgen05 (as mlp_forward),
 * 1 = warp-level mma.sync (the pre-Blackwell tensor-core path, kept for
 * comparison).  If an internal wait on the tensor cores expires (it should
 * not), the affected outputs are NaN. */
int mlp_forward_variant(const float *params, const float *x, float *y, long long n, int variant,
                        void *d_workspace, size_t workspace_bytes, pic_stream_t stream);

/* Mean squared error L = sum (y - t)^2 / (6 n) over the batch and its
 * gradient with respect to params (device float32 [MLP_NPARAMS]); loss: device
 * float32 scalar or NULL. */
int mlp_loss_grad(const float *params, const float *x, const float *t, int n, float *grad, float *loss,
                  void *d_workspace, size_t workspace_bytes, pic_stream_t stream);

/* n_steps full-batch Adam steps (Kingma & Ba 2015, Algorithm 1) on params,
 * with first and second moment estimates m, v (device float32 [MLP_NPARAMS],
 * zero before the first step) and step0 steps already taken.  loss: device
 * float32 scalar receiving the batch loss before the last update, or NULL. */
int mlp_train(float *params, float *m, float *v, int step0, const float *x, const float *t, int n, int n_steps,
              float lr, float beta1, float beta2, float eps, float *loss, void *d_workspace,
              size_t workspace_bytes, pic_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* PICMCC_H */
