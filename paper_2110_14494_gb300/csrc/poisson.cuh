// Multigrid hierarchy carved from a caller workspace (see poisson.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pic {

// State of the flexible-CG loop of a device-driven mixed solve (device
// memory): iteration index since the last refinement, cycles, decisions
// taken, cycle-limit flag, branch counts, the residual norm at the last
// refinement and the last relative residual.
// Branches of the device-driven loop: iterations 0 (first), even, odd; the
// refinement; light iterations (even, odd).
constexpr int kMxBranches = 6;
struct MxLoop {
    int it, cyc, trips, timeout;
    int n_branch[kMxBranches];
    double r_pass, rel;
};
struct MxBranchKernels {
    int k[kMxBranches];  // kernels each branch runs
};

struct MG {
    static constexpr int kMaxLevels = 12;
    int levels = 0;
    int lx[kMaxLevels], ly[kMaxLevels], lz[kMaxLevels];
    float* e[kMaxLevels];
    float* g[kMaxLevels];
    uint8_t* m[kMaxLevels];
    double* norms = nullptr;  // CG scalars: ||b||^2, ||r||^2, rho, gamma, z.r, z.q, alpha, beta
    double *r64 = nullptr, *p64 = nullptr, *q64 = nullptr;  // CG vectors (float64)
    int pre = 2, post = 2, coarse_sweeps = 4;  // coarse: red-black sweeps on the coarsest level
    // mixed solve: an iteration after the untested ones whose relative
    // residual is already within light_ratio x rtol uses a V(light_pre,
    // light_post)-cycle (0: never)
    double light_ratio = 0.0;
    int light_pre = 1, light_post = 1;
    float omega = 1.0f;          // over-relaxation of the pre- and post-smoothing sweeps (1: Gauss-Seidel)
    // mixed solve: CG iterations run before the first convergence or
    // refinement test (0 to 2; at most max_cycles).  A coupled PIC context
    // takes 2 (its warm-started solves nearly always need two), so that the
    // graph runs them without a loop trip; stateless solves take 0.
    int min_cycles = 0;
    int mixed_min_cycles(int max_cycles) const;
    int mask_min_children = 1;   // a coarse cell is an electrode cell if this many of its children are
    long long launches = 0;  // kernels launched so far
    // Reusable state for a solver owned by a long-lived caller (a PIC context):
    // the coarse masks are built once, and each CG iteration (V-cycle plus
    // vector updates) is replayed from a CUDA graph captured on a private
    // stream.  Stateless callers leave `persistent` false.
    bool persistent = false;
    bool masks_ready = false;
    cudaStream_t cap_stream = nullptr;
    cudaStream_t cap_body[3] = {nullptr, nullptr, nullptr};  // captures into conditional-node bodies
    cudaGraphExec_t g_iter[2] = {nullptr, nullptr};  // [0] first iteration, [1] later ones
    const void* g_key[3] = {nullptr, nullptr, nullptr};
    long long graph_kernels[2] = {0, 0};
    void release();
    void iteration(cudaStream_t s, double* phi, const uint8_t* mk, bool first);

    // Mixed-precision solve: float-pair potential, float32 Krylov vectors,
    // deterministic last-block reductions (scratch: ctr counters, part sums).
    bool mixed = false;
    float* d32 = nullptr;
    float* p32[2] = {nullptr, nullptr};
    float* q32 = nullptr;
    float* phi_pair = nullptr;  // pair copy for callers that hold phi in float64: hi at 0, lo 256-byte aligned after it
    unsigned* ctr = nullptr;
    double* part = nullptr;
    cudaGraphExec_t g_mx[5] = {};  // first, even, odd iterations, light even, light odd
    long long graph_kernels_mx[5] = {};
    MxLoop* loop = nullptr;
    // Creates the streams capture_solve_mixed records the loop bodies on
    // (call before the caller's capture begins).
    int prepare_capture();
    void iteration_mixed(cudaStream_t s, int it, bool light = false);
    // Records the whole mixed solve on stream cs, which must be capturing a
    // graph: the residual, a device-side while loop (a decision kernel, then
    // a switch over the first / even / odd CG iteration and the refinement),
    // the gradient and a report.  The report writes the cycles and the
    // relative residual to cycles_dst / rel_dst, ORs err_bit into *err_dst
    // when the cycle limit was reached, and adds the kernels the loop ran to
    // *kernels_dst.  No host synchronisation.  rho is h^2 rho / eps0 in
    // float; the solution goes to out (phi keeps the guess).  *fixed_kernels
    // gets the kernels recorded outside the loop.  Returns PIC_OK, or
    // PIC_ERR_CUDA when the graph could not be recorded (callers then use
    // solve_mixed).
    int capture_solve_mixed(cudaStream_t cs, const float* rho, float* phi_hi, float* phi_lo, float* out_hi,
                            float* out_lo, double h, double v_lo, double v_hi, double v_mask, double rtol,
                            int max_cycles, float* E4, int* cycles_dst, double* rel_dst, unsigned* err_dst,
                            unsigned err_bit, unsigned long long* kernels_dst, long long* fixed_kernels);
    // out = 2 cur - prev (have_prev) or cur, pair format: the warm start.
    void extrapolate_pair(const float* cur_hi, const float* cur_lo, const float* prev_hi, const float* prev_lo,
                          float* out_hi, float* out_lo, int n, bool have_prev, cudaStream_t s);
    // rho: h^2 rho / eps0 as float (rho64 false) or rho as float64 (rho64
    // true).  phi (pair) is the initial guess; with out_hi set the solution
    // goes there and phi keeps the guess, else phi is updated in place.
    // fix_mask: set phi = v_mask on electrode cells first (needed once per
    // potential buffer; later solves keep it).
    int solve_mixed(const void* rho, bool rho64, const uint8_t* mask, float* phi_hi, float* phi_lo, float* out_hi,
                    float* out_lo, bool fix_mask, double h, double v_lo, double v_hi, double v_mask, double rtol, int max_cycles,
                    float* E4, float* Ex, float* Ey, float* Ez, cudaStream_t s, int* cycles_out, double* rel_out,
                    double* host_norms);

    void plan(int nx, int ny, int nz);
    // The coarsest level must be small enough for the single-block tail
    // (its cells and those of nothing else fit in shared memory).
    static bool supported(int nx, int ny, int nz);
    // Workspace of the float64 solve (mixed false) or of the mixed one
    // (pair_copy: with room for the pair copy of a float64 potential).
    static size_t bytes(int nx, int ny, int nz, bool mixed = false, bool pair_copy = false);
    size_t carve(void* base, int nx, int ny, int nz, bool mixed = false, bool pair_copy = false);
    cudaError_t build_masks(const uint8_t* mask, cudaStream_t s);
    void vcycle(cudaStream_t s, bool light);
    int tail_level() const;
    // Returns PIC_OK, PIC_ERR_TIMEOUT or PIC_ERR_CUDA.  packed_prec selects the
    // element type (32: float, 64: double) of the optional packed field E4.
    int solve(const double* rho, const uint8_t* mask, double* phi, double h, double v_lo, double v_hi, double v_mask,
              double rtol, int max_cycles, int packed_prec, void* E4, float* Ex, float* Ey, float* Ez,
              cudaStream_t s, int* cycles_out, double* rel_out, double* host_norms);
};

}  // namespace pic
