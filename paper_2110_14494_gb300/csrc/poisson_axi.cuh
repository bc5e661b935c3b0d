// Axisymmetric Poisson solve on an (r, z) mesh (see poisson_axi.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pic {

// Loop state of a device-driven axisymmetric solve (device memory).
struct AxiLoop {
    int cyc, trips, timeout, pad;
    int n_branch[2];
    double rel;
};

struct AxiMG {
    static constexpr int kMaxLevels = 14;
    int levels = 0;
    int lr[kMaxLevels], lz[kMaxLevels];
    double* e[kMaxLevels];
    double* g[kMaxLevels];
    uint8_t* m[kMaxLevels];
    double *norms = nullptr, *r = nullptr, *p = nullptr, *q = nullptr;
    int pre = 2, post = 2, coarse_sweeps = 64;
    long long launches = 0;
    bool persistent = false, masks_ready = false;
    AxiLoop* loop = nullptr;
    // CG iterations run before the first convergence test (0 to 2, at most
    // max_cycles).  0 for every caller: the coupled axisymmetric solves often
    // converge in fewer than two, where a forced pair costs more than the
    // loop trips it saves.
    int min_cycles = 0;
    int min_cycles_for(int max_cycles) const;
    cudaStream_t cap_body[2] = {nullptr, nullptr};
    // Streams for recording loop bodies (call before the caller's capture).
    int prepare_capture();
    void release();
    // Records the solve on the capturing stream cs: residual, a device-side
    // while loop (decision, then a switch over the first and the later CG
    // iterations), the gradient and a report of cycles, relative residual,
    // cycle-limit flag (err_bit into *err_dst) and the loop's kernels (added
    // to *kernels_dst).  No host synchronisation.  Returns PIC_OK or
    // PIC_ERR_CUDA / PIC_ERR_STATE (callers then use solve).
    int capture_solve(cudaStream_t cs, const double* rho, double* phi, double h, double v_lo, double v_hi,
                      double v_mask, double rtol, int max_cycles, int packed_prec, void* E4, int* cycles_dst,
                      double* rel_dst, unsigned* err_dst, unsigned err_bit, unsigned long long* kernels_dst,
                      long long* fixed_kernels);

    void plan(int nr, int nz);
    // The coarsest level is solved by one block: at most 4096 cells.
    static bool supported(int nr, int nz);
    static size_t bytes(int nr, int nz);
    size_t carve(void* base, int nr, int nz);
    cudaError_t build_masks(const uint8_t* mask, cudaStream_t s);
    void vcycle(cudaStream_t s);
    // rho: charge density (C/m^3) [nz][nr]; phi: initial guess and solution;
    // E4 (optional): packed [nz][nr][4] (E_r, 0, E_z, 0) in float (packed_prec
    // 32) or double (64); Er, Ez: optional float planes.  Returns PIC_OK,
    // PIC_ERR_TIMEOUT or PIC_ERR_CUDA.
    int solve(const double* rho, const uint8_t* mask, double* phi, double h, double v_lo, double v_hi,
              double v_mask, double rtol, int max_cycles, int packed_prec, void* E4, float* Er, float* Ez,
              cudaStream_t s, int* cycles_out, double* rel_out, double* host_norms);
};

}  // namespace pic
