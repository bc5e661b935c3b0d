// Explicit instantiation of the push launchers for one real type.
// Included once by push_f32.cu and once by push_f64.cu.
#pragma once
#include "push.cuh"

namespace pic {

template <class T> size_t PushLaunch<T>::smem_bytes(int n_bins) {
    (void)n_bins;
    return collide_smem<T>();
}

template <class T> int PushLaunch<T>::blocks_per_sm(int mode, int n_bins) {
    constexpr bool FAST = sizeof(T) == 4;
    const size_t sm = smem_bytes(n_bins);
    int b = 0;
    if (mode == MODE_PIC) {
        cudaFuncSetAttribute(k_push<T, MODE_PIC, FAST, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_push<T, MODE_PIC, FAST, false>, kCollideThreads, sm);
    } else {
        cudaFuncSetAttribute(k_push<T, MODE_SWARM, FAST, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_push<T, MODE_SWARM, FAST, false>, kCollideThreads, sm);
    }
    return b > 0 ? b : 1;
}

template <class T, int MODE, bool FAST, bool STATS>
static cudaError_t launch_one(bool children, const PushArgs<T>& A, int grid, cudaStream_t s) {
    const size_t sm = PushLaunch<T>::smem_bytes(A.n_bins);
    cudaError_t e;
    if (children) {
        e = cudaFuncSetAttribute(k_children<T, MODE, FAST, STATS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_children<T, MODE, FAST, STATS><<<grid, kCollideThreads, sm, s>>>(A);
    } else {
        e = cudaFuncSetAttribute(k_push<T, MODE, FAST, STATS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_push<T, MODE, FAST, STATS><<<grid, kCollideThreads, sm, s>>>(A);
    }
    return cudaGetLastError();
}

template <class T>
static cudaError_t dispatch(bool children, const PushArgs<T>& A, int mode, bool stats, int grid, cudaStream_t s) {
    constexpr bool FAST = sizeof(T) == 4;  // single precision takes the total-rate early exit
    if (mode == MODE_PIC)
        return stats ? launch_one<T, MODE_PIC, FAST, true>(children, A, grid, s)
                     : launch_one<T, MODE_PIC, FAST, false>(children, A, grid, s);
    return stats ? launch_one<T, MODE_SWARM, FAST, true>(children, A, grid, s)
                 : launch_one<T, MODE_SWARM, FAST, false>(children, A, grid, s);
}

template <class T>
cudaError_t PushLaunch<T>::parents(const PushArgs<T>& A, int mode, bool stats, int grid, cudaStream_t s) {
    return dispatch<T>(false, A, mode, stats, grid, s);
}
template <class T>
cudaError_t PushLaunch<T>::children(const PushArgs<T>& A, int mode, bool stats, int grid, cudaStream_t s) {
    return dispatch<T>(true, A, mode, stats, grid, s);
}
template <class T>
cudaError_t PushLaunch<T>::deposit(const Soa<T>& p, DevState* st, const Grid& g, unsigned long long* q, int grid,
                                   cudaStream_t s) {
    k_deposit<T><<<grid, 256, 0, s>>>(p, st, (T)g.ox, (T)g.oy, (T)g.oz, (T)g.dx, g.nx, g.ny, g.nz, q, st);
    return cudaGetLastError();
}

template <class T> cudaError_t PushLaunch<T>::field_kick(const PushArgs<T>& A, int grid, cudaStream_t s) {
    k_field_kick<T><<<grid, 256, 0, s>>>(A);
    return cudaGetLastError();
}

template <class T> cudaError_t PushLaunch<T>::resample(const PushArgs<T>& A, int grid, cudaStream_t s) {
    k_resample<T><<<grid, 256, 0, s>>>(A);
    k_resample_commit<<<1, 1, 0, s>>>(A.st);
    return cudaGetLastError();
}

}  // namespace pic
