// Explicit instantiation of the push launchers for one real type.
// Included once by push_f32.cu and once by push_f64.cu.
#pragma once
#include "push.cuh"
#include "swarm_batch.cuh"

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
    k_deposit<T><<<grid, 256, 0, s>>>(p, st, (T)g.ox, (T)g.oy, (T)g.oz, (T)g.dx, g.nx, g.ny, g.nz, g.axi, q, st);
    return cudaGetLastError();
}

template <class T> cudaError_t PushLaunch<T>::field_kick(const PushArgs<T>& A, int grid, cudaStream_t s) {
    k_field_kick<T><<<grid, 256, 0, s>>>(A);
    return cudaGetLastError();
}

template <class T> cudaError_t PushLaunch<T>::photo_append(const PushArgs<T>& A, int grid, cudaStream_t s) {
    k_photo_resolve<T><<<grid, 256, 0, s>>>(A);
    k_photo_append<T><<<grid, 256, 0, s>>>(A);
    k_photo_done<<<1, 1, 0, s>>>(A.st, A.cap_photo);
    return cudaGetLastError();
}

template <class T> cudaError_t PushLaunch<T>::resample(const PushArgs<T>& A, int grid, cudaStream_t s) {
    k_resample<T><<<grid, 256, 0, s>>>(A);
    k_resample_commit<<<1, 1, 0, s>>>(A.st);
    return cudaGetLastError();
}

template <class T> int BatchLaunch<T>::max_blocks_per_sm(int block) {
    constexpr bool FAST = sizeof(T) == 4;
    const size_t sm = smem(block);
    cudaFuncSetAttribute(k_batch_collide<T, FAST, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch_collide<T, FAST, false>, block, sm);
    return b > 0 ? b : 1;
}

template <class T> cudaError_t BatchLaunch<T>::init(const BatchArgs<T>& B, long long n0, double sig, cudaStream_t s) {
    k_batch_init<T><<<1, 1024, 0, s>>>(B, n0);
    const long long total = (long long)B.n_swarms * n0;
    long long g = (total + 255) / 256;
    if (g > device_sms() * 16) g = device_sms() * 16;
    k_batch_seed<T><<<(int)(g < 1 ? 1 : g), 256, 0, s>>>(B, n0, sig);
    return cudaGetLastError();
}

template <class T> cudaError_t BatchLaunch<T>::prepare(int block) {
    constexpr bool FAST = sizeof(T) == 4;
    const size_t sm = smem(block);
    cudaError_t e = cudaFuncSetAttribute(k_batch_collide<T, FAST, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_batch_collide<T, FAST, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    return e;
}

template <class T> int BatchLaunch<T>::persistent_blocks_per_sm(int block) {
    constexpr bool FAST = sizeof(T) == 4;
    const size_t sm = smem(block);
    if (cudaFuncSetAttribute(k_batch_run<T, FAST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
        return 0;
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch_run<T, FAST>, block, sm) != cudaSuccess) return 0;
    return b;
}

template <class T>
cudaError_t BatchLaunch<T>::run_persistent(const BatchArgs<T>& B, int n_steps, int block, int grid, cudaStream_t s) {
    constexpr bool FAST = sizeof(T) == 4;
    const size_t sm = smem(block);
    cudaError_t e = cudaFuncSetAttribute(k_batch_run<T, FAST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    // barrier arrivals, generation and abort flag start at zero
    e = cudaMemsetAsync(&B.bd->bar_count, 0, 3 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_batch_run<T, FAST>, B, n_steps);
}

template <class T>
cudaError_t BatchLaunch<T>::step(BatchArgs<T> B, int block, int grid, cudaStream_t s, long long* launches) {
    constexpr bool FAST = sizeof(T) == 4;
    const size_t sm = smem(block);
    k_batch_resample<T><<<device_sms() * 8, 256, 0, s>>>(B);
    k_batch_begin<T><<<1, 1024, 0, s>>>(B);
    B.gen = 0;
    k_batch_collide<T, FAST, false><<<grid, block, sm, s>>>(B);
    for (int g = 0; g < kBatchGenerations; ++g) {
        if (g > 0) k_batch_nextgen<<<1, 1, 0, s>>>(B.bd, g);
        B.gen = g;
        k_batch_collide<T, FAST, true><<<grid, block, sm, s>>>(B);
    }
    k_batch_end<T><<<1, 1024, 0, s>>>(B);
    k_batch_step_advance<<<1, 1, 0, s>>>(B.bd, kBatchGenerations - 1);
    if (launches) *launches += 5 + 2 * kBatchGenerations;
    return cudaGetLastError();
}

}  // namespace pic
