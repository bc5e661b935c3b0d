// Shared device definitions of the PIC-MCC library (sm_103a).
//
// Layouts, the counter-based random number generator and small helpers used
// by every kernel.  Physical constants are CODATA 2018.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/picmcc.h"

namespace pic {

constexpr double kQ = 1.602176634e-19;     // elementary charge, C
constexpr double kMe = 9.1093837015e-31;   // electron mass, kg
constexpr double kEps0 = 8.8541878128e-12; // vacuum permittivity, F/m
constexpr int kMaxProc = PIC_MAX_PROC;
constexpr int kTableStride = 8;            // processes per table row (7 used + total)
constexpr int kNMom = PIC_SWARM_NMOM;
constexpr unsigned kFull = 0xffffffffu;
constexpr double kPi = 3.14159265358979323846;
constexpr int kVBinsPerOctave = 6;
constexpr int kVBins = 20 * kVBinsPerOctave;  // 2^10 .. 2^30 m/s

// Speed-histogram bin of a velocity (kVBinsPerOctave bins per octave from
// 2^10 m/s, clamped to the histogram), every operation rounded on its own so
// that kernels of units compiled with and without contraction bin alike.
__device__ __forceinline__ int speed_bin(float vx, float vy, float vz) {
    const float v2 = __fadd_rn(__fadd_rn(__fmul_rn(vx, vx), __fmul_rn(vy, vy)), __fmul_rn(vz, vz));
    if (!(v2 > 0.0f)) return 0;
    const int b = (int)floorf(__fmul_rn(__fsub_rn(__fmul_rn(0.5f, log2f(v2)), 10.0f), (float)kVBinsPerOctave));
    return b < 0 ? 0 : (b >= kVBins ? kVBins - 1 : b);
}

// Error bits raised by kernels in DevState::err.
enum : unsigned {
    kErrOutCapacity = 1u,    // output particle buffer full
    kErrChildCapacity = 2u,  // child queue full
    kErrOverflow = 4u,       // fixed-point deposit out of range
    kErrStack = 8u,          // descendant stack exhausted inside one step
    kErrSplitCapacity = 16u, // merge/split output full
    kErrPhotoCapacity = 32u, // photoelectron queue full
    kErrPoissonLimit = 64u,  // a device-driven coupled solve reached its cycle limit
    kErrBarrier = 128u,      // a grid-wide barrier of a persistent kernel gave up waiting
};

// Global loads with acquire semantics at GPU scope (flags written by other
// blocks of the same launch).
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_acquire_gpu(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// ---------------------------------------------------------------- Philox4x32-10
// Ten rounds of two 32x32 -> 64-bit multiplications (multipliers 0xD2511F53,
// 0xCD9E8D57) with a Weyl key schedule (0x9E3779B9, 0xBB67AE85), as defined by
// Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy as 1, 2, 3"
// (SC'11).  Counter = (id_lo, id_hi, step, k): a particle's k-th draw in a step.
struct u32x4 { uint32_t x, y, z, w; };

__device__ __forceinline__ u32x4 philox(u32x4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        u32x4 n;
        n.x = hi1 ^ c.y ^ k0;
        n.y = lo1;
        n.z = hi0 ^ c.w ^ k1;
        n.w = lo0;
        c = n;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Stream keys: the collision stream uses the seed; derived particle ids and the
// initial seeding use the seed xor-ed with fixed words.
struct Keys {
    uint32_t mcc0, mcc1, ids0, ids1, init0, init1;
};
inline Keys make_keys(uint64_t seed) {
    Keys k;
    k.mcc0 = (uint32_t)seed;
    k.mcc1 = (uint32_t)(seed >> 32);
    k.ids0 = (uint32_t)seed ^ 0x5A5A5A5Au;
    k.ids1 = (uint32_t)(seed >> 32) ^ 0xC3C3C3C3u;
    k.init0 = (uint32_t)seed ^ 0x1B873593u;
    k.init1 = (uint32_t)(seed >> 32) ^ 0xCC9E2D51u;
    return k;
}

// Top 23 bits of a word, centred in their bin: exact in binary32 and binary64.
template <class T> __device__ __forceinline__ T unif(uint32_t w) {
    return ((T)(w >> 9) + (T)0.5) * (T)(1.0 / 8388608.0);
}

__device__ __forceinline__ u32x4 draw_words(const Keys& K, uint64_t id, uint32_t step, uint32_t k) {
    return philox(u32x4{(uint32_t)id, (uint32_t)(id >> 32), step, k}, K.mcc0, K.mcc1);
}

__device__ __forceinline__ uint64_t derived_id(const Keys& K, uint64_t id, uint32_t step, uint32_t tag) {
    u32x4 o = philox(u32x4{(uint32_t)id, (uint32_t)(id >> 32), step, tag}, K.ids0, K.ids1);
    return (uint64_t)o.x | ((uint64_t)o.y << 32);
}

// ---------------------------------------------------------------- particle SoA
// x, y, z, vx, vy, vz, ax, ay, az, w in real type T (float or double); id uint64.
template <class T> struct Soa {
    T* r[10];
    uint64_t* id;
};
enum { PX = 0, PY, PZ, VX, VY, VZ, AX, AY, AZ, PW };

// Pending ionization products (born inside a step, still to fly for t_left).
// An entry holds the collision position x, the parent's acceleration a and
// weight w, the remaining time, the parent's id and the index k of the draw
// that ionized (the product's id and direction are derived from them when the
// entry is started), and the product's speed in the VX slot.
template <class T> struct ChildQ {
    Soa<T> p;
    T* t_left;
    uint32_t* k;
};

// Per-context device counters and statistics (lives in the workspace).
struct DevState {
    unsigned long long n_in;      // particles in the current buffer
    unsigned long long n_out;     // append cursor of the other buffer
    unsigned long long n_child;   // child queue length
    unsigned long long n_extra;   // append cursor for merge/split copies
    unsigned int err;
    unsigned int resample_mode;   // swarm: 0 none, 1 thin, 2 duplicate (decided per step)
    // statistics of the last launches (reset by the host when asked)
    unsigned long long n_events, n_null, n_clamped, n_absorbed, n_attached, n_children, n_processed;
    unsigned long long n_coll[kMaxProc];
    double w_ion, w_att, w_absorbed;
    unsigned long long n_photons; // photoelectrons created
    long long pred_total;         // merge/split: predicted count in 2^-24 units
    unsigned long long n_updates; // cumulative parents + queued children advanced
    unsigned long long n_parents; // cumulative parents advanced
    unsigned long long n_fetch;   // work cursor of the parent kernel (items handed to warps)
    unsigned long long n_fetch_c; // work cursor of the children kernel
    unsigned long long n_spill;   // products spilled to the second queue (a descendant stack ran full)
    unsigned long long n_photo;   // photoelectrons queued in this step, not yet appended
    unsigned long long n_photo_src; // emitted photons queued, paths not yet drawn
    // end-of-step statistics for the time-step control
    long long qe_max;             // largest fixed-point electron deposit of a cell
    unsigned long long qe_sum;    // sum of the deposit (two's complement)
    unsigned int vhist[kVBins];   // speeds, kVBinsPerOctave bins per octave from 2^10 m/s
    // report of the last device-driven coupled solve
    int poisson_cycles, poisson_pad;
    double poisson_rel;
    unsigned long long dev_kernels;  // kernels run by device-side loops (cumulative)
    unsigned long long n_big;        // weight update: cells left to the block-per-cell merge
    unsigned long long n_occ;        // weight update: occupied cells listed
    unsigned long long n_occ_fetch;  // weight update: work cursor over the listed cells
    // gate of the float32 field-solve graph: a speculative solve (gate_spec)
    // runs only when the step needs no weight update (count <= gate_thr) and
    // no further product generations
    double gate_thr;
    int gate_spec, gate_pad;
};

// Uniform grid description (cell-centred, cubic cells).
struct Grid {
    int nx, ny, nz;
    double dx, ox, oy, oz;
    int axi;  // 1: axisymmetric (r, z) grid, nx radial cells from the axis x = y = 0, ny = 1
    __host__ __device__ long long ncell() const { return (long long)nx * ny * nz; }
};

__device__ __forceinline__ int fold_idx(int i, int n) { return i < 0 ? 0 : (i >= n ? n - 1 : i); }

template <class T> __device__ __forceinline__ T dmax(T a, T b) { return a > b ? a : b; }

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// Streaming multiprocessors of the current device, queried once per device
// (launch shapes are sized in multiples of it).  A failed query gives 1: the
// grids stay correct, only smaller.
inline int device_sms() {
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) { cudaGetLastError(); dev = 0; }
    if (cache[dev] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
            cudaGetLastError();
            n = 1;
        }
        cache[dev] = n;
    }
    return cache[dev];
}

}  // namespace pic
