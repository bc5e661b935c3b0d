// Batched swarms: many uniform-field swarms (Sec. 2.2.2) advanced together.
//
// Swarm s owns the fixed segment [s cap_s, (s+1) cap_s) of each particle
// buffer; a step's work items are the concatenation of the swarms' live
// segments (exclusive prefix sums of the counts), so one launch advances every
// swarm and warps move from swarm to swarm as they take items.  An electron's
// random streams use the key of its swarm (seed + s, as when the swarm runs
// alone), its acceleration is that of its swarm's field, and its swarm's
// counters, moments and resampling bounds apply.  All per-step bookkeeping is
// on the device (step counter, counts, prefix sums), so a step is a fixed
// sequence of launches that is captured once in a CUDA graph and replayed.
#pragma once
#include "push.cuh"

namespace pic {

constexpr int kMaxSwarms = 4096;
constexpr int kBatchGenerations = 3;  // children generations per step inside the replayed graph
constexpr int kMaxGenerations = 62;   // product generations per step of the persistent kernel

struct BatchDev {
    unsigned long long fetch, fetch_c, n_child, n_spill;
    unsigned int err;
    unsigned int step;  // the step being run (1-based)
    // persistent kernel: fetch cursors (parents, then generation g at g + 1)
    // and product counts (gcnt[g]: products queued by generation g - 1, the
    // parents at 0), zeroed at the start of every step
    unsigned long long cur[kMaxGenerations + 1];
    unsigned long long gcnt[kMaxGenerations + 1];
    // grid barrier: arrivals, generation, abort flag
    unsigned int bar_count, bar_gen, abort;
};

template <class T> struct BatchArgs {
    PushArgs<T> P;              // rate table, process constants, dt, nu_max
    Soa<T> in, out;             // segmented buffers
    long long cap_s;            // slots per swarm segment
    int n_swarms;
    long long* cnt_in;          // [n_swarms] live items of `in`
    unsigned long long* cnt_out;// [n_swarms] append cursors of `out`
    long long* prefix;          // [n_swarms + 1] exclusive prefix of cnt_in
    ChildQ<T> cq[2];            // product queues (generation parity)
    uint32_t* csw[2];           // swarm of each queued product
    long long cap_child;
    BatchDev* bd;
    uint64_t seed;              // swarm s: seed + s
    const double* Ez;           // [n_swarms] field along z (negative: electrons drift to +z)
    double* mom;                // [n_swarms][n_steps][kNMom], z moments about the step's reference zref
    double* zref;               // [n_swarms] reference z of the current step (previous centre of mass)
    double* zref_hist;          // [n_swarms][n_steps] reference used for each step's moments
    long long* counts;          // [n_swarms][n_steps]
    int n_steps;
    long long n_lo, n_hi;
    int gen;
    // collision rates of each swarm's gas: table of swarm s at tab_s + s *
    // tab_stride (stride 0: one gas for all), nu_max and -ln 2 / nu_max
    const T* tab_s;
    long long tab_stride;
    const T* numax_s;
    const T* tau_s;
    long long warp_chunk;       // largest item range a warp takes at once (a multiple of 32)
};

// The step's input and output buffers: B.in and B.out, or swapped (FLIP) on
// the odd steps of the persistent kernel.
template <class T, bool FLIP> __device__ __forceinline__ const Soa<T>& src_buf(const BatchArgs<T>& B) {
    return FLIP ? B.out : B.in;
}
template <class T, bool FLIP> __device__ __forceinline__ const Soa<T>& dst_buf(const BatchArgs<T>& B) {
    return FLIP ? B.in : B.out;
}

template <class T> __device__ __forceinline__ Rates<T> swarm_rates(const BatchArgs<T>& B, int s) {
    return Rates<T>{B.tab_s + (long long)s * B.tab_stride, B.numax_s[s], B.tau_s[s]};
}

__device__ __forceinline__ Keys dev_keys(uint64_t seed) {
    Keys k;
    k.mcc0 = (uint32_t)seed;
    k.mcc1 = (uint32_t)(seed >> 32);
    k.ids0 = (uint32_t)seed ^ 0x5A5A5A5Au;
    k.ids1 = (uint32_t)(seed >> 32) ^ 0xC3C3C3C3u;
    k.init0 = (uint32_t)seed ^ 0x1B873593u;
    k.init1 = (uint32_t)(seed >> 32) ^ 0xCC9E2D51u;
    return k;
}

// Swarm of work item `it` by binary search in the prefix sums (prefix[s] <= it < prefix[s+1]).
__device__ __forceinline__ int swarm_of(const long long* pre, int n, long long it) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= it) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Resampling per swarm, in place (see k_resample): thinning above n_hi,
// duplication below n_lo.  Grid-stride over the step's items.
template <class T, bool FLIP> __device__ void batch_resample(const BatchArgs<T>& B, uint32_t step) {
    const long long total = B.prefix[B.n_swarms];
    for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < total;
         it += (long long)gridDim.x * blockDim.x) {
        const int s = swarm_of(B.prefix, B.n_swarms, it);
        const long long n = B.cnt_in[s];
        const bool thin = n > B.n_hi, dup = n > 0 && n < B.n_lo && 2 * n <= B.cap_s;
        if (!thin && !dup) continue;
        const long long i = s * B.cap_s + (it - B.prefix[s]);
        const Keys K = dev_keys(B.seed + (uint64_t)s);
        const Soa<T>& p = src_buf<T, FLIP>(B);
        if (thin) {
            const u32x4 r = draw_words(K, p.id[i], step, 0xA0000000u);
            if (!(unif<T>(r.x) < (T)0.5)) p.r[PW][i] = (T)0;
        } else {
            const long long j = i + n;
            for (int f = 0; f < 10; ++f) p.r[f][j] = p.r[f][i];
            p.id[j] = derived_id(K, p.id[i], step, 0xA0000000u);
        }
    }
}
template <class T> __global__ void k_batch_resample(const BatchArgs<T> B) { batch_resample<T, false>(B, B.bd->step); }

// Exclusive prefix sums of the per-swarm counts (one block calls it).
template <class T> __device__ void scan_counts(const BatchArgs<T>& B) {
    __shared__ long long carry;
    __shared__ long long wsum[32];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < B.n_swarms; base += blockDim.x) {
        const int s = base + threadIdx.x;
        const long long v = s < B.n_swarms ? B.cnt_in[s] : 0;
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        long long inc = v;
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(kFull, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) wsum[w] = inc;
        __syncthreads();
        long long woff = 0;
        for (int q = 0; q < w; ++q) woff += wsum[q];
        const long long c = carry;
        if (s < B.n_swarms) B.prefix[s] = c + woff + inc - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = c + woff + inc;
        __syncthreads();
    }
    if (threadIdx.x == 0) B.prefix[B.n_swarms] = carry;
    __syncthreads();
}

// After resampling: duplicated swarms double their counts, prefix sums of the
// step's work items, cursors and output counters reset.  One block.
template <class T> __device__ void batch_begin(const BatchArgs<T>& B, uint32_t step) {
    for (int s = threadIdx.x; s < B.n_swarms; s += blockDim.x) {
        const long long n = B.cnt_in[s];
        if (n > 0 && n < B.n_lo && 2 * n <= B.cap_s) B.cnt_in[s] = 2 * n;
        B.cnt_out[s] = 0;
        if (step >= 1 && (int)step <= B.n_steps) B.zref_hist[(size_t)s * B.n_steps + (step - 1)] = B.zref[s];
    }
    __syncthreads();
    scan_counts(B);
    if (threadIdx.x == 0) {
        B.bd->fetch = 0;
        B.bd->fetch_c = 0;
        B.bd->n_child = 0;
        B.bd->n_spill = 0;
    }
    for (int g = threadIdx.x; g <= kMaxGenerations; g += blockDim.x) {
        B.bd->cur[g] = 0;
        B.bd->gcnt[g] = 0;
    }
}
template <class T> __global__ void k_batch_begin(const BatchArgs<T> B) { batch_begin(B, B.bd->step); }

// Before children generation g >= 1.
static __global__ void k_batch_nextgen(BatchDev* bd, int gen) {
    bd->fetch_c = 0;
    if (gen & 1) bd->n_child = 0;
    else bd->n_spill = 0;
}

// End of a step: counts recorded and made the next step's input counts, with
// their prefix sums (used by the next step's resampling).  One block.
template <class T> __device__ void batch_end(const BatchArgs<T>& B, uint32_t step) {
    for (int s = threadIdx.x; s < B.n_swarms; s += blockDim.x) {
        unsigned long long n = B.cnt_out[s];
        if (n > (unsigned long long)B.cap_s) n = (unsigned long long)B.cap_s;
        B.cnt_in[s] = (long long)n;
        if (step >= 1 && (int)step <= B.n_steps) {
            B.counts[(size_t)s * B.n_steps + (step - 1)] = (long long)n;
            const double* row = B.mom + ((size_t)s * B.n_steps + (step - 1)) * kNMom;
            if (row[0] > 0.0) B.zref[s] += row[3] / row[0];
        }
    }
    __syncthreads();
    scan_counts(B);
}
template <class T> __global__ void k_batch_end(const BatchArgs<T> B) { batch_end(B, B.bd->step); }

// Initial counts: n0 per swarm, prefix sums, step 1.  One block.
template <class T> __global__ void k_batch_init(const BatchArgs<T> B, long long n0) {
    for (int s = threadIdx.x; s < B.n_swarms; s += blockDim.x) {
        B.cnt_in[s] = n0;
        B.cnt_out[s] = 0;
        B.zref[s] = 0.0;
    }
    __syncthreads();
    scan_counts(B);
    if (threadIdx.x == 0) {
        B.bd->err = 0;
        B.bd->step = 1;
    }
}

// Maxwellian start of every swarm (as for a single swarm, with key seed + s).
template <class T> __global__ void k_batch_seed(const BatchArgs<T> B, long long n0, double sig) {
    const long long total = (long long)B.n_swarms * n0;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(g / n0);
        const long long i = g - (long long)s * n0;
        const Keys K = dev_keys(B.seed + (uint64_t)s);
        const u32x4 o = draw_words(K, (uint64_t)i, 0u, 0u);
        const double u0 = unif<double>(o.x), u1 = unif<double>(o.y), u2 = unif<double>(o.z), u3 = unif<double>(o.w);
        const double r1 = sqrt(-2.0 * log(u0)), r2 = sqrt(-2.0 * log(u2));
        double s1, c1, s3, c3;
        sincospi(2.0 * u1, &s1, &c1);
        sincospi(2.0 * u3, &s3, &c3);
        const long long j = (long long)s * B.cap_s + i;
        B.in.r[VX][j] = (T)(sig * r1 * c1);
        B.in.r[VY][j] = (T)(sig * r1 * s1);
        B.in.r[VZ][j] = (T)(sig * r2 * c3);
        B.in.r[PX][j] = B.in.r[PY][j] = B.in.r[PZ][j] = (T)0;
        B.in.r[AX][j] = B.in.r[AY][j] = B.in.r[AZ][j] = (T)0;
        B.in.r[PW][j] = (T)1;
        B.in.id[j] = (uint64_t)i;
    }
}

// After the last children generation (index g_last): anything queued for a
// further generation is an error (cascade deeper than the graph allows).
static __global__ void k_batch_step_advance(BatchDev* bd, int g_last) {
    const unsigned long long pend = (g_last & 1) ? bd->n_child : bd->n_spill;
    if (pend) atomicOr(&bd->err, kErrStack);
    bd->step += 1;
}

constexpr long long kWarpChunk = 1024;  // default largest warp-private item range (BatchArgs::warp_chunk)

template <class T> struct BatchStage {
    T in[32 * kRow];
    T out[kOut * kRow];
    T ch[kCh * kRow];
    uint64_t in_id[32], out_id[kOut], ch_id[kCh];
    uint32_t ch_k[kCh];
    int in_s[32], out_s[kOut], ch_s[kCh];
    double macc[14];   // the warp's running moment sums for swarm macc_s (step macc_t)
    int macc_s;
};

// Moment contributions of the lanes' electrons (all lanes call).  When all
// 32 lanes carry electrons of one swarm (the common case: items are
// contiguous per swarm) the warp reduces them and keeps the running sums in
// its stage, writing them to the swarm's row only when the warp moves on to
// another swarm (or ends); mixed warps add per lane.
template <class T> __device__ __forceinline__ void macc_flush(const BatchArgs<T>& B, BatchStage<T>* sg, uint32_t step) {
    const int lane = threadIdx.x & 31;
    __syncwarp();
    if (sg->macc_s >= 0 && lane < 14) {
        double* row = B.mom + ((size_t)sg->macc_s * B.n_steps + (step - 1)) * kNMom;
        if (sg->macc[lane] != 0.0) atomicAdd(row + lane, sg->macc[lane]);
        sg->macc[lane] = 0.0;
    }
    __syncwarp();
}

template <class T>
__device__ __forceinline__ void swarm_moments(const BatchArgs<T>& B, BatchStage<T>* sg, bool live, int s, const T x[3],
                                              const T v[3], T wt, uint32_t step) {
    // z about the swarm's reference point: the moments of a drifting swarm
    // stay small, so float sums lose nothing to cancellation
    T m[14];
    if (live) {
        const T w = wt, X = x[0], Y = x[1], Z = x[2] - (T)B.zref[s], U = v[0], V = v[1], W = v[2];
        m[0] = w; m[1] = w * X; m[2] = w * Y; m[3] = w * Z;
        m[4] = w * X * X; m[5] = w * Y * Y; m[6] = w * Z * Z;
        m[7] = w * U; m[8] = w * V; m[9] = w * W;
        m[10] = w * X * U; m[11] = w * Y * V; m[12] = w * Z * W;
        m[13] = w * ((T)(0.5 * kMe / kQ) * (U * U + V * V + W * W));
    } else {
        for (int q = 0; q < 14; ++q) m[q] = (T)0;
    }
    // segmented warp reduction: one pass per distinct swarm among the lanes
    // (one pass in the common case), the sums kept in the warp's stage for
    // the swarm it works on and added directly for any other
    unsigned todo = __ballot_sync(kFull, live);
    while (todo) {
        const int leader = __ffs(todo) - 1;
        const int sg_s = __shfl_sync(kFull, s, leader);
        const bool mine = live && s == sg_s;
        todo &= ~__ballot_sync(kFull, mine);
        T red[14];
        for (int q = 0; q < 14; ++q) {
            T v2 = mine ? m[q] : (T)0;
            for (int o = 16; o > 0; o >>= 1) v2 += __shfl_xor_sync(kFull, v2, o);
            red[q] = v2;
        }
        if (sg->macc_s != sg_s && (sg->macc_s < 0 || todo == 0)) {
            // the warp has moved on to another swarm: write the old sums out
            macc_flush(B, sg, step);
            if ((threadIdx.x & 31) == 0) sg->macc_s = sg_s;
            __syncwarp();
        }
        const int lane = threadIdx.x & 31;
        double add = 0.0;
        for (int k = 0; k < 14; ++k)
            if (k == lane) add = (double)red[k];
        if (sg->macc_s == sg_s) {
            if (lane < 14) sg->macc[lane] += add;
        } else if (lane < 14 && add != 0.0) {
            atomicAdd(B.mom + ((size_t)sg_s * B.n_steps + (step - 1)) * kNMom + lane, add);
        }
        __syncwarp();
    }
}

template <class T>
__device__ __forceinline__ void flush_event_weights(const BatchArgs<T>& B, int s, uint32_t step, LStats& ls) {
    if (s < 0 || (ls.w_ion == 0.0 && ls.w_att == 0.0)) return;
    double* row = B.mom + ((size_t)s * B.n_steps + (step - 1)) * kNMom;
    if (ls.w_ion != 0.0) atomicAdd(row + 14, ls.w_ion);
    if (ls.w_att != 0.0) atomicAdd(row + 15, ls.w_att);
    ls.w_ion = ls.w_att = 0.0;
}

template <class T> constexpr size_t batch_smem(int warps) { return (size_t)warps * sizeof(BatchStage<T>); }

// Output flush for batched swarms: entries [0, cnt) appended to their swarms'
// segments (one cursor increment per swarm group) and their moments added.
template <class T, bool FLIP>
__device__ __forceinline__ void batch_flush_out(const BatchArgs<T>& B, BatchStage<T>* sg, int& n, int cnt,
                                                uint32_t step) {
    const int lane = threadIdx.x & 31;
    __syncwarp();
    const bool live = lane < cnt;
    T x[3] = {0, 0, 0}, v[3] = {0, 0, 0}, a[3] = {0, 0, 0}, w = (T)0;
    uint64_t id = 0;
    int s = -1;
    if (live) {
        const T* r = sg->out + lane * kRow;
        x[0] = r[0]; x[1] = r[1]; x[2] = r[2];
        v[0] = r[3]; v[1] = r[4]; v[2] = r[5];
        a[0] = r[6]; a[1] = r[7]; a[2] = r[8];
        w = r[9];
        id = sg->out_id[lane];
        s = sg->out_s[lane];
    }
    const unsigned grp = __match_any_sync(kFull, s);
    const int leader = __ffs(grp) - 1;
    unsigned long long base = 0;
    if (live && lane == leader) base = atomicAdd(&B.cnt_out[s], (unsigned long long)__popc(grp));
    base = __shfl_sync(kFull, base, leader);
    bool stored = false;
    if (live) {
        const unsigned long long slot = base + __popc(grp & ((1u << lane) - 1u));
        if ((long long)slot < B.cap_s) {
            store(dst_buf<T, FLIP>(B), (unsigned long long)(s * B.cap_s) + slot, x, v, a, w, id);
            stored = true;
        } else {
            atomicOr(&B.bd->err, kErrOutCapacity);
        }
    }
    swarm_moments(B, sg, stored, s, x, v, w, step);
    __syncwarp();
    const int rest = n - cnt;
    if (lane < rest) {
        for (int f = 0; f < 10; ++f) sg->out[lane * kRow + f] = sg->out[(cnt + lane) * kRow + f];
        sg->out_id[lane] = sg->out_id[cnt + lane];
        sg->out_s[lane] = sg->out_s[cnt + lane];
    }
    __syncwarp();
    n = rest;
}

template <class T>
__device__ __forceinline__ void batch_flush_children(const BatchArgs<T>& B, BatchStage<T>* sg, int& n, int cnt,
                                                     int dst, unsigned long long* cnt_p) {
    const int lane = threadIdx.x & 31;
    __syncwarp();
    unsigned long long s0 = 0;
    if (lane == 0) s0 = atomicAdd(cnt_p, (unsigned long long)cnt);
    s0 = __shfl_sync(kFull, s0, 0);
    if (lane < cnt) {
        const unsigned long long q = s0 + lane;
        if ((long long)q < B.cap_child) {
            const T* r = sg->ch + lane * kRow;
            const ChildQ<T>& Q = B.cq[dst];
            Q.p.r[PX][q] = r[0]; Q.p.r[PY][q] = r[1]; Q.p.r[PZ][q] = r[2];
            Q.p.r[VX][q] = r[3];
            Q.p.r[AX][q] = r[4]; Q.p.r[AY][q] = r[5]; Q.p.r[AZ][q] = r[6];
            Q.p.r[PW][q] = r[7];
            Q.t_left[q] = r[8];
            Q.p.id[q] = sg->ch_id[lane];
            Q.k[q] = sg->ch_k[lane];
            B.csw[dst][q] = (uint32_t)sg->ch_s[lane];
        } else {
            atomicOr(&B.bd->err, kErrChildCapacity);
        }
    }
    __syncwarp();
    const int rest = n - cnt;
    if (lane < rest) {
        for (int f = 0; f < 9; ++f) sg->ch[lane * kRow + f] = sg->ch[(cnt + lane) * kRow + f];
        sg->ch_id[lane] = sg->ch_id[cnt + lane];
        sg->ch_k[lane] = sg->ch_k[cnt + lane];
        sg->ch_s[lane] = sg->ch_s[cnt + lane];
    }
    __syncwarp();
    n = rest;
}

// The lane-refill collision loop of collide_loop, for batched swarms: one
// phase of a step.  CHILD = false: the work items are the swarms' electrons
// (n_items of them); their products are staged per warp and queued in queue
// dstq (append counter dst_cnt).  CHILD = true: the items are the products
// queued in srcq; their own products stay on the lane's stack, and what it
// cannot hold goes to queue dstq for the next generation.  Every warp takes
// item ranges from `cursor` until the phase runs dry.
template <class T, bool FAST, bool CHILD, bool FLIP>
__device__ void batch_phase(const BatchArgs<T>& B, const ProcSmem<T>& ps, BatchStage<T>* sg, uint32_t step,
                            long long n_items, unsigned long long* cursor, int srcq, int dstq,
                            unsigned long long* dst_cnt) {
    const int lane = threadIdx.x & 31;
    if (lane < 14) sg->macc[lane] = 0.0;
    if (lane == 0) sg->macc_s = -1;
    __syncwarp();
    const unsigned lt = (1u << lane) - 1u;
    const T qm = (T)(kQ / kMe);
    LStats ls;
    ls.zero();
    Lane<T> L;
    Keys K = dev_keys(B.seed);
    Rates<T> R = swarm_rates(B, 0);
    int s_cur = -1, s_cache = -1;
    long long w_next = 0, w_end = 0;
    bool active = false, dry = false;
    int in_head = 0, in_count = 0, n_out = 0, n_ch = 0;
    StackSink<T> stk;
    for (;;) {
        bool want = !active;
        if (CHILD && want && stk.n > 0) {
            --stk.n;
            const int t = stk.n;
            for (int d = 0; d < 3; ++d) { L.x[d] = stk.x[t][d]; L.v[d] = stk.v[t][d]; L.d[d] = (T)0; }
            L.w = stk.w[t];
            L.id = stk.id[t];
            L.t_left = stk.t[t];
            L.k = 1;
            active = true;
            want = false;
        }
        const unsigned need = __ballot_sync(kFull, want);
        const int avail = in_count - in_head;
        if (need && avail > 0) {
            const int rank = __popc(need & lt);
            if (want && rank < avail) {
                const int e = in_head + rank;
                const T* r = sg->in + e * kRow;
                const int s = sg->in_s[e];
                if (s != s_cur) {
                    flush_event_weights(B, s_cur, step, ls);
                    s_cur = s;
                    K = dev_keys(B.seed + (uint64_t)s);
                    R = swarm_rates(B, s);
                }
                for (int d = 0; d < 3; ++d) { L.x[d] = r[d]; L.v[d] = r[3 + d]; L.d[d] = (T)0; }
                L.a[0] = (T)0;
                L.a[1] = (T)0;
                L.a[2] = -qm * (T)B.Ez[s];
                L.w = r[9];
                L.t_left = r[10];
                L.id = sg->in_id[e];
                L.k = 1;
                active = L.w > (T)0;
            }
            in_head += __popc(need) < avail ? __popc(need) : avail;
        }
        if (in_head >= in_count && !dry) {
            __syncwarp();
            if (w_next >= w_end) {
                // a new warp-private range: large while much work is left (so a
                // warp's electrons share a swarm), shrinking towards 32 at the end
                unsigned long long b = 0, g = 32;
                if (lane == 0) {
                    const unsigned long long seen = *(volatile unsigned long long*)cursor;
                    const long long rem = n_items - (long long)seen;
                    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
                    long long want_g = rem > 0 ? rem / (4 * warps) : 32;
                    want_g = want_g < 32 ? 32 : (want_g > B.warp_chunk ? B.warp_chunk : want_g);
                    g = (unsigned long long)(want_g & ~31ll);
                    b = atomicAdd(cursor, g);
                }
                b = __shfl_sync(kFull, b, 0);
                g = __shfl_sync(kFull, g, 0);
                w_next = (long long)b;
                w_end = (long long)(b + g) < n_items ? (long long)(b + g) : n_items;
            }
            const long long b = w_next;
            if (b >= n_items) {
                dry = true;
                in_head = in_count = 0;
            } else {
                const long long left = w_end - b;
                const int cnt = left < 32 ? (int)left : 32;
                w_next = b + cnt;
                if (lane < cnt) {
                    const long long it = (long long)b + lane;
                    T* r = sg->in + lane * kRow;
                    if (CHILD) {
                        const ChildQ<T>& Q = B.cq[srcq];
                        const int s = (int)B.csw[srcq][it];
                        const Keys Ks = dev_keys(B.seed + (uint64_t)s);
                        T vc[3];
                        const uint64_t cid = make_child(Ks, step, Q.p.id[it], Q.k[it], Q.p.r[VX][it], vc);
                        r[0] = Q.p.r[PX][it]; r[1] = Q.p.r[PY][it]; r[2] = Q.p.r[PZ][it];
                        r[3] = vc[0]; r[4] = vc[1]; r[5] = vc[2];
                        r[9] = Q.p.r[PW][it];
                        r[10] = Q.t_left[it];
                        sg->in_id[lane] = cid;
                        sg->in_s[lane] = s;
                    } else {
                        int s = s_cache;
                        if (s < 0 || it < B.prefix[s] || it >= B.prefix[s + 1]) s = swarm_of(B.prefix, B.n_swarms, it);
                        s_cache = s;
                        const long long i = s * B.cap_s + (it - B.prefix[s]);
                        const Soa<T>& in = src_buf<T, FLIP>(B);
                        for (int f = 0; f < 6; ++f) r[f] = in.r[f][i];
                        r[9] = in.r[PW][i];
                        r[10] = B.P.dt;
                        sg->in_id[lane] = in.id[i];
                        sg->in_s[lane] = s;
                    }
                }
                in_head = 0;
                in_count = cnt;
            }
            __syncwarp();
        }
        if (!__any_sync(kFull, active || (CHILD && stk.n > 0))) {
            if (dry && in_head >= in_count) break;
            continue;
        }
        int r = EV_CONTINUE;
        T sp = (T)0;
        if (active) {
            // up to two candidate collisions per trip, as in the collision kernel
            r = event<T, MODE_SWARM, FAST, false>(B.P, R, K, step, &ps, L, ls, sp);
            if (r == EV_CONTINUE) r = event<T, MODE_SWARM, FAST, false>(B.P, R, K, step, &ps, L, ls, sp);
        }
        const bool done = r == EV_DONE, ion = r == EV_IONIZED;
        if (r == EV_DONE || r == EV_ATTACHED) active = false;
        if (CHILD && ion) {
            if (stk.n < StackSink<T>::kDepth) {
                T vc[3];
                const uint64_t cid = make_child(K, step, L.id, L.k - 1, sp, vc);
                const int t = stk.n++;
                for (int d = 0; d < 3; ++d) { stk.x[t][d] = L.x[d] + L.d[d]; stk.v[t][d] = vc[d]; }
                stk.w[t] = L.w;
                stk.id[t] = cid;
                stk.t[t] = L.t_left;
            } else {  // stack full: queue the compact entry for the next generation
                const unsigned long long q = atomicAdd(dst_cnt, 1ull);
                if ((long long)q < B.cap_child) {
                    const ChildQ<T>& Q = B.cq[dstq];
                    Q.p.r[PX][q] = L.x[0] + L.d[0]; Q.p.r[PY][q] = L.x[1] + L.d[1]; Q.p.r[PZ][q] = L.x[2] + L.d[2];
                    Q.p.r[VX][q] = sp;
                    Q.p.r[AX][q] = L.a[0]; Q.p.r[AY][q] = L.a[1]; Q.p.r[AZ][q] = L.a[2];
                    Q.p.r[PW][q] = L.w;
                    Q.t_left[q] = L.t_left;
                    Q.p.id[q] = L.id;
                    Q.k[q] = L.k - 1;
                    B.csw[dstq][q] = (uint32_t)s_cur;
                } else {
                    atomicOr(&B.bd->err, kErrChildCapacity);
                }
            }
        }
        const unsigned im = CHILD ? 0u : __ballot_sync(kFull, ion);
        if (im) {
            if (ion) {
                const int e = n_ch + __popc(im & lt);
                T* q = sg->ch + e * kRow;
                q[0] = L.x[0] + L.d[0]; q[1] = L.x[1] + L.d[1]; q[2] = L.x[2] + L.d[2];
                q[3] = sp;
                q[4] = L.a[0]; q[5] = L.a[1]; q[6] = L.a[2];
                q[7] = L.w;
                q[8] = L.t_left;
                sg->ch_id[e] = L.id;
                sg->ch_k[e] = L.k - 1;
                sg->ch_s[e] = s_cur;
            }
            n_ch += __popc(im);
            if (n_ch >= 32) batch_flush_children(B, sg, n_ch, 32, dstq, dst_cnt);
        }
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
                sg->out_s[e] = s_cur;
            }
            n_out += __popc(dm);
            if (n_out >= 32) batch_flush_out<T, FLIP>(B, sg, n_out, 32, step);
        }
    }
    if (n_out > 0) batch_flush_out<T, FLIP>(B, sg, n_out, n_out, step);
    if (!CHILD && n_ch > 0) batch_flush_children(B, sg, n_ch, n_ch, dstq, dst_cnt);
    macc_flush(B, sg, step);
    flush_event_weights(B, s_cur, step, ls);
}

template <class T> __device__ __forceinline__ void stage_proc_batch(ProcSmem<T>& ps, const BatchArgs<T>& B) {
    if (threadIdx.x < 8) {
        ps.thr[threadIdx.x] = B.P.thr[threadIdx.x];
        ps.mratio[threadIdx.x] = B.P.mratio[threadIdx.x];
        ps.kind[threadIdx.x] = B.P.kind[threadIdx.x];
    }
    __syncthreads();
}

// One phase per launch (the step replayed from a CUDA graph): generation
// B.gen reads queue B.gen & 1 and queues into the other one.
template <class T, bool FAST, bool CHILD>
__global__ void __launch_bounds__(256) k_batch_collide(const BatchArgs<T> B) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ ProcSmem<T> ps;
    stage_proc_batch(ps, B);
    BatchStage<T>* sg = reinterpret_cast<BatchStage<T>*>(smem_raw) + (threadIdx.x >> 5);
    const uint32_t step = B.bd->step;
    const int srcq = B.gen & 1, dstq = CHILD ? srcq ^ 1 : 0;
    long long n_items;
    unsigned long long* cursor;
    if (CHILD) {
        n_items = (long long)(srcq ? B.bd->n_spill : B.bd->n_child);
        if (n_items > B.cap_child) n_items = B.cap_child;
        cursor = &B.bd->fetch_c;
    } else {
        n_items = B.prefix[B.n_swarms];
        cursor = &B.bd->fetch;
    }
    unsigned long long* dst_cnt = dstq ? &B.bd->n_spill : &B.bd->n_child;
    batch_phase<T, FAST, CHILD, false>(B, ps, sg, step, n_items, cursor, srcq, dstq, dst_cnt);
}

// Grid-wide barrier of a persistent kernel (a cooperative launch: every block
// is resident).  After a block-wide barrier and a release fence, thread 0 of
// each block arrives with an atomic; the last arrival resets the count and
// opens the next barrier generation, the others poll the generation with
// acquire loads and short sleeps, at most kBarrierPolls times.  A wait that
// runs out (a block that never arrives) raises kErrBarrier and the abort
// flag, and every barrier after that returns false at once, so the kernel
// ends instead of hanging.  Returns false when the kernel must end.
constexpr long long kBarrierPolls = 1ll << 24;  // about a second of 64 ns sleeps

__device__ __forceinline__ bool grid_barrier(BatchDev* bd) {
    __shared__ int go;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned g = ld_acquire_gpu(&bd->bar_gen);
        __threadfence();
        if (atomicAdd(&bd->bar_count, 1u) == gridDim.x - 1) {
            atomicExch(&bd->bar_count, 0u);
            __threadfence();
            atomicAdd(&bd->bar_gen, 1u);
        } else {
            long long polls = 0;
            while (ld_acquire_gpu(&bd->bar_gen) == g) {
                if (ld_acquire_gpu(&bd->abort) != 0u || ++polls > kBarrierPolls) {
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        if (ok && ld_acquire_gpu(&bd->abort) != 0u) ok = 0;
        if (!ok) {
            atomicOr(&bd->err, kErrBarrier);
            atomicExch(&bd->abort, 1u);
        }
        __threadfence();
        go = ok;
    }
    __syncthreads();
    return go != 0;
}

// One step of the persistent kernel: resampling (all blocks), the step's
// prefix sums (block 0), the parents (all blocks taking item ranges from one
// cursor), then product generations until a generation queues none
// (generation g reads queue g & 1 and appends to the other; each
// generation's queue count has its own slot, so no reset separates them),
// then the counts of the step (block 0), with grid-wide barriers between the
// phases.  FLIP: the step reads B.out and writes B.in (odd steps).  Returns
// false when a barrier gave up.
template <class T, bool FAST, bool FLIP>
__device__ bool batch_run_step(const BatchArgs<T>& B, const ProcSmem<T>& ps, BatchStage<T>* sg) {
    BatchDev* bd = B.bd;
    const uint32_t step = ld_acquire_gpu(&bd->step);
    batch_resample<T, FLIP>(B, step);
    if (!grid_barrier(bd)) return false;
    if (blockIdx.x == 0) batch_begin(B, step);
    if (!grid_barrier(bd)) return false;
    batch_phase<T, FAST, false, FLIP>(B, ps, sg, step, B.prefix[B.n_swarms], &bd->cur[0], 0, 0, &bd->gcnt[0]);
    if (!grid_barrier(bd)) return false;
    for (int g = 0; g < kMaxGenerations; ++g) {
        const unsigned long long pend = ld_acquire_gpu(&bd->gcnt[g]);
        if (pend == 0) break;
        const long long n_items = (long long)pend < B.cap_child ? (long long)pend : B.cap_child;
        batch_phase<T, FAST, true, FLIP>(B, ps, sg, step, n_items, &bd->cur[g + 1], g & 1, (g + 1) & 1,
                                         &bd->gcnt[g + 1]);
        if (!grid_barrier(bd)) return false;
    }
    if (blockIdx.x == 0) {
        if (threadIdx.x == 0 && ld_acquire_gpu(&bd->gcnt[kMaxGenerations]) != 0ull) atomicOr(&bd->err, kErrStack);
        batch_end(B, step);
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(&bd->step, 1u);
    }
    return grid_barrier(bd);
}

// Every step of every swarm in one launch (cooperative: all blocks resident).
template <class T, bool FAST>
__global__ void __launch_bounds__(256) k_batch_run(const BatchArgs<T> B, int n_steps) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ ProcSmem<T> ps;
    stage_proc_batch(ps, B);
    BatchStage<T>* sg = reinterpret_cast<BatchStage<T>*>(smem_raw) + (threadIdx.x >> 5);
    for (int it = 0; it < n_steps; ++it) {
        const bool ok = (it & 1) ? batch_run_step<T, FAST, true>(B, ps, sg) : batch_run_step<T, FAST, false>(B, ps, sg);
        if (!ok) return;
    }
}

}  // namespace pic

namespace pic {

// Host-side launchers (instantiated in push_f32.cu / push_f64.cu).
template <class T> struct BatchLaunch {
    static size_t smem(int block) { return (size_t)(block / 32) * sizeof(BatchStage<T>); }
    static int max_blocks_per_sm(int block);
    static cudaError_t init(const BatchArgs<T>& B, long long n0, double sig, cudaStream_t s);
    static cudaError_t prepare(int block);  // kernel attributes for this block size (outside any capture)
    // One step: resampling, prefix sums, parents, kBatchGenerations children
    // generations, counts, step counter.  B.in / B.out are this step's buffers.
    static cudaError_t step(BatchArgs<T> B, int block, int grid, cudaStream_t s, long long* launches);
    // All n_steps steps in one cooperative launch of k_batch_run (grid at most
    // the resident blocks), recorded in a CUDA graph and launched from it.
    static int persistent_blocks_per_sm(int block);
    static cudaError_t run_persistent(const BatchArgs<T>& B, int n_steps, int block, int grid, cudaStream_t s);
};

}  // namespace pic
