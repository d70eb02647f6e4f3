// common.cuh -- device-side definitions shared by the falcON step kernels.
//
// Symmetric Cartesian tensors (Sect. 3.4.3: an order-n symmetric tensor has
// (n+1)(n+2)/2 independent components) are stored by multi-index
// alpha = (a, b, c), a + b + c = n: within order n the components run over
// k = n - a = 0..n and, for each k, c = 0..k (b = k - c).  Orders are packed
// one after the other; order n starts at n(n+1)(n+2)/6.
//   multipoles M-hat: orders 0, 2..p-1 (the dipole vanishes about the centre
//                     of mass, Sect. 3.4.3), p = 6 -> 53 values
//   locals C-hat:     orders 1..p (C^(0) is never needed), p = 6 -> 83 values
//   derivatives D:    orders 0..p
//
// Scaled storage (per cell, rho = a power of two >= max(r_max, side/256)):
//   M-hat_beta = M_beta / (beta! rho^|beta|),   C-hat_alpha = C_alpha rho^|alpha|
// which keeps every stored coefficient within a few orders of magnitude of the
// cell mass (or of the field) whatever the cell size, so that FP32 storage and
// arithmetic lose nothing to the exponent range.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ncorp {

constexpr int MAXP = 6;
constexpr int KEY_BITS = 21;                 // bits per axis of the quantised coordinates
constexpr int MAX_LEVEL = KEY_BITS;          // deepest tree level

__host__ __device__ constexpr int tri(int k) { return k * (k + 1) / 2; }
__host__ __device__ constexpr int nsym(int n) { return (n + 1) * (n + 2) / 2; }
__host__ __device__ constexpr int off(int n) { return n * (n + 1) * (n + 2) / 6; }
// packed index of multi-index (a, b, c) among all orders
__host__ __device__ constexpr int sidx(int a, int b, int c) { return off(a + b + c) + tri(b + c) + c; }
// multipole index (orders 0, 2, 3, ...)
__host__ __device__ constexpr int midx(int a, int b, int c) { return (a + b + c) >= 2 ? sidx(a, b, c) - 3 : 0; }
// local-coefficient index (orders 1..p)
__host__ __device__ constexpr int cidx(int a, int b, int c) { return sidx(a, b, c) - 1; }
__host__ __device__ constexpr int num_m(int p) { return p >= 2 ? off(p) - 3 : 1; }
__host__ __device__ constexpr int num_c(int p) { return off(p + 1) - 1; }
__host__ __device__ constexpr int num_d(int p) { return off(p + 1); }
__host__ __device__ constexpr double ifact(int n) {
    return n <= 1 ? 1.0 : n == 2 ? 0.5 : n == 3 ? 1.0 / 6.0 : n == 4 ? 1.0 / 24.0 : n == 5 ? 1.0 / 120.0
         : n == 6 ? 1.0 / 720.0 : 1.0 / 5040.0;
}
__host__ __device__ constexpr double inv_mfact(int a, int b, int c) { return ifact(a) * ifact(b) * ifact(c); }
// 1/n! for run-time n (0..7)
static __constant__ double c_ifact[8] = {1.0, 1.0, 0.5, 1.0 / 6.0, 1.0 / 24.0, 1.0 / 120.0, 1.0 / 720.0, 1.0 / 5040.0};

// ---- exactly rounded FP64 (never contracted into FMA) --------------------
// Tree geometry, walk decisions, keys, kicks/drifts and the collision test use
// these so that their results are bit-identical to a plain IEEE evaluation in
// the written order.
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double dsqrt(double a) { return __dsqrt_rn(a); }
__device__ __forceinline__ double dnorm3(double x, double y, double z) {
    return dsqrt(dadd(dadd(dmul(x, x), dmul(y, y)), dmul(z, z)));
}
__device__ __forceinline__ double dsq3(double x, double y, double z) {
    return dadd(dadd(dmul(x, x), dmul(y, y)), dmul(z, z));
}

// smallest power of two >= v (v > 0), exact; 1 for v <= 0
__device__ __forceinline__ double pow2_ceil(double v) {
    if (!(v > 0.0)) return 1.0;
    int e;
    double f = frexp(v, &e);           // v = f 2^e, f in [0.5, 1)
    return f == 0.5 ? ldexp(1.0, e - 1) : ldexp(1.0, e);
}

// ---- error word -----------------------------------------------------------
enum : int {
    ERR_CELLS = 1,        // cell capacity exceeded
    ERR_FRONTIER = 2,     // walk frontier capacity exceeded
    ERR_M2L = 4,          // M2L list capacity exceeded
    ERR_P2P = 8,          // direct list capacity exceeded
    ERR_PAIRS = 16,       // collision pair buffer exceeded
    ERR_TIMEOUT = 32,     // a bounded grid barrier gave up
    ERR_DIRECTED = 64,    // directed list capacity exceeded
    ERR_LEVEL = 128,      // internal: tree deeper than MAX_LEVEL
    ERR_NONFINITE = 256,  // a position was NaN or infinite
};

constexpr int ERR_ABORT_MASK =
    ERR_CELLS | ERR_FRONTIER | ERR_M2L | ERR_P2P | ERR_TIMEOUT | ERR_DIRECTED | ERR_LEVEL | ERR_NONFINITE;

// Device control block: counters written by kernels, read back by the host.
struct Ctrl {
    int err;
    int n_cells;
    int n_leaves;
    int max_level;
    int level_start[MAX_LEVEL + 3];
    int frontier_count[2];
    int n_m2l;             // unordered well-separated pairs
    int n_p2p;             // leaf-leaf direct pairs
    int n_self;            // leaves interacting with themselves
    int n_found;           // colliding pairs found
    int n_resolved;        // colliding pairs resolved (collision resolution on)
    int walk_iters;
    int resort_ok;         // the last key sort took the nearly-sorted path (1) or the radix sort
    int n_m2l_dir;
    int n_p2p_dir;
    unsigned bar_count;
    unsigned bar_count2;   // grid barriers of the collision climb (it may run beside another cooperative kernel
                           // of the same tree set)
    unsigned bar_gen;
    int walk_abort[3];     // walk: overflow seen in generation g, slot g mod 3
    long long dec_pairs;   // walk decisions: direct cell pairs
    long long dec_self;    // walk decisions: direct self cells
    long long n_inter;     // direct particle pairs (unordered)
    long long n_tests;     // collision tests
    long long col_pairs;   // collision walk: direct cell pairs
    long long col_self;    // collision walk: direct self cells
    long long n_m2p;       // standard tree code: moonlet-cell expansions
    int col_iters;         // collision walk: generations
    int n_cp2p;            // collision walk: leaf pairs to test
    int n_cself;           // collision walk: leaves to test within
    long long dec_pairs_c; // collision walk decisions: direct cell pairs
    long long dec_self_c;  // collision walk decisions: direct self cells
    int col_stale;         // fused walk: a moonlet's R + dt |v| exceeded the bound its tree's collision
                           // geometry used, so the collision walk is redone
    unsigned long long bbox[6];   // order-preserving encodings of min x,y,z and max x,y,z
    double root[4];        // x_lo, y_lo, z_lo, L
    // Several independent disks in one tree set (a forest): nd roots, cells 0..nd-1; disk d holds the
    // moonlets [doff[d], doff[d + 1]) in every order (the key sort orders by (disk, key)).  One disk:
    // nd = 1, disk_of = doff = null, dbox / droot point at bbox / root above.  Set once per context.
    int nd;
    const unsigned short *disk_of;   // [n] disk of each moonlet (null: one disk)
    const int *doff;                 // [nd + 1]
    unsigned long long *dbox;        // [nd][6] order-preserving encodings of each disk's box
    double *droot;                   // [nd][4] each disk's root cube: x_lo, y_lo, z_lo, L
    unsigned long long wait_ns;   // limit of a grid barrier's wait (0: one second); set once per context
    unsigned desc_epoch;   // epoch of the current descent (advanced by every M2L launch; never reset)
    int stall;             // nonzero: the grid barriers of this tree set wait for one arrival that never
                           // comes, so each gives up after wait_ns (failure-path tests; cleared per call)
};

// order-preserving map double -> uint64 (for atomicMin/atomicMax)
__device__ __forceinline__ unsigned long long ord_encode(double v) {
    unsigned long long u = __double_as_longlong(v);
    return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double ord_decode(unsigned long long u) {
    unsigned long long b = (u & 0x8000000000000000ull) ? (u & 0x7FFFFFFFFFFFFFFFull) : ~u;
    return __longlong_as_double(static_cast<long long>(b));
}

// disk of moonlet i (tree or caller order: the disks' ranges are the same) and its root cube
__device__ __forceinline__ int disk_of(const Ctrl *ctl, int i) { return ctl->disk_of ? ctl->disk_of[i] : 0; }
__device__ __forceinline__ const double *disk_root(const Ctrl *ctl, int d) { return ctl->droot + 4 * d; }

// Folds a lane's coordinates into the box of its disk d (forests: every lane of the warp calls this;
// a warp within one disk reduces first and adds one atomic per bound).
__device__ __forceinline__ void fold_disk_box(Ctrl *ctl, int d, bool valid, const unsigned long long lo[3],
                                              const unsigned long long hi[3]) {
    const unsigned same = __match_any_sync(0xffffffffu, valid ? d : -1);
    if (same == 0xffffffffu && valid) {
        unsigned long long l[3] = {lo[0], lo[1], lo[2]}, h[3] = {hi[0], hi[1], hi[2]};
#pragma unroll
        for (int k = 0; k < 3; k++)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long a = __shfl_xor_sync(0xffffffffu, l[k], o);
                const unsigned long long b = __shfl_xor_sync(0xffffffffu, h[k], o);
                l[k] = a < l[k] ? a : l[k];
                h[k] = b > h[k] ? b : h[k];
            }
        if ((threadIdx.x & 31) == 0)
#pragma unroll
            for (int k = 0; k < 3; k++) {
                atomicMin(&ctl->dbox[6 * d + k], l[k]);
                atomicMax(&ctl->dbox[6 * d + 3 + k], h[k]);
            }
    } else if (valid) {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            atomicMin(&ctl->dbox[6 * d + k], lo[k]);
            atomicMax(&ctl->dbox[6 * d + 3 + k], hi[k]);
        }
    }
}

// true when an earlier stage overflowed a buffer or timed out: later kernels
// then do nothing (their inputs may reference entries that were never
// written), and the host reruns the call with larger buffers.
__device__ __forceinline__ bool aborted(const Ctrl *ctl) {
    return (*reinterpret_cast<const volatile int *>(&ctl->err) & ERR_ABORT_MASK) != 0;
}

// ---- bounded grid barrier (cooperative launches only) ----------------------
// Every block must be resident (cudaLaunchCooperativeKernel guarantees it or
// fails).  The arrival counter only grows within a launch (it is zeroed before
// the launch): barrier k of the launch is passed when it reaches (k + 1) times
// the grid size.  Each block's thread 0 adds its arrival with release
// semantics and polls with acquire semantics, so the writes of the whole
// block before the barrier (ordered by __syncthreads) are visible to every
// block after it.  A wait longer than ctl->wait_ns (one second when 0) sets
// ERR_TIMEOUT and returns false; the kernels then leave, so no launch can
// hang.  A block that gives up also sets BAR_FAILED in the counter, so that
// a block arriving later fails at once instead of passing with the arrivals
// already counted and running on alone.  `passed` counts the grid-size steps
// of the barriers this block has passed.  With ctl->stall set the barrier
// also waits for one arrival that no block makes, so every block gives up
// after the limit (the host-armed failure of the failure-path tests).
constexpr unsigned BAR_FAILED = 1u << 30;   // (a launch's arrivals stay far below)
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add_u32(unsigned *p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Acquire-release fence at device scope: orders this thread's earlier memory
// accesses before its later ones for every thread of the GPU that
// synchronises with it through an atomic or a flag (much cheaper than the
// sequentially consistent fence of __threadfence()).
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// the barrier on any arrival counter (ctl->bar_count or a kernel's own)
__device__ __forceinline__ bool grid_sync_on(unsigned *counter, Ctrl *ctl, unsigned &passed) {
    __syncthreads();
    __shared__ int s_ok;
    passed += gridDim.x;
    if (threadIdx.x == 0) {
        red_release_add_u32(counter, 1u);
        int ok = 1;
        const unsigned long long t0 = global_ns();
        const unsigned long long limit = ctl->wait_ns ? ctl->wait_ns : 1000000000ull;
        const unsigned target = passed + (ctl->stall ? 1u : 0u);
        for (unsigned spins = 0;; spins++) {
            const unsigned v = ld_acquire_u32(counter);
            if (v & BAR_FAILED) {   // another block gave up
                ok = 0;
                break;
            }
            if (static_cast<int>(v - target) >= 0) break;
            if ((spins & 255u) == 255u && global_ns() - t0 > limit) {
                atomicOr(&ctl->err, ERR_TIMEOUT);
                atomicOr(counter, BAR_FAILED);
                ok = 0;
                break;
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ bool grid_sync(Ctrl *ctl, unsigned &passed) { return grid_sync_on(&ctl->bar_count, ctl, passed); }

// ---- warp helpers -----------------------------------------------------------
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// Warp-aggregated append: every active lane wants `k` slots in a list whose
// length is *counter; returns the lane's first slot (slots >= cap must be
// treated as overflow by the caller).  All lanes of the warp must call it.
__device__ __forceinline__ int warp_append(int *counter, int k) {
    unsigned lane = lane_id();
    int incl = k;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int v = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)lane >= o) incl += v;
    }
    int total = __shfl_sync(0xffffffffu, incl, 31);
    int base = 0;
    if (lane == 31 && total > 0) base = atomicAdd(counter, total);
    base = __shfl_sync(0xffffffffu, base, 31);
    return base + incl - k;
}

__device__ __forceinline__ int warp_sum(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace ncorp
