// sort.cu -- root cube, quantisation, 3-D Hilbert keys, their sort (LSD
// radix sort, or the merge of the few out-of-place keys of a step), and the
// gather of the moonlet state into key order.
//
// Sect. 3.4.6: cells of a level are ordered along a 3-D Hilbert curve and
// moonlets are inserted in the Hilbert order of their leaves.  Here every
// moonlet gets the 63-bit Hilbert index of its quantised position (21 bits
// per axis inside the root cube) and the state is sorted by (key, caller
// index), so that every cell of every level owns a contiguous range of
// moonlets and consecutive cells of a level are consecutive along the curve.
#include <algorithm>
#include <cfloat>
#include <cstdlib>
#include <mutex>

#include "ctx.h"

namespace ncorp {

// ---------------------------------------------------------------------------
// bounding box
// ---------------------------------------------------------------------------
// One block per SM at most; every thread folds its moonlets into running
// minima and maxima of the order-preserving integer images of the
// coordinates (integer min/max, no FP64 instruction), the block reduces them
// in shared memory and adds one atomic per bound.  A coordinate whose
// exponent field is all ones (infinite or NaN) sets ERR_NONFINITE.  With a
// gate, the launch does nothing while *gate is 0.
__global__ void __launch_bounds__(256) k_bbox(const double *__restrict__ x, const double *__restrict__ y,
                                              const double *__restrict__ z, int n, Ctrl *ctl,
                                              const int *gate = nullptr) {
    __shared__ unsigned long long s_b[6][8];
    __shared__ int s_bad;
    if ((gate && *gate == 0) || aborted(ctl)) return;
    unsigned long long lo[3] = {~0ull, ~0ull, ~0ull}, hi[3] = {0ull, 0ull, 0ull};
    bool bad = false;
    if (ctl->disk_of) {   // a forest: every disk's own box
        const int lane = threadIdx.x & 31;
        for (int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += gridDim.x * blockDim.x) {
            const int i = base + lane;
            const bool valid = i < n;
            unsigned long long l[3] = {~0ull, ~0ull, ~0ull}, h[3] = {0ull, 0ull, 0ull};
            if (valid) {
                const double v[3] = {x[i], y[i], z[i]};
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(v[k]));
                    bad |= (u & 0x7ff0000000000000ull) == 0x7ff0000000000000ull;
                    l[k] = h[k] = ord_encode(v[k]);
                }
            }
            fold_disk_box(ctl, valid ? ctl->disk_of[i] : 0, valid, l, h);
        }
        if (bad) atomicOr(&ctl->err, ERR_NONFINITE);
        return;
    }
    if (threadIdx.x == 0) s_bad = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double v[3] = {x[i], y[i], z[i]};
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(v[k]));
            bad |= (u & 0x7ff0000000000000ull) == 0x7ff0000000000000ull;
            const unsigned long long e = ord_encode(v[k]);
            lo[k] = e < lo[k] ? e : lo[k];
            hi[k] = e > hi[k] ? e : hi[k];
        }
    }
#pragma unroll
    for (int k = 0; k < 3; k++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long a = __shfl_xor_sync(0xffffffffu, lo[k], o);
            const unsigned long long b = __shfl_xor_sync(0xffffffffu, hi[k], o);
            lo[k] = a < lo[k] ? a : lo[k];
            hi[k] = b > hi[k] ? b : hi[k];
        }
    __syncthreads();
    if (__any_sync(0xffffffffu, bad) && lane_id() == 0) s_bad = 1;
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane_id() == 0)
#pragma unroll
        for (int k = 0; k < 3; k++) {
            s_b[k][w] = lo[k];
            s_b[3 + k][w] = hi[k];
        }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int k = threadIdx.x;
        unsigned long long r = s_b[k][0];
        for (int j = 1; j < nw; j++) {
            const unsigned long long v = s_b[k][j];
            r = k < 3 ? (v < r ? v : r) : (v > r ? v : r);
        }
        if (k < 3) atomicMin(&ctl->bbox[k], r);
        else atomicMax(&ctl->bbox[k], r);
    }
    if (threadIdx.x == 0 && s_bad) atomicOr(&ctl->err, ERR_NONFINITE);
}

// ---------------------------------------------------------------------------
// Hilbert index: J. Skilling, "Programming the Hilbert curve", AIP Conf. Proc.
// 707 (2004).  The axes are first brought to the curve's "transpose" form by
// walking the bit planes from the top (a set bit reflects the lower bits of
// axis 0, a clear bit swaps the lower bits of axis 0 and the current axis),
// then Gray-encoded; the key interleaves the three transposed words, axis 0
// first, most significant plane first.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t spread3(uint32_t v) {
    uint64_t x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x001f00000000ffffull;
    x = (x | (x << 16)) & 0x001f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

__device__ __forceinline__ uint64_t hilbert_key(uint32_t a0, uint32_t a1, uint32_t a2) {
    uint32_t w0 = a0, w1 = a1, w2 = a2;
    for (uint32_t Q = 1u << (KEY_BITS - 1); Q > 1u; Q >>= 1) {
        const uint32_t P = Q - 1u;
        if (w0 & Q) w0 ^= P;
        if (w1 & Q) {
            w0 ^= P;
        } else {
            uint32_t t = (w0 ^ w1) & P;
            w0 ^= t;
            w1 ^= t;
        }
        if (w2 & Q) {
            w0 ^= P;
        } else {
            uint32_t t = (w0 ^ w2) & P;
            w0 ^= t;
            w2 ^= t;
        }
    }
    w1 ^= w0;
    w2 ^= w1;
    uint32_t t = 0;
    for (uint32_t Q = 1u << (KEY_BITS - 1); Q > 1u; Q >>= 1)
        if (w2 & Q) t ^= Q - 1u;
    w0 ^= t;
    w1 ^= t;
    w2 ^= t;
    return (spread3(w0) << 2) | (spread3(w1) << 1) | spread3(w2);
}

// Root cube: centre = midpoint of the bounding box, side L = smallest power of
// two >= (max extent)(1 + 2^-20); q = floor((x - x_lo) 2^21 / L), clamped.
__device__ void root_cube(const unsigned long long *box, double out[4]) {
    double lo[3], hi[3], ext = 0.0;
    for (int k = 0; k < 3; k++) {
        lo[k] = ord_decode(box[k]);
        hi[k] = ord_decode(box[3 + k]);
        double e = dsub(hi[k], lo[k]);
        if (e > ext) ext = e;
    }
    double t = dmul(ext, 1.0 + 0x1p-20);
    double L = 1.0;
    if (t > 0.0) {
        while (L < t) L = dmul(L, 2.0);
        while (dmul(L, 0.5) >= t) L = dmul(L, 0.5);
    }
    for (int k = 0; k < 3; k++) out[k] = dsub(dmul(dadd(lo[k], hi[k]), 0.5), dmul(L, 0.5));
    out[3] = L;
}

// floor(dmul(dsub(v, lo), 2^s)) clamped to [0, 2^21 - 1], with one FP64
// instruction: the scaling by a power of two is exact, so the floor of the
// scaled difference is its significand shifted right, done in integers.
__device__ __forceinline__ uint32_t quantise(double v, double lo, int s) {
    const double d = dsub(v, lo);
    const long long u = __double_as_longlong(d);
    if (u <= 0) return 0u;                                   // d <= 0 (or -0)
    const int ex = static_cast<int>((u >> 52) & 0x7ff);
    const unsigned long long m = (static_cast<unsigned long long>(u) & 0xfffffffffffffull) | (ex ? (1ull << 52) : 0ull);
    const int sh = 1075 - (ex ? ex : 1) - s;                 // d 2^s = m 2^-sh
    const unsigned long long q = sh <= 0 ? ~0ull : (sh >= 64 ? 0ull : m >> sh);
    const unsigned long long qmax = (1u << KEY_BITS) - 1u;
    return static_cast<uint32_t>(q > qmax ? qmax : q);
}

__global__ void k_keys(const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z,
                       int n, Ctrl *ctl, uint64_t *__restrict__ key, uint32_t *__restrict__ idx,
                       uint32_t *__restrict__ qx, uint32_t *__restrict__ qy, uint32_t *__restrict__ qz,
                       const int *gate = nullptr) {
    __shared__ double s_root[4];
    __shared__ int s_shift;
    if ((gate && *gate == 0) || aborted(ctl)) return;
    if (ctl->disk_of) {   // a forest: each moonlet in its disk's root cube (k_disk_roots made them)
        if (blockIdx.x == 0 && threadIdx.x == 0) ctl->bar_count = 0;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
            const double *r = ctl->droot + 4 * ctl->disk_of[i];
            const int sh = KEY_BITS - (static_cast<int>((__double_as_longlong(r[3]) >> 52) & 0x7ff) - 1023);
            const uint32_t a = quantise(x[i], r[0], sh);
            const uint32_t b = quantise(y[i], r[1], sh);
            const uint32_t c = quantise(z[i], r[2], sh);
            qx[i] = a;
            qy[i] = b;
            qz[i] = c;
            key[i] = hilbert_key(a, b, c);
            idx[i] = static_cast<uint32_t>(i);
        }
        return;
    }
    if (threadIdx.x == 0) {
        root_cube(ctl->bbox, s_root);
        if (blockIdx.x == 0) {
            for (int k = 0; k < 4; k++) ctl->root[k] = s_root[k];
            ctl->bar_count = 0;
        }
        // L = 2^k exactly: the scale 2^21 / L is 2^(21 - k)
        s_shift = KEY_BITS - (static_cast<int>((__double_as_longlong(s_root[3]) >> 52) & 0x7ff) - 1023);
    }
    __syncthreads();
    const int sh = s_shift;
    const double x0 = s_root[0], y0 = s_root[1], z0 = s_root[2];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t a = quantise(x[i], x0, sh);
        const uint32_t b = quantise(y[i], y0, sh);
        const uint32_t c = quantise(z[i], z0, sh);
        qx[i] = a;
        qy[i] = b;
        qz[i] = c;
        key[i] = hilbert_key(a, b, c);
        idx[i] = static_cast<uint32_t>(i);
    }
}

// A forest's root cubes, one thread per disk, from the disks' boxes.
__global__ void k_disk_roots(Ctrl *ctl, const int *gate) {
    if (gate && *gate == 0) return;
    for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < ctl->nd; d += gridDim.x * blockDim.x)
        root_cube(ctl->dbox + 6 * d, ctl->droot + 4 * d);
}

// The bounding box in ctl must be empty on entry (k_reset_ctl leaves it so),
// or already hold the positions' box (bbox_done: the step's kick-drift kernel
// folds it); k_keys also zeroes the grid-barrier counter for the sort that
// follows.
void launch_bbox_keys(ncorp_ctx *c, const double *x, const double *y, const double *z, int n, uint64_t *key,
                      uint32_t *qx, uint32_t *qy, uint32_t *qz, bool bbox_done, const int *gate) {
    if (!bbox_done) {
        k_bbox<<<grid_for(n, 256, c->num_sms), 256, 0, c->stream>>>(x, y, z, n, c->ctl, gate); c->launches++;
        NCORP_CUDA_CHECK(cudaGetLastError());
    }
    if (c->nd > 1) {
        k_disk_roots<<<grid_for(c->nd, 128), 128, 0, c->stream>>>(c->ctl, gate); c->launches++;
    }
    k_keys<<<grid_for(n, 256, 16 * c->num_sms), 256, 0, c->stream>>>(x, y, z, n, c->ctl, key, c->idx, qx, qy, qz,
                                                                       gate);
    c->launches++;
    NCORP_CUDA_CHECK(cudaGetLastError());
}

__global__ void k_bbox_reset(Ctrl *ctl, const int *gate) {
    if (*gate == 0) return;
    for (int d = 0; d < ctl->nd; d++)   // (one disk: dbox is bbox)
        for (int k = 0; k < 3; k++) {
            ctl->dbox[6 * d + k] = ~0ull;
            ctl->dbox[6 * d + 3 + k] = 0ull;
        }
}

void launch_bbox_gated(ncorp_ctx *c, const double *x, const double *y, const double *z, int n, Ctrl *ctl,
                       const int *gate) {
    k_bbox_reset<<<1, 1, 0, c->stream>>>(ctl, gate); c->launches++;
    k_bbox<<<grid_for(n, 256, c->num_sms), 256, 0, c->stream>>>(x, y, z, n, ctl, gate); c->launches++;
    NCORP_CUDA_CHECK(cudaGetLastError());
}

__device__ __forceinline__ int block_excl_scan(int v, int *s_warp, int *total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int w = lane < nw ? s_warp[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < nw) s_warp[lane] = wi - w;
        if (lane == 31) s_warp[32] = wi;
    }
    __syncthreads();
    int res = s_warp[wid] + incl - v;
    if (total) *total = s_warp[32];
    __syncthreads();
    return res;
}

// ---------------------------------------------------------------------------
// LSD radix sort of (uint64 key, uint32 value), 8-bit digits, all passes in
// one cooperative launch.  A first sweep counts the digits of every pass at
// once (global histograms, hence the digit starts of each pass).  Then each
// pass ranks every tile's keys locally (stable, warp-synchronous: the lanes
// holding equal digits are found with one ballot per digit bit; each warp owns
// a contiguous slice of the tile, warps are ordered by a per-digit prefix), and finds, per digit, how many keys of the
// tiles before it carry the digit by decoupled look-back (Merrill & Garland,
// "Single-pass parallel prefix scan with decoupled look-back", 2016): a tile
// publishes its own count, reads its predecessors' words sixteen at a time
// back to the nearest published running total, then publishes its own
// running total.  A status word holds (tag, kind, value); the tag names the
// sort call and the pass, so words of other passes or calls are never
// mistaken for this one's and nothing has to be cleared.  Waits are bounded:
// a wait that runs out sets ERR_TIMEOUT and the call fails.  One grid
// barrier ends each pass.
// ---------------------------------------------------------------------------
constexpr int RS_T = 256, RS_I = 8, RS_TILE = RS_T * RS_I, RS_W = RS_T / 32, RS_SLICE = RS_TILE / RS_W;
constexpr int RS_MAX_PASSES = 10;   // 8 key passes, and for a forest the disk pass and a copy pass
constexpr unsigned long long RS_AGG = 0ull, RS_INC = 1ull << 31;   // kind bit of a status word

struct RadixArgs {
    uint64_t *k0, *k1;
    uint32_t *v0, *v1;
    int n, ntiles, passes;
    unsigned long long *status;   // [ntiles][256]: tag << 32 | kind << 31 | value
    long long status_words;       // size of the whole status region (>= ntiles * 256)
    int *ghist;                   // [2][RS_MAX_PASSES][256]: half (epoch & 1) zero on entry, the other
                                  // half zeroed by the call for the next one
    unsigned *epoch;              // device counter: this call's tag base, advanced by the call
    unsigned epoch_limit;         // at this epoch the call clears the status region and restarts from 0
    Ctrl *ctl;
    const int *gate;              // k_radix: nothing to do while *gate is 0 (null: always sort)
};

// Tags are (epoch + 1) * 8 + pass in 32 bits; well before they would wrap, the
// sort that reaches the limit clears every status word and restarts the epoch.
constexpr unsigned RS_EPOCH_LIMIT = 1u << 28;

__device__ __forceinline__ unsigned long long ld_status(const unsigned long long *p) {
    return *reinterpret_cast<const volatile unsigned long long *>(p);
}

// The whole sort, run by every block of a cooperative grid of any size (256
// threads per block); bar counts the grid barriers the blocks have passed.
// Returns false if a grid barrier gave up (the call has failed).
__device__ bool radix_body(const RadixArgs &A, unsigned &bar) {
    __shared__ int s_cnt[RS_W][256];
    __shared__ int s_start[256];
    __shared__ int s_excl[256];
    __shared__ int s_warp[33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int n = A.n, ntiles = A.ntiles;
    // every block reads the call's epoch before the first barrier; block 0 advances it after
    const unsigned epoch = *reinterpret_cast<volatile unsigned *>(A.epoch);
    int *const ghist = A.ghist + (epoch & 1u) * (RS_MAX_PASSES * 256);
    {   // the next call's histograms (nobody reads them in this call)
        int *const nxt = A.ghist + ((epoch + 1u) & 1u) * (RS_MAX_PASSES * 256);
        for (int i = blockIdx.x * RS_T + threadIdx.x; i < RS_MAX_PASSES * 256; i += gridDim.x * RS_T) nxt[i] = 0;
    }
    // ---- 0. digit counts of every key pass (s_cnt reused as [8][256]); a forest's disk pass counts
    // are the disks' sizes and its copy pass has the one digit 0, written by block 0
    const int kpasses = min(A.passes, 8);
    {
        int *s_h = &s_cnt[0][0];
        for (int i = threadIdx.x; i < 8 * 256; i += RS_T) s_h[i] = 0;
        __syncthreads();
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            const long long base = static_cast<long long>(tile) * RS_TILE;
            for (int k = 0; k < RS_I; k++) {
                const long long i = base + static_cast<long long>(k) * RS_T + threadIdx.x;
                if (i < n) {
                    const uint64_t key = A.k0[i];
                    for (int p = 0; p < kpasses; p++) atomicAdd(&s_h[p * 256 + ((key >> (8 * p)) & 0xffu)], 1);
                }
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kpasses * 256; i += RS_T)
            if (s_h[i]) atomicAdd(&ghist[i], s_h[i]);
        if (A.passes > 8 && blockIdx.x == 0) {
            const int t = threadIdx.x;   // RS_T = 256 threads: one digit each
            ghist[8 * 256 + t] = t < A.ctl->nd ? A.ctl->doff[t + 1] - A.ctl->doff[t] : 0;
            ghist[9 * 256 + t] = t == 0 ? n : 0;
        }
    }
    if (!grid_sync(A.ctl, bar)) return false;
    const bool wrap = epoch + 1 >= A.epoch_limit;
    if (blockIdx.x == 0 && threadIdx.x == 0) *A.epoch = wrap ? 0u : epoch + 1;
    for (int ps = 0; ps < A.passes; ps++) {
        const int shift = 8 * ps;
        const uint64_t *kin = (ps & 1) ? A.k1 : A.k0;
        const uint32_t *vin = (ps & 1) ? A.v1 : A.v0;
        uint64_t *kout = (ps & 1) ? A.k0 : A.k1;
        uint32_t *vout = (ps & 1) ? A.v0 : A.v1;
        const unsigned long long tag = static_cast<unsigned long long>((epoch + 1) * RS_MAX_PASSES + ps) << 32;
        s_start[threadIdx.x] = block_excl_scan(__ldcg(&ghist[ps * 256 + threadIdx.x]), s_warp, nullptr);
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            for (int d = lane; d < 256; d += 32) s_cnt[w][d] = 0;
            __syncwarp();
            const long long base = static_cast<long long>(tile) * RS_TILE + static_cast<long long>(w) * RS_SLICE;
            uint64_t kk[RS_I];
            uint32_t vv[RS_I];
            int rank[RS_I];
#pragma unroll
            for (int r = 0; r < RS_I; r++) {   // all loads first: they are in flight together
                const long long i = base + r * 32 + lane;
                kk[r] = i < n ? __ldcg(&kin[i]) : 0ull;
                vv[r] = i < n ? __ldcg(&vin[i]) : 0u;
            }
#pragma unroll
            for (int r = 0; r < RS_I; r++) {
                const long long i = base + r * 32 + lane;
                const bool ok = i < n;
                const int d = ps < 8 ? static_cast<int>((kk[r] >> shift) & 0xffu)
                                     : (ps == 8 && ok ? A.ctl->disk_of[vv[r]] : 0);   // disk pass, copy pass
                // lanes holding the same digit: one ballot per digit bit, every lane of the warp taking part
                // in every ballot (lanes past n start from the mask of valid lanes and keep only themselves)
                unsigned peers = __ballot_sync(0xffffffffu, ok);
#pragma unroll
                for (int bit = 0; bit < 8; bit++) {
                    const bool set = (d >> bit) & 1;
                    const unsigned m = __ballot_sync(0xffffffffu, set);
                    peers &= set ? m : ~m;
                }
                if (!ok) peers = 1u << lane;
                const int before = ok ? s_cnt[w][d] : 0;
                rank[r] = before + __popc(peers & lt);
                __syncwarp();
                if (ok && (__ffs(peers) - 1) == lane) s_cnt[w][d] = before + __popc(peers);
                __syncwarp();
            }
            __syncthreads();
            {
                const int d = threadIdx.x;
                int acc = 0;   // exclusive prefix over warps; acc ends as the tile's count of digit d
                for (int ww = 0; ww < RS_W; ww++) {
                    const int t = s_cnt[ww][d];
                    s_cnt[ww][d] = acc;
                    acc += t;
                }
                unsigned long long *st = A.status + static_cast<size_t>(tile) * 256 + d;
                if (tile == 0) {
                    *reinterpret_cast<volatile unsigned long long *>(st) = tag | RS_INC | static_cast<unsigned>(acc);
                    s_excl[d] = 0;
                } else {
                    *reinterpret_cast<volatile unsigned long long *>(st) = tag | RS_AGG | static_cast<unsigned>(acc);
                    // look back, sixteen predecessors at a time, to the nearest running total
                    int excl = 0, t = tile - 1;
                    bool done = false;
                    while (!done) {
                        const int m = min(16, t + 1);
                        unsigned long long wv[16];
#pragma unroll
                        for (int u = 0; u < 16; u++)
                            wv[u] = u < m ? ld_status(A.status + static_cast<size_t>(t - u) * 256 + d) : 0ull;
                        for (int u = 0; u < m && !done; u++) {
                            long long spins = 0;
                            while ((wv[u] & 0xffffffff00000000ull) != tag) {
                                if (++spins > (1ll << 22)) {
                                    atomicOr(&A.ctl->err, ERR_TIMEOUT);
                                    wv[u] = tag | RS_INC;
                                    break;
                                }
                                __nanosleep(32);
                                wv[u] = ld_status(A.status + static_cast<size_t>(t - u) * 256 + d);
                            }
                            excl += static_cast<int>(wv[u] & 0x7fffffffull);
                            if (wv[u] & RS_INC) done = true;
                        }
                        t -= m;
                        if (t < 0) done = true;
                    }
                    *reinterpret_cast<volatile unsigned long long *>(st) =
                        tag | RS_INC | static_cast<unsigned>(excl + acc);
                    s_excl[d] = excl;
                }
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < RS_I; r++) {
                const long long i = base + r * 32 + lane;
                if (i < n) {
                    const int d = ps < 8 ? static_cast<int>((kk[r] >> shift) & 0xffu)
                                         : (ps == 8 ? A.ctl->disk_of[vv[r]] : 0);
                    const int pos = s_start[d] + s_excl[d] + s_cnt[w][d] + rank[r];
                    // always in range for a consistent prefix; a look-back that gave up (ERR_TIMEOUT, the
                    // call fails) must not write outside the arrays
                    if (static_cast<unsigned>(pos) < static_cast<unsigned>(n)) {
                        kout[pos] = kk[r];
                        vout[pos] = vv[r];
                    }
                }
            }
            __syncthreads();
        }
        if (ps + 1 < A.passes && !grid_sync(A.ctl, bar)) return false;
    }
    if (wrap) {   // every look-back of the call is over after this barrier: no status word is read again
        if (!grid_sync(A.ctl, bar)) return false;
        for (long long i = static_cast<long long>(blockIdx.x) * RS_T + threadIdx.x; i < A.status_words;
             i += static_cast<long long>(gridDim.x) * RS_T)
            A.status[i] = 0ull;
        for (int i = blockIdx.x * RS_T + threadIdx.x; i < RS_MAX_PASSES * 256; i += gridDim.x * RS_T)
            ghist[i] = 0;   // the next call (epoch 0) takes the first half
    }
    return true;
}

__global__ void __launch_bounds__(RS_T) k_radix(RadixArgs A) {
    // every block returns before the first barrier (an aborted step's keys are never used)
    if ((A.gate && *A.gate == 0) || aborted(A.ctl)) return;
    unsigned bar = 0;
    radix_body(A, bar);
}

// Sorts keys/vals in place (the alt buffers are scratch); `bits` low bits of
// the key are significant (rounded up to an even number of 8-bit passes, so
// the result ends in the input buffers).  bar_zeroed: the caller's stream has
// already zeroed ctl->bar_count since the last cooperative kernel.
// The epoch at which a context's sorts clear their status words: the constant
// above, or a smaller value from NCORP_RADIX_EPOCH_LIMIT (read at context
// creation; lets a test reach the clearing path in a few calls).
unsigned radix_epoch_limit() {
    const char *e = std::getenv("NCORP_RADIX_EPOCH_LIMIT");
    if (e) {
        const long long v = std::atoll(e);
        if (v >= 1 && v <= static_cast<long long>(RS_EPOCH_LIMIT)) return static_cast<unsigned>(v);
    }
    return RS_EPOCH_LIMIT;
}

// Layout of the context's radix scratch (ints): two sets of digit histograms
// of every pass at [0, 2 RS_MAX_PASSES 256), the epoch counter at RS_EPOCH_AT, the tile
// status words from RS_STATUS_AT on.  The status words never share memory with anything
// else, so a word left by an earlier sort (of any size) carries an older tag.
constexpr int RS_EPOCH_AT = 2 * RS_MAX_PASSES * 256;
constexpr int RS_STATUS_AT = 2 * RS_MAX_PASSES * 256 + 64;

void ensure_radix_scratch(ncorp_ctx *c, int n) {
    const int ntiles = std::max(1, (n + RS_TILE - 1) / RS_TILE);
    const int need = RS_STATUS_AT + 2 * 256 * ntiles;   // status words take two ints each
    if (c->tile_hist_cap < need) {
        // the capacity is recorded only once the buffer exists, so a failed allocation leaves none
        if (c->tile_hist) cudaFree(c->tile_hist);
        c->tile_hist = nullptr;
        c->tile_hist_cap = 0;
        bump_alloc_generation();
        int *p = nullptr;
        const cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&p), sizeof(int) * (need + 4096));
        if (e != cudaSuccess) {
            cudaGetLastError();   // (reported here; a later check must not see it again)
            throw CudaError(e, "cudaMalloc", __FILE__, __LINE__);
        }
        c->tile_hist = p;
        // on the context's stream, ordered before the sorts that use it (the legacy stream is not
        // ordered with the non-blocking streams the library is driven on)
        NCORP_CUDA_CHECK(cudaMemsetAsync(c->tile_hist, 0, sizeof(int) * (need + 4096), c->stream));
        c->tile_hist_cap = need + 4096;
    }
}

static RadixArgs radix_args(ncorp_ctx *c, uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt,
                            int n, int bits, bool by_disk = false) {
    ensure_radix_scratch(c, n);
    if (c->radix_dirty) {
        // A sort of an earlier call may have stopped at a timed-out barrier before advancing the epoch,
        // leaving counts in the histograms the next sort would take as zeroed: start from clean scratch
        // (epoch 0, zero histograms, status words with tag 0, which no sort uses).
        NCORP_CUDA_CHECK(cudaMemsetAsync(c->tile_hist, 0, sizeof(int) * c->tile_hist_cap, c->stream));
        c->radix_dirty = false;
    }
    int passes = (bits + 7) / 8;
    if (passes & 1) passes++;
    if (by_disk) passes = RS_MAX_PASSES;   // the key passes, the disk pass and the copy pass
    RadixArgs A;
    A.k0 = keys; A.k1 = keys_alt; A.v0 = vals; A.v1 = vals_alt;
    A.n = n; A.ntiles = (n + RS_TILE - 1) / RS_TILE; A.passes = passes;
    A.status = reinterpret_cast<unsigned long long *>(c->tile_hist + RS_STATUS_AT);
    A.status_words = (c->tile_hist_cap - RS_STATUS_AT) / 2;
    A.ghist = c->tile_hist;
    A.epoch = reinterpret_cast<unsigned *>(c->tile_hist + RS_EPOCH_AT);
    A.epoch_limit = c->radix_epoch_limit;
    A.ctl = c->ctl;
    A.gate = nullptr;
    return A;
}

void radix_sort_u64(ncorp_ctx *c, uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, int n,
                    int bits, bool bar_zeroed, const int *gate, bool by_disk) {
    if (n <= 1) return;
    RadixArgs A = radix_args(c, keys, vals, keys_alt, vals_alt, n, bits, by_disk && c->nd > 1);
    A.gate = gate;
    int per_sm = 0;
    NCORP_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, reinterpret_cast<const void *>(k_radix),
                                                                   RS_T, 0));
    if (per_sm < 1) per_sm = 1;
    if (per_sm > 2) per_sm = 2;
    const int grid = std::min(A.ntiles, coop_blocks(c, per_sm));
    if (!bar_zeroed) NCORP_CUDA_CHECK(cudaMemsetAsync(&c->ctl->bar_count, 0, sizeof(unsigned), c->stream));
    void *args[] = {&A};
    NCORP_CUDA_CHECK(cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(k_radix), dim3(grid), dim3(RS_T), args,
                                                 0, c->stream));
    c->launches++;
}

// ---------------------------------------------------------------------------
// Sorting keys that are nearly sorted already.  In a step the keys are
// computed in the previous step's tree order; a drift moves most moonlets
// by a small fraction of their spacing, so only a few keys are out of place
// (at dt = 1e-3 on the 1e5 disk: 627 of 1e5, i.e. n minus the longest
// sorted subsequence).  One cooperative launch:
//   1. every key adjacent to a descent (k[i] > k[i+1]) is a "mover", and so
//      is a key out of order with the nearest non-adjacent keys on either
//      side (a second round: a few keys that moved together leave the inner
//      ones of their run behind; on the 1e6 disk at dt = 1e-3 the first
//      round leaves 46 of them out of order, the second none); the rest are
//      "stayers"; per-block counts;
//   2. stayers and movers are compacted in input order (stayer keys and
//      indices into the radix sort's scratch arrays, movers into a small
//      buffer);
//   3. the stayers are checked to be sorted, and the movers are sorted: by
//      rank in shared memory when they are few (the count of movers with a
//      smaller key, one warp per mover), else by the radix sort of the movers
//      alone;
//   4. the two sorted sequences are merged: a stayer goes to its rank among
//      the stayers plus the number of movers with a smaller key (each block
//      takes a contiguous run of stayers and the movers whose keys fall in
//      its key range), a mover to its rank among the movers plus the number
//      of stayers with a key not larger than its own.
// The result is sorted by key (equal keys in any order: the gather ranks
// them by caller index).  If there are more than RS_MOVERS_MAX movers or
// the stayers are not sorted, nothing has been written to the keys or the
// index (the index must be the identity on entry) and the same launch sorts
// them with the full radix sort; ctl->resort_ok tells which path ran (1
// fast with the movers ranked, 2 fast with the movers' radix sort, 0 or -1
// the full radix sort).
// ---------------------------------------------------------------------------
constexpr int RS_MOVERS_MAX = RESORT_MOVERS_CAP;
constexpr int RS_MOVERS_SMEM = 4096;  // movers ranked in shared memory; larger counts take the movers' radix sort
constexpr int RS_MSLICE = 4096;       // movers of a block's key range searched in shared memory
constexpr int RS_SAMPLES = 2048;      // stayer keys sampled into shared memory for the movers' searches
constexpr int RZ_T = 256;

struct ResortArgs {
    RadixArgs radix;      // the full sort of the same arrays (its alt buffers are the stayer scratch)
    RadixArgs movers;     // the radix sort of the movers (m_key, m_idx; alt m_key2, m_idx2), n set on the device
    uint64_t *key;        // [n] in: keys in input order; out: sorted
    uint32_t *idx;        // [n] in: identity; out: input index of every sorted key
    uint64_t *s_key;      // [n] scratch: stayer keys
    uint32_t *s_idx;      // [n] scratch: stayer input indices
    uint64_t *m_key;      // [RS_MOVERS_MAX] movers in input order
    uint32_t *m_idx;
    uint64_t *m_key2;     // [RS_MOVERS_MAX] movers sorted by key (rank path) / scratch (radix path)
    uint32_t *m_idx2;
    int *bcount;          // [gridDim.x] movers per block
    int n;
    Ctrl *ctl;
};

__device__ __forceinline__ bool next_to_descent(const uint64_t *k, int i, int n) {
    const uint64_t v = k[i];
    return (i > 0 && k[i - 1] > v) || (i + 1 < n && v > k[i + 1]);
}

constexpr int RZ_REACH = 16;   // a key with this many keys next to descents beside it is a mover

__device__ __forceinline__ bool is_mover(const uint64_t *k, int i, int n) {
    if (next_to_descent(k, i, n)) return true;
    const uint64_t v = k[i];
    int j = i - 1;   // the nearest key before i that is not next to a descent
    for (int steps = 0; j >= 0 && next_to_descent(k, j, n); j--)
        if (++steps == RZ_REACH) return true;
    if (j >= 0 && k[j] > v) return true;
    j = i + 1;       // and after i
    for (int steps = 0; j < n && next_to_descent(k, j, n); j++)
        if (++steps == RZ_REACH) return true;
    return j < n && v > k[j];
}

// number of a[lo, hi) (sorted) smaller than v, plus lo
__device__ __forceinline__ int count_below(const unsigned long long *a, int lo, int hi, unsigned long long v) {
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldcg(&a[mid]) < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(RZ_T) k_resort(ResortArgs A) {
    extern __shared__ unsigned long long rz_smem[];
    __shared__ int s_warp[33];
    __shared__ int s_range[2];
    if (aborted(A.ctl)) return;   // every block, before the first barrier
    const int n = A.n, G = gridDim.x, b = blockIdx.x, t = threadIdx.x;
    const int chunk = (n + G - 1) / G, c0 = min(n, b * chunk), c1 = min(n, c0 + chunk);
    unsigned bar = 0;
    if (b == 0 && t == 0) A.ctl->resort_ok = 0;
    // ---- 1. movers per block
    int mine = 0;
    for (int i = c0 + t; i < c1; i += RZ_T) mine += is_mover(A.key, i, n) ? 1 : 0;
    int cnt = 0;
    block_excl_scan(mine, s_warp, &cnt);
    if (t == 0) A.bcount[b] = cnt;
    if (!grid_sync(A.ctl, bar)) return;
    // ---- 2. prefix over the blocks, total; compaction in input order
    int before = 0, total = 0;
    for (int j = t; j < G; j += RZ_T) {
        const int v = __ldcg(&A.bcount[j]);
        total += v;
        if (j < b) before += v;
    }
    block_excl_scan(before, s_warp, &before);
    block_excl_scan(total, s_warp, &total);
    if (total > RS_MOVERS_MAX) {           // uniform: every block computed the same total
        radix_body(A.radix, bar);
        return;
    }
    const int nm = total, ns = n - nm;
    {
        int mb = before, sb = c0 - before;   // this block's first mover and stayer slots
        for (int base = c0; base < c1; base += RZ_T) {
            const int i = base + t;
            const bool ok = i < c1;
            const bool mv = ok && is_mover(A.key, i, n);
            int tot_m = 0;
            const int rm = block_excl_scan(mv ? 1 : 0, s_warp, &tot_m);
            const int nok = min(RZ_T, c1 - base);
            if (mv) {
                A.m_key[mb + rm] = A.key[i];
                A.m_idx[mb + rm] = static_cast<uint32_t>(i);
            } else if (ok) {
                const int rs = t - rm;
                A.s_key[sb + rs] = A.key[i];
                A.s_idx[sb + rs] = static_cast<uint32_t>(i);
            }
            mb += tot_m;
            sb += nok - tot_m;
        }
    }
    if (!grid_sync(A.ctl, bar)) return;
    // ---- 3. stayers sorted?  movers sorted (stable: equal keys keep their input order)
    {
        bool bad = false;
        for (int p = b * RZ_T + t; p + 1 < ns; p += G * RZ_T) bad |= __ldcg(&A.s_key[p]) > __ldcg(&A.s_key[p + 1]);
        if (__syncthreads_or(bad) && t == 0) A.ctl->resort_ok = -1;
    }
    const bool by_rank = nm <= RS_MOVERS_SMEM;   // uniform
    if (by_rank) {
        // a mover's place is the number of movers with a smaller key, or an equal key and a smaller
        // slot; one warp per mover, the keys in shared memory
        unsigned long long *mk = rz_smem;
        for (int q = t; q < nm; q += RZ_T) mk[q] = __ldcg(&A.m_key[q]);
        __syncthreads();
        const int lane = t & 31, gw = (b * RZ_T + t) >> 5, nwarps = (G * RZ_T) >> 5;
        for (int q = gw; q < nm; q += nwarps) {
            const unsigned long long v = mk[q];
            int r = 0;
            for (int j = lane; j < nm; j += 32) {
                const unsigned long long u = mk[j];
                r += (u < v || (u == v && j < q)) ? 1 : 0;
            }
            r = warp_sum(r);
            if (lane == 0) {
                A.m_key2[r] = v;
                A.m_idx2[r] = __ldcg(&A.m_idx[q]);
            }
        }
    } else {
        RadixArgs R = A.movers;   // sorts m_key / m_idx in place
        R.n = nm;
        R.ntiles = (nm + RS_TILE - 1) / RS_TILE;
        if (!radix_body(R, bar)) return;
    }
    if (!grid_sync(A.ctl, bar)) return;
    if (*reinterpret_cast<volatile int *>(&A.ctl->resort_ok) != 0) {   // stayers out of order (uniform)
        radix_body(A.radix, bar);
        return;
    }
    // the sorted movers
    const unsigned long long *mks = reinterpret_cast<const unsigned long long *>(by_rank ? A.m_key2 : A.m_key);
    const uint32_t *mis = by_rank ? A.m_idx2 : A.m_idx;
    // ---- 4. merge
    unsigned long long *sl = rz_smem;                   // the movers of this block's key range
    unsigned long long *smp = rz_smem + RS_MSLICE;      // every step-th stayer key
    const int step = max(1, (ns + RS_SAMPLES - 1) / RS_SAMPLES), nsmp = (ns + step - 1) / step;
    __syncthreads();   // the rank phase's reads of rz_smem are over in this block
    const int sc = (ns + G - 1) / G, p0 = min(ns, b * sc), p1 = min(ns, p0 + sc);
    if (t == 0) {
        // movers below this block's first stayer, and below its last one
        s_range[0] = p0 < p1 ? count_below(mks, 0, nm, __ldcg(&A.s_key[p0])) : 0;
        s_range[1] = p0 < p1 ? count_below(mks, s_range[0], nm, __ldcg(&A.s_key[p1 - 1])) : 0;
    }
    for (int q = t; q < nsmp; q += RZ_T) smp[q] = __ldcg(&A.s_key[q * step]);
    __syncthreads();
    const int mlo = s_range[0], mhi = s_range[1];
    const bool in_smem = mhi - mlo <= RS_MSLICE;  // uniform in the block
    if (in_smem)
        for (int q = mlo + t; q < mhi; q += RZ_T) sl[q - mlo] = __ldcg(&mks[q]);
    __syncthreads();
    for (int p = p0 + t; p < p1; p += RZ_T) {
        const unsigned long long v = __ldcg(&A.s_key[p]);
        int below;                                  // movers with a key < v: in [mlo, mhi]
        if (in_smem) {
            int lo = 0, hi = mhi - mlo;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (sl[mid] < v) lo = mid + 1;
                else hi = mid;
            }
            below = mlo + lo;
        } else {
            below = count_below(mks, mlo, mhi, v);
        }
        A.key[p + below] = v;
        A.idx[p + below] = __ldcg(&A.s_idx[p]);
    }
    // movers: one thread each; the sample search in shared memory brackets the stayers with a key <= v,
    // a binary search inside the bracket counts them
    const unsigned long long *skey = reinterpret_cast<const unsigned long long *>(A.s_key);
    for (int q = b * RZ_T + t; q < nm; q += G * RZ_T) {
        const unsigned long long v = __ldcg(&mks[q]);
        int lo = 0, hi = nsmp;                      // samples with a key <= v
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (smp[mid] <= v) lo = mid + 1;
            else hi = mid;
        }
        // stayers [0, (lo - 1) step] have keys <= v; the count ends in [(lo - 1) step + 1, lo step]
        int r = lo == 0 ? 0 : (lo - 1) * step + 1, e = min(ns, lo * step);
        while (r < e) {                             // first stayer in [r, e) with a key > v
            const int mid = (r + e) >> 1;
            if (__ldcg(&skey[mid]) <= v) r = mid + 1;
            else e = mid;
        }
        A.key[q + r] = v;
        A.idx[q + r] = __ldcg(&mis[q]);
    }
    if (b == 0 && t == 0) A.ctl->resort_ok = by_rank ? 1 : 2;
}

// Sorts keys (with idx = identity on entry) like radix_sort_u64 with the
// key bits of a Hilbert key, taking the fast path above when the keys are
// nearly sorted.  ctl->bar_count must be zero on entry (k_keys zeroes it).
void sort_near_sorted(ncorp_ctx *c, uint64_t *keys, uint32_t *idx, uint64_t *keys_alt, uint32_t *idx_alt, int n,
                      int bits) {
    if (n <= 1) return;
    ResortArgs A;
    A.radix = radix_args(c, keys, idx, keys_alt, idx_alt, n, bits);
    A.key = keys; A.idx = idx;
    A.s_key = keys_alt; A.s_idx = idx_alt;
    A.m_key = c->resort_mkey; A.m_idx = c->resort_midx; A.bcount = c->resort_bcount;
    A.m_key2 = c->resort_mkey + RESORT_MOVERS_CAP; A.m_idx2 = c->resort_midx + RESORT_MOVERS_CAP;
    A.movers = radix_args(c, A.m_key, A.m_idx, A.m_key2, A.m_idx2, std::min(n, RESORT_MOVERS_CAP), bits);
    A.n = n;
    A.ctl = c->ctl;
    const size_t smem = sizeof(unsigned long long) * (RS_MSLICE + RS_SAMPLES);
    NCORP_CUDA_CHECK(cudaFuncSetAttribute(reinterpret_cast<const void *>(k_resort),
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
    // about 512 keys per block (short compaction loops), at most one block per SM: the collision
    // search's kernels run beside this launch, and a second block of this size would not fit with
    // them on an SM (the launch would wait for them to drain); the fallback runs with the same grid
    const int want = std::max((n + 511) / 512, A.radix.ntiles);
    const int grid = std::max(1, std::min({coop_blocks(c, 1), want, RESORT_BLOCKS_CAP}));
    void *args[] = {&A};
    NCORP_CUDA_CHECK(cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(k_resort), dim3(grid), dim3(RZ_T),
                                                 args, smem, c->stream));
    c->launches++;
}

__global__ void k_iota(uint32_t *idx, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) idx[i] = i;
}

void launch_iota(ncorp_ctx *c, uint32_t *idx, int n) {
    k_iota<<<grid_for(n, 256, 8 * c->num_sms), 256, 0, c->stream>>>(idx, n); c->launches++;
    NCORP_CUDA_CHECK(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// gather: dst[i] = src[idx[i]] for the state (positions and velocities from
// src_xv, the rest from src_rest), the caller index and the quantised coords.
// Ties: the radix sort keeps moonlets with equal keys in their input order
// (the previous step's tree order), while the order is defined by (key,
// caller index).  A moonlet inside a run of equal keys therefore goes to the
// run's first slot plus its rank by caller index within the run; runs are
// found from the sorted keys (they are rare: equal keys mean the same
// quantised cell of side L / 2^21).
// ---------------------------------------------------------------------------
struct GatherArgs {
    const double *x, *y, *z, *vx, *vy, *vz, *m, *R;
    const int *perm;
    const uint32_t *qx, *qy, *qz;
    double *ox, *oy, *oz, *ovx, *ovy, *ovz, *om, *oR;
    int *operm;
    uint32_t *oqx, *oqy, *oqz;
    float4 *hi4, *lo4;
    const uint32_t *idx;
    const uint64_t *key;   // sorted keys
    const unsigned short *disk_of;   // a forest: disk of each position (equal keys of two disks are no run)
    const Ctrl *ctl;       // the tree set being built (an aborted step gathers nothing)
    double G;
    int n;
    const int *gate;       // nothing to do while *gate is 0 (null: always)
    // fused walk (nullable rc_spec): each moonlet's bound R + dt (|v + dt a| + dt |a| / 2) on its R + dt |v|
    // at the next step, from the source's velocity v and acceleration a, into rc_spec (tree order)
    const double *ax, *ay, *az;
    double *rc_spec;
    double dt;
};

__global__ void k_gather(GatherArgs g) {
    if ((g.gate && *g.gate == 0) || aborted(g.ctl)) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += gridDim.x * blockDim.x) {
        const int j = static_cast<int>(g.idx[i]);
        int d = i;
        const uint64_t k = g.key[i];
        const int dk = g.disk_of ? g.disk_of[i] : 0;
        auto same = [&](int u) { return g.key[u] == k && (!g.disk_of || g.disk_of[u] == dk); };
        if ((i > 0 && same(i - 1)) || (i + 1 < g.n && same(i + 1))) {
            int s = i, e = i + 1;
            while (s > 0 && same(s - 1)) s--;
            while (e < g.n && same(e)) e++;
            const int pj = g.perm[j];
            int r = 0;
            for (int u = s; u < e; u++) r += g.perm[g.idx[u]] < pj;
            d = s + r;
        }
        g.ox[d] = g.x[j];
        g.oy[d] = g.y[j];
        g.oz[d] = g.z[j];
        g.ovx[d] = g.vx[j];
        g.ovy[d] = g.vy[j];
        g.ovz[d] = g.vz[j];
        g.om[d] = g.m[j];
        g.oR[d] = g.R[j];
        g.operm[d] = g.perm[j];
        g.oqx[d] = g.qx[j];
        g.oqy[d] = g.qy[j];
        g.oqz[d] = g.qz[j];
        // double-float copy of the position: x = hi + lo with both parts FP32
        const double X = g.x[j], Y = g.y[j], Z = g.z[j];
        const float hx = static_cast<float>(X), hy = static_cast<float>(Y), hz = static_cast<float>(Z);
        g.hi4[d] = make_float4(hx, hy, hz, static_cast<float>(g.G * g.m[j]));
        g.lo4[d] = make_float4(static_cast<float>(X - static_cast<double>(hx)), static_cast<float>(Y - static_cast<double>(hy)),
                               static_cast<float>(Z - static_cast<double>(hz)), 0.0f);
        if (g.rc_spec) {
            const double ax = g.ax[j], ay = g.ay[j], az = g.az[j];
            const double sp = dnorm3(dadd(g.vx[j], dmul(g.dt, ax)), dadd(g.vy[j], dmul(g.dt, ay)),
                                     dadd(g.vz[j], dmul(g.dt, az)));
            g.rc_spec[d] = dadd(g.R[j], dmul(g.dt, dadd(sp, dmul(0.5 * g.dt, dnorm3(ax, ay, az)))));
        }
    }
}

void launch_gather(ncorp_ctx *c, const ParticleSet &src_xv, const ParticleSet &src_rest, ParticleSet &dst, int n,
                   const uint32_t *idx, double G, const int *gate, double spec_dt) {
    GatherArgs g;
    g.gate = gate;
    g.rc_spec = spec_dt > 0.0 ? c->cells.rc_spec : nullptr;
    g.ax = src_rest.ax; g.ay = src_rest.ay; g.az = src_rest.az;
    g.dt = spec_dt;
    g.x = src_xv.x; g.y = src_xv.y; g.z = src_xv.z;
    g.vx = src_xv.vx; g.vy = src_xv.vy; g.vz = src_xv.vz;
    g.m = src_rest.m; g.R = src_rest.R; g.perm = src_rest.perm;
    g.qx = src_xv.qx; g.qy = src_xv.qy; g.qz = src_xv.qz;
    g.ox = dst.x; g.oy = dst.y; g.oz = dst.z;
    g.ovx = dst.vx; g.ovy = dst.vy; g.ovz = dst.vz;
    g.om = dst.m; g.oR = dst.R; g.operm = dst.perm;
    g.oqx = dst.qx; g.oqy = dst.qy; g.oqz = dst.qz;
    g.hi4 = dst.hi4; g.lo4 = dst.lo4;
    g.idx = idx;
    g.key = dst.key;
    g.disk_of = c->nd > 1 ? c->disk_of : nullptr;
    g.ctl = c->ctl;
    g.G = G;
    g.n = n;
    k_gather<<<grid_for(n, 256, 16 * c->num_sms), 256, 0, c->stream>>>(g); c->launches++;
    NCORP_CUDA_CHECK(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Allocation-free keys + sort (ncorp_hilbert_sort_static): the same kernels
// as the step's key and sort stages, with every scratch buffer in one
// file-scope device array.
// ---------------------------------------------------------------------------
constexpr int STATIC_MAX_N = NCORP_STATIC_MAX_N;
constexpr int STATIC_TILES = (STATIC_MAX_N + RS_TILE - 1) / RS_TILE;

struct StaticScratch {
    Ctrl ctl;                          // bounding box, status word, barrier
    double x[STATIC_MAX_N], y[STATIC_MAX_N], z[STATIC_MAX_N];
    uint64_t key_alt[STATIC_MAX_N];
    uint32_t idx[STATIC_MAX_N], idx_alt[STATIC_MAX_N];
    uint32_t qx[STATIC_MAX_N], qy[STATIC_MAX_N], qz[STATIC_MAX_N];
    unsigned long long status[256 * STATIC_TILES];
    int ghist[2 * RS_MAX_PASSES * 256];
    unsigned epoch;                   // radix sort calls so far (tags the status words)
};

static __device__ __align__(256) StaticScratch g_static_scratch;

__global__ void k_static_reset(StaticScratch *S) {
    for (int i = 0; i < 2 * RS_MAX_PASSES * 256; i++) S->ghist[i] = 0;
    Ctrl &c = S->ctl;
    c.err = 0;
    c.bar_count = 0;
    c.nd = 1;   // one disk: the box and root cube of the control block itself
    c.disk_of = nullptr;
    c.doff = nullptr;
    c.dbox = c.bbox;
    c.droot = c.root;
    for (int k = 0; k < 3; k++) {
        c.bbox[k] = ~0ull;
        c.bbox[3 + k] = 0ull;
    }
}

__global__ void k_static_split(const double *__restrict__ pos, StaticScratch *S, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        S->x[i] = pos[3 * i];
        S->y[i] = pos[3 * i + 1];
        S->z[i] = pos[3 * i + 2];
    }
}

__global__ void k_static_order(const StaticScratch *S, int64_t *order, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        order[i] = static_cast<int64_t>(S->idx[i]);
}

struct StaticDevice {
    StaticScratch *ptr = nullptr;
    int num_sms = 0;
    int radix_per_sm = 0;
};

static std::mutex g_static_mutex;
static StaticDevice g_static_dev[128];

// Per-device set-up, done once with the device current.
static cudaError_t static_setup(int dev, StaticDevice &out) {
    std::lock_guard<std::mutex> lock(g_static_mutex);
    StaticDevice &d = g_static_dev[dev];
    if (!d.ptr) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, reinterpret_cast<const void *>(k_radix), RS_T, 0);
        if (e != cudaSuccess) return e;
        d.num_sms = sms;
        d.radix_per_sm = std::max(1, std::min(per_sm, 2));
        d.ptr = static_cast<StaticScratch *>(p);
    }
    out = d;
    return cudaSuccess;
}

static bool on_device(const void *p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace ncorp

extern "C" int ncorp_hilbert_sort_static(const double *positions, int64_t n64, uint64_t *keys, int64_t *order,
                                         void *cuda_stream) {
    using namespace ncorp;
    if (n64 < 1 || n64 > STATIC_MAX_N || !positions || !keys || !order) return NCORP_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return NCORP_ECUDA;
    if (!on_device(positions, dev) || !on_device(keys, dev) || !on_device(order, dev)) return NCORP_EINVAL;
    StaticDevice d;
    if (static_setup(dev, d) != cudaSuccess) return NCORP_ECUDA;
    const int n = static_cast<int>(n64);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    StaticScratch *S = d.ptr;
    const int g = std::max(1, std::min((n + 255) / 256, 4 * d.num_sms));
    // Launched through cudaLaunchKernel, whose return value is this launch's own
    // error (cudaGetLastError could report an earlier, unrelated failure).
    Ctrl *ctl = &S->ctl;
    double *sx = S->x, *sy = S->y, *sz = S->z;
    uint32_t *sidx = S->idx, *qx = S->qx, *qy = S->qy, *qz = S->qz;
    int ni = n;
    {
        const int *no_gate = nullptr;
        void *a_reset[] = {&S};
        void *a_split[] = {const_cast<double **>(&positions), &S, &ni};
        void *a_bbox[] = {&sx, &sy, &sz, &ni, &ctl, &no_gate};
        void *a_keys[] = {&sx, &sy, &sz, &ni, &ctl, &keys, &sidx, &qx, &qy, &qz, &no_gate};
        if (cudaLaunchKernel(reinterpret_cast<const void *>(k_static_reset), dim3(1), dim3(1), a_reset, 0, s) !=
                cudaSuccess ||
            cudaLaunchKernel(reinterpret_cast<const void *>(k_static_split), dim3(g), dim3(256), a_split, 0, s) !=
                cudaSuccess ||
            cudaLaunchKernel(reinterpret_cast<const void *>(k_bbox), dim3(g), dim3(256), a_bbox, 0, s) != cudaSuccess ||
            cudaLaunchKernel(reinterpret_cast<const void *>(k_keys), dim3(g), dim3(256), a_keys, 0, s) != cudaSuccess)
            return NCORP_ECUDA;
    }
    if (n > 1) {
        RadixArgs A;
        A.k0 = keys; A.k1 = S->key_alt; A.v0 = S->idx; A.v1 = S->idx_alt;
        A.n = n;
        A.ntiles = (n + RS_TILE - 1) / RS_TILE;
        A.passes = 8;   // 3 x 21 key bits, rounded up to an even number of 8-bit passes
        A.status = S->status;
        A.status_words = 256ll * STATIC_TILES;
        A.ghist = S->ghist;
        A.epoch = &S->epoch;
        A.epoch_limit = RS_EPOCH_LIMIT;
        A.ctl = &S->ctl;
        A.gate = nullptr;
        const int grid = std::min(A.ntiles, d.radix_per_sm * d.num_sms);
        void *args[] = {&A};
        if (cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(k_radix), dim3(grid), dim3(RS_T), args, 0, s) !=
            cudaSuccess)
            return NCORP_ECUDA;
    }
    {
        void *a_order[] = {&S, &order, &ni};
        if (cudaLaunchKernel(reinterpret_cast<const void *>(k_static_order), dim3(g), dim3(256), a_order, 0, s) !=
            cudaSuccess)
            return NCORP_ECUDA;
    }
    int err = 0;
    if (cudaMemcpyAsync(&err, &S->ctl.err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return NCORP_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return NCORP_ECUDA;
    if (err & ERR_NONFINITE) return NCORP_EINVAL;
    if (err & ERR_TIMEOUT) return NCORP_ETIMEOUT;
    return NCORP_OK;
}
