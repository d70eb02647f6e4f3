// tree.cu -- octree build from sorted Hilbert keys (Sect. 3.4.1, 3.4.6) and
// the two tree climbs of Sect. 3.4.2 (collision search: Eqs. center, rmax,
// rcrit; gravity: Eqs. expansion_center, rmax_2, rcrit_2 with the corner cap,
// the opening angle theta(M) of Dehnen 2002 Eq. 13) with P2M
// (Eq. multipole_moment) at the leaves and M2M (App. C) at the parents.
//
// Cells are stored level-major, in Hilbert order within a level, children of a
// cell contiguous; every cell owns a contiguous range of the key-sorted
// moonlets.  All geometry that decides the walk (centres, r_max, r_crit) is
// computed with exactly rounded FP64 operations in the same order as a plain
// sequential evaluation (moonlets in key order, children in cell order), so
// it is reproducible bit for bit.
#include "ctx.h"

namespace ncorp {

// exponents (a, b, c) of every packed symmetric index up to order 7
struct ExpTable {
    unsigned char e[off(MAXP + 2)][3];
};
constexpr ExpTable make_exp_table() {
    ExpTable t{};
    for (int n = 0; n <= MAXP + 1; n++)
        for (int k = 0; k <= n; k++)
            for (int c = 0; c <= k; c++) {
                int idx = off(n) + tri(k) + c;
                t.e[idx][0] = static_cast<unsigned char>(n - k);
                t.e[idx][1] = static_cast<unsigned char>(k - c);
                t.e[idx][2] = static_cast<unsigned char>(c);
            }
    return t;
}
__constant__ ExpTable c_exp = make_exp_table();

__device__ __forceinline__ int lower_bound_u64(const uint64_t *__restrict__ a, int lo, int hi, uint64_t t) {
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] < t) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// Build: one cooperative launch, one grid barrier per level.  The cells of a
// level are shared evenly among the blocks.  Per level, a block
//   1. places the children of its cells: a cell's children follow the level
//      in the order of their parents, at
//        level end + (children of the cells made by blocks before the cell's
//        maker) + (children of the cells its maker made before it),
//      both terms published before the barrier; then writes them;
//   2. for each child it made with more than s moonlets, finds the
//      boundaries of its octants on the next 3 key bits (the Hilbert digit of
//      the grandchild), so the children of every cell come out in Hilbert
//      order, and publishes, for the next level, the running count of
//      grandchildren over the cells it made and its total.
// Octant boundaries: boundary o (o = 1..7) is the first moonlet whose key is
// >= (prefix, o); four lanes search for it together, cutting the range in
// five per round.
// ---------------------------------------------------------------------------
struct BuildArgs {
    const uint64_t *key;
    const uint32_t *qx, *qy, *qz;
    int n, s, cap;
    int *level, *first, *count, *child0, *nchild, *parent, *arrive, *arrive_m;
    uint32_t *cx, *cy, *cz;
    int *bounds, *blocksum;
    int *maker, *before;    // per cell: the block that made it, children of its maker's earlier cells
    Ctrl *ctl;
    const int *gate;        // nothing to do while *gate is 0 (null: always build)
};

// The roots: one per disk (cell d holds disk d's moonlets; one disk: cell 0 holds all).
__global__ void k_build_init(BuildArgs A) {
    if ((A.gate && *A.gate == 0) || aborted(A.ctl)) return;
    const int nd = A.ctl->nd;
    for (int d = 0; d < nd; d++) {
        A.level[d] = 0;
        A.first[d] = A.ctl->doff ? A.ctl->doff[d] : 0;
        A.count[d] = A.ctl->doff ? A.ctl->doff[d + 1] - A.ctl->doff[d] : A.n;
        A.child0[d] = -1;
        A.nchild[d] = 0;
        A.parent[d] = -1;
        A.cx[d] = A.cy[d] = A.cz[d] = 0;
        A.maker[d] = 0;
        A.before[d] = 0;
        A.arrive[d] = 0;     // arrival counters of the collision climb and of the multipoles,
        A.arrive_m[d] = 0;   // zeroed as cells are made
    }
    A.ctl->col_stale = 1;   // a new tree: no collision pairs listed for it yet
    A.ctl->level_start[0] = 0;
    A.ctl->level_start[1] = nd;
    A.ctl->n_cells = nd;
    A.ctl->max_level = 0;
    A.ctl->n_leaves = 0;
    A.ctl->bar_count = 0;
}

// Octant boundaries of cell c (level lev, moonlets [f, f + cnt)), written to
// bounds[c][0..8] (b_0 = f, b_8 = f + cnt), and its number of non-empty
// octants (returned on every lane).  Called by a whole warp.
__device__ int octant_bounds(const BuildArgs &A, int c, int f, int cnt, int lev, int lane) {
    const uint64_t pref = __ldg(&A.key[f]) >> (63 - 3 * lev);
    const int shift = 60 - 3 * lev;
    const int grp = lane >> 2, j = lane & 3;           // boundary o = grp + 1 for grp < 7
    const bool searching = grp < 7;
    const uint64_t target = ((pref << 3) | static_cast<uint64_t>(grp + 1)) << shift;
    int lo = f, hi = f + cnt;                          // the boundary lies in [lo, hi]
    while (true) {
        const bool wide = searching && hi - lo > 4;
        if (!__any_sync(0xffffffffu, wide)) break;
        bool less = false;
        int sj = 0;
        if (wide) {
            sj = lo + static_cast<int>((static_cast<long long>(hi - lo) * (j + 1)) / 5);
            less = __ldg(&A.key[sj]) < target;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, less);
        const int cl = __popc((bal >> (4 * grp)) & 0xfu);    // samples below the target (monotone)
        const int s_lo = __shfl_sync(0xffffffffu, sj, (lane & ~3) + max(cl - 1, 0));
        const int s_hi = __shfl_sync(0xffffffffu, sj, (lane & ~3) + min(cl, 3));
        if (wide) {
            const int nlo = cl > 0 ? s_lo + 1 : lo;
            const int nhi = cl < 4 ? s_hi : hi;
            lo = nlo;
            hi = nhi;
        }
    }
    const bool below = searching && lo + j < hi && __ldg(&A.key[lo + j]) < target;
    const unsigned bal = __ballot_sync(0xffffffffu, below);
    const int b_o = lo + __popc((bal >> (4 * grp)) & 0xfu);
    // lane k < 9 holds b_k: b_0 = f, b_1..b_7 from the groups, b_8 = f + cnt
    const int from_grp = __shfl_sync(0xffffffffu, b_o, 4 * max(lane - 1, 0));
    const int b = lane == 0 ? f : (lane < 8 ? from_grp : f + cnt);
    const int bn = __shfl_down_sync(0xffffffffu, b, 1);
    const unsigned ne = __ballot_sync(0xffffffffu, lane < 8 && bn > b);
    if (lane < 9) A.bounds[(size_t)c * 9 + lane] = b;
    return __popc(ne);
}

// For the cells [cb, ce) this block made (level lev): octant bounds, children
// counts, and the running count over them (before[]); returns the total.
__device__ int made_cells(const BuildArgs &A, int cb, int ce, int lev, int *s_red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c = cb + wid; c < ce; c += nw) {
        if (c >= A.cap) break;
        const int cnt = __ldcg(&A.count[c]), f = __ldcg(&A.first[c]);
        int nch = 0;
        if (cnt > A.s && lev < MAX_LEVEL) nch = octant_bounds(A, c, f, cnt, lev, lane);
        if (lane == 0) A.nchild[c] = nch;
    }
    __syncthreads();
    int run = 0;
    if (wid == 0) {
        for (int c0 = cb; c0 < ce; c0 += 32) {
            const int c = c0 + lane;
            const int v = (c < ce && c < A.cap) ? __ldcg(&A.nchild[c]) : 0;
            int incl = v;
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += u;
            }
            if (c < ce && c < A.cap) {
                A.before[c] = run + incl - v;
                A.maker[c] = blockIdx.x;
            }
            run += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (lane == 0) s_red[0] = run;
    }
    __syncthreads();
    const int t = s_red[0];
    __syncthreads();
    return t;
}

__global__ void __launch_bounds__(256) k_build(BuildArgs A) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __shared__ int s_red[32];
    __shared__ int s_pre[4097];      // children made by blocks before each block (grid <= 4096)
    __shared__ int s_lo, s_hi;
    volatile Ctrl *vc = A.ctl;
    const int G = gridDim.x;
    unsigned bar = 0;
    if ((A.gate && *A.gate == 0) || aborted(A.ctl)) return;   // every block, before the first barrier
    {   // block 0 makes the roots' children counts
        const int t = made_cells(A, 0, blockIdx.x == 0 ? vc->level_start[1] : 0, 0, s_red);
        if (threadIdx.x == 0) A.blocksum[blockIdx.x] = t;
    }
    if (!grid_sync(A.ctl, bar)) return;
    for (int lev = 0; lev < MAX_LEVEL; lev++) {
        const int ls = vc->level_start[lev], le = vc->level_start[lev + 1];
        if (ls >= le) break;
        const int *bsum = A.blocksum + (lev & 1) * G;
        // prefix of the published totals (every block computes it; each thread a run of them)
        {
            const int T = blockDim.x, per = (G + T - 1) / T;
            const int b0 = min(G, (int)threadIdx.x * per), b1 = min(G, b0 + per);
            int sum = 0;
            for (int b = b0; b < b1; b++) sum += ((volatile const int *)bsum)[b];
            int incl = sum;
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += u;
            }
            if (lane == 31) s_red[wid] = incl;
            __syncthreads();
            if (wid == 0) {
                const int v = lane < nw ? s_red[lane] : 0;
                int wi = v;
                for (int o = 1; o < 32; o <<= 1) {
                    const int u = __shfl_up_sync(0xffffffffu, wi, o);
                    if (lane >= o) wi += u;
                }
                if (lane < nw) s_red[lane] = wi - v;
                if (lane == nw - 1) s_pre[G] = wi;
            }
            __syncthreads();
            int run = s_red[wid] + incl - sum;
            for (int b = b0; b < b1; b++) {
                const int v = ((volatile const int *)bsum)[b];
                s_pre[b] = run;
                run += v;
            }
        }
        __syncthreads();
        const int total = s_pre[G];
        // this block's share of the level, and the children it will make
        const int ncl = le - ls;
        const int chunk = (ncl + G - 1) / G;
        const int cb = min(le, ls + (int)blockIdx.x * chunk), ce = min(le, cb + chunk);
        if (threadIdx.x == 0) {
            s_lo = 1 << 30;
            s_hi = -1;
        }
        __syncthreads();
        // ---- 1. place and write the children of the block's cells
        for (int c = cb + wid; c < ce; c += nw) {
            if (c >= A.cap) break;
            const int nch = __ldcg(&A.nchild[c]);
            if (nch == 0) {
                if (lane == 0) A.child0[c] = -1;
                continue;
            }
            const int c0 = le + s_pre[__ldcg(&A.maker[c])] + __ldcg(&A.before[c]);
            if (lane == 0) {
                A.child0[c] = c0;
                atomicMin(&s_lo, c0);
                atomicMax(&s_hi, c0 + nch);
            }
            int b = 0;
            if (lane < 9) b = __ldcg(&A.bounds[(size_t)c * 9 + lane]);
            const int bn = __shfl_down_sync(0xffffffffu, b, 1);
            const bool ne = lane < 8 && bn > b;
            const unsigned mask = __ballot_sync(0xffffffffu, ne);
            if (ne) {
                const int ci = c0 + __popc(mask & ((1u << lane) - 1u));
                if (ci < A.cap) {
                    const int sh = KEY_BITS - (lev + 1);
                    A.level[ci] = lev + 1;
                    A.first[ci] = b;
                    A.count[ci] = bn - b;
                    A.child0[ci] = -1;
                    A.nchild[ci] = 0;
                    A.parent[ci] = c;
                    A.arrive[ci] = 0;
                    A.arrive_m[ci] = 0;
                    A.cx[ci] = A.qx[b] >> sh;
                    A.cy[ci] = A.qy[b] >> sh;
                    A.cz[ci] = A.qz[b] >> sh;
                } else {
                    atomicOr(&A.ctl->err, ERR_CELLS);
                }
            }
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            A.ctl->level_start[lev + 2] = le + total;
            A.ctl->n_cells = le + total;
            if (total > 0) A.ctl->max_level = lev + 1;
        }
        __syncthreads();
        // ---- 2. the children this block made (a contiguous range): bounds, running counts
        const int mb = s_hi >= 0 ? s_lo : 0, me = s_hi >= 0 ? s_hi : 0;
        {
            const int t = made_cells(A, mb, me, lev + 1, s_red);
            if (threadIdx.x == 0) A.blocksum[((lev + 1) & 1) * G + blockIdx.x] = t;
        }
        if (!grid_sync(A.ctl, bar)) return;
    }
}

// The leaf list, and the leaf of every moonlet (leaf_of, tree order).  Also
// zeroes the grid-barrier counter for the cooperative kernel that follows.
__global__ void k_collect_leaves(const int *__restrict__ nchild, const int *__restrict__ first,
                                 const int *__restrict__ count, Ctrl *ctl, int cap, int *leaves, int *n_leaves,
                                 int *leaf_of, const int *gate) {
    if (gate && *gate == 0) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->bar_count = 0;
    if (aborted(ctl)) return;
    const int nc = min(ctl->n_cells, cap);
    for (int base = blockIdx.x * blockDim.x; base < nc; base += gridDim.x * blockDim.x) {
        const int i = base + threadIdx.x;
        const int is_leaf = (i < nc && nchild[i] == 0) ? 1 : 0;
        const int slot = warp_append(n_leaves, is_leaf);
        if (is_leaf) {
            leaves[slot] = i;
            const int f = first[i], e = f + count[i];
            for (int k = f; k < e; k++) leaf_of[k] = i;
        }
    }
}

static int coop_grid(ncorp_ctx *c, const void *kernel, int block, size_t smem) {
    int per_sm = 0;
    NCORP_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem));
    if (per_sm < 1) per_sm = 1;
    if (per_sm > 2) per_sm = 2;
    return coop_blocks(c, per_sm);
}

void launch_build(ncorp_ctx *c, const ParticleSet &P, int n, int s, const int *gate) {
    Cells &C = c->cells;
    BuildArgs A;
    A.gate = gate;
    A.key = P.key;
    A.qx = P.qx; A.qy = P.qy; A.qz = P.qz;
    A.n = n; A.s = s; A.cap = C.cap;
    A.level = C.level; A.first = C.first; A.count = C.count; A.child0 = C.child0; A.nchild = C.nchild;
    A.parent = C.parent; A.cx = C.cx; A.cy = C.cy; A.cz = C.cz;
    A.bounds = C.bounds; A.blocksum = C.blocksum; A.maker = C.maker; A.before = C.before; A.ctl = c->ctl;
    A.arrive = C.arrive;
    A.arrive_m = C.arrive_m;
    k_build_init<<<1, 1, 0, c->stream>>>(A); c->launches++;
    NCORP_CUDA_CHECK(cudaGetLastError());
    const int block = 256;
    // about one block per thousand moonlets (a level holds at most ~n/s*8 cells): enough warps for the
    // widest level, and few blocks at small n so that the per-level barriers stay short
    int grid = std::min(coop_grid(c, reinterpret_cast<const void *>(k_build), block, 0), std::max(16, n / 1024));
    void *args[] = {&A};
    NCORP_CUDA_CHECK(cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(k_build), dim3(grid), dim3(block),
                                                 args, 0, c->stream));
    c->launches++;
    k_collect_leaves<<<grid_for(C.cap, 256, 4 * c->num_sms), 256, 0, c->stream>>>(
        C.nchild, C.first, C.count, c->ctl, C.cap, C.leaves, &c->ctl->n_leaves, C.leaf_of, gate);
    c->launches++;
    NCORP_CUDA_CHECK(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Corner cap (Sect. 3.4.2): distance from s to the farthest corner of the
// cell's cube, the cube widened by L 2^-48 on each side.
// ---------------------------------------------------------------------------
// root: the cube of the cell's disk (x_lo, y_lo, z_lo, L)
__device__ __forceinline__ double cell_side(const double *root, int lev) { return ldexp(root[3], -lev); }

// the root cube of cell c's disk
__device__ __forceinline__ const double *cell_root(const Ctrl *ctl, const int *first, int c) {
    return disk_root(ctl, disk_of(ctl, first[c]));
}

__device__ __forceinline__ double corner_axis(const double *root, int k, double h, uint32_t c, double s) {
    const double eps = dmul(root[3], 0x1p-48);
    const double lo = dadd(root[k], dmul(static_cast<double>(c), h));
    const double a = dsub(s, dsub(lo, eps));
    const double b = dsub(dadd(dadd(lo, h), eps), s);
    return a > b ? a : b;
}

__device__ __forceinline__ double corner_distance(const double *root, int lev, uint32_t cx, uint32_t cy, uint32_t cz,
                                                  double sx, double sy, double sz) {
    const double h = cell_side(root, lev);
    return dnorm3(corner_axis(root, 0, h, cx, sx), corner_axis(root, 1, h, cy, sy), corner_axis(root, 2, h, cz, sz));
}

// Power-of-two scale of a cell's expansions: >= r_max (so |x - s|/rho <= 1)
// and >= side/256, so that the scale ratios met in M2M, M2L and L2L stay
// below 2^(level difference + 8) even for one-moonlet cells (r_max ~ 0).
__device__ __forceinline__ double cell_scale(const double *root, int lev, double rmax) {
    return pow2_ceil(fmax(rmax, cell_side(root, lev) * 0x1p-8));
}

// FP32 double-float copy of a centre: hi = fl32(s), lo = fl32(s - hi)
__device__ __forceinline__ void split3(double x, double y, double z, float4 &hi, float4 &lo) {
    hi.x = static_cast<float>(x);
    hi.y = static_cast<float>(y);
    hi.z = static_cast<float>(z);
    lo.x = static_cast<float>(x - static_cast<double>(hi.x));
    lo.y = static_cast<float>(y - static_cast<double>(hi.y));
    lo.z = static_cast<float>(z - static_cast<double>(hi.z));
}

// ---------------------------------------------------------------------------
// Climbs.  GB300 executes an FP64 warp instruction in the same time whatever
// the number of active lanes, so the sequential, order-fixed FP64 sums that
// make the geometry reproducible bit for bit are spread one cell per thread
// (leaves) or one sum per lane (parents), never run on a single lane.
// r_max of a leaf is sqrt(max_i |x_i - s|^2): a correctly rounded square root
// is non-decreasing, so this equals max_i sqrt(|x_i - s|^2) exactly.
// ---------------------------------------------------------------------------
struct ClimbArgs {
    const double *x, *y, *z, *m;
    const float4 *hi4, *lo4;
    const double *vx, *vy, *vz, *R;
    int *first, *count, *child0, *nchild, *parent, *level, *arrive;
    uint32_t *cx, *cy, *cz;
    double *M, *sx, *sy, *sz, *rmax, *rcrit, *rho;
    float4 *gh, *gl;
    void *Mh;
    float4 *cv4;
    const int *leaves;
    Ctrl *ctl;
    double G, dt, theta;
    int cap;
    const double *rc_given;   // collision climb (nullable): each moonlet's R + dt |v| given (tree order)
    const int *gate;          // collision climb (nullable): nothing to do while *gate is 0
};

constexpr int CLIMB_WARPS_COOP = 8;

template <typename real>
__device__ __forceinline__ real warp_sum_r(real v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---- leaves: eight leaves per warp, four lanes per leaf.  The centre's
// sums run in the oracle's order, one sum per lane (q = 0: the weights,
// q = 1..3: the weighted coordinates), so a warp instruction advances 32
// independent sums; the maxima over the moonlets are exact in any order and
// are split over the four lanes.
constexpr int LEAF_GROUP = 8;

struct LeafSlot {
    int sub, q, base, t, c, f, cnt;
    bool valid;
};

__device__ __forceinline__ LeafSlot leaf_slot(const ClimbArgs &A, int gw, int lane, int n_leaves) {
    LeafSlot L;
    L.sub = lane >> 2;
    L.q = lane & 3;
    L.base = lane & ~3;
    L.t = gw * LEAF_GROUP + L.sub;
    L.valid = L.t < n_leaves;
    L.c = L.valid ? A.leaves[L.t] : 0;
    L.f = L.valid ? A.first[L.c] : 0;
    L.cnt = L.valid ? A.count[L.c] : 0;
    return L;
}

__device__ __forceinline__ double quad_max(double v) {
    v = fmax(v, __shfl_xor_sync(0xffffffffu, v, 1));
    return fmax(v, __shfl_xor_sync(0xffffffffu, v, 2));
}

// Corner cap of the leaf (lanes q = 0..2 take one axis each), returned on every lane of the quad.
__device__ __forceinline__ double quad_corner(const ClimbArgs &A, const LeafSlot &L, double sx, double sy, double sz) {
    double d = 0.0;
    if (L.valid && L.q < 3) {
        const int lev = A.level[L.c];
        const double *rt = disk_root(A.ctl, disk_of(A.ctl, L.f));
        const double h = cell_side(rt, lev);
        d = corner_axis(rt, L.q, h, L.q == 0 ? A.cx[L.c] : (L.q == 1 ? A.cy[L.c] : A.cz[L.c]),
                        L.q == 0 ? sx : (L.q == 1 ? sy : sz));
    }
    const double d0 = __shfl_sync(0xffffffffu, d, L.base), d1 = __shfl_sync(0xffffffffu, d, L.base + 1),
                 d2 = __shfl_sync(0xffffffffu, d, L.base + 2);
    return dnorm3(d0, d1, d2);
}

// ---- gravity leaves (Eqs. expansion_center, rmax_2, corner cap): the
// group of LEAF_GROUP leaves of warp-group gw.
__device__ __forceinline__ void leaf_gravity_group(const ClimbArgs &A, int gw, int lane, int n_leaves) {
    const LeafSlot L = leaf_slot(A, gw, lane, n_leaves);
    const double *coord = L.q == 1 ? A.x : (L.q == 2 ? A.y : A.z);
    double acc = 0.0;
    for (int k = L.f; k < L.f + L.cnt; k++) {
        const double m = A.m[k];
        acc = L.q == 0 ? dadd(acc, m) : dadd(acc, dmul(m, coord[k]));
    }
    const double M = __shfl_sync(0xffffffffu, acc, L.base);
    const double sq = L.q == 0 ? M : ddiv(acc, M);
    const double sx = __shfl_sync(0xffffffffu, sq, L.base + 1), sy = __shfl_sync(0xffffffffu, sq, L.base + 2),
                 sz = __shfl_sync(0xffffffffu, sq, L.base + 3);
    double d2 = 0.0;
    for (int k = L.f + L.q; k < L.f + L.cnt; k += 4)
        d2 = fmax(d2, dsq3(dsub(A.x[k], sx), dsub(A.y[k], sy), dsub(A.z[k], sz)));
    d2 = quad_max(d2);
    double rmax = dsqrt(d2);
    const double cap = quad_corner(A, L, sx, sy, sz);
    if (cap < rmax) rmax = cap;
    if (L.valid && L.q == 0) {
        const int c = L.c;
        const double rho = cell_scale(cell_root(A.ctl, A.first, c), A.level[c], rmax);
        A.M[c] = M;
        A.sx[c] = sx;
        A.sy[c] = sy;
        A.sz[c] = sz;
        A.rmax[c] = rmax;
        A.rho[c] = rho;
        float4 hi, lo;
        split3(sx, sy, sz, hi, lo);
        hi.w = 0.f;
        lo.w = static_cast<float>(rho);
        A.gh[c] = hi;
        A.gl[c] = lo;
    }
}

// acc[midx(beta)] += mu d^beta for orders 0 and 2..P-1
template <int P, typename real>
__device__ __forceinline__ void p2m_add(real dx, real dy, real dz, real mu, real *acc) {
    real px[P], py[P], pz[P];
    px[0] = py[0] = pz[0] = real(1);
#pragma unroll
    for (int k = 1; k < P; k++) {
        px[k] = px[k - 1] * dx;
        py[k] = py[k - 1] * dy;
        pz[k] = pz[k - 1] * dz;
    }
    acc[0] += mu;
#pragma unroll
    for (int n = 2; n < P; n++)
#pragma unroll
        for (int k = 0; k <= n; k++)
#pragma unroll
            for (int c = 0; c <= k; c++) acc[midx(n - k, k - c, c)] += mu * px[n - k] * py[k - c] * pz[c];
}

template <int P, typename real>
__device__ __forceinline__ void store_reduced(real *acc, real *dst, int lane) {
    constexpr int NM = num_m(P);
#pragma unroll
    for (int j = 0; j < NM; j++) {
        const real v = warp_sum_r(acc[j]);
        if (lane == (j & 31)) dst[j] = v;
    }
}

// ---- gravity geometry of parents from their children (Eqs. expansion_center,
// rmax_2, corner cap), four parents per warp, eight lanes each (a parent has
// at most eight children), so that one FP64 warp instruction advances four
// parents.  Lane j of a group holds child j; lanes
// j = 0..3 form the centre's sums over the children in child order (lane 0
// the mass, as w * 1 = w exactly, lanes 1..3 the weighted coordinates).  c is
// the group's parent, -1 for none; every lane of the warp calls this.
constexpr int PARENT_GROUP = 4;

__device__ __forceinline__ void parent_gravity_group(const ClimbArgs &A, int c, int lane) {
    const int j = lane & 7, base = lane & ~7;
    const bool valid = c >= 0;
    const int c0 = valid ? A.child0[c] : 0, nch = valid ? A.nchild[c] : 0;
    double cm = 0.0, csx = 0.0, csy = 0.0, csz = 0.0, crm = 0.0;
    if (j < nch) {
        cm = __ldcg(&A.M[c0 + j]);
        csx = __ldcg(&A.sx[c0 + j]);
        csy = __ldcg(&A.sy[c0 + j]);
        csz = __ldcg(&A.sz[c0 + j]);
        crm = __ldcg(&A.rmax[c0 + j]);
    }
    double acc = 0.0;
#pragma unroll
    for (int ch = 0; ch < 8; ch++) {
        const double w = __shfl_sync(0xffffffffu, cm, base + ch);
        const double bx = __shfl_sync(0xffffffffu, csx, base + ch);
        const double by = __shfl_sync(0xffffffffu, csy, base + ch);
        const double bz = __shfl_sync(0xffffffffu, csz, base + ch);
        const double coord = j == 1 ? bx : (j == 2 ? by : (j == 3 ? bz : 1.0));
        const double t = dmul(w, coord);
        if (ch < nch) acc = dadd(acc, t);
    }
    const double M = __shfl_sync(0xffffffffu, acc, base);
    const double q = ddiv(acc, M);
    const double px = __shfl_sync(0xffffffffu, q, base + 1), py = __shfl_sync(0xffffffffu, q, base + 2),
                 pz = __shfl_sync(0xffffffffu, q, base + 3);
    double rm = 0.0;
    if (j < nch) rm = dadd(crm, dnorm3(dsub(csx, px), dsub(csy, py), dsub(csz, pz)));
    rm = fmax(rm, __shfl_xor_sync(0xffffffffu, rm, 1));
    rm = fmax(rm, __shfl_xor_sync(0xffffffffu, rm, 2));
    rm = fmax(rm, __shfl_xor_sync(0xffffffffu, rm, 4));
    const int plev = valid ? A.level[c] : 0;
    double d = 0.0;
    if (valid && j < 3) {
        const double *rt = cell_root(A.ctl, A.first, c);
        const double h = cell_side(rt, plev);
        d = corner_axis(rt, j, h, j == 0 ? A.cx[c] : (j == 1 ? A.cy[c] : A.cz[c]), j == 0 ? px : (j == 1 ? py : pz));
    }
    const double d0 = __shfl_sync(0xffffffffu, d, base), d1 = __shfl_sync(0xffffffffu, d, base + 1),
                 d2 = __shfl_sync(0xffffffffu, d, base + 2);
    const double pcap = dnorm3(d0, d1, d2);
    if (pcap < rm) rm = pcap;
    if (valid && j == 0) {
        const double prho = cell_scale(cell_root(A.ctl, A.first, c), plev, rm);
        A.M[c] = M;
        A.sx[c] = px;
        A.sy[c] = py;
        A.sz[c] = pz;
        A.rmax[c] = rm;
        A.rho[c] = prho;
        float4 hi, lo;
        split3(px, py, pz, hi, lo);
        hi.w = 0.f;
        lo.w = static_cast<float>(prho);
        A.gh[c] = hi;
        A.gl[c] = lo;
    }
}

// ---- multipoles (Eq. multipole_moment, scaled: M-hat_beta = sum mu (d/rho)^beta / beta!,
// orders 0 and 2..p-1; the dipole vanishes about the centre of mass).
// Leaves take the sum over their moonlets (one warp per leaf, lanes over the
// moonlets, a butterfly sum per coefficient).  A parent takes its children's
// moments translated to its own centre (the M2M shift of App. C), which in
// scaled form reads, with delta = (s_c - s_P)/rho_P and r = rho_c/rho_P,
//   M-hat_P(beta) = sum_children sum_{gamma <= beta, |gamma| != 1}
//                   M-hat_c(gamma) r^|gamma| delta^(beta - gamma) / (beta - gamma)!
// (the multinomial expansion of (d_c + delta)^beta / beta!, axis by axis).
// The children are added in child order.
struct P2MArgs {
    const double *x, *y, *z, *m;
    const float4 *hi4, *lo4;
    const int *first, *count, *child0, *nchild, *parent, *leaves;
    int *arrive;       // per cell: children whose moments are done (zeroed by the build)
    const double *sx, *sy, *sz, *rho;
    const float4 *gh, *gl;
    void *Mh;
    double G;
    Ctrl *ctl;
};

constexpr int P2M_WARPS = 4;

template <int P, typename real>
struct M2MShared {
    real a[P2M_WARPS][8][off(P) < 1 ? 1 : off(P)];   // per child: full storage, orders 0..P-1
    real b[P2M_WARPS][8][off(P) < 1 ? 1 : off(P)];
};

// (n, b + c, c) of slot j of the full storage (orders 0..P-1): order n starts
// at n(n+1)(n+2)/6, and within it k = b + c runs 0..n with c = 0..k
template <int P>
__device__ __forceinline__ void full_exps(int j, int &n, int &kk, int &c) {
    n = 0;
    while (n + 1 < P && off(n + 1) <= j) n++;
    const int rem = j - off(n);
    kk = 0;
    while (kk < n && tri(kk + 1) <= rem) kk++;
    c = rem - tri(kk);
}

// One-dimensional shift of full-storage moments along AXIS: out(a,b,c) = sum_{k <= exponent} in(... - k e_axis) w_k
template <int P, int AXIS, typename real>
__device__ __forceinline__ real m_shift(const real *in, const real (&w)[P], int n, int kk, int c) {
    const int ax = AXIS == 0 ? n - kk : (AXIS == 1 ? kk - c : c);   // the exponent along the axis
    real s = real(0);
#pragma unroll
    for (int k = 0; k < P; k++) {
        if (k > ax) break;
        const int m = n - k, t = AXIS == 0 ? kk : kk - k, cc = AXIS == 2 ? c - k : c;
        s += in[m * (m + 1) * (m + 2) / 6 + t * (t + 1) / 2 + cc] * w[k];
    }
    return s;
}

// Eight leaves per warp, four lanes per leaf: each lane sums a quarter of its
// leaf's moonlets, then the four partial sums are added by two butterfly
// steps and each lane stores a quarter of the coefficients.  Every lane of
// the warp calls this (valid: the lane's group has a leaf).
template <int P, typename real>
__device__ __forceinline__ void leaf_moments(const P2MArgs &A, int c, bool valid, int q, real *Mh) {
    constexpr int NM = num_m(P);
    real acc[NM];
#pragma unroll
    for (int j = 0; j < NM; j++) acc[j] = real(0);
    if (valid) {
        const int f = A.first[c], e = f + A.count[c];
        if constexpr (sizeof(real) == 4) {   // double-float difference, no FP64 work
            const float4 gh = A.gh[c], gl = A.gl[c];
            const float ir = 1.0f / gl.w;   // exact: rho is a power of two
            for (int k = f + q; k < e; k += 4) {
                const float4 h = A.hi4[k], l = A.lo4[k];
                p2m_add<P, real>(((h.x - gh.x) + (l.x - gl.x)) * ir, ((h.y - gh.y) + (l.y - gl.y)) * ir,
                                 ((h.z - gh.z) + (l.z - gl.z)) * ir, h.w, acc);
            }
        } else {
            const double irho = 1.0 / A.rho[c], sx = A.sx[c], sy = A.sy[c], sz = A.sz[c];
            for (int k = f + q; k < e; k += 4)
                p2m_add<P, real>((A.x[k] - sx) * irho, (A.y[k] - sy) * irho, (A.z[k] - sz) * irho, A.G * A.m[k], acc);
        }
    }
#pragma unroll
    for (int n = 0; n < P; n++) {
        if (n == 1) continue;
#pragma unroll
        for (int k = 0; k <= n; k++)
#pragma unroll
            for (int cc = 0; cc <= k; cc++) {
                const int j = midx(n - k, k - cc, cc);
                real v = acc[j] * static_cast<real>(inv_mfact(n - k, k - cc, cc));
                v += __shfl_xor_sync(0xffffffffu, v, 1);
                v += __shfl_xor_sync(0xffffffffu, v, 2);
                if (valid && (j & 3) == q) Mh[(size_t)c * NM + j] = v;
            }
    }
}

// M2M of a parent from its children, as three one-dimensional shifts per
// child (the expansion of (d_c + delta)^beta / beta! factorises over the
// axes): the child's moments scaled by r^|gamma| go into full storage with
// zero dipole slots, are shifted along x, y and z by delta, and the slots of
// orders 0 and 2..P-1 are summed over the children in child order (the
// parent's dipole about its own centre of mass vanishes).  The children are
// shifted side by side: four lanes per child (a parent has at most eight),
// each lane a quarter of the child's slots.
template <int P, typename real>
__device__ __forceinline__ void parent_moments(const P2MArgs &A, M2MShared<P, real> &S, int wl, int pc, int lane,
                                               real *Mh) {
    constexpr int NM = num_m(P), NF = off(P);
    constexpr int PER4 = (NF + 3) / 4;   // slots per lane of a child's quad
    const int ch = lane >> 2, sub = lane & 3;
    const int c0 = A.child0[pc], nch = A.nchild[pc];
    const bool act = ch < nch;
    const int c = act ? c0 + ch : c0;
    real ipr, dx, dy, dz, rr;
    if constexpr (sizeof(real) == 4) {
        const float4 ch_h = A.gh[c], ch_l = A.gl[c], p_h = A.gh[pc], p_l = A.gl[pc];
        ipr = 1.0f / p_l.w;   // exact: rho is a power of two
        dx = ((ch_h.x - p_h.x) + (ch_l.x - p_l.x)) * ipr;
        dy = ((ch_h.y - p_h.y) + (ch_l.y - p_l.y)) * ipr;
        dz = ((ch_h.z - p_h.z) + (ch_l.z - p_l.z)) * ipr;
        rr = ch_l.w * ipr;
    } else {
        ipr = 1.0 / A.rho[pc];
        dx = (A.sx[c] - A.sx[pc]) * ipr;
        dy = (A.sy[c] - A.sy[pc]) * ipr;
        dz = (A.sz[c] - A.sz[pc]) * ipr;
        rr = A.rho[c] * ipr;
    }
    real wx[P], wy[P], wz[P];
    wx[0] = wy[0] = wz[0] = real(1);
#pragma unroll
    for (int k = 1; k < P; k++) {
        wx[k] = wx[k - 1] * dx;
        wy[k] = wy[k - 1] * dy;
        wz[k] = wz[k - 1] * dz;
    }
#pragma unroll
    for (int k = 2; k < P; k++) {
        const real f = static_cast<real>(ifact(k));
        wx[k] *= f; wy[k] *= f; wz[k] *= f;
    }
    int en[PER4], ek[PER4], ec[PER4];
#pragma unroll
    for (int q = 0; q < PER4; q++) full_exps<P>(sub + 4 * q, en[q], ek[q], ec[q]);
    real *sa = S.a[wl][ch], *sb = S.b[wl][ch];
    __syncwarp();
    if (act) {
#pragma unroll
        for (int q = 0; q < PER4; q++) {   // the child's moments, scaled by r^n, dipole slots zero
            const int j = sub + 4 * q;
            if (j >= NF) continue;
            real v = real(0);
            if (en[q] != 1) {
                v = __ldcg(&Mh[(size_t)c * NM + (en[q] == 0 ? 0 : j - 3)]);
                for (int t = 0; t < en[q]; t++) v *= rr;
            }
            sa[j] = v;
        }
    }
    __syncwarp();
    if (act) {
#pragma unroll
        for (int q = 0; q < PER4; q++)
            if (sub + 4 * q < NF) sb[sub + 4 * q] = m_shift<P, 0>(sa, wx, en[q], ek[q], ec[q]);
    }
    __syncwarp();
    if (act) {
#pragma unroll
        for (int q = 0; q < PER4; q++)
            if (sub + 4 * q < NF) sa[sub + 4 * q] = m_shift<P, 1>(sb, wy, en[q], ek[q], ec[q]);
    }
    __syncwarp();
    if (act) {
#pragma unroll
        for (int q = 0; q < PER4; q++)
            if (sub + 4 * q < NF) sb[sub + 4 * q] = m_shift<P, 2>(sa, wz, en[q], ek[q], ec[q]);
    }
    __syncwarp();
    // sums over the children in child order; lane j takes slots j, j + 32
    for (int j = lane; j < NF; j += 32) {
        int n, kk, cc;
        full_exps<P>(j, n, kk, cc);
        if (n == 1) continue;
        real acc = real(0);
        for (int k = 0; k < nch; k++) acc += S.b[wl][k][j];
        Mh[(size_t)pc * NM + (n == 0 ? 0 : j - 3)] = acc;
    }
}

// One launch, no waiting: the leaves' moments from their moonlets (eight
// leaves per warp), then the parents up the tree.  A warp that has finished a
// cell adds its arrival to the parent's counter (release); the warp that
// arrives last (acquire) computes the parent, whose children are then all
// done, and goes on up.  The children are added in child order, so the
// result does not depend on which warp arrives last.
template <int P, typename real>
__device__ __forceinline__ int arrive_last(const P2MArgs &A, int c) {
    const int pc = A.parent[c];
    if (pc < 0) return -1;
    fence_acq_rel_gpu();   // release: the cell's moments before the arrival
    if (atomicAdd(&A.arrive[pc], 1) != A.nchild[pc] - 1) return -1;
    fence_acq_rel_gpu();   // acquire: the other children's moments
    return pc;
}

template <int P, typename real>
__global__ void __launch_bounds__(32 * P2M_WARPS) k_multipoles(P2MArgs A) {
    __shared__ M2MShared<P, real> S;
    if (aborted(A.ctl)) return;
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int gw0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
    const int nl = A.ctl->n_leaves;
    real *Mh = static_cast<real *>(A.Mh);
    for (int base = gw0 * 8; base < nl; base += nwarps * 8) {   // eight leaves per warp, four lanes each
        const int li = base + (lane >> 2);
        const bool valid = li < nl;
        const int c = valid ? A.leaves[li] : 0;
        leaf_moments<P, real>(A, c, valid, lane & 3, Mh);
        __syncwarp();
        int up = -1;   // the parent this quad's leaf completed, if any
        if (valid && (lane & 3) == 0) up = arrive_last<P, real>(A, c);
        unsigned todo = __ballot_sync(0xffffffffu, up >= 0);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            int pc = __shfl_sync(0xffffffffu, up, src);
            __syncwarp();   // orders the quad leader's acquire before every lane's reads
            while (true) {
                parent_moments<P, real>(A, S, wl, pc, lane, Mh);
                __syncwarp();
                int next = -1;
                if (lane == 0) next = arrive_last<P, real>(A, pc);
                next = __shfl_sync(0xffffffffu, next, 0);
                if (next < 0) break;
                __syncwarp();
                pc = next;
            }
        }
    }
}

template <int P, typename real>
static void p2m_t(ncorp_ctx *c, const P2MArgs &B) {
    k_multipoles<P, real><<<4 * c->num_sms, 32 * P2M_WARPS, 0, c->stream>>>(B); c->launches++;
}

// theta(M) of Dehnen (2002) Eq. 13: theta^5/(1-theta)^2 = K (M/M_tot)^(-1/3),
// K = theta_min^5/(1-theta_min)^2, i.e. the root in [theta_min, 1) of the
// increasing f(theta) = theta^15 M - K^3 M_tot (1-theta)^6: 12 bisection
// steps, then 4 Newton steps kept inside the final bracket (+ - x / only).
__device__ double theta_of(double M, double Mtot, double tmin) {
    const double t2 = dmul(tmin, tmin), t4 = dmul(t2, t2), t5 = dmul(t4, tmin);
    const double u = dsub(1.0, tmin), u2 = dmul(u, u);
    const double K = ddiv(t5, u2);
    const double K3 = dmul(dmul(K, K), K);
    const double rhs = dmul(K3, Mtot);
    double lo = tmin, hi = 1.0;
    for (int it = 0; it < 12; it++) {
        const double mid = dmul(dadd(lo, hi), 0.5);
        const double m2 = dmul(mid, mid), m3 = dmul(m2, mid), m6 = dmul(m3, m3), m12 = dmul(m6, m6),
                     m15 = dmul(m12, m3);
        const double w = dsub(1.0, mid), w2 = dmul(w, w), w3 = dmul(w2, w), w6 = dmul(w3, w3);
        const double f = dsub(dmul(m15, M), dmul(rhs, w6));
        if (f > 0.0) hi = mid;
        else lo = mid;
    }
    double th = dmul(dadd(lo, hi), 0.5);
    for (int it = 0; it < 4; it++) {
        const double w = dsub(1.0, th);
        const double q2 = dmul(th, th), q3 = dmul(q2, th), q6 = dmul(q3, q3), q12 = dmul(q6, q6),
                     q14 = dmul(q12, q2), q15 = dmul(q14, th);
        const double w2 = dmul(w, w), w3 = dmul(w2, w), w5 = dmul(w3, w2), w6 = dmul(w3, w3);
        const double f = dsub(dmul(q15, M), dmul(rhs, w6));
        const double fp = dadd(dmul(dmul(15.0, q14), M), dmul(dmul(6.0, rhs), w5));
        double nt = dsub(th, ddiv(f, fp));
        if (nt < lo) nt = lo;
        if (nt > hi) nt = hi;
        th = nt;
    }
    return th;
}

// ---- gravity geometry in one cooperative launch: the leaves, then the
// parents level by level from the deepest (each needs its children's), then
// theta(M) and r_crit = r_max / theta (which need the root's mass).  One FP64
// warp instruction costs the same whatever the number of active lanes, so the
// leaves go eight to a warp with four lanes each, theta(M) 32 cells to a
// warp, and the parents four to a warp with eight lanes each.
__global__ void __launch_bounds__(32 * CLIMB_WARPS_COOP) k_geometry(ClimbArgs A) {
    if (aborted(A.ctl)) return;
    const int lane = threadIdx.x & 31;
    // warps numbered across the blocks first, so that consecutive work items land on different SMs
    const int gw0 = (threadIdx.x >> 5) * gridDim.x + blockIdx.x, nwarps = (gridDim.x * blockDim.x) >> 5;
    unsigned bar = 0;
    const int n_leaves = A.ctl->n_leaves;
    for (int gw = gw0; gw * LEAF_GROUP < n_leaves; gw += nwarps) leaf_gravity_group(A, gw, lane, n_leaves);
    if (!grid_sync(A.ctl, bar)) return;
    const int maxl = A.ctl->max_level;
    for (int lev = maxl - 1; lev >= 0; lev--) {
        const int ls = A.ctl->level_start[lev], le = A.ctl->level_start[lev + 1];
        for (int g = gw0; ls + g * PARENT_GROUP < le; g += nwarps) {
            const int cc = ls + g * PARENT_GROUP + (lane >> 3);
            const int c = (cc < le && A.nchild[cc] > 0) ? cc : -1;
            if (__any_sync(0xffffffffu, c >= 0)) parent_gravity_group(A, c, lane);
        }
        if (!grid_sync(A.ctl, bar)) return;
    }
    const int nc = min(A.ctl->n_cells, A.cap);
    // theta(M): every lane one cell; the dependent FP64 chain of a warp bounds this phase, so fewer,
    // fuller warps (at most one per sub-partition) finish first.  M_tot is the mass of the cell's disk
    // (its root: cell d of disk d).
    {
        for (int i = gw0 * 32 + lane; i < nc; i += nwarps * 32) {
            const double Mtot = __ldcg(&A.M[disk_of(A.ctl, A.first[i])]);
            const double rc = ddiv(__ldcg(&A.rmax[i]), theta_of(__ldcg(&A.M[i]), Mtot, A.theta));
            A.rcrit[i] = rc;
            A.gh[i].w = static_cast<float>(rc);
        }
    }
}


void launch_climb_geometry(ncorp_ctx *c, const ParticleSet &P, double G, double theta) {
    Cells &C = c->cells;
    ClimbArgs A{};
    A.x = P.x; A.y = P.y; A.z = P.z; A.m = P.m; A.hi4 = P.hi4; A.lo4 = P.lo4;
    A.first = C.first; A.count = C.count; A.child0 = C.child0; A.nchild = C.nchild; A.parent = C.parent;
    A.level = C.level; A.arrive = C.arrive; A.cx = C.cx; A.cy = C.cy; A.cz = C.cz;
    A.M = C.M; A.sx = C.sx; A.sy = C.sy; A.sz = C.sz; A.rmax = C.rmax; A.rcrit = C.rcrit; A.rho = C.rho;
    A.gh = C.gh; A.gl = C.gl;
    A.Mh = C.Mh; A.leaves = C.leaves; A.ctl = c->ctl; A.G = G; A.theta = theta; A.cap = C.cap;
    const int block = 32 * CLIMB_WARPS_COOP;
    // every SM: the FP64 work of the leaves and of theta(M) is bound by the FP64 units of the
    // sub-partitions, so it is spread over all of them
    const int grid = coop_grid(c, reinterpret_cast<const void *>(k_geometry), block, 0);
    void *args[] = {&A};   // ctl->bar_count was zeroed by k_collect_leaves
    NCORP_CUDA_CHECK(cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(k_geometry), dim3(grid), dim3(block),
                                                 args, 0, c->stream));
    c->launches++;
}

void launch_multipoles(ncorp_ctx *c, const ParticleSet &P, int p, bool mixed, double G) {
    Cells &C = c->cells;
    P2MArgs B;
    B.x = P.x; B.y = P.y; B.z = P.z; B.m = P.m; B.hi4 = P.hi4; B.lo4 = P.lo4;
    B.first = C.first; B.count = C.count; B.child0 = C.child0; B.nchild = C.nchild; B.parent = C.parent;
    B.leaves = C.leaves; B.arrive = C.arrive_m;
    B.sx = C.sx; B.sy = C.sy; B.sz = C.sz; B.rho = C.rho; B.gh = C.gh; B.gl = C.gl;
    B.Mh = C.Mh;
    B.G = G; B.ctl = c->ctl;
#define NCORP_P2M_CASE(PP)                     \
    case PP:                                   \
        if (mixed) p2m_t<PP, float>(c, B);     \
        else p2m_t<PP, double>(c, B);          \
        break;
    switch (p) {
        NCORP_P2M_CASE(1)
        NCORP_P2M_CASE(2)
        NCORP_P2M_CASE(3)
        NCORP_P2M_CASE(4)
        NCORP_P2M_CASE(5)
        NCORP_P2M_CASE(6)
        default: break;
    }
#undef NCORP_P2M_CASE
    NCORP_CUDA_CHECK(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Collision climb (Eqs. center, rmax, rcrit): s-bar is the mean moonlet
// position (children weighted by their moonlet counts); r_crit = r_max + max
// over children of (r_crit - r_max), a moonlet's being R + dt |v| (stored,
// rounded up to FP32, with the velocity rounded to FP32, for the pair
// prefilter).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(64) k_leaf_collision(ClimbArgs A) {
    if (A.gate && *A.gate == 0) return;
    // the grid barrier counter of the parents' cooperative climb that follows on this stream
    if (blockIdx.x == 0 && threadIdx.x == 0) A.ctl->bar_count2 = 0;
    if (aborted(A.ctl)) return;
    const int lane = threadIdx.x & 31;
    const int n_leaves = A.ctl->n_leaves;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; gw * LEAF_GROUP < n_leaves; gw += nwarps) {
        const LeafSlot L = leaf_slot(A, gw, lane, n_leaves);
        const double *coord = L.q == 0 ? A.x : (L.q == 1 ? A.y : A.z);
        double acc = 0.0;
        if (L.q < 3)
            for (int k = L.f; k < L.f + L.cnt; k++) acc = dadd(acc, coord[k]);
        const double sq = L.q < 3 ? ddiv(acc, static_cast<double>(L.cnt)) : 0.0;
        const double sx = __shfl_sync(0xffffffffu, sq, L.base), sy = __shfl_sync(0xffffffffu, sq, L.base + 1),
                     sz = __shfl_sync(0xffffffffu, sq, L.base + 2);
        double d2 = 0.0, ex = 0.0;
        for (int k = L.f + L.q; k < L.f + L.cnt; k += 4) {
            d2 = fmax(d2, dsq3(dsub(A.x[k], sx), dsub(A.y[k], sy), dsub(A.z[k], sz)));
            if (A.rc_given) {   // bounds given: the pair test's per-moonlet values come later
                ex = fmax(ex, A.rc_given[k]);
                continue;
            }
            const double vx = A.vx[k], vy = A.vy[k], vz = A.vz[k];
            const double e = dadd(A.R[k], dmul(A.dt, dnorm3(vx, vy, vz)));
            ex = fmax(ex, e);
            A.cv4[k] = make_float4(static_cast<float>(vx), static_cast<float>(vy), static_cast<float>(vz),
                                   __double2float_ru(e));
        }
        d2 = quad_max(d2);
        ex = quad_max(ex);
        double rmax = dsqrt(d2);
        const double cap = quad_corner(A, L, sx, sy, sz);
        if (cap < rmax) rmax = cap;
        if (L.valid && L.q == 0) {
            const int c = L.c;
            const double rc = dadd(rmax, ex);
            A.sx[c] = sx;
            A.sy[c] = sy;
            A.sz[c] = sz;
            A.rmax[c] = rmax;
            A.rcrit[c] = rc;
            float4 hi, lo;
            split3(sx, sy, sz, hi, lo);
            hi.w = static_cast<float>(rc);
            lo.w = 0.f;
            A.gh[c] = hi;
            A.gl[c] = lo;
        }
    }
}

// ---- collision geometry of parents from their children (Eqs. center, rmax,
// rcrit, corner cap), four parents per warp, eight lanes each, as for gravity
// (parent_gravity_group) with the children's moonlet counts as weights and
// the parent's count as divisor; r_crit = r_max + the largest (r_crit - r_max)
// of the children.  c is the group's parent, -1 for none; every lane of the
// warp calls this.
__device__ __forceinline__ void parent_collision_group(const ClimbArgs &A, int c, int lane) {
    const int j = lane & 7, base = lane & ~7;
    const bool valid = c >= 0;
    const int c0 = valid ? A.child0[c] : 0, nch = valid ? A.nchild[c] : 0;
    double cw = 0.0, csx = 0.0, csy = 0.0, csz = 0.0, crm = 0.0, cex = 0.0;
    if (j < nch) {
        cw = static_cast<double>(A.count[c0 + j]);
        csx = __ldcg(&A.sx[c0 + j]);
        csy = __ldcg(&A.sy[c0 + j]);
        csz = __ldcg(&A.sz[c0 + j]);
        crm = __ldcg(&A.rmax[c0 + j]);
        cex = dsub(__ldcg(&A.rcrit[c0 + j]), crm);
    }
    double acc = 0.0;
#pragma unroll
    for (int ch = 0; ch < 8; ch++) {
        const double w = __shfl_sync(0xffffffffu, cw, base + ch);
        const double bx = __shfl_sync(0xffffffffu, csx, base + ch);
        const double by = __shfl_sync(0xffffffffu, csy, base + ch);
        const double bz = __shfl_sync(0xffffffffu, csz, base + ch);
        const double coord = j == 1 ? bx : (j == 2 ? by : (j == 3 ? bz : 1.0));
        const double t = dmul(w, coord);
        if (ch < nch) acc = dadd(acc, t);
    }
    const double q = ddiv(acc, valid ? static_cast<double>(A.count[c]) : 1.0);
    const double px = __shfl_sync(0xffffffffu, q, base + 1), py = __shfl_sync(0xffffffffu, q, base + 2),
                 pz = __shfl_sync(0xffffffffu, q, base + 3);
    double rm = 0.0;
    if (j < nch) rm = dadd(crm, dnorm3(dsub(csx, px), dsub(csy, py), dsub(csz, pz)));
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
        rm = fmax(rm, __shfl_xor_sync(0xffffffffu, rm, o));
        cex = fmax(cex, __shfl_xor_sync(0xffffffffu, cex, o));
    }
    double d = 0.0;
    if (valid && j < 3) {
        const double *rt = cell_root(A.ctl, A.first, c);
        const double h = cell_side(rt, A.level[c]);
        d = corner_axis(rt, j, h, j == 0 ? A.cx[c] : (j == 1 ? A.cy[c] : A.cz[c]), j == 0 ? px : (j == 1 ? py : pz));
    }
    const double d0 = __shfl_sync(0xffffffffu, d, base), d1 = __shfl_sync(0xffffffffu, d, base + 1),
                 d2 = __shfl_sync(0xffffffffu, d, base + 2);
    const double pcap = dnorm3(d0, d1, d2);
    if (pcap < rm) rm = pcap;
    if (valid && j == 0) {
        const double rc = dadd(rm, cex);
        A.sx[c] = px;
        A.sy[c] = py;
        A.sz[c] = pz;
        A.rmax[c] = rm;
        A.rcrit[c] = rc;
        float4 hi, lo;
        split3(px, py, pz, hi, lo);
        hi.w = static_cast<float>(rc);
        lo.w = 0.f;
        A.gh[c] = hi;
        A.gl[c] = lo;
    }
}

// The parents, level by level from the deepest, in one cooperative launch
// (the leaves were done by k_leaf_collision, which also zeroed the barrier
// counter).  Four parents per warp, so that one FP64 warp instruction
// advances four parents.
__global__ void __launch_bounds__(32 * CLIMB_WARPS_COOP) k_climb_collision(ClimbArgs A) {
    if ((A.gate && *A.gate == 0) || aborted(A.ctl)) return;
    const int lane = threadIdx.x & 31;
    // warps numbered across the blocks first, so that consecutive work items land on different SMs
    const int gw0 = (threadIdx.x >> 5) * gridDim.x + blockIdx.x, nwarps = (gridDim.x * blockDim.x) >> 5;
    unsigned bar = 0;
    const int maxl = A.ctl->max_level;
    for (int lev = maxl - 1; lev >= 0; lev--) {
        const int ls = A.ctl->level_start[lev], le = A.ctl->level_start[lev + 1];
        for (int g = gw0; ls + g * PARENT_GROUP < le; g += nwarps) {
            const int cc = ls + g * PARENT_GROUP + (lane >> 3);
            const int c = (cc < le && A.nchild[cc] > 0) ? cc : -1;
            if (__any_sync(0xffffffffu, c >= 0)) parent_collision_group(A, c, lane);
        }
        if (lev > 0 && !grid_sync_on(&A.ctl->bar_count2, A.ctl, bar)) return;
    }
}

void launch_climb_collision(ncorp_ctx *c, const ParticleSet &P, const double *vx, const double *vy,
                            const double *vz, double dt, const double *rc_given, const int *gate) {
    Cells &C = c->cells;
    ClimbArgs A{};
    A.x = P.x; A.y = P.y; A.z = P.z; A.R = P.R; A.vx = vx; A.vy = vy; A.vz = vz;
    A.first = C.first; A.count = C.count; A.child0 = C.child0; A.nchild = C.nchild; A.parent = C.parent;
    A.level = C.level; A.arrive = C.arrive; A.cx = C.cx; A.cy = C.cy; A.cz = C.cz;
    A.sx = C.bx; A.sy = C.by; A.sz = C.bz; A.rmax = C.bmax; A.rcrit = C.bcrit;
    A.gh = C.bh; A.gl = C.bl;
    A.leaves = C.leaves; A.ctl = c->ctl; A.dt = dt; A.cv4 = c->cv4;
    A.rc_given = rc_given;
    A.gate = gate;
    k_leaf_collision<<<8 * c->num_sms, 64, 0, c->stream>>>(A); c->launches++;
    NCORP_CUDA_CHECK(cudaGetLastError());
    const int block = 32 * CLIMB_WARPS_COOP;
    const int grid = coop_grid(c, reinterpret_cast<const void *>(k_climb_collision), block, 0);
    void *args[] = {&A};   // ctl->bar_count2 was zeroed by k_leaf_collision
    NCORP_CUDA_CHECK(cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(k_climb_collision), dim3(grid),
                                                 dim3(block), args, 0, c->stream));
    c->launches++;
}

}  // namespace ncorp
