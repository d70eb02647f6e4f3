// walk.cu -- the symmetric dual-tree walk of Algorithm TreeWalk (Sect. 3.4.5)
// for mutual gravity and for collision search, run breadth first.
//
// The recursive walk is replaced by a frontier of pending (A, B) cell pairs
// that is expanded one generation per pass of a single cooperative launch;
// every pair takes the branch the algorithm gives it, in the algorithm's
// order:
//   A == B : N_A <= N_cs or A a leaf -> direct self interaction,
//            else all pairs (a, b), a <= b, of children (up to 36);
//   A != B : N_A N_B < N_cc,pre      -> direct;
//            well separated          -> M2L (gravity) / nothing (collisions);
//            N_A N_B < N_cc,post or both leaves -> direct;
//            split A if A is not a leaf and (r_crit,A > r_crit,B or B is a
//            leaf), else split B.
// Well separated: (r_crit,A + r_crit,B)^2 <= |s_A - s_B|^2 for gravity; for
// collisions the pair is pruned only if ((r_crit,A + r_crit,B)(1 + 2^-40))^2
// < |s_A - s_B|^2, a margin that keeps rounding from dropping a pair that the
// pairwise test would accept.
//
// A direct interaction between cells that are not both leaves is refined into
// leaf-leaf and leaf-self pieces covering exactly the same moonlet pairs (a
// "forced" frontier entry that is only ever split), so that the direct lists
// only hold leaves; the decision itself is counted once, where it is taken.
#include "ctx.h"

namespace ncorp {

// One criterion of the walk: the geometry it separates cells by and its thresholds.
struct WalkCrit {
    long long n_cs, pre, post;
    const double *sx, *sy, *sz, *rcrit;
    const float4 *H, *Lo;      // FP32 centre hi + r_crit, centre lo
};

struct WalkArgs {
    int gravity;               // the gravity criterion is walked (its lists, per-target lists, statistics)
    int collisions;            // the collision criterion is walked (pairs into cp2p / cself)
    WalkCrit g, c;             // gravity and collision criteria
    const int *gate;           // nullable: the walk does nothing while *gate is 0
    int2 *cp2p;                // collision walk: leaf pairs to test (count ctl->n_cp2p)
    int *cself;                // collision walk: leaves to test within (count ctl->n_cself)
    int cp2p_cap, cself_cap;
    const int *count, *child0, *nchild;
    int2 *front0, *front1;
    int *fcount;
    int front_cap;
    int2 *m2l;
    int m2l_cap;
    int2 *p2p;
    int p2p_cap;
    int *self;
    int self_cap;
    // per-target lists (gravity): counting sort by target cell
    int *cnt, *offs, *cursor, *p2p_off;
    int2 *p2p_src;             // per directed near-field entry: the source leaf's (first, count)
    const int *first;
    int2 *m2l_dir;
    int m2l_dir_cap, p2p_dir_cap;
    int *work;                 // gravity: the near-field kernel's work counter, zeroed by k_walk_init
    Ctrl *ctl;
};

// Frontier entries (x, y): x = cell A | flags, y = cell B | gravity forced.  Forced: the pair was
// decided direct above the leaves and is only split into leaf pieces.  The flags say which criterion
// still acts on the pair (a walk of both criteria follows gravity's choice of the cell to split while
// gravity acts, and the collision criterion's once gravity is done with the pair).
constexpr int FORCED = static_cast<int>(0x80000000u);   // y: gravity forced
constexpr int C_FORCED = static_cast<int>(0x80000000u); // x: collisions forced
constexpr int G_DONE = 1 << 30;                          // x: gravity has decided the pair
constexpr int C_DONE = 1 << 29;                          // x: the collision criterion has decided the pair
constexpr int CELL_MASK = (1 << 29) - 1;

// One thread: the root pairs, zeroed frontier counts and counters, and (for
// gravity) the work counter of the near-field kernel that reads the lists.
__global__ void k_walk_init(WalkArgs A) {
    if ((A.gate && *A.gate == 0) || aborted(A.ctl)) return;
    const int nd = A.ctl->nd;   // one root pair per disk (a forest's disks never interact)
    for (int d = 0; d < nd; d++) A.front0[d] = make_int2(d, d);
    A.ctl->n_cp2p = 0;
    A.ctl->n_cself = 0;
    // a walk of both criteria lists the next collision search's pairs; a gravity walk alone does not
    if (A.gravity) A.ctl->col_stale = A.collisions ? 0 : 1;
    A.ctl->dec_pairs_c = 0;
    A.ctl->dec_self_c = 0;
    for (int i = 1; i <= WALK_MAX_ITERS; i++) A.fcount[i] = 0;
    A.fcount[0] = nd;
    if (A.work) *A.work = 0;
    A.ctl->n_m2l = 0;
    A.ctl->n_p2p = 0;
    A.ctl->n_self = 0;
    A.ctl->dec_pairs = 0;
    A.ctl->dec_self = 0;
    A.ctl->n_inter = 0;
    A.ctl->walk_iters = 0;
    A.ctl->bar_count = 0;
    A.ctl->walk_abort[0] = A.ctl->walk_abort[1] = A.ctl->walk_abort[2] = 0;
}

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Exclusive prefix of v over the block; *total receives the block's sum.
__device__ int block_prefix(int v, int *s_tmp, int *total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    __syncthreads();
    if (lane == 31) s_tmp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int w = lane < nw ? s_tmp[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += u;
        }
        if (lane < nw) s_tmp[lane] = wi - w;
        if (lane == 31) s_tmp[32] = wi;
    }
    __syncthreads();
    const int r = s_tmp[wid] + incl - v;
    if (total) *total = s_tmp[32];
    return r;
}

// One end of a walk entry: the target's counter, key = 2 target + (0: M2L
// list, 1: direct list), -1 for none.  Lanes of a warp holding the same key
// are served by one atomic (entries of a split arrive together, so a target
// often appears several times in a warp); returns the lane's slot.
__device__ __forceinline__ int aggregated_add(int *m2l_ctr, int *p2p_ctr, int key) {
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
    int at = 0;
    if (key >= 0 && lane == leader) at = atomicAdd((key & 1) ? &p2p_ctr[key >> 1] : &m2l_ctr[key >> 1], __popc(peers));
    at = __shfl_sync(0xffffffffu, at, leader);
    return at + __popc(peers & ((1u << lane) - 1u));
}

// Directed lists from the walk's output (gravity): M2L (A, B) gives A <- B
// and B <- A grouped by target; leaf pairs give A <- B and B <- A, self
// leaves A <- A, grouped by target leaf.  Counting sort: counts (warp-
// aggregated atomics), prefix sums over all blocks (chunk sums, a barrier,
// chunk scans), scatter (aggregated again: entries of one target in an order
// set by the atomics).  The frontier buffers, idle after the walk, hold the
// chunk sums.
__device__ void walk_lists(const WalkArgs &A, int *s_tmp, unsigned &bar) {
    const int nm = min(A.ctl->n_m2l, A.m2l_cap), np = min(A.ctl->n_p2p, A.p2p_cap),
              ns = min(A.ctl->n_self, A.self_cap);
    const int nc = A.ctl->n_cells + 1, total = nm + np + ns;
    const int lane = threadIdx.x & 31;
    const int wbase = (blockIdx.x * blockDim.x + threadIdx.x - lane), wstride = gridDim.x * blockDim.x;
    for (int base = wbase; base < total; base += wstride) {
        const int i = base + lane;
        int k0 = -1, k1 = -1;
        if (i < nm) {
            const int2 e = __ldcg(&A.m2l[i]);
            k0 = 2 * e.x;
            k1 = 2 * e.y;
        } else if (i < nm + np) {
            const int2 e = __ldcg(&A.p2p[i - nm]);
            k0 = 2 * e.x + 1;
            k1 = 2 * e.y + 1;
        } else if (i < total) {
            k0 = 2 * __ldcg(&A.self[i - nm - np]) + 1;
        }
        aggregated_add(A.cnt, A.p2p_off, k0);
        aggregated_add(A.cnt, A.p2p_off, k1);
    }
    if (!grid_sync(A.ctl, bar)) return;
    // chunk sums of both count arrays
    int *bs = reinterpret_cast<int *>(A.front0);   // [2][gridDim.x]
    const int G = gridDim.x, ch = (nc + G - 1) / G;
    const int c0 = min(nc, static_cast<int>(blockIdx.x) * ch), c1 = min(nc, c0 + ch);
    {
        int sm = 0, sp = 0;
        for (int i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
            sm += __ldcg(&A.cnt[i]);
            sp += __ldcg(&A.p2p_off[i]);
        }
        int tm = 0, tp = 0;
        block_prefix(sm, s_tmp, &tm);
        block_prefix(sp, s_tmp, &tp);
        if (threadIdx.x == 0) {
            bs[blockIdx.x] = tm;
            bs[G + blockIdx.x] = tp;
        }
    }
    if (!grid_sync(A.ctl, bar)) return;
    {
        int pm = 0, pp = 0;
        for (int b = threadIdx.x; b < static_cast<int>(blockIdx.x); b += blockDim.x) {
            pm += __ldcg(&bs[b]);
            pp += __ldcg(&bs[G + b]);
        }
        block_prefix(pm, s_tmp, &pm);
        block_prefix(pp, s_tmp, &pp);
        for (int t0 = c0; t0 < c1; t0 += blockDim.x) {
            const int i = t0 + threadIdx.x;
            const bool ok = i < c1;
            const int vm = ok ? __ldcg(&A.cnt[i]) : 0, vp = ok ? __ldcg(&A.p2p_off[i]) : 0;
            int sm = 0, sp = 0;
            const int xm = block_prefix(vm, s_tmp, &sm), xp = block_prefix(vp, s_tmp, &sp);
            if (ok) {
                A.offs[i] = pm + xm;      // M2L: offsets and cursors
                A.cursor[i] = pm + xm;
                A.p2p_off[i] = pp + xp;   // direct: offsets (in place), cursors in cnt
                A.cnt[i] = pp + xp;
            }
            pm += sm;
            pp += sp;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            A.ctl->n_m2l_dir = 2 * nm;
            A.ctl->n_p2p_dir = 2 * np + ns;
        }
    }
    if (!grid_sync(A.ctl, bar)) return;
    for (int base = wbase; base < total; base += wstride) {
        const int i = base + lane;
        int k0 = -1, k1 = -1;
        int2 e = make_int2(0, 0);
        if (i < nm) {
            e = __ldcg(&A.m2l[i]);
            k0 = 2 * e.x;
            k1 = 2 * e.y;
        } else if (i < nm + np) {
            e = __ldcg(&A.p2p[i - nm]);
            k0 = 2 * e.x + 1;
            k1 = 2 * e.y + 1;
        } else if (i < total) {
            e.x = e.y = __ldcg(&A.self[i - nm - np]);
            k0 = 2 * e.x + 1;
        }
        const int a = aggregated_add(A.cursor, A.cnt, k0), b = aggregated_add(A.cursor, A.cnt, k1);
        if (i < nm) {
            if (a < A.m2l_dir_cap && b < A.m2l_dir_cap) {
                A.m2l_dir[a] = make_int2(e.x, e.y);
                A.m2l_dir[b] = make_int2(e.y, e.x);
            } else {
                atomicOr(&A.ctl->err, ERR_DIRECTED);
            }
        } else if (i < nm + np) {
            if (a < A.p2p_dir_cap && b < A.p2p_dir_cap) {
                A.p2p_src[a] = make_int2(__ldg(&A.first[e.y]), __ldg(&A.count[e.y]));
                A.p2p_src[b] = make_int2(__ldg(&A.first[e.x]), __ldg(&A.count[e.x]));
            } else {
                atomicOr(&A.ctl->err, ERR_DIRECTED);
            }
        } else if (i < total) {
            if (a < A.p2p_dir_cap) A.p2p_src[a] = make_int2(__ldg(&A.first[e.x]), __ldg(&A.count[e.x]));
            else atomicOr(&A.ctl->err, ERR_DIRECTED);
        }
    }
}

constexpr int WALK_THREADS = 256, WALK_WARPS = WALK_THREADS / 32, WALK_LISTS = 6;

// Per block: the slots one iteration's warps want in the six append lists
// (M2L, direct pairs, self leaves, next frontier, and the collision
// criterion's pairs and self leaves), reserved with one atomic per list for
// the whole block (a global counter that every warp hit in turn was the
// walk's bottleneck at N = 1e6).
struct WalkSlots {
    int want[WALK_WARPS][WALK_LISTS];
    int base[WALK_WARPS][WALK_LISTS];
};

// The outcome of one criterion for a pair of cells (Algorithm TreeWalk).
enum : int { O_NONE = 0, O_M2L, O_P2P, O_SELF, O_SPLIT_SELF, O_SPLIT_A, O_SPLIT_B };

struct WalkDec {
    int kind;                  // O_*: O_M2L for a separated pair (gravity: an M2L; collisions: pruned)
    bool child_forced;         // the children pairs are pieces of a direct interaction
    long long dpair, dself, inter;
};

// The decision of criterion K for (cA, cB): cells with nA, nB moonlets and chA, chB children, K's
// centres (hi, lo) and r_crit in FP32 (ha, la, hb, lb) and r_crit in FP64 (rA, rB).
__device__ __forceinline__ WalkDec walk_decide(const WalkCrit &K, bool grav, int cA, int cB, bool forced, int nA,
                                               int nB, int chA, int chB, const float4 &ha, const float4 &la,
                                               const float4 &hb, const float4 &lb, double rA, double rB) {
    WalkDec d{O_NONE, false, 0, 0, 0};
    const bool leafA = chA == 0, leafB = chB == 0;
    if (cA == cB) {
        if (forced || nA <= K.n_cs || leafA) {
            if (!forced) {
                d.dself = 1;
                d.inter = static_cast<long long>(nA) * (nA - 1) / 2;
            }
            if (leafA) d.kind = O_SELF;
            else { d.kind = O_SPLIT_SELF; d.child_forced = true; }
        } else {
            d.kind = O_SPLIT_SELF;
        }
        return d;
    }
    if (forced) {
        if (leafA && leafB) d.kind = O_P2P;
        else { d.kind = leafA ? O_SPLIT_B : O_SPLIT_A; d.child_forced = true; }
        return d;
    }
    const long long prod = static_cast<long long>(nA) * nB;
    bool direct = false;
    if (prod < K.pre) {
        direct = true;
    } else {
        // FP32 first: centres as hi + lo pairs give |s_A - s_B|^2 to ~1e-6
        // relative and r_crit is rounded once; outside a band of
        // +-2^-14 around the threshold the FP32 answer is the FP64 one,
        // inside it the exact FP64 test decides.
        const float fx = (ha.x - hb.x) + (la.x - lb.x);
        const float fy = (ha.y - hb.y) + (la.y - lb.y);
        const float fz = (ha.z - hb.z) + (la.z - lb.z);
        const float d2f = fx * fx + fy * fy + fz * fz;
        const float tf = ha.w + hb.w, t2f = tf * tf;
        // (the hi + lo pairs carry an absolute error ~2^-47 |s|: separations below
        // ~2^-26 |s| go to FP64)
        const float fl = (fabsf(ha.x) + fabsf(ha.y) + fabsf(ha.z)) * 0x1p-26f, fl2 = fl * fl + 1e-30f;
        bool sep;
        if (d2f > fl2 && d2f > t2f * (1.0f + 0x1p-14f)) {
            sep = true;
        } else if (d2f > fl2 && d2f < t2f * (1.0f - 0x1p-14f)) {
            sep = false;
        } else {
            const double dx = dsub(K.sx[cA], K.sx[cB]);
            const double dy = dsub(K.sy[cA], K.sy[cB]);
            const double dz = dsub(K.sz[cA], K.sz[cB]);
            const double d2 = dsq3(dx, dy, dz);
            if (grav) {
                const double t = dadd(rA, rB);
                sep = dmul(t, t) <= d2;
            } else {
                const double t = dmul(dadd(rA, rB), 1.0 + 0x1p-40);
                sep = dmul(t, t) < d2;
            }
        }
        if (sep) d.kind = O_M2L;
        else if (prod < K.post || (leafA && leafB)) direct = true;
        else if (!leafA && (rA > rB || leafB)) d.kind = O_SPLIT_A;
        else d.kind = O_SPLIT_B;
    }
    if (direct) {
        d.dpair = 1;
        d.inter = prod;
        if (leafA && leafB) d.kind = O_P2P;
        else { d.kind = leafA ? O_SPLIT_B : O_SPLIT_A; d.child_forced = true; }
    }
    return d;
}

__device__ __forceinline__ bool is_split(int k) { return k >= O_SPLIT_SELF; }

// One generation of the walk: the pairs cur[0, nf) of generation it, taken
// a block of WALK_THREADS at a time (warp w of the block takes the w-th 32);
// outcomes appended to the lists and children pairs to the next frontier.
// The decision statistics are added to the thread's totals st[5] (gravity:
// direct pairs, direct self cells, moonlet pairs; collisions: direct pairs,
// direct self cells).
template <bool GRAV, bool COL>
__device__ __forceinline__ void walk_generation(const WalkArgs &A, int it, int nf, long long *st, WalkSlots &S) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int2 *cur = (it & 1) ? A.front1 : A.front0;
    int2 *nxt = (it & 1) ? A.front0 : A.front1;
    int *ncount = A.fcount + it + 1;
    // the loop bounds are the same for every thread of the block (block barriers inside)
    for (int bbase = blockIdx.x * WALK_THREADS; bbase < nf; bbase += gridDim.x * WALK_THREADS) {
        const int i = bbase + w * 32 + lane;
        const bool valid = i < nf;
        int cA = 0, cB = 0;
        bool g_act = false, c_act = false, g_forced = false, c_forced = false;
        if (valid) {
            const int2 e = __ldcg(&cur[i]);
            cA = e.x & CELL_MASK;
            cB = e.y & 0x7fffffff;
            g_act = GRAV && !(e.x & G_DONE);
            c_act = COL && !(e.x & C_DONE);
            g_forced = (e.y & FORCED) != 0;
            c_forced = (e.x & C_FORCED) != 0;
        }
        // every cell field this lane may need, loaded in one round
        int nA = 0, nB = 0, chA = 0, chB = 0, c0A = 0, c0B = 0;
        float4 ha = make_float4(0.f, 0.f, 0.f, 0.f), hb = ha, la = ha, lb = ha, ka = ha, kb = ha, ma = ha, mb = ha;
        double rA = 0.0, rB = 0.0, qA = 0.0, qB = 0.0;
        if (valid) {
            nA = __ldg(&A.count[cA]);
            nB = __ldg(&A.count[cB]);
            chA = __ldg(&A.nchild[cA]);
            chB = __ldg(&A.nchild[cB]);
            c0A = __ldg(&A.child0[cA]);
            c0B = __ldg(&A.child0[cB]);
        }
        if (GRAV && g_act) {
            ha = __ldg(&A.g.H[cA]);
            hb = __ldg(&A.g.H[cB]);
            la = __ldg(&A.g.Lo[cA]);
            lb = __ldg(&A.g.Lo[cB]);
            rA = __ldg(&A.g.rcrit[cA]);
            rB = __ldg(&A.g.rcrit[cB]);
        }
        if (COL && c_act) {
            ka = __ldg(&A.c.H[cA]);
            kb = __ldg(&A.c.H[cB]);
            ma = __ldg(&A.c.Lo[cA]);
            mb = __ldg(&A.c.Lo[cB]);
            qA = __ldg(&A.c.rcrit[cA]);
            qB = __ldg(&A.c.rcrit[cB]);
        }
        WalkDec gd{O_NONE, false, 0, 0, 0}, cd{O_NONE, false, 0, 0, 0};
        if (GRAV && g_act) gd = walk_decide(A.g, true, cA, cB, g_forced, nA, nB, chA, chB, ha, la, hb, lb, rA, rB);
        if (COL && c_act) cd = walk_decide(A.c, false, cA, cB, c_forced, nA, nB, chA, chB, ka, ma, kb, mb, qA, qB);
        st[0] += gd.dpair;
        st[1] += gd.dself;
        st[2] += gd.inter;
        st[3] += cd.dpair;
        st[4] += cd.dself;
        const int emit_m2l = gd.kind == O_M2L, emit_p2p = gd.kind == O_P2P, emit_self = gd.kind == O_SELF;
        const int emit_cp2p = cd.kind == O_P2P, emit_cself = cd.kind == O_SELF;
        // the split: gravity's choice while gravity acts on the pair, else the collision criterion's
        const bool gs = is_split(gd.kind), cs = is_split(cd.kind);
        const int split = gs ? gd.kind : (cs ? cd.kind : O_NONE);
        // flags of the children: each criterion that split goes on, with its forced state
        int fx = 0, fy = 0;
        if (split != O_NONE) {
            if (!gs) fx |= G_DONE;
            else if (gd.child_forced) fy |= FORCED;
            if (!cs) fx |= C_DONE;
            else if (cd.child_forced) fx |= C_FORCED;
        }
        int c0 = 0, nch = 0, k = 0;
        if (split == O_SPLIT_SELF) {
            c0 = c0A;
            nch = chA;
            k = nch * (nch + 1) / 2;
        } else if (split == O_SPLIT_A) {
            c0 = c0A;
            nch = chA;
            k = nch;
        } else if (split == O_SPLIT_B) {
            c0 = c0B;
            nch = chB;
            k = nch;
        }
        // outputs: the block's warps reserve their slots together, one atomic per list
        const unsigned bm = __ballot_sync(0xffffffffu, emit_m2l), bp = __ballot_sync(0xffffffffu, emit_p2p),
                       bs = __ballot_sync(0xffffffffu, emit_self), bcp = __ballot_sync(0xffffffffu, emit_cp2p),
                       bcs = __ballot_sync(0xffffffffu, emit_cself);
        int kin = k;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, kin, o);
            if (lane >= o) kin += v;
        }
        const int ktot = __shfl_sync(0xffffffffu, kin, 31);
        if (lane == 0) {
            S.want[w][0] = __popc(bm);
            S.want[w][1] = __popc(bp);
            S.want[w][2] = __popc(bs);
            S.want[w][3] = ktot;
            S.want[w][4] = __popc(bcp);
            S.want[w][5] = __popc(bcs);
        }
        __syncthreads();
        if (threadIdx.x < WALK_LISTS) {   // one thread per list: the warps' offsets, one atomic for the block
            const int q = threadIdx.x;
            int tot = 0;
#pragma unroll
            for (int ww = 0; ww < WALK_WARPS; ww++) {
                S.base[ww][q] = tot;
                tot += S.want[ww][q];
            }
            int *ctr = q == 0 ? &A.ctl->n_m2l
                     : q == 1 ? &A.ctl->n_p2p
                     : q == 2 ? &A.ctl->n_self
                     : q == 3 ? ncount
                     : q == 4 ? &A.ctl->n_cp2p : &A.ctl->n_cself;
            const int b0 = tot ? atomicAdd(ctr, tot) : 0;
#pragma unroll
            for (int ww = 0; ww < WALK_WARPS; ww++) S.base[ww][q] += b0;
        }
        __syncthreads();
        const int base_m = S.base[w][0], base_p = S.base[w][1], base_s = S.base[w][2], base_f = S.base[w][3],
                  base_cp = S.base[w][4], base_cs = S.base[w][5];
        const unsigned lt = (1u << lane) - 1u;
        if (emit_m2l) {
            const int slot = base_m + __popc(bm & lt);
            if (slot < A.m2l_cap) A.m2l[slot] = make_int2(cA, cB);
            else { atomicOr(&A.ctl->err, ERR_M2L); A.ctl->walk_abort[it % 3] = 1; }
        }
        if (emit_p2p) {
            const int slot = base_p + __popc(bp & lt);
            if (slot < A.p2p_cap) A.p2p[slot] = make_int2(cA, cB);
            else { atomicOr(&A.ctl->err, ERR_P2P); A.ctl->walk_abort[it % 3] = 1; }
        }
        if (emit_self) {
            const int slot = base_s + __popc(bs & lt);
            if (slot < A.self_cap) A.self[slot] = cA;
            else { atomicOr(&A.ctl->err, ERR_P2P); A.ctl->walk_abort[it % 3] = 1; }
        }
        if (emit_cp2p) {
            const int slot = base_cp + __popc(bcp & lt);
            if (slot < A.cp2p_cap) A.cp2p[slot] = make_int2(cA, cB);
            else { atomicOr(&A.ctl->err, ERR_P2P); A.ctl->walk_abort[it % 3] = 1; }
        }
        if (emit_cself) {
            const int slot = base_cs + __popc(bcs & lt);
            if (slot < A.cself_cap) A.cself[slot] = cA;
            else { atomicOr(&A.ctl->err, ERR_P2P); A.ctl->walk_abort[it % 3] = 1; }
        }
        if (k > 0) {
            int slot = base_f + kin - k;
            if (slot + k > A.front_cap) {
                atomicOr(&A.ctl->err, ERR_FRONTIER);
                A.ctl->walk_abort[it % 3] = 1;
            } else {
                if (split == O_SPLIT_SELF) {
                    for (int a = 0; a < nch; a++)
                        for (int b = a; b < nch; b++) nxt[slot++] = make_int2((c0 + a) | fx, (c0 + b) | fy);
                } else if (split == O_SPLIT_A) {
                    for (int a = 0; a < nch; a++) nxt[slot++] = make_int2((c0 + a) | fx, cB | fy);
                } else {
                    for (int b = 0; b < nch; b++) nxt[slot++] = make_int2(cA | fx, (c0 + b) | fy);
                }
            }
        }
    }
}

template <bool GRAV, bool COL>
__global__ void __launch_bounds__(WALK_THREADS) k_walk(WalkArgs A) {
    __shared__ int s_tmp[33];
    __shared__ WalkSlots S;
    __shared__ long long s_stat[WALK_WARPS][5];
    if ((A.gate && *A.gate == 0) || aborted(A.ctl)) return;   // (every block, before the first barrier)
    if (A.gravity) {   // list counters, zeroed before the first barrier of the walk
        const int nc = A.ctl->n_cells + 1;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
            A.cnt[i] = 0;
            A.p2p_off[i] = 0;
        }
    }
    volatile int *vcount = A.fcount;
    unsigned bar = 0;
    int it = 0;
    long long st[5] = {0, 0, 0, 0, 0};   // decision statistics of this thread's pairs
    for (; it < WALK_MAX_ITERS; it++) {
        const int nf = min(vcount[it], A.front_cap);
        if (nf == 0) break;
        if (blockIdx.x == 0 && threadIdx.x == 0) A.ctl->walk_abort[(it + 1) % 3] = 0;   // slot of the next generation
        walk_generation<GRAV, COL>(A, it, nf, st, S);
        if (!grid_sync(A.ctl, bar)) return;
        // overflow in this generation (slot it mod 3: identical for every block after the barrier)
        if (((volatile int *)A.ctl->walk_abort)[it % 3]) { it++; break; }
    }
    {   // the statistics: one atomic per block and counter
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
        for (int k = 0; k < 5; k++) {
            const long long v = warp_sum_ll(st[k]);
            if (lane == 0) s_stat[w][k] = v;
        }
        __syncthreads();
        if (threadIdx.x < 5) {
            long long v = 0;
#pragma unroll
            for (int ww = 0; ww < WALK_WARPS; ww++) v += s_stat[ww][threadIdx.x];
            long long *dst = threadIdx.x == 0 ? &A.ctl->dec_pairs
                           : threadIdx.x == 1 ? &A.ctl->dec_self
                           : threadIdx.x == 2 ? &A.ctl->n_inter
                           : threadIdx.x == 3 ? &A.ctl->dec_pairs_c : &A.ctl->dec_self_c;
            if (v) atomicAdd(reinterpret_cast<unsigned long long *>(dst), static_cast<unsigned long long>(v));
        }
        // the collision statistics' copies below read every block's totals
        if (A.collisions && !grid_sync(A.ctl, bar)) return;
    }
    // the generation count and the barrier snapshot are the same in every block
    if (A.gravity && it < WALK_MAX_ITERS && !((volatile int *)A.ctl->walk_abort)[(it + 2) % 3]) walk_lists(A, s_tmp, bar);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (A.gravity) A.ctl->walk_iters = it;
        if (A.collisions) {
            A.ctl->col_pairs = A.ctl->dec_pairs_c;
            A.ctl->col_self = A.ctl->dec_self_c;
            A.ctl->col_iters = it;
        }
        if (it >= WALK_MAX_ITERS) atomicOr(&A.ctl->err, ERR_FRONTIER);
    }
}

static WalkCrit walk_crit(const ncorp_ctx *c, bool gravity) {
    const Cells &C = c->cells;
    WalkCrit K;
    K.n_cs = gravity ? c->g_cs : c->c_cs;
    K.pre = gravity ? c->g_pre : c->c_pre;
    K.post = gravity ? c->g_post : c->c_post;
    K.sx = gravity ? C.sx : C.bx;
    K.sy = gravity ? C.sy : C.by;
    K.sz = gravity ? C.sz : C.bz;
    K.rcrit = gravity ? C.rcrit : C.bcrit;
    K.H = gravity ? C.gh : C.bh;
    K.Lo = gravity ? C.gl : C.bl;
    return K;
}

void launch_walk(ncorp_ctx *c, bool gravity, bool collisions, const int *gate) {
    Cells &C = c->cells;
    WalkLists &W = c->wl;
    WalkArgs A;
    A.gravity = gravity ? 1 : 0;
    A.collisions = collisions ? 1 : 0;
    A.g = walk_crit(c, true);
    A.c = walk_crit(c, false);
    A.gate = gate;
    A.count = C.count; A.first = C.first; A.child0 = C.child0; A.nchild = C.nchild;
    A.front0 = W.front[0]; A.front1 = W.front[1]; A.fcount = W.front_count; A.front_cap = W.front_cap;
    A.m2l = W.m2l; A.m2l_cap = W.m2l_cap;
    A.p2p = W.p2p; A.p2p_cap = W.p2p_cap;
    A.self = W.self; A.self_cap = W.self_cap;
    A.cp2p = W.cp2p; A.cp2p_cap = W.p2p_cap;
    A.cself = W.cself; A.cself_cap = W.self_cap;
    A.cnt = W.cnt; A.offs = W.offs; A.cursor = W.cursor; A.p2p_off = W.p2p_off; A.p2p_src = W.p2p_src;
    A.m2l_dir = W.m2l_dir; A.m2l_dir_cap = W.m2l_dir_cap; A.p2p_dir_cap = W.p2p_dir_cap;
    A.work = gravity ? c->work_counter : nullptr;
    A.ctl = c->ctl;
    k_walk_init<<<1, 1, 0, c->stream>>>(A); c->launches++;
    NCORP_CUDA_CHECK(cudaGetLastError());
    const void *kern = gravity && collisions ? reinterpret_cast<const void *>(k_walk<true, true>)
                     : gravity              ? reinterpret_cast<const void *>(k_walk<true, false>)
                                            : reinterpret_cast<const void *>(k_walk<false, true>);
    int per_sm = 0;
    NCORP_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WALK_THREADS, 0));
    if (per_sm < 1) per_sm = 1;
    if (per_sm > 2) per_sm = 2;
    // about one block per 640 moonlets (frontiers peak near a third of n pairs), 32 to the cooperative limit
    const int grid = std::min(coop_blocks(c, per_sm), std::max(32, c->cur_n / 640));
    void *args[] = {&A};
    NCORP_CUDA_CHECK(cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(WALK_THREADS), args, 0, c->stream));
    c->launches++;
}

}  // namespace ncorp
