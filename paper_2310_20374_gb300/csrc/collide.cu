// collide.cu -- the pairwise collision test of Sect. 3.1 over the direct lists
// of the collision walk, the resolution of the colliding pairs (Sect. 5.1,
// 5.2) and the sorting of the pairs for output.
//
// Straight-line trajectories over the step: with dr = r1 - r2, dv = v1 - v2,
//   Delta = (dr.dv)^2 + dv^2 ((R1 + R2)^2 - dr^2),
//   dt_c  = -(dr.dv + sqrt(Delta)) / dv^2,
// the pair collides within the step iff Delta >= 0 and 0 <= dt_c <= dt
// (dv = 0: no collision).  Evaluated in FP64 with exactly rounded operations
// in a fixed order, (1, 2) being the pair in increasing caller index, so that
// the set of pairs is reproducible bit for bit.
#include <algorithm>

#include "ctx.h"

namespace ncorp {

// Impact time of the straight-line trajectories: false when dv = 0 or Delta < 0.
__device__ __forceinline__ bool impact_time(double x1, double y1, double z1, double u1, double v1, double w1,
                                            double R1, double x2, double y2, double z2, double u2, double v2,
                                            double w2, double R2, double &tc) {
    const double dx = dsub(x1, x2), dy = dsub(y1, y2), dz = dsub(z1, z2);
    const double ux = dsub(u1, u2), uy = dsub(v1, v2), uz = dsub(w1, w2);
    const double b = dadd(dadd(dmul(dx, ux), dmul(dy, uy)), dmul(dz, uz));
    const double dr2 = dsq3(dx, dy, dz);
    const double dv2 = dsq3(ux, uy, uz);
    if (dv2 == 0.0) return false;
    const double Rs = dadd(R1, R2);
    const double Delta = dadd(dmul(b, b), dmul(dv2, dsub(dmul(Rs, Rs), dr2)));
    if (Delta < 0.0) return false;
    tc = ddiv(-dadd(b, dsqrt(Delta)), dv2);
    return true;
}

__device__ __forceinline__ bool collide_test(double x1, double y1, double z1, double u1, double v1, double w1,
                                             double R1, double x2, double y2, double z2, double u2, double v2,
                                             double w2, double R2, double dt) {
    double tc;
    if (!impact_time(x1, y1, z1, u1, v1, w1, R1, x2, y2, z2, u2, v2, w2, R2, tc)) return false;
    return tc >= 0.0 && tc <= dt;
}

struct CollideArgs {
    const int2 *p2p;
    const int *self;
    const int *first, *count;
    const double *x, *y, *z, *vx, *vy, *vz, *R;
    const float4 *hi4, *lo4;
    const float4 *cv;          // velocity rounded to FP32 (xyz), R + dt |v| rounded up to FP32 (w)
    const float4 *bh, *bl;     // per cell: collision centre hi (xyz) and r_crit in FP32 (w); centre lo
    const int *perm;
    double dt;
    uint64_t *pairs;
    int2 *where;               // nullable: the pair's positions in this order (lower caller index first)
    int cap, self_cap, p2p_cap;
    Ctrl *ctl;
};

__device__ __forceinline__ void test_and_emit(const CollideArgs &A, int u, int v) {
    int a = u, b = v;
    if (A.perm[a] > A.perm[b]) {
        a = v;
        b = u;
    }
    if (collide_test(A.x[a], A.y[a], A.z[a], A.vx[a], A.vy[a], A.vz[a], A.R[a], A.x[b], A.y[b], A.z[b], A.vx[b],
                     A.vy[b], A.vz[b], A.R[b], A.dt)) {
        const int slot = atomicAdd(&A.ctl->n_found, 1);
        if (slot < A.cap) {
            A.pairs[slot] = (static_cast<unsigned long long>(A.perm[a]) << 32) | static_cast<unsigned>(A.perm[b]);
            if (A.where) A.where[slot] = make_int2(a, b);
        } else
            atomicOr(&A.ctl->err, ERR_PAIRS);
    }
}

// Two FP32 prefilters in front of the exact FP64 test, each keeping every pair
// the FP64 test can accept, so the pair set is the one the FP64 test alone
// gives.
//  1. A pair can only collide within the step if |dr| <= R1 + R2 + dt |dv| <=
//     rc1 + rc2 (rc = R + dt |v|): the separation from the double-float
//     positions (relative error ~1e-7) against (rc1 + rc2)^2 (1 + 2^-10).
//  2. The trajectories come within R1 + R2 of each other at the impact time
//     dt_c in [0, dt], so the least distance over [0, dt] is at most R1 + R2:
//     with t* = clamp(-dr.dv / dv^2, 0, dt), |dr + t* dv|^2 against
//     (R1 + R2)^2 (1 + 2^-10) plus 2^-12 (|dr|^2 + dt^2 |dv|^2).  The margin
//     exceeds the FP32 evaluation's error (velocities rounded to FP32: ~1e-7
//     relative; the terms of the quadratic are bounded by that scale) by
//     orders of magnitude, and the FP64 predicate's rounding likewise.
__device__ __forceinline__ bool may_touch(const float4 &h, const float4 &l, float r, const float4 &th,
                                          const float4 &tl, float tr, float &dx, float &dy, float &dz) {
    dx = (h.x - th.x) + (l.x - tl.x);
    dy = (h.y - th.y) + (l.y - tl.y);
    dz = (h.z - th.z) + (l.z - tl.z);
    const float s = r + tr;
    return dx * dx + dy * dy + dz * dz <= s * s * (1.0f + 0x1p-10f);
}

__device__ __forceinline__ bool may_meet(float dx, float dy, float dz, const float4 &v, const float4 &tv, float Rs,
                                         float dt) {
    const float ux = v.x - tv.x, uy = v.y - tv.y, uz = v.z - tv.z;
    const float b = dx * ux + dy * uy + dz * uz;
    const float u2 = ux * ux + uy * uy + uz * uz;
    const float t = u2 > 0.0f ? fminf(fmaxf(-b / u2, 0.0f), dt) : 0.0f;
    const float ex = dx + t * ux, ey = dy + t * uy, ez = dz + t * uz;
    const float d2 = dx * dx + dy * dy + dz * dz;
    const float margin = 0x1p-12f * (d2 + dt * dt * u2) + 1e-30f;
    return ex * ex + ey * ey + ez * ez <= Rs * Rs * (1.0f + 0x1p-10f) + margin;
}

constexpr int COL_WARPS = 8;

// 3. Before the pairs of two different leaves A and B are formed, each
//    moonlet is tested against the other leaf's sphere: a pair (a, b) can
//    only collide if |x_a - x_b| <= rc_a + rc_b, and every moonlet b of B has
//    |x_b - sbar_B| <= r_max,B <= r_crit,B - rc_b, so |x_a - sbar_B| <= rc_a +
//    r_crit,B (and the same with A and B exchanged).  In FP32 with the
//    margins of test 1; the moonlets of A and B that fail take no part in the
//    item's pairs.  Tests are still counted per item (n_A n_B pairs), as the
//    walk defines them.
__device__ __forceinline__ bool near_sphere(const float4 &h, const float4 &l, float r, const float4 &ch,
                                            const float4 &cl) {
    const float dx = (h.x - ch.x) + (l.x - cl.x);
    const float dy = (h.y - ch.y) + (l.y - cl.y);
    const float dz = (h.z - ch.z) + (l.z - cl.z);
    const float s = r + ch.w;
    return dx * dx + dy * dy + dz * dz <= s * s * (1.0f + 0x1p-10f);
}

// Warp per direct item (a leaf with itself, or a pair of leaves).  The
// item's targets are taken 32 at a time and, for a pair of leaves, only those
// near the source leaf's sphere are kept; the m kept targets occupy T =
// pow2ceil(m) lanes and the warp's lanes form G = 32 / T groups.  The source
// leaf is staged COL_STAGE moonlets at a time, compacted to those near the
// target leaf's sphere; lane (g, t) tests target t against the staged sources
// k = g, g + G, ...  so small leaves keep the lanes busy.
constexpr int COL_STAGE = 64;

__global__ void __launch_bounds__(32 * COL_WARPS, 4) k_collide(CollideArgs A) {
    __shared__ float4 s_h[COL_WARPS][COL_STAGE], s_l[COL_WARPS][COL_STAGE], s_v[COL_WARPS][COL_STAGE];
    __shared__ float s_R[COL_WARPS][COL_STAGE];
    __shared__ int s_j[COL_WARPS][COL_STAGE];
    const float dtf = static_cast<float>(A.dt) * (1.0f + 0x1p-20f);
    if (aborted(A.ctl)) return;
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const unsigned below = (1u << lane) - 1u;
    const int ns = min(A.ctl->n_cself, A.self_cap), np = min(A.ctl->n_cp2p, A.p2p_cap);
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    long long tests = 0;
    for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < ns + np; w += nwarps) {
        int ct, cs;
        if (w < ns) {
            ct = cs = A.self[w];
        } else {
            const int2 e = A.p2p[w - ns];
            ct = e.x;
            cs = e.y;
        }
        const bool self = ct == cs;
        const int ft = A.first[ct], nt = A.count[ct], fs = A.first[cs], nsrc = A.count[cs];
        if (lane == 0) tests += self ? static_cast<long long>(nt) * (nt - 1) / 2 : static_cast<long long>(nt) * nsrc;
        float4 tch = make_float4(0.f, 0.f, 0.f, 0.f), tcl = tch, sch = tch, scl = tch;   // leaves' spheres
        if (!self) {
            tch = A.bh[ct];
            tcl = A.bl[ct];
            sch = A.bh[cs];
            scl = A.bl[cs];
        }
        for (int t0 = 0; t0 < nt; t0 += 32) {
            bool keep = t0 + lane < nt;
            if (keep && !self)
                keep = near_sphere(A.hi4[ft + t0 + lane], A.lo4[ft + t0 + lane], A.cv[ft + t0 + lane].w, sch, scl);
            const unsigned kept = __ballot_sync(0xffffffffu, keep);
            const int m = __popc(kept);
            if (m == 0) continue;
            int lg = 0;
            while ((1 << lg) < m) lg++;
            const int T = 1 << lg, G = 32 >> lg, tt = lane & (T - 1), g = lane >> lg;
            const bool act = tt < m;
            const int u = act ? t0 + static_cast<int>(__fns(kept, 0, tt + 1)) : 0;
            float4 th = make_float4(0.f, 0.f, 0.f, 0.f), tl = th, tv = th;
            float tR = 0.f;
            if (act) {
                th = A.hi4[ft + u];
                tl = A.lo4[ft + u];
                tv = A.cv[ft + u];
                tR = static_cast<float>(A.R[ft + u]);
            }
            for (int j0 = 0; j0 < nsrc; j0 += COL_STAGE) {
                const int lim = min(COL_STAGE, nsrc - j0);
                __syncwarp();
                int cnt = 0;
#pragma unroll
                for (int r = 0; r < COL_STAGE / 32; r++) {
                    const int k = r * 32 + lane;
                    bool in = k < lim;
                    float4 h = make_float4(0.f, 0.f, 0.f, 0.f), l = h, v = h;
                    if (in) {
                        h = A.hi4[fs + j0 + k];
                        l = A.lo4[fs + j0 + k];
                        v = A.cv[fs + j0 + k];
                        if (!self) in = near_sphere(h, l, v.w, tch, tcl);
                    }
                    const unsigned bal = __ballot_sync(0xffffffffu, in);
                    if (in) {
                        const int slot = cnt + __popc(bal & below);
                        s_h[wl][slot] = h;
                        s_l[wl][slot] = l;
                        s_v[wl][slot] = v;
                        s_R[wl][slot] = static_cast<float>(A.R[fs + j0 + k]);
                        s_j[wl][slot] = j0 + k;
                    }
                    cnt += __popc(bal);
                }
                __syncwarp();
                if (act) {
                    for (int k = g; k < cnt; k += G) {
                        const int v = s_j[wl][k];
                        float dx, dy, dz;
                        if ((!self || v > u) && may_touch(s_h[wl][k], s_l[wl][k], s_v[wl][k].w, th, tl, tv.w, dx, dy, dz) &&
                            may_meet(dx, dy, dz, s_v[wl][k], tv, (s_R[wl][k] + tR) * (1.0f + 0x1p-20f), dtf))
                            test_and_emit(A, ft + u, fs + v);
                    }
                }
            }
        }
    }
    if (lane == 0 && tests)
        atomicAdd(reinterpret_cast<unsigned long long *>(&A.ctl->n_tests), static_cast<unsigned long long>(tests));
}

void launch_collide(ncorp_ctx *c, const ParticleSet &P, const double *vx, const double *vy, const double *vz,
                    double dt, bool wide) {
    CollideArgs A;
    A.p2p = c->wl.cp2p; A.self = c->wl.cself;   // the collision walk's lists
    A.first = c->cells.first; A.count = c->cells.count;
    A.x = P.x; A.y = P.y; A.z = P.z; A.vx = vx; A.vy = vy; A.vz = vz; A.R = P.R;
    A.hi4 = P.hi4; A.lo4 = P.lo4; A.cv = c->cv4;
    A.bh = c->cells.bh; A.bl = c->cells.bl;
    A.perm = P.perm;
    A.dt = dt;
    A.pairs = c->pairs;
    A.where = c->cfg.resolve_f > 0.0 ? c->pair_where : nullptr;
    A.cap = c->pair_cap;
    A.self_cap = c->wl.self_cap;
    A.p2p_cap = c->wl.p2p_cap;
    A.ctl = c->ctl;
    // two blocks per SM beside the main chain (its cooperative kernels must find room on every SM
    // while the search runs); four (the register file's limit) when nothing else runs
    k_collide<<<(wide ? 4 : 2) * c->num_sms, 32 * COL_WARPS, 0, c->stream>>>(A); c->launches++;
    NCORP_CUDA_CHECK(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Collision search by the standard tree code (Algorithm StandardTree, Sect.
// 3.4.4, the instructions for collisions).  Every moonlet a is walked from the
// root with its own r_crit,a = R_a + dt |v_a| (a point: r_max = 0): a cell B
// with fewer than N_cb,pre moonlets is searched directly; B is skipped when
// ((r_crit,a + r_crit,B)(1 + 2^-40))^2 < |x_a - sbar_B|^2 (the dual walk's
// pruning rule); a cell with fewer than N_cb,post moonlets, or a leaf, is
// searched directly; any other is opened, children in order.  Searching B
// directly tests a against the moonlets of B with a larger caller index, so
// every pair is tested once, from the walk of its lower index.
//
// Work layout as for the standard gravity code: a warp walks 32 consecutive
// moonlets of the key order together with a (cell, lanes) stack; each lane
// takes its own moonlet's decisions.  The pruning test is decided in FP32
// only where it is clear by a 2^-16 relative margin (the double-float
// separation and the FP32 radii are accurate to ~1e-7), in FP64 in the
// oracle's order of operations otherwise, so the walk is the oracle's.  The
// moonlet pairs go through the same two FP32 prefilters and the exact FP64
// test as the dual walk's pairs.
// ---------------------------------------------------------------------------
constexpr int SC_WARPS = 4;
constexpr int SC_STACK = 8 * (MAX_LEVEL + 3);

struct StdCollideArgs {
    CollideArgs C;
    const int *child0, *nchild;
    const double *bx, *by, *bz, *bcrit;
    const float4 *bh, *bl;    // collision centre hi (xyz), r_crit in FP32 (w); centre lo
    int pre, post, n;
};

__global__ void __launch_bounds__(32 * SC_WARPS) k_standard_collide(StdCollideArgs S) {
    constexpr unsigned FULL = 0xffffffffu;
    __shared__ int s_cell[SC_WARPS][SC_STACK];
    __shared__ unsigned s_mask[SC_WARPS][SC_STACK];
    const CollideArgs &A = S.C;
    if (aborted(A.ctl)) return;
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const float dtf = static_cast<float>(A.dt) * (1.0f + 0x1p-20f);
    long long n_dir = 0, n_tests = 0;
    bool overflow = false;
    for (int base = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < S.n; base += nwarps * 32) {
        const int i = base + lane;
        const bool valid = i < S.n;
        const int a = valid ? i : base;
        const double X = A.x[a], Y = A.y[a], Z = A.z[a];
        const double rca = dadd(A.R[a], dmul(A.dt, dnorm3(A.vx[a], A.vy[a], A.vz[a])));
        const float4 th = A.hi4[a], tl = A.lo4[a], tv = A.cv[a];
        const float tR = static_cast<float>(A.R[a]), rcf = static_cast<float>(rca);
        const int pa = A.perm[a];
        const unsigned lanes = __ballot_sync(FULL, valid);
        __syncwarp();
        if (lane == 0) {
            s_cell[wl][0] = 0;
            s_mask[wl][0] = lanes;
        }
        __syncwarp();
        int sp = 1;
        while (sp > 0) {
            sp--;
            const int c = s_cell[wl][sp];
            const unsigned mask = s_mask[wl][sp];
            __syncwarp();
            const bool mine = (mask >> lane) & 1u;
            const int nb = A.count[c], f = A.first[c];
            const bool leaf = S.nchild[c] == 0;
            int d = -1;   // 0: search directly, 1: pruned, 2: open
            if (mine) {
                if (nb < S.pre) {
                    d = 0;
                } else {
                    const float4 ch = S.bh[c], cl = S.bl[c];
                    const float dx = (th.x - ch.x) + (tl.x - cl.x);
                    const float dy = (th.y - ch.y) + (tl.y - cl.y);
                    const float dz = (th.z - ch.z) + (tl.z - cl.z);
                    const float d2f = dx * dx + dy * dy + dz * dz, tf = rcf + ch.w, t2f = tf * tf;
                    const float fl = (fabsf(th.x) + fabsf(th.y) + fabsf(th.z)) * 0x1p-26f;
                    bool pruned;
                    if (d2f > fl * fl && d2f > t2f * (1.0f + 0x1p-16f)) {
                        pruned = true;
                    } else if (d2f > fl * fl && d2f < t2f * (1.0f - 0x1p-16f)) {
                        pruned = false;
                    } else {
                        const double ex = dsub(X, S.bx[c]), ey = dsub(Y, S.by[c]), ez = dsub(Z, S.bz[c]);
                        const double t = dmul(dadd(rca, S.bcrit[c]), 1.0 + 0x1p-40);
                        pruned = dmul(t, t) < dsq3(ex, ey, ez);
                    }
                    d = pruned ? 1 : ((nb < S.post || leaf) ? 0 : 2);
                }
            }
            const unsigned m_dir = __ballot_sync(FULL, d == 0);
            const unsigned m_open = __ballot_sync(FULL, d == 2);
            if (m_dir) {   // the cell's moonlets, read once for the warp
                if (d == 0) n_dir++;
                for (int k = f; k < f + nb; k++) {
                    const float4 h = A.hi4[k], l = A.lo4[k], v = A.cv[k];
                    const int pk = A.perm[k];
                    const float Rk = static_cast<float>(A.R[k]);
                    if (d == 0 && pk > pa) {
                        n_tests++;
                        float dx, dy, dz;
                        if (may_touch(h, l, v.w, th, tl, tv.w, dx, dy, dz) &&
                            may_meet(dx, dy, dz, v, tv, (Rk + tR) * (1.0f + 0x1p-20f), dtf))
                            test_and_emit(A, a, k);
                    }
                }
            }
            if (m_open) {
                const int c0 = S.child0[c], nch = S.nchild[c];
                if (sp + nch > SC_STACK) {   // cannot happen within MAX_LEVEL levels; never write past the stack
                    overflow = true;
                    break;
                }
                if (lane < nch) {   // children pushed last first, so the first is taken next
                    s_cell[wl][sp + nch - 1 - lane] = c0 + lane;
                    s_mask[wl][sp + nch - 1 - lane] = m_open;
                }
                sp += nch;
                __syncwarp();
            }
        }
    }
    if (__any_sync(FULL, overflow) && lane == 0) atomicOr(&A.ctl->err, ERR_LEVEL);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        n_dir += __shfl_xor_sync(FULL, n_dir, o);
        n_tests += __shfl_xor_sync(FULL, n_tests, o);
    }
    if (lane == 0) {
        atomicAdd(reinterpret_cast<unsigned long long *>(&A.ctl->col_pairs), static_cast<unsigned long long>(n_dir));
        atomicAdd(reinterpret_cast<unsigned long long *>(&A.ctl->n_tests), static_cast<unsigned long long>(n_tests));
    }
}

void launch_standard_collide(ncorp_ctx *c, const ParticleSet &P, double dt, int n, int pre, int post) {
    StdCollideArgs S;
    CollideArgs &A = S.C;
    A.p2p = nullptr; A.self = nullptr;
    A.first = c->cells.first; A.count = c->cells.count;
    A.x = P.x; A.y = P.y; A.z = P.z; A.vx = P.vx; A.vy = P.vy; A.vz = P.vz; A.R = P.R;
    A.hi4 = P.hi4; A.lo4 = P.lo4; A.cv = c->cv4;
    A.bh = c->cells.bh; A.bl = c->cells.bl;
    A.perm = P.perm;
    A.dt = dt;
    A.pairs = c->pairs;
    A.where = nullptr;
    A.cap = c->pair_cap;
    A.self_cap = 0;
    A.p2p_cap = 0;
    A.ctl = c->ctl;
    S.child0 = c->cells.child0; S.nchild = c->cells.nchild;
    S.bx = c->cells.bx; S.by = c->cells.by; S.bz = c->cells.bz; S.bcrit = c->cells.bcrit;
    S.bh = c->cells.bh; S.bl = c->cells.bl;
    S.pre = pre; S.post = post; S.n = n;
    const int warps = (n + 31) / 32;
    const int grid = std::max(1, std::min((warps + SC_WARPS - 1) / SC_WARPS, 16 * c->num_sms));
    k_standard_collide<<<grid, 32 * SC_WARPS, 0, c->stream>>>(S); c->launches++;
    NCORP_CUDA_CHECK(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Collision resolution (Sect. 5.1 elastic, 5.2 inelastic).  For a pair (1, 2)
// in increasing caller index, both moonlets travel in straight lines to the
// impact at t_c, where with dr = r1 - r2 and dv = v1 - v2 taken there
//   J = alpha (dr.dv) dr,  alpha = f m1 m2 / ((m1 + m2)(R1 + R2)^2),
//   v1' = v1 - J / m1,     v2' = v2 + J / m2,
// and the rest of the step is travelled at v': the drift starts from
// x + t_c (v - v'), i.e. x_new = (x + t_c (v - v')) + dt v'.  Every operation
// is an exactly rounded FP64 one in a fixed order, so resolved states are
// reproducible bit for bit.
//
// A moonlet takes at most one impact per step: pairs are taken in increasing
// (t_c, i, j) and a pair is resolved only if neither moonlet was resolved by
// an earlier pair.  That sequential greedy matching is computed in rounds: in
// each, every undecided pair whose key is the least of the undecided pairs at
// both its moonlets is resolved (all earlier pairs there were skipped), then
// every undecided pair at a moonlet just taken is skipped.  The least
// undecided pair always wins, so the rounds end, usually after one or two.
// One block does it all: the pairs of a disk's step are few (ones to tens),
// and a block needs no grid-wide barrier between the rounds.
// ---------------------------------------------------------------------------
constexpr int RES_THREADS = 512;
enum { RES_UNDECIDED = 0, RES_RESOLVED = 1, RES_SKIPPED = 2 };

struct ResolveArgs {
    const uint64_t *pairs;     // packed caller indices (i << 32 | j), i < j
    const int2 *where;         // their positions in the search tree's order
    const double *x, *y, *z;   // positions at the start of the drift
    const double *m, *R;
    double *vx, *vy, *vz;      // half-kicked velocities in, resolved ones out
    double *ox, *oy, *oz;      // drifted positions, rewritten for resolved moonlets
    double f, dt;
    int cap;
    double *tc;
    int *state;
    unsigned long long *node_tc, *node_ij;
    int *owner;
    Ctrl *ctl;                 // the search's control block: n_found in, n_resolved out
};

__device__ __forceinline__ unsigned long long tc_key(double tc) {
    return static_cast<unsigned long long>(__double_as_longlong(tc == 0.0 ? 0.0 : tc));   // -0 sorts as +0
}

__global__ void __launch_bounds__(RES_THREADS) k_resolve(ResolveArgs A) {
    __shared__ int s_count;
    const int found = A.ctl->n_found;
    // an overflowed search (pairs missing) is rerun by the host with more room: resolve nothing now
    if (found == 0 || found > A.cap || aborted(A.ctl)) {
        if (threadIdx.x == 0) A.ctl->n_resolved = 0;
        return;
    }
    if (threadIdx.x == 0) s_count = 0;
    for (int k = threadIdx.x; k < found; k += blockDim.x) {
        const int2 w = A.where[k];
        const int a = w.x, b = w.y;
        double tc = 0.0;
        const bool ok = impact_time(A.x[a], A.y[a], A.z[a], A.vx[a], A.vy[a], A.vz[a], A.R[a], A.x[b], A.y[b],
                                    A.z[b], A.vx[b], A.vy[b], A.vz[b], A.R[b], tc);
        A.tc[k] = tc;
        A.state[k] = ok ? RES_UNDECIDED : RES_SKIPPED;
        A.owner[a] = 0;
        A.owner[b] = 0;
    }
    __syncthreads();
    for (int round = 0; round <= found; round++) {
        for (int k = threadIdx.x; k < found; k += blockDim.x) {
            if (A.state[k] != RES_UNDECIDED) continue;
            const int2 w = A.where[k];
            A.node_tc[w.x] = A.node_tc[w.y] = ~0ull;
            A.node_ij[w.x] = A.node_ij[w.y] = ~0ull;
        }
        __syncthreads();
        for (int k = threadIdx.x; k < found; k += blockDim.x) {
            if (A.state[k] != RES_UNDECIDED) continue;
            const int2 w = A.where[k];
            const unsigned long long t = tc_key(A.tc[k]);
            atomicMin(&A.node_tc[w.x], t);
            atomicMin(&A.node_tc[w.y], t);
        }
        __syncthreads();
        for (int k = threadIdx.x; k < found; k += blockDim.x) {
            if (A.state[k] != RES_UNDECIDED) continue;
            const int2 w = A.where[k];
            const unsigned long long t = tc_key(A.tc[k]), ij = A.pairs[k];
            if (A.node_tc[w.x] == t) atomicMin(&A.node_ij[w.x], ij);
            if (A.node_tc[w.y] == t) atomicMin(&A.node_ij[w.y], ij);
        }
        __syncthreads();
        for (int k = threadIdx.x; k < found; k += blockDim.x) {
            if (A.state[k] != RES_UNDECIDED) continue;
            const int2 w = A.where[k];
            const unsigned long long t = tc_key(A.tc[k]), ij = A.pairs[k];
            if (A.node_tc[w.x] == t && A.node_ij[w.x] == ij && A.node_tc[w.y] == t && A.node_ij[w.y] == ij) {
                // (a duplicated pair would tie with itself: the first copy claims the moonlets)
                if (atomicCAS(&A.owner[w.x], 0, k + 1) == 0) {
                    A.owner[w.y] = k + 1;
                    A.state[k] = RES_RESOLVED;
                } else {
                    A.state[k] = RES_SKIPPED;
                }
            }
        }
        __syncthreads();
        int left = 0;
        for (int k = threadIdx.x; k < found; k += blockDim.x) {
            if (A.state[k] != RES_UNDECIDED) continue;
            const int2 w = A.where[k];
            if (A.owner[w.x] || A.owner[w.y]) A.state[k] = RES_SKIPPED;
            else left = 1;
        }
        if (!__syncthreads_or(left)) break;
    }
    for (int k = threadIdx.x; k < found; k += blockDim.x) {
        if (A.state[k] != RES_RESOLVED) continue;
        const int2 w = A.where[k];
        const int a = w.x, b = w.y;
        const double tc = A.tc[k];
        const double m1 = A.m[a], m2 = A.m[b];
        const double Rs = dadd(A.R[a], A.R[b]);
        const double x1[3] = {A.x[a], A.y[a], A.z[a]}, x2[3] = {A.x[b], A.y[b], A.z[b]};
        const double v1[3] = {A.vx[a], A.vy[a], A.vz[a]}, v2[3] = {A.vx[b], A.vy[b], A.vz[b]};
        double dr[3], dv[3];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            dr[d] = dsub(dadd(x1[d], dmul(tc, v1[d])), dadd(x2[d], dmul(tc, v2[d])));
            dv[d] = dsub(v1[d], v2[d]);
        }
        const double alpha = ddiv(dmul(dmul(A.f, m1), m2), dmul(dadd(m1, m2), dmul(Rs, Rs)));
        const double cj = dmul(alpha, dadd(dadd(dmul(dr[0], dv[0]), dmul(dr[1], dv[1])), dmul(dr[2], dv[2])));
        double w1[3], w2[3], o1[3], o2[3];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const double J = dmul(cj, dr[d]);
            w1[d] = dsub(v1[d], ddiv(J, m1));
            w2[d] = dadd(v2[d], ddiv(J, m2));
            o1[d] = dadd(dadd(x1[d], dmul(tc, dsub(v1[d], w1[d]))), dmul(A.dt, w1[d]));
            o2[d] = dadd(dadd(x2[d], dmul(tc, dsub(v2[d], w2[d]))), dmul(A.dt, w2[d]));
        }
        A.vx[a] = w1[0]; A.vy[a] = w1[1]; A.vz[a] = w1[2];
        A.vx[b] = w2[0]; A.vy[b] = w2[1]; A.vz[b] = w2[2];
        A.ox[a] = o1[0]; A.oy[a] = o1[1]; A.oz[a] = o1[2];
        A.ox[b] = o2[0]; A.oy[b] = o2[1]; A.oz[b] = o2[2];
        atomicAdd(&s_count, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) A.ctl->n_resolved = s_count;
}

// S: the searched state (positions at the start of the drift, masses, radii,
// in the search tree's order); D: the half-kicked velocities and drifted
// positions in the same order, rewritten for the resolved moonlets.  The
// count goes to the search's control block (n_resolved), where the caller's
// gated launches read it.
void launch_resolve(ncorp_ctx *c, const ParticleSet &S, ParticleSet &D, int n, double dt) {
    (void)n;
    ResolveArgs A;
    A.pairs = c->pairs; A.where = c->pair_where;
    A.x = S.x; A.y = S.y; A.z = S.z; A.m = S.m; A.R = S.R;
    A.vx = D.vx; A.vy = D.vy; A.vz = D.vz;
    A.ox = D.x; A.oy = D.y; A.oz = D.z;
    A.f = c->cfg.resolve_f;
    A.dt = dt;
    A.cap = c->pair_cap;
    A.tc = c->res_tc; A.state = c->res_state;
    A.node_tc = c->node_tc; A.node_ij = c->node_ij; A.owner = c->node_owner;
    A.ctl = c->ctl;
    k_resolve<<<1, RES_THREADS, 0, c->stream>>>(A); c->launches++;
    NCORP_CUDA_CHECK(cudaGetLastError());
}

__global__ void k_unpack_pairs(const uint64_t *__restrict__ packed, int64_t *__restrict__ out, int count) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const uint64_t v = packed[i];
        out[2 * i] = static_cast<int64_t>(v >> 32);
        out[2 * i + 1] = static_cast<int64_t>(v & 0xffffffffull);
    }
}

void launch_sort_pairs(ncorp_ctx *c, int count) {
    if (count <= 0) return;
    launch_iota(c, c->pair_idx, count);
    radix_sort_u64(c, c->pairs, c->pair_idx, c->pairs_alt, c->pair_idx_alt, count, 64);
}

void launch_unpack_pairs(ncorp_ctx *c, const uint64_t *packed, int64_t *out, int count) {
    if (count <= 0) return;
    k_unpack_pairs<<<grid_for(count, 256, 4 * c->num_sms), 256, 0, c->stream>>>(packed, out, count); c->launches++;
    NCORP_CUDA_CHECK(cudaGetLastError());
}

}  // namespace ncorp
