// ncorp.cu -- C ABI entry points (include/ncorp.h) and the order in which one
// falcON step runs its kernels.
//
// Step (SBAB1 with merged kicks, Sect. 4.1), on the state A kept in tree order:
//   B.v = A.v + dt/2 A.a                         half kick
//   collision climb + walk + pair test on (A.x, B.v) with A's tree (Sect. 3.1)
//   B.x = A.x + dt B.v                           drift
//   keys -> radix sort -> gather into C -> build  (Sect. 3.4.1, 3.4.6)
//   climb (geometry, P2M/M2M) -> walk -> lists -> M2L -> L2L/L2P + P2P + external
//   C.v += dt/2 C.a                              half kick
//   A <-> C
// A is never written during a step, so a step whose lists overflowed is rerun
// from it with larger buffers.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "ctx.h"

using namespace ncorp;

static std::atomic<unsigned long long> g_alloc_gen{0};
unsigned long long ncorp::alloc_generation() { return g_alloc_gen.load(); }
void ncorp::bump_alloc_generation() { g_alloc_gen++; }

namespace {

int fail(ncorp_ctx *c, int code, const char *fmt, ...) {
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

template <typename T>
void dalloc(T *&p, size_t count) {
    g_alloc_gen++;
    if (p) cudaFree(p);
    p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&p), sizeof(T) * count);
    if (e != cudaSuccess) {
        p = nullptr;
        cudaGetLastError();   // (the failure is reported here; a later check must not see it again)
        throw CudaError(e, "cudaMalloc", __FILE__, __LINE__);
    }
}

template <typename T>
void dfree(T *&p) {
    if (p) cudaFree(p);
    p = nullptr;
}

void alloc_set(ParticleSet &S, size_t n) {
    dalloc(S.x, n); dalloc(S.y, n); dalloc(S.z, n);
    dalloc(S.vx, n); dalloc(S.vy, n); dalloc(S.vz, n);
    dalloc(S.m, n); dalloc(S.R, n);
    dalloc(S.ax, n); dalloc(S.ay, n); dalloc(S.az, n);
    dalloc(S.perm, n);
    dalloc(S.qx, n); dalloc(S.qy, n); dalloc(S.qz, n);
    dalloc(S.key, n);
    dalloc(S.hi4, n);
    dalloc(S.lo4, n);
}

void free_set(ParticleSet &S) {
    dfree(S.x); dfree(S.y); dfree(S.z); dfree(S.vx); dfree(S.vy); dfree(S.vz); dfree(S.m); dfree(S.R);
    dfree(S.ax); dfree(S.ay); dfree(S.az); dfree(S.perm); dfree(S.qx); dfree(S.qy); dfree(S.qz); dfree(S.key);
    dfree(S.hi4); dfree(S.lo4);
}

// Every allocator below records a capacity only after all its buffers exist:
// an allocation that fails leaves the capacity at 0, so the next call
// allocates again instead of using a buffer that is missing or too small.
void ensure_particles(ncorp_ctx *c, int64_t n) {
    if (n <= c->n_cap) return;
    int64_t cap = std::max<int64_t>(n, c->n_cap * 3 / 2);
    c->n_cap = 0;
    c->have_state = false;
    c->tree_valid = false;
    alloc_set(c->A, cap);
    alloc_set(c->B, cap);
    alloc_set(c->Cset, cap);
    dalloc(c->amx, cap); dalloc(c->amy, cap); dalloc(c->amz, cap);
    dalloc(c->cv4, cap);
    dalloc(c->key_alt, cap);
    dalloc(c->idx, cap); dalloc(c->idx_alt, cap);
    if (!c->resort_mkey) {
        dalloc(c->resort_mkey, 2 * RESORT_MOVERS_CAP);   // input order, then sorted
        dalloc(c->resort_midx, 2 * RESORT_MOVERS_CAP);
        dalloc(c->resort_bcount, RESORT_BLOCKS_CAP);
    }
    dalloc(c->stage, 3 * cap);
    dalloc(c->stage2, 3 * cap);
    if (c->cfg.resolve_f > 0.0) {
        dalloc(c->node_tc, cap);
        dalloc(c->node_ij, cap);
        dalloc(c->node_owner, cap);
    }
    c->n_cap = cap;
    c->have_state = false;
    c->tree_valid = false;
}

void alloc_cells(ncorp_ctx *c, int cap) {
    Cells &C = c->cells;
    C.cap = 0;
    c->tree_valid = false;
    dalloc(C.level, cap); dalloc(C.first, cap); dalloc(C.count, cap); dalloc(C.child0, cap);
    dalloc(C.nchild, cap); dalloc(C.parent, cap); dalloc(C.arrive, cap); dalloc(C.arrive_m, cap);
    dalloc(C.cx, cap); dalloc(C.cy, cap); dalloc(C.cz, cap);
    dalloc(C.M, cap); dalloc(C.sx, cap); dalloc(C.sy, cap); dalloc(C.sz, cap);
    dalloc(C.rmax, cap); dalloc(C.rcrit, cap); dalloc(C.rho, cap);
    dalloc(C.bx, cap); dalloc(C.by, cap); dalloc(C.bz, cap); dalloc(C.bmax, cap); dalloc(C.bcrit, cap);
    dalloc(C.gh, cap); dalloc(C.gl, cap); dalloc(C.bh, cap); dalloc(C.bl, cap);
    // each new buffer is stored as soon as it exists, so that an allocation failing part-way leaves
    // nothing unowned (ncorp_free releases whatever the context holds)
    for (void **slot : {&C.Mh, &C.Ch, &C.Cf}) {
        if (*slot) cudaFree(*slot);
        *slot = nullptr;
    }
    double *mh = nullptr, *ch = nullptr, *cf = nullptr;
    dalloc(mh, static_cast<size_t>(cap) * num_m(MAXP));
    C.Mh = mh;
    dalloc(ch, static_cast<size_t>(cap) * num_c(MAXP));
    C.Ch = ch;
    dalloc(cf, static_cast<size_t>(cap) * num_c(MAXP));
    C.Cf = cf;
    dalloc(C.leaves, cap);
    dalloc(C.bounds, static_cast<size_t>(cap) * 9);
    dalloc(C.blocksum, 8192);
    dalloc(C.maker, cap);
    dalloc(C.before, cap);
    dalloc(C.Cf_lo, 3 * static_cast<size_t>(cap));
    dalloc(C.Ch_lo, 3 * static_cast<size_t>(cap));
    dalloc(C.done, cap);   // descent epochs start at 1: zeroed words never match
    // (on the context's stream, ahead of every kernel that reads them: a plain memset would run on the
    // legacy stream, which is not ordered with the non-blocking streams the library is driven on)
    NCORP_CUDA_CHECK(cudaMemsetAsync(C.done, 0, sizeof(unsigned) * cap, c->stream));
    WalkLists &W = c->wl;
    dalloc(W.cnt, cap + 1); dalloc(W.offs, cap + 1); dalloc(W.cursor, cap + 1); dalloc(W.p2p_off, cap + 1);
    C.cap = cap;
    c->tree_valid = false;
}

void alloc_lists(ncorp_ctx *c, int front, int m2l, int p2p, int self) {
    WalkLists &W = c->wl;
    if (front != W.front_cap) {
        W.front_cap = 0;
        dalloc(W.front[0], front);
        dalloc(W.front[1], front);
        W.front_cap = front;
    }
    if (!W.front_count) dalloc(W.front_count, WALK_MAX_ITERS + 2);
    if (m2l != W.m2l_cap) {
        W.m2l_cap = 0;
        W.m2l_dir_cap = 0;
        dalloc(W.m2l, m2l);
        dalloc(W.m2l_dir, 2 * static_cast<size_t>(m2l));
        W.m2l_cap = m2l;
        W.m2l_dir_cap = 2 * m2l;
    }
    if (p2p != W.p2p_cap || self != W.self_cap) {
        W.p2p_cap = 0;
        W.self_cap = 0;
        W.p2p_dir_cap = 0;
        dalloc(W.p2p, p2p);
        dalloc(W.self, self);
        dalloc(W.p2p_src, 2 * static_cast<size_t>(p2p) + self);   // int2
        dalloc(W.cp2p, p2p);
        dalloc(W.cself, self);
        W.p2p_cap = p2p;
        W.self_cap = self;
        W.p2p_dir_cap = 2 * p2p + self;
    }
}

void alloc_pairs(ncorp_ctx *c, int cap) {
    c->pair_cap = 0;
    dalloc(c->pairs, cap);
    dalloc(c->pairs_alt, cap);
    dalloc(c->pair_idx, cap);
    dalloc(c->pair_idx_alt, cap);
    dalloc(c->pairs_out, 2 * static_cast<size_t>(cap));
    if (c->cfg.resolve_f > 0.0) {
        dalloc(c->pair_where, cap);
        dalloc(c->res_tc, cap);
        dalloc(c->res_state, cap);
    }
    c->pair_cap = cap;
}

// leaf size and thresholds for expansion order p (config values win when set)
void choose_parameters(ncorp_ctx *c, int p) {
    const ncorp_config &g = c->cfg;
    c->s = g.leaf_size > 0 ? g.leaf_size : (c->s_tuned > 0 ? c->s_tuned : (p <= 3 ? 32 : 64));
    if (g.n_cs || g.n_cc_pre || g.n_cc_post) {
        c->g_cs = g.n_cs; c->g_pre = g.n_cc_pre; c->g_post = g.n_cc_post;
    } else if (p >= 6) {
        c->g_cs = 256; c->g_pre = 256; c->g_post = 512;   // Sect. 4.2, p = 6
    } else {
        c->g_cs = 64; c->g_pre = 8; c->g_post = 64;        // Sect. 4.2, p = 3
    }
    if (g.c_cs || g.c_cc_pre || g.c_cc_post) {
        c->c_cs = g.c_cs; c->c_pre = g.c_cc_pre; c->c_post = g.c_cc_post;
    } else {
        c->c_cs = 12; c->c_pre = 0; c->c_post = 16;        // Sect. 4.2, collisions
    }
}

void ensure_tree_capacity(ncorp_ctx *c, int n) {
    int want = std::max({4096, 4 * (n / std::max(1, c->s)) + 1024, c->floor_cells});
    if (c->cells.cap < want) alloc_cells(c, want);
    if (c->cells.leaf_of_cap < n) {
        c->cells.leaf_of_cap = 0;
        dalloc(c->cells.leaf_of, static_cast<size_t>(n));
        dalloc(c->cells.rc_spec, static_cast<size_t>(n));
        c->cells.leaf_of_cap = n;
    }
    const int cc = c->cells.cap;
    int front = std::max({1 << 16, 48 * cc, c->floor_front}), m2l = std::max({1 << 16, 64 * cc, c->floor_m2l}),
        p2p = std::max({1 << 16, 48 * cc, c->floor_p2p});
    if (c->test_list_cap > 0) {   // failure-path tests: lists too small until they first overflow
        m2l = std::min(m2l, c->test_list_cap);
        p2p = std::min(p2p, c->test_list_cap);
    }
    const int self = std::max(cc, c->floor_self);
    if (c->wl.front_cap < front || c->wl.m2l_cap < m2l || c->wl.p2p_cap < p2p || c->wl.self_cap < self)
        alloc_lists(c, std::max(front, c->wl.front_cap), std::max(m2l, c->wl.m2l_cap), std::max(p2p, c->wl.p2p_cap),
                    std::max(self, c->wl.self_cap));
    int pc = std::max(1 << 16, 4 * n);
    if (c->test_pair_cap > 0) pc = std::min(pc, c->test_pair_cap);
    if (c->pair_cap < pc) alloc_pairs(c, pc);
    ensure_radix_scratch(c, std::max(n, pc));
}

// The current tree set (cells, wl, ctl, ctl_h) and the other one trade places.
void swap_sets(ncorp_ctx *c) {
    std::swap(c->cells, c->alt.cells);
    std::swap(c->wl, c->alt.wl);
    std::swap(c->ctl, c->alt.ctl);
    std::swap(c->ctl_h, c->alt.ctl_h);
}

// Runs f with the other tree set as the current one (the resident flags
// describe the current tree and are left as they were).
template <class F>
void on_alt(ncorp_ctx *c, F f) {
    const bool tv = c->tree_valid;
    swap_sets(c);
    try {
        f();
    } catch (...) {
        swap_sets(c);
        c->tree_valid = tv;
        throw;
    }
    swap_sets(c);
    c->tree_valid = tv;
}

void ensure_both_capacities(ncorp_ctx *c, int n) {
    ensure_tree_capacity(c, n);
    on_alt(c, [&] { ensure_tree_capacity(c, n); });
}

// grows whatever overflowed; returns false if nothing can be grown
bool grow_after(ncorp_ctx *c, int err) {
    bool grew = false;
    if (err & ERR_CELLS) {
        alloc_cells(c, std::max(2 * c->cells.cap, c->ctl_h->n_cells + 1024));
        c->floor_cells = std::max(c->floor_cells, c->cells.cap);
        grew = true;
    }
    WalkLists &W = c->wl;
    int front = W.front_cap, m2l = W.m2l_cap, p2p = W.p2p_cap, self = W.self_cap;
    if (err & ERR_FRONTIER) { front *= 2; grew = true; }
    if (err & (ERR_M2L | ERR_DIRECTED)) { m2l = std::max(2 * m2l, c->ctl_h->n_m2l + 1024); grew = true; }
    if (err & (ERR_P2P | ERR_DIRECTED)) {
        p2p = std::max(2 * p2p, c->ctl_h->n_p2p + 1024);
        self = std::max(2 * self, c->ctl_h->n_self + 1024);
        grew = true;
    }
    if (grew) {
        alloc_lists(c, front, m2l, p2p, self);
        c->test_list_cap = 0;
        c->floor_front = std::max(c->floor_front, front);
        c->floor_m2l = std::max(c->floor_m2l, m2l);
        c->floor_p2p = std::max(c->floor_p2p, p2p);
        c->floor_self = std::max(c->floor_self, self);
    }
    if (err & ERR_PAIRS) {
        c->test_pair_cap = 0;
        alloc_pairs(c, std::max(2 * c->pair_cap, c->ctl_h->n_found + 1024));
        grew = true;
    }
    return grew;
}

bool is_device_ptr(ncorp_ctx *c, const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeDevice) {
        if (a.device != c->device) throw CudaError(cudaErrorInvalidDevicePointer, "pointer on another device",
                                                   __FILE__, __LINE__);
        return true;
    }
    return a.type == cudaMemoryTypeManaged;
}

void upload_vec(ncorp_ctx *c, const double *user, double *x, double *y, double *z, int n) {
    if (is_device_ptr(c, user)) {
        launch_aos_to_soa(c, user, x, y, z, n);
    } else {
        NCORP_CUDA_CHECK(cudaMemcpyAsync(c->stage, user, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, c->stream));
        launch_aos_to_soa(c, c->stage, x, y, z, n);
    }
}

void upload_scalar(ncorp_ctx *c, const double *user, double *dst, int n) {
    NCORP_CUDA_CHECK(cudaMemcpyAsync(dst, user, sizeof(double) * n, cudaMemcpyDefault, c->stream));
}

// abort_a / abort_b (nullable): error words that stop the write when they hold an abort flag
void download_vec(ncorp_ctx *c, const double *x, const double *y, const double *z, const int *perm, double *user,
                  int n, double *stage, const int *abort_a = nullptr, const int *abort_b = nullptr) {
    if (is_device_ptr(c, user)) {
        launch_scatter_aos(c, x, y, z, perm, user, n, abort_a, abort_b);
    } else {
        launch_scatter_aos(c, x, y, z, perm, stage, n, abort_a, abort_b);
        NCORP_CUDA_CHECK(cudaMemcpyAsync(user, stage, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c->stream));
    }
}

ExtForce external(ncorp_ctx *c, double t) {
    ExtForce e{};
    const ncorp_config &g = c->cfg;
    e.GMc = g.G * g.central_mass;
    e.bulge = g.G * g.central_mass * g.central_radius * g.central_radius * g.central_J2;
    if (g.star_mass != 0.0) {
        const double a = g.star_a;
        const double nsun = std::sqrt(g.G * g.star_mass / (a * a * a));
        const double lam = nsun * t;
        e.sx = a * std::cos(lam);
        e.sy = a * std::sin(lam) * std::cos(g.star_obliquity);
        e.sz = a * std::sin(lam) * std::sin(g.star_obliquity);
        const double rs2 = e.sx * e.sx + e.sy * e.sy + e.sz * e.sz;
        e.star_k = (g.G * g.star_mass) / (rs2 * std::sqrt(rs2));
        e.inv_rs2 = 1.0 / rs2;
    }
    return e;
}

// Clears the error word and the per-call counters and sets the bounding box
// to empty; the tree description (cell and leaf counts, levels, root cube)
// of a resident tree is kept.  With fold, the cleared error word is first
// or-ed into the context's accumulator (a tree set recycled in the middle of
// a call keeps its errors visible).  ctl2 (optional) is cleared the same way
// and clear (optional) is zeroed: one launch resets both tree sets and the
// accumulator at the start of a step.
__device__ void reset_one(Ctrl *ctl, int *fold) {
    if (fold) {
        *fold |= ctl->err;
        // a run of steps that aborted stays aborted: the set is not reused, so that no later step of the
        // run computes from the results the aborted step never wrote (the run is redone by the host)
        if (*fold & ERR_ABORT_MASK) {
            ctl->err = *fold & ERR_ABORT_MASK;
            return;
        }
    }
    ctl->err = 0;
    ctl->n_found = 0;
    ctl->n_resolved = 0;
    ctl->n_tests = 0;
    ctl->dec_pairs = 0;
    ctl->col_pairs = 0;
    ctl->col_self = 0;
    ctl->n_inter = 0;
    ctl->n_m2p = 0;
    ctl->bar_count = 0;
    ctl->resort_ok = 0;
    if (!fold) ctl->stall = 0;   // a set recycled within a call (fold) keeps the call's armed stall
    for (int d = 0; d < ctl->nd; d++)   // every disk's box (one disk: dbox is bbox)
        for (int k = 0; k < 3; k++) {
            ctl->dbox[6 * d + k] = ~0ull;
            ctl->dbox[6 * d + 3 + k] = 0ull;
        }
}

__global__ void k_arm_stall(Ctrl *ctl, Ctrl *ctl2) {
    ctl->stall = 1;
    ctl2->stall = 1;
}

// inherit (nullable, with fold): the control block of the tree whose results the cleared set's work
// starts from (the opening kick reads that tree's accelerations); its abort bits are folded first, so
// that nothing is computed from an evaluation that never ran.
__global__ void k_reset_ctl(Ctrl *ctl, Ctrl *ctl2, int *fold, int *clear, const Ctrl *inherit) {
    if (fold && inherit) *fold |= inherit->err & ERR_ABORT_MASK;
    reset_one(ctl, fold);
    if (ctl2) reset_one(ctl2, nullptr);
    if (clear) *clear = 0;
}

// The disk layout of a tree set (one disk: null arrays, the control block's own box and root cube).
__global__ void k_set_disks(Ctrl *ctl, int nd, const unsigned short *disk_of, const int *doff,
                            unsigned long long *dbox, double *droot) {
    ctl->nd = nd;
    ctl->disk_of = disk_of;
    ctl->doff = doff;
    ctl->dbox = dbox ? dbox : ctl->bbox;
    ctl->droot = droot ? droot : ctl->root;
}

// disk_of[i] = the d with doff[d] <= i < doff[d + 1]
__global__ void k_fill_disk_of(const int *__restrict__ doff, int nd, unsigned short *disk_of, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int lo = 0, hi = nd - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (doff[mid] <= i) lo = mid;
            else hi = mid - 1;
        }
        disk_of[i] = static_cast<unsigned short>(lo);
    }
}

// Lays the context's moonlets out as nd independent disks of sizes[d]
// moonlets each, disk d taking [sum of the earlier sizes, + sizes[d]) in the
// caller's arrays and in every internal order; nd = 1 returns to one disk.
// The resident state and tree are dropped (the next call reads the caller's
// arrays).  Synchronous.
void drop_graph(StepGraph &g);

void configure_disks(ncorp_ctx *c, int nd, const int64_t *sizes) {
    std::vector<int> off(nd + 1, 0);
    for (int d = 0; d < nd && sizes; d++) off[d + 1] = off[d] + static_cast<int>(sizes[d]);
    const int n = off[nd];
    NCORP_CUDA_CHECK(cudaStreamSynchronize(c->stream));
    for (StepGraph &g : c->graphs) drop_graph(g);
    if (nd == 1) {   // (the layout buffers are kept for the next forest layout)
        k_set_disks<<<1, 1, 0, c->stream>>>(c->ctl, 1, nullptr, nullptr, nullptr, nullptr);
        k_set_disks<<<1, 1, 0, c->stream>>>(c->alt.ctl, 1, nullptr, nullptr, nullptr, nullptr);
    } else {
        // grown, never shrunk: a re-layout of a batch's forest allocates nothing in the common case
        if (c->disk_of_cap < n) {
            c->disk_of_cap = 0;
            dalloc(c->disk_of, n);
            c->disk_of_cap = n;
        }
        if (c->nd_cap < nd) {
            c->nd_cap = 0;
            dalloc(c->doff, NCORP_MAX_DISKS + 1);
            for (int s = 0; s < 2; s++) {
                dalloc(c->fbox[s], 6 * static_cast<size_t>(NCORP_MAX_DISKS));
                dalloc(c->froot[s], 4 * static_cast<size_t>(NCORP_MAX_DISKS));
            }
            c->nd_cap = NCORP_MAX_DISKS;
        }
        NCORP_CUDA_CHECK(cudaMemcpyAsync(c->doff, off.data(), sizeof(int) * (nd + 1), cudaMemcpyHostToDevice, c->stream));
        k_fill_disk_of<<<grid_for(n, 256, 4 * c->num_sms), 256, 0, c->stream>>>(c->doff, nd, c->disk_of, n);
        k_set_disks<<<1, 1, 0, c->stream>>>(c->ctl, nd, c->disk_of, c->doff, c->fbox[0], c->froot[0]);
        k_set_disks<<<1, 1, 0, c->stream>>>(c->alt.ctl, nd, c->disk_of, c->doff, c->fbox[1], c->froot[1]);
    }
    NCORP_CUDA_CHECK(cudaGetLastError());
    NCORP_CUDA_CHECK(cudaStreamSynchronize(c->stream));
    c->nd = nd;
    c->forest_n = nd > 1 ? n : 0;
    c->have_state = false;
    c->tree_valid = false;
}

// fold: the set is recycled within a call (called with the other tree set as c->alt, the one the
// recycled set's next work starts from)
void reset_ctl(ncorp_ctx *c, bool fold = false) {
    k_reset_ctl<<<1, 1, 0, c->stream>>>(c->ctl, nullptr, fold ? c->err_acc : nullptr, nullptr,
                                        fold ? c->alt.ctl : nullptr);
    c->launches++;
    NCORP_CUDA_CHECK(cudaGetLastError());
}

// Both tree sets and the error accumulator, before a step.
void reset_ctls(ncorp_ctx *c) {
    k_reset_ctl<<<1, 1, 0, c->stream>>>(c->ctl, c->alt.ctl, nullptr, c->err_acc, nullptr);
    c->launches++;
    NCORP_CUDA_CHECK(cudaGetLastError());
}

// ---- stage timers (CUDA events on the context's stream, only when profiling)
void stage_begin(ncorp_ctx *c, int st) {
    if (!c->profile || c->ev_used[st] >= 8) return;
    cudaEvent_t &e = c->ev[st][c->ev_used[st]][0];
    if (!e) NCORP_CUDA_CHECK(cudaEventCreate(&e));
    NCORP_CUDA_CHECK(cudaEventRecord(e, c->stream));
}

void stage_end(ncorp_ctx *c, int st) {
    if (!c->profile || c->ev_used[st] >= 8) return;
    cudaEvent_t &e = c->ev[st][c->ev_used[st]][1];
    if (!e) NCORP_CUDA_CHECK(cudaEventCreate(&e));
    NCORP_CUDA_CHECK(cudaEventRecord(e, c->stream));
    c->ev_used[st]++;
}

struct Stage {
    ncorp_ctx *c;
    int st;
    Stage(ncorp_ctx *c_, int st_) : c(c_), st(st_) { stage_begin(c, st); }
    ~Stage() { stage_end(c, st); }
};

void begin_call(ncorp_ctx *c) {
    c->launches = 0;
    c->graph_used = false;
    for (int i = 0; i < NCORP_NSTAGES; i++) {
        c->ev_used[i] = 0;
        c->stage_ms[i] = 0.0;
    }
}

// Waits for the call's work and returns its error word: the current tree
// set's, and with both also the other set's and the accumulator's.
int finish(ncorp_ctx *c, bool both = false) {
    NCORP_CUDA_CHECK(cudaMemcpyAsync(c->ctl_h, c->ctl, sizeof(Ctrl), cudaMemcpyDeviceToHost, c->stream));
    if (both) {
        NCORP_CUDA_CHECK(cudaMemcpyAsync(c->alt.ctl_h, c->alt.ctl, sizeof(Ctrl), cudaMemcpyDeviceToHost, c->stream));
        NCORP_CUDA_CHECK(cudaMemcpyAsync(c->err_acc_h, c->err_acc, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    }
    NCORP_CUDA_CHECK(cudaStreamSynchronize(c->stream));
    if (c->profile)
        for (int i = 0; i < NCORP_NSTAGES; i++) {
            double sum = 0;
            for (int k = 0; k < c->ev_used[i]; k++) {
                float ms = 0;
                NCORP_CUDA_CHECK(cudaEventElapsedTime(&ms, c->ev[i][k][0], c->ev[i][k][1]));
                sum += ms;
            }
            c->stage_ms[i] = sum;
        }
    const int err = c->ctl_h->err | (both ? (c->alt.ctl_h->err | *c->err_acc_h) : 0);
    if (err & ERR_TIMEOUT) c->radix_dirty = true;
    return err;
}

// keys of (x from sx, v from sv, m/R/perm from sr) -> radix sort -> gather into dst -> build
// near_sorted: the positions are in the previous tree order of nearby
// positions (a drift), so the keys are nearly sorted.
// gate (nullable, radix sort only): every kernel does nothing while *gate is 0.
// spec_dt > 0 (fused walk): the gather also bounds every moonlet's next R + dt |v| (velocities of sv,
// accelerations of sr)
void build_tree(ncorp_ctx *c, const ParticleSet &sx, const ParticleSet &sv, const ParticleSet &sr, ParticleSet &dst,
                int n, bool near_sorted = false, bool bbox_done = false, const int *gate = nullptr,
                double spec_dt = 0.0) {
    c->cur_n = n;
    {
        Stage st(c, NCORP_STAGE_SORT);
        launch_bbox_keys(c, sx.x, sx.y, sx.z, n, dst.key, c->B.qx, c->B.qy, c->B.qz, bbox_done, gate);
        // (a forest's keys restart in every disk: they are sorted by (disk, key) with the full radix sort)
        if (near_sorted && c->nd == 1) sort_near_sorted(c, dst.key, c->idx, c->key_alt, c->idx_alt, n, 3 * KEY_BITS);
        else radix_sort_u64(c, dst.key, c->idx, c->key_alt, c->idx_alt, n, 3 * KEY_BITS, true, gate, true);
        ParticleSet view = sr;
        view.x = sx.x; view.y = sx.y; view.z = sx.z;
        view.vx = sv.vx; view.vy = sv.vy; view.vz = sv.vz;
        view.qx = c->B.qx; view.qy = c->B.qy; view.qz = c->B.qz;
        launch_gather(c, view, view, dst, n, c->idx, c->cfg.G, gate, spec_dt);
    }
    Stage st(c, NCORP_STAGE_BUILD);
    launch_build(c, dst, n, c->s, gate);
}

// Runs body with c->stream set to s (launchers enqueue on c->stream).
template <class F>
void on_stream(ncorp_ctx *c, cudaStream_t s, F body) {
    cudaStream_t main = c->stream;
    c->stream = s;
    try {
        body();
    } catch (...) {
        c->stream = main;
        throw;
    }
    c->stream = main;
}

// Gravity of the tree in the current set.  Two streams: the main one runs the
// geometry climb (with theta(M)), the walk (with its lists), M2L, the descent
// and the far-field evaluation; the second one runs the multipoles beside the
// walk, then the near field (which needs only the lists) beside M2L and the
// descent.
// kick_h != 0: the evaluation also applies the closing half kick v += kick_h a.
// fused_dt > 0 (fused walk): the walk also collects the collision pairs of the next step, with the
// collision geometry of the bounds the gather wrote (its climb runs on the second stream beside the
// gravity geometry).
void gravity(ncorp_ctx *c, ParticleSet &S, int p, double theta, double t, bool want_mutual, double kick_h = 0.0,
             double fused_dt = 0.0) {
    const bool mixed = c->cfg.precision == NCORP_MIXED;
    const double G = c->cfg.G;
    const bool fused = fused_dt > 0.0;
    c->grav_p = p;
    c->grav_mixed = mixed;
    c->grav_local = true;
    if (fused) {
        NCORP_CUDA_CHECK(cudaEventRecord(c->ev_spec0, c->stream));
        NCORP_CUDA_CHECK(cudaStreamWaitEvent(c->side2, c->ev_spec0, 0));
        const int cap = c->coop_max;
        c->coop_max = cap > 0 ? std::min(cap, c->side_blocks) : c->side_blocks;   // beside the geometry
        try {
            on_stream(c, c->side2, [&] {
                Stage st(c, NCORP_STAGE_COLLIDE);
                launch_climb_collision(c, S, S.vx, S.vy, S.vz, fused_dt, c->cells.rc_spec);
                NCORP_CUDA_CHECK(cudaEventRecord(c->ev_spec, c->stream));
            });
        } catch (...) {
            c->coop_max = cap;
            throw;
        }
        c->coop_max = cap;
    }
    { Stage st(c, NCORP_STAGE_CLIMB); launch_climb_geometry(c, S, G, theta); }
    NCORP_CUDA_CHECK(cudaEventRecord(c->ev_geo, c->stream));
    NCORP_CUDA_CHECK(cudaStreamWaitEvent(c->side2, c->ev_geo, 0));
    on_stream(c, c->side2, [&] {
        Stage st(c, NCORP_STAGE_CLIMB);
        launch_multipoles(c, S, p, mixed, G);
        NCORP_CUDA_CHECK(cudaEventRecord(c->ev_p2m, c->stream));
    });
    if (fused) NCORP_CUDA_CHECK(cudaStreamWaitEvent(c->stream, c->ev_spec, 0));
    { Stage st(c, NCORP_STAGE_WALK); launch_walk(c, true, fused); }
    NCORP_CUDA_CHECK(cudaEventRecord(c->ev_lists, c->stream));
    NCORP_CUDA_CHECK(cudaStreamWaitEvent(c->side2, c->ev_lists, 0));
    on_stream(c, c->side2, [&] {
        Stage st(c, NCORP_STAGE_NEAR);
        launch_near(c, S, p, mixed, G);
        NCORP_CUDA_CHECK(cudaEventRecord(c->ev_near, c->stream));
    });
    NCORP_CUDA_CHECK(cudaStreamWaitEvent(c->stream, c->ev_p2m, 0));
    { Stage st(c, NCORP_STAGE_M2L); launch_m2l(c, p, mixed); }
    { Stage st(c, NCORP_STAGE_DESCEND); launch_descend(c, p, mixed); }
    NCORP_CUDA_CHECK(cudaStreamWaitEvent(c->stream, c->ev_near, 0));
    { Stage st(c, NCORP_STAGE_EVAL); launch_far(c, S, p, mixed, G, external(c, t), want_mutual, kick_h); }
}

// Gravity of the tree in the current set by the standard tree code: the
// geometry climb (with theta(M)), the multipoles, then one walk per moonlet.
void gravity_standard(ncorp_ctx *c, ParticleSet &S, int n, int p, double theta, double t, bool want_mutual) {
    const bool mixed = c->cfg.precision == NCORP_MIXED;
    const double G = c->cfg.G;
    c->grav_p = p;
    c->grav_mixed = mixed;
    c->grav_local = false;
    { Stage st(c, NCORP_STAGE_CLIMB); launch_climb_geometry(c, S, G, theta); }
    { Stage st(c, NCORP_STAGE_CLIMB); launch_multipoles(c, S, p, mixed, G); }
    Stage st(c, NCORP_STAGE_EVAL);
    launch_standard(c, S, n, p, mixed, G, external(c, t), want_mutual, c->cfg.n_cb_pre, c->cfg.n_cb_post);
}

// wide: nothing else runs on the device meanwhile (the pair test takes every SM)
// gate (nullable): the climb and the walk run only while *gate is set (fused walk: the pairs to test
// are already listed unless a bound was exceeded); the pair test always runs
void collisions(ncorp_ctx *c, const ParticleSet &S, const double *vx, const double *vy, const double *vz, double dt,
                bool wide, const int *gate = nullptr) {
    Stage st(c, NCORP_STAGE_COLLIDE);
    launch_climb_collision(c, S, vx, vy, vz, dt, nullptr, gate);
    launch_walk(c, false, true, gate);
    launch_collide(c, S, vx, vy, vz, dt, wide);
}

// The same search by the standard tree code (Algorithm StandardTree): the collision climb, then one walk
// per moonlet.  S's velocities are the ones searched.
void collisions_standard(ncorp_ctx *c, const ParticleSet &S, int n, double dt) {
    Stage st(c, NCORP_STAGE_COLLIDE);
    launch_climb_collision(c, S, S.vx, S.vy, S.vz, dt);
    launch_standard_collide(c, S, dt, n, c->cfg.c_cb_pre, c->cfg.c_cb_post);
}


// One SBAB1 step of the resident state A (its tree, in the current tree set,
// and its acceleration valid): half kick, collision search on A's tree, drift,
// tree of the new positions in the other tree set, gravity, half kick.  With
// overlap, the collision search runs on the context's side stream while the
// main stream drifts, sorts, builds and walks the new tree (the two touch
// disjoint buffers); its cooperative grids are kept small enough that both
// streams' cooperative kernels fit on the device together.  With collision
// resolution the side stream also resolves the pairs it found, which
// rewrites the drift of the resolved moonlets while the main stream may be
// reading it: after the new tree is built the main stream joins the side
// stream, and if anything was resolved (a device counter) it folds the box
// and builds the tree again from the resolved drift (gated launches that
// return at once otherwise).  Without overlap (batches) the search and the
// resolution run before the keys.  On return the
// tree sets have traded places (the current one describes the new positions)
// and the new state is in Cset (not yet swapped with A); nothing is copied to
// the caller and nothing waits: the caller reads the status.
void enqueue_kdk(ncorp_ctx *c, int n, int p, double theta, double dt, bool overlap) {
    const double h = 0.5 * dt;
    ParticleSet &A = c->A, &B = c->B, &Cn = c->Cset;
    const bool resolve = c->cfg.collisions && c->cfg.resolve_f > 0.0;
    const bool side = overlap && c->cfg.collisions;
    // fused walk: A's tree set lists the pairs to test unless its bounds were exceeded (or never made:
    // a tree set whose last walk was not a fused one is marked stale)
    const bool fused = c->cfg.fused_walk && side && !resolve && c->nd == 1;
    // the other tree set becomes the new tree's: cleared (its errors kept) before the kick-drift
    // kernel folds the drifted positions' bounding box into its control block.  It also takes over
    // the abort bits of A's tree: if A's acceleration was never computed (an overflow in the same
    // call), the kick-drift and everything built from it do nothing.
    on_alt(c, [&] { reset_ctl(c, true); });
    {
        Stage st(c, NCORP_STAGE_KDK);
        KickDriftArgs K;
        K.x = A.x; K.y = A.y; K.z = A.z; K.vx = A.vx; K.vy = A.vy; K.vz = A.vz;
        K.ax = A.ax; K.ay = A.ay; K.az = A.az;
        K.h = h; K.dt = dt;
        K.ox = B.x; K.oy = B.y; K.oz = B.z; K.ovx = B.vx; K.ovy = B.vy; K.ovz = B.vz;
        K.n = n;
        K.ctl = c->alt.ctl;
        K.R = A.R;
        K.rc_spec = fused ? c->cells.rc_spec : nullptr;
        K.stale = &c->ctl->col_stale;
        K.cv4 = c->cv4;
        launch_kick_drift(c, K);
    }
    if (c->cfg.collisions) {
        if (side) {
            cudaStream_t main = c->stream;
            const int cap = c->coop_max;
            NCORP_CUDA_CHECK(cudaEventRecord(c->ev_fork, main));
            NCORP_CUDA_CHECK(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
            c->stream = c->side;
            c->coop_max = cap > 0 ? std::min(cap, c->side_blocks) : c->side_blocks;
            try {
                collisions(c, A, B.vx, B.vy, B.vz, dt, false, fused ? &c->ctl->col_stale : nullptr);
                if (resolve) launch_resolve(c, A, B, n, dt);   // may rewrite the drift the main stream reads
                NCORP_CUDA_CHECK(cudaEventRecord(c->ev_join, c->side));
            } catch (...) {
                c->stream = main;
                c->coop_max = cap;
                throw;
            }
            c->stream = main;
            c->coop_max = cap;
        } else {
            collisions(c, A, B.vx, B.vy, B.vz, dt, false);   // (no overlap: a batch's streams share the GPU)
            if (resolve) {
                Stage st(c, NCORP_STAGE_COLLIDE);
                launch_resolve(c, A, B, n, dt);
                // the drifted box again, if a moonlet's drift changed (the new tree set's control block)
                launch_bbox_gated(c, B.x, B.y, B.z, n, c->alt.ctl, &c->ctl->n_resolved);
            }
        }
    }
    swap_sets(c);
    build_tree(c, B, B, A, Cn, n, true, true, nullptr, fused ? dt : 0.0);
    if (side && resolve) {
        // The tree above was built beside the search from the unresolved drift.  A step that resolved an
        // impact builds it again from the resolved one; otherwise these launches return at once.
        NCORP_CUDA_CHECK(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
        const int *moved = &c->alt.ctl->n_resolved;   // the search's control block
        {
            Stage st(c, NCORP_STAGE_SORT);
            launch_bbox_gated(c, B.x, B.y, B.z, n, c->ctl, moved);
        }
        build_tree(c, B, B, A, Cn, n, false, true, moved);
    }
    gravity(c, Cn, p, theta, c->time + dt, false, h, fused ? dt : 0.0);   // with the closing half kick
    if (side && !resolve) NCORP_CUDA_CHECK(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
}

// col: the control block of the tree the collision search ran on (NULL: the current one)
void record_stats(ncorp_ctx *c, bool grav, const Ctrl *col = nullptr) {
    const Ctrl &h = *c->ctl_h;
    const Ctrl &hc = col ? *col : h;
    c->stats[NCORP_STAT_LAUNCHES] = c->launches;
    c->stats[NCORP_STAT_GRAPH] = c->graph_used ? 1 : 0;
    c->stats[NCORP_STAT_SORT_PATH] = h.resort_ok;
    c->stats[NCORP_STAT_RESOLVED] = c->cfg.collisions ? hc.n_resolved : 0;
    c->stats[NCORP_STAT_CELLS] = h.n_cells;
    c->stats[NCORP_STAT_LEAVES] = h.n_leaves;
    c->stats[NCORP_STAT_DEPTH] = h.max_level;
    c->stats[NCORP_STAT_WALK_ITERS] = h.walk_iters;
    if (grav) {
        c->stats[NCORP_STAT_M2L] = h.n_m2l;
        c->stats[NCORP_STAT_P2P_PAIRS] = h.dec_pairs;
        c->stats[NCORP_STAT_P2P_SELF] = h.dec_self;
        c->stats[NCORP_STAT_P2P_INTER] = h.n_inter;
        c->stats[NCORP_STAT_M2L_DIRECTED] = h.n_m2l_dir;
        c->stats[NCORP_STAT_P2P_DIRECTED] = h.n_p2p_dir;
    }
    c->stats[NCORP_STAT_FUSED] = (c->cfg.fused_walk && c->cfg.collisions && col && !hc.col_stale) ? 1 : 0;
    if (!grav || c->cfg.collisions) {
        c->stats[NCORP_STAT_COL_PAIRS] = hc.col_pairs;
        c->stats[NCORP_STAT_COL_SELF] = hc.col_self;
        c->stats[NCORP_STAT_COL_TESTS] = hc.n_tests;
        c->stats[NCORP_STAT_COL_FOUND] = hc.n_found;
        c->stats[NCORP_STAT_COL_ITERS] = hc.col_iters;
    }
}

bool finite_ok(ncorp_ctx *c) { return (c->ctl_h->err & ERR_NONFINITE) == 0; }

int check_common(ncorp_ctx *c, int64_t n, int p, double theta) {
    if (!c) return NCORP_EINVAL;
    if (n < 1 || n > (int64_t(1) << 30)) return fail(c, NCORP_EINVAL, "n = %lld out of range", (long long)n);
    if (p < 1 || p > MAXP) return fail(c, NCORP_EINVAL, "p = %d outside 1..6", p);
    if (!(theta > 0.0 && theta < 1.0)) return fail(c, NCORP_EINVAL, "theta = %g outside (0, 1)", theta);
    if (c->nd > 1 && n != c->forest_n)
        return fail(c, NCORP_EINVAL, "n = %lld is not the %d disks' total of %d", (long long)n, c->nd, c->forest_n);
    return NCORP_OK;
}

// ---- CUDA graphs of resident steps ------------------------------------------
// A resident step (state, tree and acceleration already on the device) makes
// the same launches with the same arguments every other call: the two tree
// sets and the two particle sets trade places once per step.  Such a step is
// captured once per rotation into a CUDA graph and then replayed, which takes
// the host's launch overhead out of the step and lets the device start
// dependent launches back to back.  A graph is valid for everything its
// launches read from the host: the buffer pointers (and the allocation
// generation, which every device (re)allocation bumps), n, p, theta, dt, the
// precision, the collision switch, the cooperative grid cap and whether the
// caller's arrays are on the device.  The star's position depends on the time,
// so steps with a star are never captured.

void step_graph_key(ncorp_ctx *c, const double *pos, const double *vel, int n, int p, double theta, double dt,
                    bool dev_x, bool dev_v, StepGraph &k) {
    const void *ptrs[6] = {pos, vel, c->A.x, c->Cset.x, c->ctl, c->alt.ctl};
    long long tb, db;
    std::memcpy(&tb, &theta, sizeof tb);
    std::memcpy(&db, &dt, sizeof db);
    const long long nums[10] = {n, p, tb, db, static_cast<long long>(alloc_generation()), c->cfg.precision,
                                c->cfg.collisions, (dev_x ? 2 : 0) | (dev_v ? 1 : 0), c->coop_max, c->num_sms};
    std::memcpy(k.key, ptrs, sizeof ptrs);
    std::memcpy(k.nums, nums, sizeof nums);
}

bool same_key(const StepGraph &a, const StepGraph &b) {
    return std::memcmp(a.key, b.key, sizeof a.key) == 0 && std::memcmp(a.nums, b.nums, sizeof a.nums) == 0;
}

void drop_graph(StepGraph &g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g = StepGraph{};
}

// The device work of one resident step up to the scatter of the new state
// into the caller's order (into the caller's arrays when they are on the
// device, else into the staging buffers).
void resident_step_body(ncorp_ctx *c, double *pos, double *vel, int n, int p, double theta, double dt, bool dev_x,
                        bool dev_v) {
    reset_ctls(c);
    enqueue_kdk(c, n, p, theta, dt, true);
    Stage st(c, NCORP_STAGE_KDK);
    ParticleSet &Cn = c->Cset;
    // a step that aborted (overflow, time-out) writes nothing to the caller's arrays
    launch_scatter_state(c, Cn, dev_x ? pos : c->stage, dev_v ? vel : c->stage2, n, &c->ctl->err, &c->alt.ctl->err);
}

// Enqueues a resident step on c->stream through a cached graph (capturing it
// first if no cached graph fits).  Host side effects are those of the direct
// path: the tree sets trade places.  Returns false, with nothing enqueued and
// the host state unchanged, if the step could not be captured.
bool resident_step_graph(ncorp_ctx *c, double *pos, double *vel, int n, int p, double theta, double dt, bool dev_x,
                         bool dev_v) {
    StepGraph want;
    step_graph_key(c, pos, vel, n, p, theta, dt, dev_x, dev_v, want);
    for (StepGraph &g : c->graphs)
        if (g.exec && same_key(g, want)) {
            NCORP_CUDA_CHECK(cudaGraphLaunch(g.exec, c->stream));
            swap_sets(c);
            c->cur_n = n;
            c->grav_p = p;
            c->grav_mixed = c->cfg.precision == NCORP_MIXED;
            c->launches += g.launches;
            return true;
        }
    if (!c->gstream) {   // highest priority: the step's main chain (captured from it) goes first
        int least = 0, greatest = 0;
        NCORP_CUDA_CHECK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        NCORP_CUDA_CHECK(cudaStreamCreateWithPriority(&c->gstream, cudaStreamNonBlocking, greatest));
    }
    const Ctrl *ctl0 = c->ctl;
    const int launches0 = c->launches;
    cudaStream_t main = c->stream;
    cudaGraph_t graph = nullptr;
    NCORP_CUDA_CHECK(cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeRelaxed));
    c->stream = c->gstream;
    bool ok = true;
    try {
        resident_step_body(c, pos, vel, n, p, theta, dt, dev_x, dev_v);
    } catch (const CudaError &) {
        ok = false;
    }
    c->stream = main;
    const cudaError_t end = cudaStreamEndCapture(c->gstream, &graph);
    cudaGraphExec_t exec = nullptr;
    // kernel nodes keep the priority of the stream they were captured from
    if (ok && end == cudaSuccess && graph)
        ok = cudaGraphInstantiateWithFlags(&exec, graph, cudaGraphInstantiateFlagUseNodePriority) == cudaSuccess;
    else ok = false;
    if (graph) cudaGraphDestroy(graph);
    if (!ok) {
        cudaGetLastError();
        if (exec) cudaGraphExecDestroy(exec);
        if (c->ctl != ctl0) swap_sets(c);
        c->launches = launches0;
        return false;
    }
    NCORP_CUDA_CHECK(cudaGraphLaunch(exec, main));
    StepGraph &slot = c->graphs[c->graph_next];
    c->graph_next ^= 1;
    drop_graph(slot);
    slot = want;
    slot.exec = exec;
    slot.launches = c->launches - launches0;
    return true;
}

constexpr int MAX_RETRIES = 6;

// integer environment variable, clamped to [lo, hi]; dflt when unset or not a number
long long env_int(const char *name, long long dflt, long long lo, long long hi) {
    const char *v = std::getenv(name);
    if (!v || !*v) return dflt;
    char *end = nullptr;
    const long long x = std::strtoll(v, &end, 10);
    if (end == v) return dflt;
    return std::min(hi, std::max(lo, x));
}

#define NCORP_API_BODY(ctxp, ...)                                                               \
    try {                                                                                       \
        NCORP_CUDA_CHECK(cudaSetDevice((ctxp)->device));                                        \
        __VA_ARGS__                                                                             \
    } catch (const CudaError &e) {                                                              \
        cudaGetLastError();   /* a non-sticky error is reported once, by this call */           \
        (ctxp)->have_state = false;                                                             \
        (ctxp)->tree_valid = false;                                                             \
        return fail((ctxp), e.code == cudaErrorMemoryAllocation ? NCORP_ENOMEM : NCORP_ECUDA,   \
                    "%s: %s (%s:%d)", e.expr, cudaGetErrorString(e.code), e.file, e.line);       \
    } catch (const std::bad_alloc &) {                                                          \
        return fail((ctxp), NCORP_ENOMEM, "host allocation failed");                             \
    }

}  // namespace

extern "C" {

void ncorp_config_default(ncorp_config *cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->G = 1.0;
    cfg->central_mass = 1.0;
    cfg->central_radius = 1.0;
    cfg->precision = NCORP_MIXED;
    cfg->collisions = 1;
    cfg->n_cb_pre = 6;
    cfg->n_cb_post = 16;
    cfg->c_cb_pre = 0;
    cfg->c_cb_post = 16;
}

int ncorp_init(ncorp_ctx **out, const ncorp_config *cfg, int64_t n_max, int device, void *cuda_stream) {
    if (!out || !cfg || n_max < 1) return NCORP_EINVAL;
    if (cfg->precision != NCORP_FP64 && cfg->precision != NCORP_MIXED) return NCORP_EINVAL;
    if (!(cfg->G > 0.0) || !(cfg->central_mass >= 0.0) || cfg->leaf_size < 0) return NCORP_EINVAL;
    if (!(cfg->resolve_f == 0.0 || (cfg->resolve_f >= 1.0 && cfg->resolve_f <= 2.0))) return NCORP_EINVAL;
    if (cfg->n_cb_pre < 0 || cfg->n_cb_post < 0 || cfg->c_cb_pre < 0 || cfg->c_cb_post < 0) return NCORP_EINVAL;
    *out = nullptr;
    ncorp_ctx *c = new (std::nothrow) ncorp_ctx();
    if (!c) return NCORP_ENOMEM;
    c->cfg = *cfg;
    c->device = device;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    c->time = cfg->t0;
    c->radix_epoch_limit = radix_epoch_limit();
    try {
        NCORP_CUDA_CHECK(cudaSetDevice(device));
        NCORP_CUDA_CHECK(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device));
        int coop = 0;
        NCORP_CUDA_CHECK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device));
        if (!coop) throw CudaError(cudaErrorNotSupported, "cooperative launch unsupported", __FILE__, __LINE__);
        // Failure-path test knobs (off unless set): NCORP_WAIT_LIMIT_MS bounds every grid barrier's wait
        // (default 1000), NCORP_TEST_STALL_STEP=k makes the k-th ncorp_step's barriers wait for an arrival
        // that never comes, NCORP_TEST_LIST_CAP / NCORP_TEST_PAIR_CAP start the walk lists / pair buffer at
        // that many entries so that they overflow and grow.
        const unsigned long long wait_ns = static_cast<unsigned long long>(env_int("NCORP_WAIT_LIMIT_MS", 1000, 1,
                                                                                    60000)) * 1000000ull;
        c->stall_call = env_int("NCORP_TEST_STALL_STEP", 0, 0, 1 << 30);
        c->side_blocks = static_cast<int>(env_int("NCORP_SIDE_BLOCKS", 64, 8, 1024));
        c->test_list_cap = static_cast<int>(env_int("NCORP_TEST_LIST_CAP", 0, 0, 1 << 30));
        c->test_pair_cap = static_cast<int>(env_int("NCORP_TEST_PAIR_CAP", 0, 0, 1 << 30));
        for (int set = 0; set < 2; set++) {
            dalloc(c->ctl, 1);
            NCORP_CUDA_CHECK(cudaMallocHost(reinterpret_cast<void **>(&c->ctl_h), sizeof(Ctrl)));
            std::memset(c->ctl_h, 0, sizeof(Ctrl));
            c->ctl_h->wait_ns = wait_ns;
            c->ctl_h->nd = 1;   // one disk: its box and root cube are the control block's own
            c->ctl_h->col_stale = 1;   // no fused walk has listed this tree set's collision pairs
            c->ctl_h->dbox = c->ctl->bbox;
            c->ctl_h->droot = c->ctl->root;
            NCORP_CUDA_CHECK(cudaMemcpy(c->ctl, c->ctl_h, sizeof(Ctrl), cudaMemcpyHostToDevice));
            swap_sets(c);
        }
        dalloc(c->work_counter, 4);
        dalloc(c->err_acc, 1);
        NCORP_CUDA_CHECK(cudaMemsetAsync(c->err_acc, 0, sizeof(int), c->stream));
        NCORP_CUDA_CHECK(cudaMallocHost(reinterpret_cast<void **>(&c->err_acc_h), sizeof(int)));
        *c->err_acc_h = 0;
        // side streams at the lowest priority: when blocks of both wait for room on the SMs, the main
        // chain's go first
        int least = 0, greatest = 0;
        NCORP_CUDA_CHECK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        NCORP_CUDA_CHECK(cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, least));
        NCORP_CUDA_CHECK(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
        NCORP_CUDA_CHECK(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
        NCORP_CUDA_CHECK(cudaStreamCreateWithPriority(&c->side2, cudaStreamNonBlocking, least));
        for (cudaEvent_t *e : {&c->ev_geo, &c->ev_p2m, &c->ev_lists, &c->ev_near, &c->ev_spec0, &c->ev_spec})
            NCORP_CUDA_CHECK(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
        ensure_particles(c, n_max);
        choose_parameters(c, 6);
        ensure_both_capacities(c, static_cast<int>(n_max));
        NCORP_CUDA_CHECK(cudaStreamSynchronize(c->stream));   // the clears above, before any other stream's use
    } catch (const CudaError &e) {
        cudaGetLastError();   // (a non-sticky error is reported once, here)
        int code = (e.code == cudaErrorMemoryAllocation) ? NCORP_ENOMEM : NCORP_ECUDA;
        ncorp_free(c);
        return code;
    }
    *out = c;
    return NCORP_OK;
}

int ncorp_set_stream(ncorp_ctx *c, void *cuda_stream) {
    if (!c) return NCORP_EINVAL;
    // work already enqueued on the old stream (buffer clears included) ends before the new one's
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return fail(c, NCORP_ECUDA, "%s", "stream synchronize failed");
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    return NCORP_OK;
}

int ncorp_set_graphs(ncorp_ctx *c, int enable) {
    if (!c) return NCORP_EINVAL;
    c->graphs_on = enable != 0;
    if (!c->graphs_on) {
        NCORP_API_BODY(c, {
            NCORP_CUDA_CHECK(cudaStreamSynchronize(c->stream));
            for (StepGraph &g : c->graphs) drop_graph(g);
        })
    }
    return NCORP_OK;
}

int ncorp_reset(ncorp_ctx *c) {
    if (!c) return NCORP_EINVAL;
    c->have_state = false;
    c->tree_valid = false;
    return NCORP_OK;
}

int ncorp_set_disks(ncorp_ctx *c, int n_disks, const int64_t *sizes) {
    if (!c) return NCORP_EINVAL;
    if (n_disks < 1 || n_disks > NCORP_MAX_DISKS)
        return fail(c, NCORP_EINVAL, "n_disks = %d outside 1..%d", n_disks, NCORP_MAX_DISKS);
    if (n_disks > 1 && !sizes) return fail(c, NCORP_EINVAL, "null pointer");
    int64_t total = 0;
    for (int d = 0; sizes && d < n_disks; d++) {
        if (sizes[d] < 1) return fail(c, NCORP_EINVAL, "disk %d has %lld moonlets", d, (long long)sizes[d]);
        total += sizes[d];
    }
    if (total > (int64_t(1) << 30)) return fail(c, NCORP_EINVAL, "%lld moonlets in all", (long long)total);
    NCORP_API_BODY(c, {
        configure_disks(c, n_disks, n_disks > 1 ? sizes : nullptr);
        return NCORP_OK;
    })
}

int ncorp_accel(ncorp_ctx *c, const double *positions, const double *masses, int64_t n64, int p, double theta,
                double *acc, double *acc_mutual) {
    int st = check_common(c, n64, p, theta);
    if (st) return st;
    if (!positions || !masses || !acc) return fail(c, NCORP_EINVAL, "null pointer");
    NCORP_API_BODY(c, {
        begin_call(c);
        const int n = static_cast<int>(n64);
        ensure_particles(c, n);
        choose_parameters(c, p);
        c->have_state = false;
        c->tree_valid = false;
        for (int attempt = 0;; attempt++) {
            ensure_tree_capacity(c, n);
            reset_ctl(c);
            ParticleSet &A = c->A;
            upload_vec(c, positions, A.x, A.y, A.z, n);
            upload_scalar(c, masses, A.m, n);
            NCORP_CUDA_CHECK(cudaMemsetAsync(A.vx, 0, sizeof(double) * n, c->stream));
            NCORP_CUDA_CHECK(cudaMemsetAsync(A.vy, 0, sizeof(double) * n, c->stream));
            NCORP_CUDA_CHECK(cudaMemsetAsync(A.vz, 0, sizeof(double) * n, c->stream));
            NCORP_CUDA_CHECK(cudaMemsetAsync(A.R, 0, sizeof(double) * n, c->stream));
            launch_iota(c, reinterpret_cast<uint32_t *>(A.perm), n);
            build_tree(c, A, A, A, c->Cset, n);
            std::swap(c->A, c->Cset);
            gravity(c, c->A, p, theta, c->time, true);
            download_vec(c, c->A.ax, c->A.ay, c->A.az, c->A.perm, acc, n, c->stage);
            if (acc_mutual) download_vec(c, c->amx, c->amy, c->amz, c->A.perm, acc_mutual, n, c->stage2);
            int err = finish(c);
            if (!finite_ok(c)) return fail(c, NCORP_EINVAL, "non-finite position");
            if (err & ERR_TIMEOUT) return fail(c, NCORP_ETIMEOUT, "device-side barrier timed out");
            if (err == 0) break;
            if (attempt >= MAX_RETRIES || !grow_after(c, err))
                return fail(c, NCORP_EOVERFLOW, "internal list overflow (flags 0x%x)", err);
        }
        c->n = n;
        c->tree_kind = 1;
        record_stats(c, true);
        return NCORP_OK;
    })
}

int ncorp_accel_standard(ncorp_ctx *c, const double *positions, const double *masses, int64_t n64, int p,
                         double theta, double *acc, double *acc_mutual) {
    int st = check_common(c, n64, p, theta);
    if (st) return st;
    if (c->nd > 1) return fail(c, NCORP_EINVAL, "the standard tree code walks one disk: ncorp_set_disks(ctx, 1, ...)");
    if (!positions || !masses || !acc) return fail(c, NCORP_EINVAL, "null pointer");
    NCORP_API_BODY(c, {
        begin_call(c);
        const int n = static_cast<int>(n64);
        ensure_particles(c, n);
        choose_parameters(c, p);
        c->have_state = false;
        c->tree_valid = false;
        for (int attempt = 0;; attempt++) {
            ensure_tree_capacity(c, n);
            reset_ctl(c);
            ParticleSet &A = c->A;
            upload_vec(c, positions, A.x, A.y, A.z, n);
            upload_scalar(c, masses, A.m, n);
            NCORP_CUDA_CHECK(cudaMemsetAsync(A.vx, 0, sizeof(double) * n, c->stream));
            NCORP_CUDA_CHECK(cudaMemsetAsync(A.vy, 0, sizeof(double) * n, c->stream));
            NCORP_CUDA_CHECK(cudaMemsetAsync(A.vz, 0, sizeof(double) * n, c->stream));
            NCORP_CUDA_CHECK(cudaMemsetAsync(A.R, 0, sizeof(double) * n, c->stream));
            launch_iota(c, reinterpret_cast<uint32_t *>(A.perm), n);
            build_tree(c, A, A, A, c->Cset, n);
            std::swap(c->A, c->Cset);
            gravity_standard(c, c->A, n, p, theta, c->time, acc_mutual != nullptr);
            download_vec(c, c->A.ax, c->A.ay, c->A.az, c->A.perm, acc, n, c->stage);
            if (acc_mutual) download_vec(c, c->amx, c->amy, c->amz, c->A.perm, acc_mutual, n, c->stage2);
            int err = finish(c);
            if (!finite_ok(c)) return fail(c, NCORP_EINVAL, "non-finite position");
            if (err & ERR_TIMEOUT) return fail(c, NCORP_ETIMEOUT, "device-side barrier timed out");
            if (err == 0) break;
            if (attempt >= MAX_RETRIES || !grow_after(c, err))
                return fail(c, NCORP_EOVERFLOW, "internal list overflow (flags 0x%x)", err);
        }
        c->n = n;
        c->tree_kind = 1;
        record_stats(c, true);
        const Ctrl &h = *c->ctl_h;
        c->stats[NCORP_STAT_M2L] = h.n_m2p;
        c->stats[NCORP_STAT_P2P_SELF] = 0;
        c->stats[NCORP_STAT_M2L_DIRECTED] = 0;
        c->stats[NCORP_STAT_P2P_DIRECTED] = 0;
        c->stats[NCORP_STAT_WALK_ITERS] = 0;
        return NCORP_OK;
    })
}

// Collision search alone, by falcON's dual walk (standard = false) or by the standard tree code.
static int collide_call(ncorp_ctx *c, const double *positions, const double *velocities, const double *radii, int64_t n64,
                 double dt, bool standard) {
    if (!c) return NCORP_EINVAL;
    if (n64 < 1 || n64 > (int64_t(1) << 30)) return fail(c, NCORP_EINVAL, "n out of range");
    if (!positions || !velocities || !radii) return fail(c, NCORP_EINVAL, "null pointer");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, NCORP_EINVAL, "dt must be > 0");
    if (c->nd > 1 && n64 != c->forest_n)
        return fail(c, NCORP_EINVAL, "n = %lld is not the %d disks' total of %d", (long long)n64, c->nd, c->forest_n);
    if (standard && c->nd > 1)
        return fail(c, NCORP_EINVAL, "the standard tree code walks one disk: ncorp_set_disks(ctx, 1, ...)");
    NCORP_API_BODY(c, {
        begin_call(c);
        const int n = static_cast<int>(n64);
        ensure_particles(c, n);
        if (c->s == 0) choose_parameters(c, 6);
        c->have_state = false;
        c->tree_valid = false;
        for (int attempt = 0;; attempt++) {
            ensure_tree_capacity(c, n);
            reset_ctl(c);
            ParticleSet &A = c->A;
            upload_vec(c, positions, A.x, A.y, A.z, n);
            upload_vec(c, velocities, A.vx, A.vy, A.vz, n);
            upload_scalar(c, radii, A.R, n);
            NCORP_CUDA_CHECK(cudaMemsetAsync(A.m, 0, sizeof(double) * n, c->stream));
            launch_iota(c, reinterpret_cast<uint32_t *>(A.perm), n);
            build_tree(c, A, A, A, c->Cset, n);
            std::swap(c->A, c->Cset);
            if (standard) collisions_standard(c, c->A, n, dt);
            else collisions(c, c->A, c->A.vx, c->A.vy, c->A.vz, dt, true);
            int err = finish(c);
            if (!finite_ok(c)) return fail(c, NCORP_EINVAL, "non-finite position");
            if (err & ERR_TIMEOUT) return fail(c, NCORP_ETIMEOUT, "device-side barrier timed out");
            if (err == 0) break;
            if (attempt >= MAX_RETRIES || !grow_after(c, err))
                return fail(c, NCORP_EOVERFLOW, "internal list overflow (flags 0x%x)", err);
        }
        c->n = n;
        c->n_found = c->ctl_h->n_found;
        c->pairs_sorted = false;
        c->tree_kind = 2;
        record_stats(c, false);
        return NCORP_OK;
    })
}

int ncorp_collide(ncorp_ctx *c, const double *positions, const double *velocities, const double *radii, int64_t n64,
                  double dt) {
    return collide_call(c, positions, velocities, radii, n64, dt, false);
}

int ncorp_collide_standard(ncorp_ctx *c, const double *positions, const double *velocities, const double *radii,
                           int64_t n64, double dt) {
    return collide_call(c, positions, velocities, radii, n64, dt, true);
}

int ncorp_step(ncorp_ctx *c, double *positions, double *velocities, const double *masses, const double *radii,
               int64_t n64, int p, double theta, double dt) {
    int st = check_common(c, n64, p, theta);
    if (st) return st;
    if (!positions || !velocities || !masses || !radii) return fail(c, NCORP_EINVAL, "null pointer");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, NCORP_EINVAL, "dt must be > 0");
    NCORP_API_BODY(c, {
        begin_call(c);
        const int n = static_cast<int>(n64);
        const bool resident = c->have_state && c->tree_valid && c->n == n && c->last_pos == positions &&
                              c->last_vel == velocities && c->last_m == masses && c->last_R == radii &&
                              c->last_p == p && c->last_theta == theta;
        ensure_particles(c, n);
        choose_parameters(c, p);
        bool have = resident && c->have_state;
        bool tree = resident;
        const bool stall = c->stall_call > 0 && ++c->step_calls == c->stall_call;
        for (int attempt = 0;; attempt++) {
            ensure_both_capacities(c, n);
            c->graph_used = false;
            if (attempt == 0 && have && tree && c->graphs_on && !c->profile && c->cfg.star_mass == 0.0 && !stall) {
                const bool dev_x = is_device_ptr(c, positions), dev_v = is_device_ptr(c, velocities);
                c->graph_used = resident_step_graph(c, positions, velocities, n, p, theta, dt, dev_x, dev_v);
                if (c->graph_used && !dev_x)
                    NCORP_CUDA_CHECK(cudaMemcpyAsync(positions, c->stage, sizeof(double) * 3 * n,
                                                     cudaMemcpyDeviceToHost, c->stream));
                if (c->graph_used && !dev_v)
                    NCORP_CUDA_CHECK(cudaMemcpyAsync(velocities, c->stage2, sizeof(double) * 3 * n,
                                                     cudaMemcpyDeviceToHost, c->stream));
            }
            if (!c->graph_used) {
                reset_ctls(c);
                if (stall && attempt == 0) {   // failure-path test: this step's grid barriers give up
                    k_arm_stall<<<1, 1, 0, c->stream>>>(c->ctl, c->alt.ctl);
                    c->launches++;
                    NCORP_CUDA_CHECK(cudaGetLastError());
                }
                if (!have) {   // read the caller's state (caller order)
                    Stage st(c, NCORP_STAGE_KDK);
                    ParticleSet &A = c->A;
                    upload_vec(c, positions, A.x, A.y, A.z, n);
                    upload_vec(c, velocities, A.vx, A.vy, A.vz, n);
                    upload_scalar(c, masses, A.m, n);
                    upload_scalar(c, radii, A.R, n);
                    launch_iota(c, reinterpret_cast<uint32_t *>(A.perm), n);
                    tree = false;
                }
                if (!tree) {   // tree and acceleration of the current positions
                    build_tree(c, c->A, c->A, c->A, c->Cset, n);
                    std::swap(c->A, c->Cset);
                    gravity(c, c->A, p, theta, c->time, false);
                }
                enqueue_kdk(c, n, p, theta, dt, true);
                Stage st(c, NCORP_STAGE_KDK);
                ParticleSet &Cn = c->Cset;
                // nothing is written to the caller's arrays if the step aborted
                download_vec(c, Cn.x, Cn.y, Cn.z, Cn.perm, positions, n, c->stage, &c->ctl->err, &c->alt.ctl->err);
                download_vec(c, Cn.vx, Cn.vy, Cn.vz, Cn.perm, velocities, n, c->stage2, &c->ctl->err,
                             &c->alt.ctl->err);
            }
            const int err = finish(c, true);
            // the current tree set now holds the new tree, the other one A's tree
            const int e_new = c->ctl_h->err, e_old = c->alt.ctl_h->err, e_acc = *c->err_acc_h;
            if (err & ERR_NONFINITE) {
                c->have_state = false;
                c->tree_valid = false;
                return fail(c, NCORP_EINVAL, "non-finite position");
            }
            if (err & ERR_TIMEOUT) {
                c->have_state = false;
                c->tree_valid = false;
                return fail(c, NCORP_ETIMEOUT, "device-side barrier timed out");
            }
            if (err == 0) break;
            // A was not written: rerun from it with larger buffers (its tree is rebuilt)
            swap_sets(c);
            have = true;
            tree = false;
            bool grew = grow_after(c, e_old | e_acc);
            on_alt(c, [&] { grew = grow_after(c, e_new | e_acc) || grew; });
            if (attempt >= MAX_RETRIES || !grew) {
                c->tree_valid = false;
                return fail(c, NCORP_EOVERFLOW, "internal list overflow (flags 0x%x)", err);
            }
        }
        if (c->cfg.collisions) {
            c->n_found = c->alt.ctl_h->n_found;
            c->pairs_sorted = false;
        } else {
            c->n_found = 0;
        }
        std::swap(c->A, c->Cset);
        c->time += dt;
        c->n = n;
        c->have_state = true;
        c->tree_valid = true;
        c->tree_kind = 1;
        c->last_pos = positions;
        c->last_vel = velocities;
        c->last_m = masses;
        c->last_R = radii;
        c->last_p = p;
        c->last_theta = theta;
        record_stats(c, true, c->alt.ctl_h);
        c->stats[NCORP_STAT_COL_FOUND] = c->n_found;
        return NCORP_OK;
    })
}

int ncorp_collisions(ncorp_ctx *c, int64_t *pairs, int64_t cap, int64_t *n_pairs) {
    if (!c || cap < 0 || (cap > 0 && !pairs)) return NCORP_EINVAL;
    NCORP_API_BODY(c, {
        const int found = c->n_found;
        const int stored = std::min(found, c->pair_cap);
        if (!c->pairs_sorted) {
            launch_sort_pairs(c, stored);
            launch_unpack_pairs(c, c->pairs, c->pairs_out, stored);
            c->pairs_sorted = true;
        }
        const int64_t k = std::min<int64_t>(cap, stored);
        if (k > 0)
            NCORP_CUDA_CHECK(cudaMemcpyAsync(pairs, c->pairs_out, sizeof(int64_t) * 2 * k, cudaMemcpyDefault, c->stream));
        NCORP_CUDA_CHECK(cudaStreamSynchronize(c->stream));
        if (n_pairs) *n_pairs = found;
        if (found > c->pair_cap) return fail(c, NCORP_EOVERFLOW, "pair buffer overflowed (%d found)", found);
        if (found > cap) return fail(c, NCORP_EOVERFLOW, "%d pairs found, room for %lld", found, (long long)cap);
        return NCORP_OK;
    })
}

int ncorp_get_state(ncorp_ctx *c, double *positions, double *velocities) {
    if (!c || !positions || !velocities) return NCORP_EINVAL;
    if (!c->have_state) return fail(c, NCORP_ESTATE, "no resident state");
    NCORP_API_BODY(c, {
        download_vec(c, c->A.x, c->A.y, c->A.z, c->A.perm, positions, c->n, c->stage);
        download_vec(c, c->A.vx, c->A.vy, c->A.vz, c->A.perm, velocities, c->n, c->stage2);
        NCORP_CUDA_CHECK(cudaStreamSynchronize(c->stream));
        return NCORP_OK;
    })
}

int ncorp_stats(ncorp_ctx *c, int64_t *stats, int n_stats) {
    if (!c || !stats || n_stats < 0) return NCORP_EINVAL;
    for (int i = 0; i < n_stats && i < NCORP_NSTATS; i++) stats[i] = c->stats[i];
    return NCORP_OK;
}

int ncorp_tree_export(ncorp_ctx *c, int64_t *order, uint64_t *keys, double *root, int64_t *cells, double *ggeo,
                      double *cgeo, int64_t cap, int64_t *n_cells) {
    if (!c || cap < 0) return NCORP_EINVAL;
    if (c->n <= 0 || c->tree_kind == 0) return fail(c, NCORP_ESTATE, "no tree yet");
    NCORP_API_BODY(c, {
        const int n = c->n;
        const int nc = std::min(c->ctl_h->n_cells, c->cells.cap);
        const Cells &C = c->cells;
        if (n_cells) *n_cells = nc;
        if (order) {
            std::vector<int> perm(n);
            std::vector<int64_t> o(n);
            NCORP_CUDA_CHECK(cudaMemcpy(perm.data(), c->A.perm, sizeof(int) * n, cudaMemcpyDeviceToHost));
            for (int i = 0; i < n; i++) o[i] = perm[i];
            NCORP_CUDA_CHECK(cudaMemcpy(order, o.data(), sizeof(int64_t) * n, cudaMemcpyDefault));
        }
        if (keys) NCORP_CUDA_CHECK(cudaMemcpy(keys, c->A.key, sizeof(uint64_t) * n, cudaMemcpyDefault));
        if (root) {   // one root cube per disk (a forest's are in the current tree set's own array)
            const double *src = c->nd > 1 ? c->ctl_h->droot : c->ctl->root;
            NCORP_CUDA_CHECK(cudaMemcpy(root, src, sizeof(double) * 4 * c->nd, cudaMemcpyDefault));
        }
        const int k = static_cast<int>(std::min<int64_t>(cap, nc));
        if (k > 0 && cells) {
            std::vector<int> lv(k), f(k), cnt(k), nch(k);
            std::vector<uint32_t> x(k), y(k), z(k);
            NCORP_CUDA_CHECK(cudaMemcpy(lv.data(), C.level, sizeof(int) * k, cudaMemcpyDeviceToHost));
            NCORP_CUDA_CHECK(cudaMemcpy(f.data(), C.first, sizeof(int) * k, cudaMemcpyDeviceToHost));
            NCORP_CUDA_CHECK(cudaMemcpy(cnt.data(), C.count, sizeof(int) * k, cudaMemcpyDeviceToHost));
            NCORP_CUDA_CHECK(cudaMemcpy(nch.data(), C.nchild, sizeof(int) * k, cudaMemcpyDeviceToHost));
            NCORP_CUDA_CHECK(cudaMemcpy(x.data(), C.cx, sizeof(uint32_t) * k, cudaMemcpyDeviceToHost));
            NCORP_CUDA_CHECK(cudaMemcpy(y.data(), C.cy, sizeof(uint32_t) * k, cudaMemcpyDeviceToHost));
            NCORP_CUDA_CHECK(cudaMemcpy(z.data(), C.cz, sizeof(uint32_t) * k, cudaMemcpyDeviceToHost));
            std::vector<int64_t> rows(7 * static_cast<size_t>(k));
            for (int i = 0; i < k; i++) {
                int64_t *r = &rows[7 * static_cast<size_t>(i)];
                r[0] = lv[i]; r[1] = x[i]; r[2] = y[i]; r[3] = z[i]; r[4] = f[i]; r[5] = cnt[i]; r[6] = nch[i];
            }
            NCORP_CUDA_CHECK(cudaMemcpy(cells, rows.data(), sizeof(int64_t) * rows.size(), cudaMemcpyDefault));
        }
        auto pack = [&](double *dst, std::initializer_list<const double *> cols) {
            const int w = static_cast<int>(cols.size());
            std::vector<double> tmp(k), out(static_cast<size_t>(k) * w);
            int j = 0;
            for (const double *col : cols) {
                NCORP_CUDA_CHECK(cudaMemcpy(tmp.data(), col, sizeof(double) * k, cudaMemcpyDeviceToHost));
                for (int i = 0; i < k; i++) out[static_cast<size_t>(i) * w + j] = tmp[i];
                j++;
            }
            NCORP_CUDA_CHECK(cudaMemcpy(dst, out.data(), sizeof(double) * out.size(), cudaMemcpyDefault));
        };
        if (k > 0 && ggeo && (c->tree_kind & 1)) pack(ggeo, {C.M, C.sx, C.sy, C.sz, C.rmax, C.rcrit});
        if (k > 0 && cgeo && (c->tree_kind & 2)) pack(cgeo, {C.bx, C.by, C.bz, C.bmax, C.bcrit});
        if (nc > cap) return fail(c, NCORP_EOVERFLOW, "%d cells, room for %lld", nc, (long long)cap);
        return NCORP_OK;
    })
}

int ncorp_expansions(ncorp_ctx *c, double *mult, double *local, double *rho, int64_t cap, int64_t *n_cells, int *p) {
    if (!c || cap < 0) return NCORP_EINVAL;
    if (c->grav_p <= 0 || !(c->tree_kind & 1)) return fail(c, NCORP_ESTATE, "no gravity evaluation yet");
    NCORP_API_BODY(c, {
        const int P = c->grav_p;
        const int nm = num_m(P), nc_ = num_c(P);
        const int ncell = std::min(c->ctl_h->n_cells, c->cells.cap);
        const int k = static_cast<int>(std::min<int64_t>(cap, ncell));
        if (n_cells) *n_cells = ncell;
        if (p) *p = P;
        std::vector<double> r(std::max(k, 1));
        if (k > 0) NCORP_CUDA_CHECK(cudaMemcpy(r.data(), c->cells.rho, sizeof(double) * k, cudaMemcpyDeviceToHost));
        auto fetch = [&](const void *src, int w) {
            std::vector<double> out(static_cast<size_t>(k) * w);
            if (c->grav_mixed) {
                std::vector<float> f(out.size());
                if (k > 0) NCORP_CUDA_CHECK(cudaMemcpy(f.data(), src, sizeof(float) * f.size(), cudaMemcpyDeviceToHost));
                for (size_t i = 0; i < f.size(); i++) out[i] = f[i];
            } else if (k > 0) {
                NCORP_CUDA_CHECK(cudaMemcpy(out.data(), src, sizeof(double) * out.size(), cudaMemcpyDeviceToHost));
            }
            return out;
        };
        // exponents of the packed components
        auto exps = [](int idx, int &a, int &b, int &cc) {
            int n = 0;
            while (off(n + 1) <= idx) n++;
            int rem = idx - off(n), kk = 0;
            while (tri(kk + 1) <= rem) kk++;
            cc = rem - tri(kk);
            b = kk - cc;
            a = n - kk;
        };
        if (mult) {
            std::vector<double> M = fetch(c->cells.Mh, nm);
            for (int i = 0; i < k; i++)
                for (int j = 0; j < nm; j++) {
                    int a, b, cc;
                    exps(j == 0 ? 0 : j + 3, a, b, cc);
                    double f = 1.0 / inv_mfact(a, b, cc);
                    for (int t = 0; t < a + b + cc; t++) f *= r[i];
                    M[static_cast<size_t>(i) * nm + j] *= f;
                }
            NCORP_CUDA_CHECK(cudaMemcpy(mult, M.data(), sizeof(double) * M.size(), cudaMemcpyDefault));
        }
        if (local && !c->grav_local)
            return fail(c, NCORP_ESTATE, "the last evaluation (standard tree code) made no local expansions");
        if (local) {   // the evaluation's descent completed every cell's expansion
            std::vector<double> Cl = fetch(c->cells.Cf, nc_);
            if (c->grav_mixed && k > 0) {   // the order-1 coefficients are double-float
                std::vector<float> lo(static_cast<size_t>(k) * 3);
                NCORP_CUDA_CHECK(cudaMemcpy(lo.data(), c->cells.Cf_lo, sizeof(float) * lo.size(), cudaMemcpyDeviceToHost));
                for (int i = 0; i < k; i++)
                    for (int j = 0; j < 3; j++) Cl[static_cast<size_t>(i) * nc_ + j] += static_cast<double>(lo[3 * i + j]);
            }
            for (int i = 0; i < k; i++)
                for (int j = 0; j < nc_; j++) {
                    int a, b, cc;
                    exps(j + 1, a, b, cc);
                    double f = 1.0;
                    for (int t = 0; t < a + b + cc; t++) f /= r[i];
                    Cl[static_cast<size_t>(i) * nc_ + j] *= f;
                }
            NCORP_CUDA_CHECK(cudaMemcpy(local, Cl.data(), sizeof(double) * Cl.size(), cudaMemcpyDefault));
        }
        if (rho && k > 0) NCORP_CUDA_CHECK(cudaMemcpy(rho, r.data(), sizeof(double) * k, cudaMemcpyDefault));
        if (ncell > cap) return fail(c, NCORP_EOVERFLOW, "%d cells, room for %lld", ncell, (long long)cap);
        return NCORP_OK;
    })
}

int ncorp_profile(ncorp_ctx *c, int enable) {
    if (!c) return NCORP_EINVAL;
    c->profile = enable != 0;
    return NCORP_OK;
}

int ncorp_stage_times(ncorp_ctx *c, double *ms, int n) {
    if (!c || !ms || n < 0) return NCORP_EINVAL;
    for (int i = 0; i < n && i < NCORP_NSTAGES; i++) ms[i] = c->stage_ms[i];
    return NCORP_OK;
}

void ncorp_free(ncorp_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    if (c->side) cudaStreamSynchronize(c->side);
    if (c->side2) cudaStreamSynchronize(c->side2);
    free_set(c->A);
    free_set(c->B);
    free_set(c->Cset);
    dfree(c->amx); dfree(c->amy); dfree(c->amz); dfree(c->cv4);
    dfree(c->key_alt); dfree(c->idx); dfree(c->idx_alt);
    dfree(c->resort_mkey); dfree(c->resort_midx); dfree(c->resort_bcount);
    dfree(c->tile_hist); dfree(c->stage); dfree(c->stage2);
    for (int set = 0; set < 2; set++) {
        Cells &C = c->cells;
        dfree(C.level); dfree(C.first); dfree(C.count); dfree(C.child0); dfree(C.nchild); dfree(C.parent);
        dfree(C.arrive); dfree(C.arrive_m); dfree(C.cx); dfree(C.cy); dfree(C.cz); dfree(C.M); dfree(C.sx); dfree(C.sy); dfree(C.sz);
        dfree(C.rmax); dfree(C.rcrit); dfree(C.rho); dfree(C.bx); dfree(C.by); dfree(C.bz); dfree(C.bmax);
        dfree(C.bcrit); dfree(C.gh); dfree(C.gl); dfree(C.bh); dfree(C.bl); dfree(C.Mh); dfree(C.Ch); dfree(C.Cf); dfree(C.Cf_lo); dfree(C.Ch_lo);
        dfree(C.leaves); dfree(C.leaf_of); dfree(C.rc_spec); dfree(C.bounds); dfree(C.blocksum); dfree(C.maker); dfree(C.before); dfree(C.done);
        WalkLists &W = c->wl;
        dfree(W.front[0]); dfree(W.front[1]); dfree(W.front_count); dfree(W.m2l); dfree(W.p2p); dfree(W.self);
        dfree(W.cnt); dfree(W.offs); dfree(W.cursor); dfree(W.m2l_dir); dfree(W.p2p_off); dfree(W.p2p_src);
        dfree(W.cp2p); dfree(W.cself);
        dfree(c->ctl);
        if (c->ctl_h) cudaFreeHost(c->ctl_h);
        c->ctl_h = nullptr;
        swap_sets(c);
    }
    dfree(c->pairs); dfree(c->pairs_alt); dfree(c->pair_idx); dfree(c->pair_idx_alt); dfree(c->pairs_out);
    dfree(c->pair_where); dfree(c->res_tc); dfree(c->res_state);
    dfree(c->node_tc); dfree(c->node_ij); dfree(c->node_owner);
    dfree(c->disk_of); dfree(c->doff);
    for (int s = 0; s < 2; s++) {
        dfree(c->fbox[s]);
        dfree(c->froot[s]);
    }
    dfree(c->err_acc);
    if (c->err_acc_h) cudaFreeHost(c->err_acc_h);
    if (c->side) {
        cudaStreamSynchronize(c->side);
        cudaStreamDestroy(c->side);
    }
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->side2) {
        cudaStreamSynchronize(c->side2);
        cudaStreamDestroy(c->side2);
    }
    for (cudaEvent_t e : {c->ev_geo, c->ev_p2m, c->ev_lists, c->ev_near, c->ev_spec0, c->ev_spec})
        if (e) cudaEventDestroy(e);
    for (StepGraph &g : c->graphs) drop_graph(g);
    if (c->gstream) cudaStreamDestroy(c->gstream);
    dfree(c->work_counter);
    for (int i = 0; i < NCORP_NSTAGES; i++)
        for (int k = 0; k < 8; k++)
            for (int e = 0; e < 2; e++)
                if (c->ev[i][k][e]) cudaEventDestroy(c->ev[i][k][e]);
    delete c;
}

const char *ncorp_last_error(const ncorp_ctx *c) {
    if (!c) return "null context";
    return c->err[0] ? c->err : "no error";
}

}  // extern "C"

// ===========================================================================
// Batches of independent disks.  The disks that share (p, theta, dt) form a
// forest: one context whose arrays hold the disks side by side
// (configure_disks), so that every stage of a step is one launch over all of
// them, whatever their number.  ncorp_batch_run advances each forest by k
// steps through one CUDA graph (a snapshot of the state for a rerun, then
// the k steps), cached per (k, buffer rotation); forests run one after
// another on the batch's stream.  A forest whose membership changed is laid out anew
// and its tree and acceleration recomputed at the start of the next run.
// ===========================================================================
namespace {

// Forests run one after another on one stream: each forest's launches cover
// all its disks and fill the GPU, and no forest's cooperative grids then
// share the SMs with another forest's kernels (a grid whose blocks could not
// all be resident together would give up at its first barrier).
constexpr int BATCH_STREAMS = 1;
constexpr double BATCH_DEFAULT_BYTES_PER_MOONLET = 4096.0;   // admission estimate before any measurement
constexpr int64_t BATCH_MEASURE_MIN = 1 << 16;               // forests measured for the estimate: n at least this

// Device arrays owned by the batch: plain allocations that leave the
// context allocation counter alone (the cached graphs of other forests stay
// valid; a forest's own graphs name its arrays).
void balloc(double *&p, size_t count) {
    p = nullptr;
    const cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&p), sizeof(double) * std::max<size_t>(count, 1));
    if (e != cudaSuccess) {
        p = nullptr;
        cudaGetLastError();   // (the failure is reported here; a later check must not see it again)
        throw CudaError(e, "cudaMalloc", __FILE__, __LINE__);
    }
}

void bfree(double *&p) {
    if (p) cudaFree(p);
    p = nullptr;
}

struct BatchDisk {
    int32_t id = 0;
    int64_t n = 0;
    int64_t off = 0;   // first moonlet in the forest's arrays
};

struct RunGraph {
    cudaGraphExec_t exec = nullptr;
    const void *key[4] = {};
    long long nums[4] = {};
    int launches = 0;
};

struct Forest {
    int p = 0;
    double theta = 0.5, dt = 0.0;
    int stream = 0;
    ncorp_ctx *c = nullptr;
    std::vector<BatchDisk> disks;   // in array order
    int64_t n = 0, cap = 0;         // moonlets of all disks; room in the arrays below
    double *pos = nullptr, *vel = nullptr, *m = nullptr, *R = nullptr;   // [cap] side by side, caller order
    bool synced = true;    // pos / vel hold the current state (else it is resident in the context only)
    bool primed = false;   // the context holds the tree and acceleration of the current layout
    size_t ctx_bytes = 0;  // device bytes the context took when created or grown (measured)
    RunGraph graphs[2];
    int graph_next = 0;
    std::vector<int64_t> pairs;   // the last step's pairs of all disks, host copy
    bool pairs_valid = false;
    int64_t n_found = 0;
    int64_t tuned_n = 0;          // moonlets the leaf size was tuned for (0: not tuned)
};

}  // namespace

struct ncorp_batch {
    ncorp_config cfg;
    int device = 0;
    int num_sms = 0;
    cudaStream_t user = nullptr;
    size_t budget = 0;
    double bytes_per_moonlet = BATCH_DEFAULT_BYTES_PER_MOONLET;   // the largest measured so far
    bool measured = false;
    int *flag = nullptr;   // device word of the input check
    bool validate = false; // NCORP_VALIDATE set: check the resident state around every forest step
    bool autotune = true;  // NCORP_AUTOTUNE=0 turns the leaf-size tuner off
    cudaStream_t pool[BATCH_STREAMS] = {};
    cudaEvent_t ev_start = nullptr, ev_done[BATCH_STREAMS] = {};
    std::vector<Forest *> forests;
    std::vector<std::pair<int32_t, Forest *>> where;   // disk id -> forest
    int32_t next_id = 0;
    int64_t fallbacks = 0;
    int64_t launches = 0;
    int64_t tuned = 0;
    char err[512] = {0};
};

namespace {

int batch_fail(ncorp_batch *b, int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b->err, sizeof(b->err), fmt, ap);
    va_end(ap);
    return code;
}

size_t free_bytes() {
    size_t f = 0, t = 0;
    cudaMemGetInfo(&f, &t);
    return f;
}

size_t array_bytes(const Forest &f) { return static_cast<size_t>(f.cap) * 8 * sizeof(double); }

size_t batch_used(const ncorp_batch *b) {
    size_t u = 0;
    for (const Forest *f : b->forests) u += f->ctx_bytes + array_bytes(*f);
    return u;
}

Forest *forest_of(ncorp_batch *b, int32_t id, BatchDisk **disk) {
    for (auto &w : b->where)
        if (w.first == id) {
            for (BatchDisk &d : w.second->disks)
                if (d.id == id) {
                    *disk = &d;
                    return w.second;
                }
        }
    return nullptr;
}

void drop_run_graphs(Forest &f) {
    for (RunGraph &g : f.graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g = RunGraph{};
    }
}

void free_forest(Forest *f) {
    drop_run_graphs(*f);
    if (f->c) ncorp_free(f->c);
    f->c = nullptr;
    bfree(f->pos); bfree(f->vel); bfree(f->m); bfree(f->R);
    delete f;
}

// Arrays of room for `cap` moonlets holding the first `keep` of the old ones.
void regrow_arrays(Forest &f, int64_t cap, int64_t keep, cudaStream_t s) {
    double *np = nullptr, *nv = nullptr, *nm = nullptr, *nr = nullptr;
    try {
        balloc(np, 3 * cap); balloc(nv, 3 * cap); balloc(nm, cap); balloc(nr, cap);
        if (keep > 0) {
            NCORP_CUDA_CHECK(cudaMemcpyAsync(np, f.pos, sizeof(double) * 3 * keep, cudaMemcpyDeviceToDevice, s));
            NCORP_CUDA_CHECK(cudaMemcpyAsync(nv, f.vel, sizeof(double) * 3 * keep, cudaMemcpyDeviceToDevice, s));
            NCORP_CUDA_CHECK(cudaMemcpyAsync(nm, f.m, sizeof(double) * keep, cudaMemcpyDeviceToDevice, s));
            NCORP_CUDA_CHECK(cudaMemcpyAsync(nr, f.R, sizeof(double) * keep, cudaMemcpyDeviceToDevice, s));
        }
        NCORP_CUDA_CHECK(cudaStreamSynchronize(s));
    } catch (...) {
        bfree(np); bfree(nv); bfree(nm); bfree(nr);
        throw;
    }
    bfree(f.pos); bfree(f.vel); bfree(f.m); bfree(f.R);
    f.pos = np; f.vel = nv; f.m = nm; f.R = nr;
    f.cap = cap;
}

// The forest's current state into its arrays (caller order), if it is resident only.
void sync_state(Forest &f) {
    if (f.synced) return;
    ncorp_ctx *c = f.c;
    const int n = static_cast<int>(f.n);
    launch_scatter_aos(c, c->A.x, c->A.y, c->A.z, c->A.perm, f.pos, n, nullptr, nullptr);
    launch_scatter_aos(c, c->A.vx, c->A.vy, c->A.vz, c->A.perm, f.vel, n, nullptr, nullptr);
    NCORP_CUDA_CHECK(cudaStreamSynchronize(c->stream));
    f.synced = true;
}

// Cooperative grids of forests that share the GPU at the same time would be
// capped so that all of them fit on the device together; with the forests
// one after another every forest runs uncapped, with its collision search
// beside the gravity pipeline as in ncorp_step.
int coop_cap(const ncorp_batch *b) {
    const int nf = std::min(static_cast<int>(b->forests.size()), BATCH_STREAMS);
    return nf > 1 ? std::max(16, b->num_sms / nf) : 0;
}

// Lays the forest out for its current disks and computes their tree and
// acceleration from the arrays (which must hold the state); creates the
// context, or creates it anew (returning the memory) when its buffers hold
// more than four times the moonlets the forest has left, and over a million.
// Synchronous.
int prime_forest(ncorp_batch *b, Forest &f) {
    const int n = static_cast<int>(f.n);
    const size_t free0 = free_bytes();
    const int s_tuned = f.c ? f.c->s_tuned : 0;   // (kept by a context created anew)
    if (f.c && f.c->n_cap > 4 * f.n && f.c->n_cap > (1 << 20)) {
        drop_run_graphs(f);
        ncorp_free(f.c);
        f.c = nullptr;
        f.ctx_bytes = 0;
    }
    if (!f.c) {
        const int st = ncorp_init(&f.c, &b->cfg, f.n, b->device, b->pool[f.stream]);
        if (st != NCORP_OK) {
            f.c = nullptr;
            return batch_fail(b, st, "context for %lld moonlets: allocation failed", (long long)f.n);
        }
        f.c->s_tuned = s_tuned;
    }
    ncorp_ctx *c = f.c;
    c->stream = b->pool[f.stream];
    c->coop_max = coop_cap(b);
    drop_run_graphs(f);
    int status = NCORP_OK;
    try {
        std::vector<int64_t> sizes;
        for (const BatchDisk &d : f.disks) sizes.push_back(d.n);
        configure_disks(c, static_cast<int>(sizes.size()), sizes.data());
        ensure_particles(c, n);
        choose_parameters(c, f.p);
        for (int attempt = 0;; attempt++) {
            begin_call(c);
            ensure_both_capacities(c, n);
            reset_ctl(c);
            ParticleSet &A = c->A;
            launch_aos_to_soa(c, f.pos, A.x, A.y, A.z, n);
            launch_aos_to_soa(c, f.vel, A.vx, A.vy, A.vz, n);
            NCORP_CUDA_CHECK(cudaMemcpyAsync(A.m, f.m, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
            NCORP_CUDA_CHECK(cudaMemcpyAsync(A.R, f.R, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
            launch_iota(c, reinterpret_cast<uint32_t *>(A.perm), n);
            build_tree(c, c->A, c->A, c->A, c->Cset, n);
            std::swap(c->A, c->Cset);
            gravity(c, c->A, f.p, f.theta, c->time, false);
            const int err = finish(c);
            if (!finite_ok(c)) {
                status = fail(c, NCORP_EINVAL, "non-finite position");
                break;
            }
            if (err & ERR_TIMEOUT) {
                status = fail(c, NCORP_ETIMEOUT, "device-side barrier timed out");
                break;
            }
            if (err == 0) break;
            if (attempt >= MAX_RETRIES || !grow_after(c, err)) {
                status = fail(c, NCORP_EOVERFLOW, "internal list overflow (flags 0x%x)", err);
                break;
            }
        }
    } catch (const CudaError &e) {
        cudaGetLastError();   // (a non-sticky error is reported once, here)
        status = fail(c, e.code == cudaErrorMemoryAllocation ? NCORP_ENOMEM : NCORP_ECUDA, "%s: %s (%s:%d)", e.expr,
                      cudaGetErrorString(e.code), e.file, e.line);
    }
    const size_t free1 = free_bytes();
    if (free0 > free1) f.ctx_bytes += free0 - free1;
    // footprint per moonlet, from layouts that succeeded (a failed one held whatever it had grabbed) and
    // forests large enough that the fixed minimum capacities do not dominate
    // per moonlet of the context's capacity (a forest that shrank keeps its context's capacity) plus the
    // forest's arrays per moonlet
    if (status == NCORP_OK && f.n >= BATCH_MEASURE_MIN) {
        const double per = static_cast<double>(f.ctx_bytes) / static_cast<double>(std::max<int64_t>(f.n, c->n_cap)) +
                           static_cast<double>(array_bytes(f)) / static_cast<double>(std::max<int64_t>(f.n, f.cap));
        b->bytes_per_moonlet = b->measured ? std::max(b->bytes_per_moonlet, per) : per;
        b->measured = true;
    }
    if (status != NCORP_OK) {
        batch_fail(b, status, "%s", ncorp_last_error(c));
        c->have_state = false;
        c->tree_valid = false;
        if (status == NCORP_ENOMEM) {   // release what the context holds; the next layout starts afresh
            drop_run_graphs(f);
            ncorp_free(c);
            f.c = nullptr;
            f.ctx_bytes = 0;
        }
        return status;
    }
    c->n = n;
    c->have_state = true;
    c->tree_valid = true;
    c->tree_kind = 1;
    c->last_pos = f.pos;
    c->last_vel = f.vel;
    c->last_m = f.m;
    c->last_R = f.R;
    c->last_p = f.p;
    c->last_theta = f.theta;
    c->n_found = 0;
    f.primed = true;
    f.pairs_valid = false;
    f.n_found = 0;
    return NCORP_OK;
}

// The device work of one run: snapshot of the state at its start (into the
// forest's arrays, for a rerun), cleared control blocks, k steps.
void run_body(Forest &f, int k) {
    ncorp_ctx *c = f.c;
    const int n = static_cast<int>(f.n);
    const bool overlap = c->coop_max == 0;
    launch_scatter_aos(c, c->A.x, c->A.y, c->A.z, c->A.perm, f.pos, n, nullptr, nullptr);
    launch_scatter_aos(c, c->A.vx, c->A.vy, c->A.vz, c->A.perm, f.vel, n, nullptr, nullptr);
    reset_ctls(c);
    for (int s = 0; s < k; s++) {
        enqueue_kdk(c, n, f.p, f.theta, f.dt, overlap);
        std::swap(c->A, c->Cset);
    }
}

void run_key(Forest &f, int k, RunGraph &g) {
    ncorp_ctx *c = f.c;
    const void *ptrs[4] = {c->A.x, c->ctl, f.pos, c->stream};
    const long long nums[4] = {k, static_cast<long long>(alloc_generation()), c->coop_max, f.n};
    std::memcpy(g.key, ptrs, sizeof ptrs);
    std::memcpy(g.nums, nums, sizeof nums);
}

// Enqueues a run of k steps on the forest's stream through a cached graph,
// capturing it first when none fits; a run that cannot be captured is
// launched directly.  On return the host state describes the state after
// the run (tree sets and particle sets traded k times).
void enqueue_run(Forest &f, int k) {
    ncorp_ctx *c = f.c;
    RunGraph want;
    run_key(f, k, want);
    for (RunGraph &g : f.graphs)
        if (g.exec && std::memcmp(g.key, want.key, sizeof g.key) == 0 &&
            std::memcmp(g.nums, want.nums, sizeof g.nums) == 0) {
            NCORP_CUDA_CHECK(cudaGraphLaunch(g.exec, c->stream));
            for (int s = 0; s < k; s++) {
                swap_sets(c);
                std::swap(c->A, c->Cset);
            }
            c->cur_n = static_cast<int>(f.n);
            c->grav_p = f.p;
            c->grav_mixed = c->cfg.precision == NCORP_MIXED;
            c->grav_local = true;
            c->launches += g.launches;
            return;
        }
    const Ctrl *ctl0 = c->ctl;
    const double *ax0 = c->A.x;
    const int launches0 = c->launches;
    cudaGraph_t graph = nullptr;
    NCORP_CUDA_CHECK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed));
    bool ok = true;
    try {
        run_body(f, k);
    } catch (const CudaError &) {
        ok = false;
    }
    const cudaError_t end = cudaStreamEndCapture(c->stream, &graph);
    cudaGraphExec_t exec = nullptr;
    if (ok && end == cudaSuccess && graph)
        ok = cudaGraphInstantiateWithFlags(&exec, graph, cudaGraphInstantiateFlagUseNodePriority) == cudaSuccess;
    else ok = false;
    if (graph) cudaGraphDestroy(graph);
    if (!ok) {   // back to the state before the capture, then the same work launched directly
        cudaGetLastError();
        if (exec) cudaGraphExecDestroy(exec);
        if (c->ctl != ctl0) swap_sets(c);
        if (c->A.x != ax0) std::swap(c->A, c->Cset);
        c->launches = launches0;
        run_body(f, k);
        return;
    }
    NCORP_CUDA_CHECK(cudaGraphLaunch(exec, c->stream));
    RunGraph &slot = f.graphs[f.graph_next];
    f.graph_next ^= 1;
    if (slot.exec) cudaGraphExecDestroy(slot.exec);
    slot = want;
    slot.exec = exec;
    slot.launches = c->launches - launches0;
}

// ---- autotuner of the leaf size s (Sect. 3.4.1: cells with more than s
// moonlets are split).  The best s depends on p, on the disks' sizes and on
// how the work spreads over the SMs, so for a forest of TUNE_MIN_MOONLETS to
// TUNE_MAX_MOONLETS moonlets (and again when its size has changed more than
// fourfold) each candidate lays the forest out and times two steps from the
// same state; the fastest is kept.  The candidates are around the default
// for p (32 for p <= 3, else 64).  A configured leaf size disables
// the tuner, as does NCORP_AUTOTUNE=0.
constexpr int64_t TUNE_MIN_MOONLETS = 1 << 15, TUNE_MAX_MOONLETS = 1 << 22;

bool needs_tuning(const ncorp_batch *b, const Forest &f) {
    // (above TUNE_MAX_MOONLETS the trials' larger trees are not worth their memory)
    if (!b->autotune || b->cfg.leaf_size > 0 || f.n < TUNE_MIN_MOONLETS || f.n > TUNE_MAX_MOONLETS) return false;
    return f.tuned_n == 0 || f.n > 4 * f.tuned_n || 4 * f.n < f.tuned_n;
}

int tune_forest(ncorp_batch *b, Forest &f) {
    const int base = f.p <= 3 ? 32 : 64;
    const int cand[4] = {base / 2, (3 * base) / 4, base, (3 * base) / 2};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    NCORP_CUDA_CHECK(cudaEventCreate(&e0));
    NCORP_CUDA_CHECK(cudaEventCreate(&e1));
    float best_ms = 0.0f;
    int best = base, st = NCORP_OK;
    for (int s : cand) {
        if (f.c) f.c->s_tuned = s;
        f.primed = false;
        if ((st = prime_forest(b, f)) != NCORP_OK) break;   // lays out from the arrays (the state to keep)
        ncorp_ctx *c = f.c;
        begin_call(c);
        choose_parameters(c, f.p);
        NCORP_CUDA_CHECK(cudaEventRecord(e0, c->stream));
        run_body(f, 2);   // its snapshot rewrites the arrays with the same state
        NCORP_CUDA_CHECK(cudaEventRecord(e1, c->stream));
        const int err = finish(c, true);
        float ms = 0.0f;
        NCORP_CUDA_CHECK(cudaEventElapsedTime(&ms, e0, e1));
        if (err == 0 && (best_ms == 0.0f || ms < best_ms)) {
            best_ms = ms;
            best = s;
        }
        f.synced = true;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != NCORP_OK) return st;
    f.c->s_tuned = best;
    f.tuned_n = f.n;
    b->tuned++;
    // the capacities the trials needed are not the chosen leaf size's
    f.c->floor_cells = f.c->floor_front = f.c->floor_m2l = f.c->floor_p2p = f.c->floor_self = 0;
    f.primed = false;
    return prime_forest(b, f);
}

// ---- validation mode: invariants of a forest's resident state, checked by
// kernels that only read inside the bounds they check (a violated invariant
// is recorded, never followed).  bad[0] = first violated invariant, bad[1] =
// its index, bad[2] = the offending value, bad[3] = violations.
struct ValidateArgs {
    const int *perm;
    int n;
    const unsigned short *disk_of;
    const int *doff;
    int nd;
    const int *first, *count, *nchild, *child0, *parent, *leaves, *leaf_of;
    int cap;
    const Ctrl *ctl;
    int *hist;   // [n], zero on entry
    int *bad;    // [4], zero on entry
};

__device__ void report(int *bad, int code, int idx, int val) {
    if (atomicCAS(&bad[0], 0, code) == 0) {
        bad[1] = idx;
        bad[2] = val;
    }
    atomicAdd(&bad[3], 1);
}

__global__ void k_validate(ValidateArgs V) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    const int nc = V.ctl->n_cells, nl = V.ctl->n_leaves, roots = V.ctl->nd;
    if (tid == 0) {
        if (nc < 1 || nc > V.cap) report(V.bad, 3, nc, V.cap);
        if (nl < 1 || nl > nc) report(V.bad, 7, nl, nc);
        if (roots != V.nd) report(V.bad, 11, roots, V.nd);
    }
    for (int i = tid; i < V.n; i += nt) {
        const int u = V.perm[i];
        if (u < 0 || u >= V.n) report(V.bad, 1, i, u);
        else atomicAdd(&V.hist[u], 1);
        if (V.disk_of) {
            const int d = V.disk_of[i];
            if (d >= V.nd || V.doff[d] > i || V.doff[d + 1] <= i) report(V.bad, 2, i, d);
        }
    }
    const int ncv = min(max(nc, 0), V.cap);
    for (int c = tid; c < ncv; c += nt) {
        const int f = V.first[c], k = V.count[c];
        if (f < 0 || k < 1 || f > V.n - k) report(V.bad, 4, c, f);
        const int ch = V.nchild[c];
        if (ch < 0 || ch > 8) report(V.bad, 12, c, ch);
        else if (ch > 0) {
            const int c0 = V.child0[c];
            if (c0 <= c || c0 > ncv - ch) report(V.bad, 5, c, c0);
        }
        const int pa = V.parent[c];
        if (c < V.nd ? pa != -1 : (pa < 0 || pa >= c)) report(V.bad, 6, c, pa);
    }
    const int nlv = min(max(nl, 0), ncv);
    for (int t = tid; t < nlv; t += nt) {
        const int l = V.leaves[t];
        if (l < 0 || l >= ncv || V.nchild[l] != 0) report(V.bad, 8, t, l);
    }
    for (int i = tid; i < V.n; i += nt) {
        const int l = V.leaf_of[i];
        if (l < 0 || l >= ncv || V.first[l] > i || i - V.first[l] >= V.count[l]) report(V.bad, 9, i, l);
    }
}

__global__ void k_validate_perm(ValidateArgs V) {
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < V.n; u += gridDim.x * blockDim.x)
        if (V.hist[u] != 1) report(V.bad, 10, u, V.hist[u]);
}

// NCORP_OK, or NCORP_ESTATE with the first violated invariant in the batch's message.
int validate_forest(ncorp_batch *b, Forest &f, const char *when) {
    ncorp_ctx *c = f.c;
    const int n = static_cast<int>(f.n);
    if (c->n != n || c->n_cap < n || c->nd != static_cast<int>(f.disks.size()))
        return batch_fail(b, NCORP_ESTATE, "validation %s: host state n %d / %lld, cap %lld, disks %d / %zu", when,
                          c->n, (long long)f.n, (long long)c->n_cap, c->nd, f.disks.size());
    int *scratch = nullptr;
    int hbad[4] = {0, 0, 0, 0};
    NCORP_CUDA_CHECK(cudaMalloc(reinterpret_cast<void **>(&scratch), sizeof(int) * (n + 4)));
    try {
        NCORP_CUDA_CHECK(cudaMemsetAsync(scratch, 0, sizeof(int) * (n + 4), c->stream));
        ValidateArgs V;
        V.perm = c->A.perm;
        V.n = n;
        V.disk_of = c->nd > 1 ? c->disk_of : nullptr;
        V.doff = c->doff;
        V.nd = c->nd;
        const Cells &C = c->cells;
        V.first = C.first; V.count = C.count; V.nchild = C.nchild; V.child0 = C.child0; V.parent = C.parent;
        V.leaves = C.leaves; V.leaf_of = C.leaf_of; V.cap = C.cap;
        V.ctl = c->ctl;
        V.hist = scratch;
        V.bad = scratch + n;
        k_validate<<<4 * b->num_sms, 256, 0, c->stream>>>(V);
        k_validate_perm<<<4 * b->num_sms, 256, 0, c->stream>>>(V);
        NCORP_CUDA_CHECK(cudaGetLastError());
        NCORP_CUDA_CHECK(cudaMemcpyAsync(hbad, scratch + n, sizeof(hbad), cudaMemcpyDeviceToHost, c->stream));
        NCORP_CUDA_CHECK(cudaStreamSynchronize(c->stream));
    } catch (...) {
        cudaFree(scratch);
        throw;
    }
    cudaFree(scratch);
    if (hbad[0])
        return batch_fail(b, NCORP_ESTATE, "validation %s (forest p = %d, %zu disks, n = %d): invariant %d at %d "
                          "(value %d), %d violations", when, f.p, f.disks.size(), n, hbad[0], hbad[1], hbad[2],
                          hbad[3]);
    return NCORP_OK;
}

__global__ void k_count_nonfinite(const double *__restrict__ a, int64_t n, int *bad) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(a[i]));
        if ((u & 0x7ff0000000000000ull) == 0x7ff0000000000000ull) atomicOr(bad, 1);
    }
}

}  // namespace

extern "C" {

int ncorp_batch_create(ncorp_batch **out, const ncorp_config *cfg, size_t hbm_budget_bytes, void *cuda_stream) {
    if (!out || !cfg) return NCORP_EINVAL;
    *out = nullptr;
    if (cfg->precision != NCORP_FP64 && cfg->precision != NCORP_MIXED) return NCORP_EINVAL;
    if (!(cfg->resolve_f == 0.0 || (cfg->resolve_f >= 1.0 && cfg->resolve_f <= 2.0))) return NCORP_EINVAL;
    if (cfg->star_mass != 0.0) return NCORP_EINVAL;   // the star's tide needs each disk's own time
    ncorp_batch *b = new (std::nothrow) ncorp_batch();
    if (!b) return NCORP_ENOMEM;
    b->cfg = *cfg;
    b->budget = hbm_budget_bytes;
    b->user = static_cast<cudaStream_t>(cuda_stream);
    b->validate = env_int("NCORP_VALIDATE", 0, 0, 1) != 0;
    b->autotune = env_int("NCORP_AUTOTUNE", 1, 0, 1) != 0;
    int least = 0, greatest = 0;
    bool ok = cudaGetDevice(&b->device) == cudaSuccess &&
              cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device) == cudaSuccess &&
              cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->ev_start, cudaEventDisableTiming) == cudaSuccess &&
              cudaMalloc(reinterpret_cast<void **>(&b->flag), sizeof(int)) == cudaSuccess;
    // the forests' main chains at the highest priority (their side streams are at the lowest)
    for (int s = 0; ok && s < BATCH_STREAMS; s++)
        ok = cudaStreamCreateWithPriority(&b->pool[s], cudaStreamNonBlocking, greatest) == cudaSuccess &&
             cudaEventCreateWithFlags(&b->ev_done[s], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        ncorp_batch_free(b);
        return NCORP_ECUDA;
    }
    *out = b;
    return NCORP_OK;
}

int ncorp_batch_add_disk(ncorp_batch *b, const double *positions, const double *velocities, const double *masses,
                         const double *radii, int64_t n, int p, double theta, double dt, int32_t *disk_id) {
    if (!b) return NCORP_EINVAL;
    if (!positions || !velocities || !masses || !radii || !disk_id)
        return batch_fail(b, NCORP_EINVAL, "null pointer");
    if (n < 1 || n > (int64_t(1) << 30)) return batch_fail(b, NCORP_EINVAL, "n = %lld out of range", (long long)n);
    if (p < 1 || p > MAXP) return batch_fail(b, NCORP_EINVAL, "p = %d outside 1..6", p);
    if (!(theta > 0.0 && theta < 1.0)) return batch_fail(b, NCORP_EINVAL, "theta = %g outside (0, 1)", theta);
    if (!(dt > 0.0) || !std::isfinite(dt)) return batch_fail(b, NCORP_EINVAL, "dt must be > 0");
    if (cudaSetDevice(b->device) != cudaSuccess) return batch_fail(b, NCORP_ECUDA, "cudaSetDevice failed");
    Forest *f = nullptr;
    // the forest of (p, theta, dt) with room for one more disk (a full one: the disk starts another)
    for (Forest *g : b->forests)
        if (g->p == p && g->theta == theta && g->dt == dt && static_cast<int>(g->disks.size()) < NCORP_MAX_DISKS &&
            g->n + n <= (int64_t(1) << 30))
            f = g;
    // admission by device memory: what the batch holds plus the new disk's share at the largest
    // footprint per moonlet measured so far
    // (with a margin of one half: a forest's buffers grow in steps, and an overflow doubles a list)
    const size_t used = batch_used(b);
    const size_t need = static_cast<size_t>(1.5 * b->bytes_per_moonlet * static_cast<double>(n));
    if (b->budget && used + need > b->budget)
        return batch_fail(b, NCORP_ENOMEM, "device-memory budget exceeded: %zu + %zu > %zu bytes", used, need,
                          b->budget);
    if (b->budget && free_bytes() < need)
        return batch_fail(b, NCORP_ENOMEM, "device-memory budget: %zu bytes free, %zu needed", free_bytes(), need);
    const bool fresh = f == nullptr;
    if (fresh) {
        f = new (std::nothrow) Forest();
        if (!f) return batch_fail(b, NCORP_ENOMEM, "host allocation failed");
        f->p = p;
        f->theta = theta;
        f->dt = dt;
        f->stream = static_cast<int>(b->forests.size()) % BATCH_STREAMS;
    }
    cudaStream_t s = b->pool[f->stream];
    int *bad = b->flag;
    try {
        if (fresh) {   // the context now, so that it reads the environment at the time of the first add
            const size_t free0 = free_bytes();
            const int st = ncorp_init(&f->c, &b->cfg, n, b->device, s);
            if (st != NCORP_OK) {
                f->c = nullptr;
                free_forest(f);
                return batch_fail(b, st, "context for %lld moonlets: allocation failed", (long long)n);
            }
            const size_t free1 = free_bytes();
            f->ctx_bytes = free0 > free1 ? free0 - free1 : 0;
        } else {
            sync_state(*f);
        }
        if (f->n + n > f->cap) regrow_arrays(*f, std::max(f->n + n, f->cap * 3 / 2), f->n, s);
        const int64_t o = f->n;
        NCORP_CUDA_CHECK(cudaMemcpyAsync(f->pos + 3 * o, positions, sizeof(double) * 3 * n, cudaMemcpyDefault, s));
        NCORP_CUDA_CHECK(cudaMemcpyAsync(f->vel + 3 * o, velocities, sizeof(double) * 3 * n, cudaMemcpyDefault, s));
        NCORP_CUDA_CHECK(cudaMemcpyAsync(f->m + o, masses, sizeof(double) * n, cudaMemcpyDefault, s));
        NCORP_CUDA_CHECK(cudaMemcpyAsync(f->R + o, radii, sizeof(double) * n, cudaMemcpyDefault, s));
        NCORP_CUDA_CHECK(cudaMemsetAsync(bad, 0, sizeof(int), s));
        const int g = std::max(1, std::min(static_cast<int>((3 * n + 255) / 256), 4 * b->num_sms));
        k_count_nonfinite<<<g, 256, 0, s>>>(f->pos + 3 * o, 3 * n, bad);
        k_count_nonfinite<<<g, 256, 0, s>>>(f->vel + 3 * o, 3 * n, bad);
        NCORP_CUDA_CHECK(cudaGetLastError());
        int hbad = 0;
        NCORP_CUDA_CHECK(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
        NCORP_CUDA_CHECK(cudaStreamSynchronize(s));
        if (hbad) {   // the disk is not added (its rows past f->n are ignored)
            if (fresh) free_forest(f);
            return batch_fail(b, NCORP_EINVAL, "non-finite position or velocity");
        }
    } catch (const CudaError &e) {
        cudaGetLastError();   // (a non-sticky error is reported once, here)
        if (fresh) free_forest(f);
        return batch_fail(b, e.code == cudaErrorMemoryAllocation ? NCORP_ENOMEM : NCORP_ECUDA, "%s: %s", e.expr,
                          cudaGetErrorString(e.code));
    }
    BatchDisk d;
    d.id = b->next_id++;
    d.n = n;
    d.off = f->n;
    f->disks.push_back(d);
    f->n += n;
    f->primed = false;
    f->pairs_valid = false;
    if (fresh) b->forests.push_back(f);
    b->where.emplace_back(d.id, f);
    *disk_id = d.id;
    return NCORP_OK;
}

int ncorp_batch_run(ncorp_batch *b, int n_steps) {
    if (!b) return NCORP_EINVAL;
    if (n_steps < 0) return batch_fail(b, NCORP_EINVAL, "n_steps < 0");
    b->launches = 0;
    if (b->forests.empty()) return NCORP_OK;
    try {
        NCORP_CUDA_CHECK(cudaSetDevice(b->device));
        // forests whose disks changed: new layout, tree and acceleration
        for (Forest *f : b->forests)
            if (!f->primed) {
                int st = prime_forest(b, *f);
                if (st != NCORP_OK) return st;
                b->launches += f->c->launches;
                if (b->validate && (st = validate_forest(b, *f, "after the layout")) != NCORP_OK) return st;
            }
        for (Forest *f : b->forests)
            if (needs_tuning(b, *f)) {
                const int st = tune_forest(b, *f);
                if (st != NCORP_OK) return st;
            }
        if (n_steps == 0) return NCORP_OK;
        if (b->validate) {   // one forest and one step at a time, the resident state checked around each
            for (int k = 0; k < n_steps; k++)
                for (Forest *f : b->forests) {
                    ncorp_ctx *c = f->c;
                    c->stream = b->pool[f->stream];
                    c->coop_max = coop_cap(b);
                    int st = validate_forest(b, *f, "before a step");
                    if (st != NCORP_OK) return st;
                    begin_call(c);
                    choose_parameters(c, f->p);
                    run_body(*f, 1);
                    const int err = finish(c, true);
                    f->synced = false;
                    f->pairs_valid = false;
                    b->launches += c->launches;
                    if (err != 0) {   // the step again from its snapshot, buffers growing, as after a run
                        b->fallbacks++;
                        c->have_state = false;
                        c->tree_valid = false;
                        st = ncorp_step(c, f->pos, f->vel, f->m, f->R, f->n, f->p, f->theta, f->dt);
                        if (st != NCORP_OK)
                            return batch_fail(b, st == NCORP_ENOMEM ? NCORP_EOVERFLOW : st, "validation step: %s",
                                              ncorp_last_error(c));
                        f->synced = true;
                        f->n_found = c->n_found;
                    } else {
                        c->n_found = c->cfg.collisions ? c->alt.ctl_h->n_found : 0;
                        c->pairs_sorted = false;
                        c->time += f->dt;
                        f->n_found = c->n_found;
                    }
                    st = validate_forest(b, *f, "after a step");
                    if (st != NCORP_OK) return st;
                }
            return NCORP_OK;
        }
        NCORP_CUDA_CHECK(cudaEventRecord(b->ev_start, b->user));
        for (int s = 0; s < BATCH_STREAMS; s++) NCORP_CUDA_CHECK(cudaStreamWaitEvent(b->pool[s], b->ev_start, 0));
        const int cap = coop_cap(b);
        for (Forest *f : b->forests) {
            ncorp_ctx *c = f->c;
            c->stream = b->pool[f->stream];
            if (c->coop_max != cap) {
                c->coop_max = cap;
                drop_run_graphs(*f);
            }
            begin_call(c);
            choose_parameters(c, f->p);
            enqueue_run(*f, n_steps);
            NCORP_CUDA_CHECK(cudaMemcpyAsync(c->ctl_h, c->ctl, sizeof(Ctrl), cudaMemcpyDeviceToHost, c->stream));
            NCORP_CUDA_CHECK(cudaMemcpyAsync(c->alt.ctl_h, c->alt.ctl, sizeof(Ctrl), cudaMemcpyDeviceToHost, c->stream));
            NCORP_CUDA_CHECK(cudaMemcpyAsync(c->err_acc_h, c->err_acc, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        }
        for (int s = 0; s < BATCH_STREAMS; s++) {
            NCORP_CUDA_CHECK(cudaEventRecord(b->ev_done[s], b->pool[s]));
            NCORP_CUDA_CHECK(cudaStreamWaitEvent(b->user, b->ev_done[s], 0));
        }
        for (int s = 0; s < BATCH_STREAMS; s++) NCORP_CUDA_CHECK(cudaStreamSynchronize(b->pool[s]));
    } catch (const CudaError &e) {
        cudaGetLastError();   // (a non-sticky error is reported once, here)
        for (Forest *f : b->forests) {
            f->primed = false;   // the arrays hold the state at the start of the run at the latest
            f->synced = true;
            if (f->c) {
                f->c->have_state = false;
                f->c->tree_valid = false;
            }
        }
        return batch_fail(b, NCORP_ECUDA, "%s: %s (%s:%d)", e.expr, cudaGetErrorString(e.code), e.file, e.line);
    }
    for (Forest *f : b->forests) {
        ncorp_ctx *c = f->c;
        b->launches += c->launches;
        f->synced = false;
        f->pairs_valid = false;
        const int err = c->ctl_h->err | c->alt.ctl_h->err | *c->err_acc_h;
        if (err & ERR_TIMEOUT) c->radix_dirty = true;
        if (err == 0) {
            c->n_found = c->cfg.collisions ? c->alt.ctl_h->n_found : 0;
            c->pairs_sorted = false;
            c->time += n_steps * f->dt;
            record_stats(c, true, c->alt.ctl_h);
            c->stats[NCORP_STAT_COL_FOUND] = c->n_found;
            f->n_found = c->n_found;
            continue;
        }
        // A list overflowed or a barrier gave up in some step: rerun the forest from the state at the
        // start of the run (in its arrays), one synchronous step at a time, buffers growing as needed.
        b->fallbacks++;
        f->synced = true;
        c->have_state = false;
        c->tree_valid = false;
        drop_run_graphs(*f);
        const size_t free0 = free_bytes();
        for (int k = 0; k < n_steps; k++) {
            const int st = ncorp_step(c, f->pos, f->vel, f->m, f->R, f->n, f->p, f->theta, f->dt);
            if (st != NCORP_OK) {
                f->primed = false;
                // (NCORP_ENOMEM is kept for runs that stepped nothing: here other forests have run)
                return batch_fail(b, st == NCORP_ENOMEM ? NCORP_EOVERFLOW : st, "forest of %zu disks (p = %d): %s",
                                  f->disks.size(), f->p, ncorp_last_error(c));
            }
            b->launches += c->launches;
        }
        const size_t free1 = free_bytes();
        if (free0 > free1) f->ctx_bytes += free0 - free1;
        f->primed = true;
        f->synced = true;
        f->n_found = c->n_found;
    }
    return NCORP_OK;
}

int ncorp_batch_get_state(ncorp_batch *b, int32_t disk_id, double *positions, double *velocities) {
    if (!b) return NCORP_EINVAL;
    BatchDisk *d = nullptr;
    Forest *f = forest_of(b, disk_id, &d);
    if (!f) return batch_fail(b, NCORP_EINVAL, "no disk %d", disk_id);
    if (!positions || !velocities) return batch_fail(b, NCORP_EINVAL, "null pointer");
    try {
        NCORP_CUDA_CHECK(cudaSetDevice(b->device));
        sync_state(*f);
        cudaStream_t s = b->pool[f->stream];
        NCORP_CUDA_CHECK(cudaMemcpyAsync(positions, f->pos + 3 * d->off, sizeof(double) * 3 * d->n, cudaMemcpyDefault, s));
        NCORP_CUDA_CHECK(cudaMemcpyAsync(velocities, f->vel + 3 * d->off, sizeof(double) * 3 * d->n, cudaMemcpyDefault,
                                         s));
        NCORP_CUDA_CHECK(cudaStreamSynchronize(s));
    } catch (const CudaError &e) {
        cudaGetLastError();   // (a non-sticky error is reported once, here)
        return batch_fail(b, NCORP_ECUDA, "%s: %s (%s:%d)", e.expr, cudaGetErrorString(e.code), e.file, e.line);
    }
    return NCORP_OK;
}

int ncorp_batch_collisions(ncorp_batch *b, int32_t disk_id, int64_t *pairs, int64_t cap, int64_t *n_pairs) {
    if (!b) return NCORP_EINVAL;
    BatchDisk *d = nullptr;
    Forest *f = forest_of(b, disk_id, &d);
    if (!f) return batch_fail(b, NCORP_EINVAL, "no disk %d", disk_id);
    if (cap < 0 || (cap > 0 && !pairs)) return batch_fail(b, NCORP_EINVAL, "bad pair buffer");
    if (!f->pairs_valid) {   // the forest's pairs of its last step, once per run (indices of its arrays)
        f->pairs.assign(2 * static_cast<size_t>(f->n_found), 0);
        if (f->n_found > 0 && f->primed) {
            int64_t got = 0;
            const int st = ncorp_collisions(f->c, f->pairs.data(), f->n_found, &got);
            if (st != NCORP_OK) return batch_fail(b, st, "%s", ncorp_last_error(f->c));
        } else {
            f->pairs.clear();
        }
        f->pairs_valid = true;
    }
    // rows are sorted by their first index and a pair never spans two disks: the disk's rows are one range
    const int64_t rows = static_cast<int64_t>(f->pairs.size() / 2);
    int64_t lo = 0, hi = rows;
    while (lo < hi) {
        const int64_t mid = (lo + hi) / 2;
        if (f->pairs[2 * mid] < d->off) lo = mid + 1;
        else hi = mid;
    }
    int64_t e = lo;
    while (e < rows && f->pairs[2 * e] < d->off + d->n) e++;
    const int64_t k = e - lo;
    if (n_pairs) *n_pairs = k;
    const int64_t w = std::min(k, cap);
    if (w > 0) {
        std::vector<int64_t> out(2 * w);
        for (int64_t r = 0; r < w; r++) {
            out[2 * r] = f->pairs[2 * (lo + r)] - d->off;
            out[2 * r + 1] = f->pairs[2 * (lo + r) + 1] - d->off;
        }
        if (cudaMemcpy(pairs, out.data(), sizeof(int64_t) * 2 * w, cudaMemcpyDefault) != cudaSuccess)
            return batch_fail(b, NCORP_ECUDA, "copy of the pairs failed");
    }
    if (k > cap) return batch_fail(b, NCORP_EOVERFLOW, "%lld pairs found, room for %lld", (long long)k, (long long)cap);
    return NCORP_OK;
}

int ncorp_batch_remove_disk(ncorp_batch *b, int32_t disk_id, double *positions, double *velocities) {
    if (!b) return NCORP_EINVAL;
    BatchDisk *dp = nullptr;
    Forest *f = forest_of(b, disk_id, &dp);
    if (!f) return batch_fail(b, NCORP_EINVAL, "no disk %d", disk_id);
    if ((positions == nullptr) != (velocities == nullptr))
        return batch_fail(b, NCORP_EINVAL, "give both output arrays or neither");
    if (positions) {
        const int st = ncorp_batch_get_state(b, disk_id, positions, velocities);
        if (st != NCORP_OK) return st;
    }
    const BatchDisk d = *dp;
    try {
        NCORP_CUDA_CHECK(cudaSetDevice(b->device));
        for (size_t i = 0; i < b->where.size(); i++)
            if (b->where[i].first == disk_id) {
                b->where.erase(b->where.begin() + i);
                break;
            }
        if (f->disks.size() == 1) {   // the forest's last disk: release all of it
            for (size_t i = 0; i < b->forests.size(); i++)
                if (b->forests[i] == f) {
                    b->forests.erase(b->forests.begin() + i);
                    break;
                }
            free_forest(f);
            return NCORP_OK;
        }
        sync_state(*f);
        // the disks after it move down by d.n moonlets (through a copy: the ranges may overlap)
        const int64_t tail = f->n - (d.off + d.n);
        if (tail > 0) {
            cudaStream_t s = b->pool[f->stream];
            double *tmp = nullptr;
            const bool own = !f->c || f->c->n_cap < tail;   // the context's staging buffer: 3 n_cap doubles
            if (own) balloc(tmp, 3 * tail);
            else tmp = f->c->stage;
            double *src[4] = {f->pos + 3 * (d.off + d.n), f->vel + 3 * (d.off + d.n), f->m + d.off + d.n,
                              f->R + d.off + d.n};
            double *dst[4] = {f->pos + 3 * d.off, f->vel + 3 * d.off, f->m + d.off, f->R + d.off};
            const int64_t len[4] = {3 * tail, 3 * tail, tail, tail};
            try {
                for (int a = 0; a < 4; a++) {
                    NCORP_CUDA_CHECK(cudaMemcpyAsync(tmp, src[a], sizeof(double) * len[a], cudaMemcpyDeviceToDevice, s));
                    NCORP_CUDA_CHECK(cudaMemcpyAsync(dst[a], tmp, sizeof(double) * len[a], cudaMemcpyDeviceToDevice, s));
                }
                NCORP_CUDA_CHECK(cudaStreamSynchronize(s));
            } catch (...) {
                if (own) bfree(tmp);
                throw;
            }
            if (own) bfree(tmp);
        }
    } catch (const CudaError &e) {
        cudaGetLastError();   // (a non-sticky error is reported once, here)
        return batch_fail(b, NCORP_ECUDA, "%s: %s (%s:%d)", e.expr, cudaGetErrorString(e.code), e.file, e.line);
    }
    for (size_t i = 0; i < f->disks.size(); i++)
        if (f->disks[i].id == disk_id) {
            f->disks.erase(f->disks.begin() + i);
            break;
        }
    for (BatchDisk &o : f->disks)
        if (o.off > d.off) o.off -= d.n;
    f->n -= d.n;
    f->primed = false;
    f->pairs_valid = false;
    return NCORP_OK;
}

int ncorp_batch_info(const ncorp_batch *b, int64_t *info, int n_info) {
    if (!b || !info || n_info < 0) return NCORP_EINVAL;
    int64_t moonlets = 0, disks = 0, leaf = 0, largest = -1;
    for (const Forest *f : b->forests) {
        moonlets += f->n;
        disks += static_cast<int64_t>(f->disks.size());
        if (f->n > largest && f->c) {
            largest = f->n;
            leaf = f->c->s;
        }
    }
    const int64_t v[NCORP_BATCH_NINFO] = {disks, moonlets, static_cast<int64_t>(batch_used(b)),
                                          static_cast<int64_t>(b->forests.size()), b->fallbacks, b->launches,
                                          b->tuned, leaf};
    for (int i = 0; i < n_info && i < NCORP_BATCH_NINFO; i++) info[i] = v[i];
    return NCORP_OK;
}

void ncorp_batch_free(ncorp_batch *b) {
    if (!b) return;
    cudaSetDevice(b->device);
    for (int s = 0; s < BATCH_STREAMS; s++)
        if (b->pool[s]) cudaStreamSynchronize(b->pool[s]);
    for (Forest *f : b->forests) free_forest(f);
    b->forests.clear();
    for (int s = 0; s < BATCH_STREAMS; s++) {
        if (b->pool[s]) cudaStreamDestroy(b->pool[s]);
        if (b->ev_done[s]) cudaEventDestroy(b->ev_done[s]);
    }
    if (b->ev_start) cudaEventDestroy(b->ev_start);
    if (b->flag) cudaFree(b->flag);
    delete b;
}

const char *ncorp_batch_last_error(const ncorp_batch *b) {
    if (!b) return "null batch";
    return b->err[0] ? b->err : "no error";
}

}  // extern "C"
