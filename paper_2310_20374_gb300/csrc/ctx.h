// ctx.h -- host-side context of the falcON step library and the launchers
// each translation unit provides.
#pragma once
#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>

#include "../../include/ncorp.h"
#include "common.cuh"

namespace ncorp {

// One set of per-moonlet arrays in tree (Hilbert) order, SoA.
struct ParticleSet {
    double *x = nullptr, *y = nullptr, *z = nullptr;
    double *vx = nullptr, *vy = nullptr, *vz = nullptr;
    double *m = nullptr, *R = nullptr;
    double *ax = nullptr, *ay = nullptr, *az = nullptr;   // total acceleration (mutual + external)
    int *perm = nullptr;                                   // caller index of each moonlet
    uint32_t *qx = nullptr, *qy = nullptr, *qz = nullptr; // quantised coordinates
    uint64_t *key = nullptr;                               // Hilbert key
    float4 *hi4 = nullptr;    // (x, y, z) rounded to FP32, and mu = G m
    float4 *lo4 = nullptr;    // (x, y, z) - hi, rounded to FP32 (double-float position)
};

struct Cells {
    int cap = 0;
    int *level = nullptr, *first = nullptr, *count = nullptr, *child0 = nullptr, *nchild = nullptr,
        *parent = nullptr, *arrive = nullptr, *arrive_m = nullptr;   // arrival counters: collision climb, multipoles
    uint32_t *cx = nullptr, *cy = nullptr, *cz = nullptr;
    double *M = nullptr, *sx = nullptr, *sy = nullptr, *sz = nullptr, *rmax = nullptr, *rcrit = nullptr,
           *rho = nullptr;                                 // gravity climb
    double *bx = nullptr, *by = nullptr, *bz = nullptr, *bmax = nullptr, *bcrit = nullptr;  // collision climb
    // FP32 copies for the walk's first test and the FP32 kernels:
    float4 *gh = nullptr;     // gravity centre rounded to FP32 (xyz), r_crit rounded to FP32 (w)
    float4 *gl = nullptr;     // centre - hi (xyz), rho (w, exact power of two)
    float4 *bh = nullptr;     // collision centre hi (xyz), collision r_crit (w)
    float4 *bl = nullptr;     // collision centre lo (xyz)
    void *Mh = nullptr;       // [cap][num_m(p)] multipoles (float or double)
    void *Ch = nullptr;       // [cap][num_c(p)] local coefficients of the cell's own M2L (float or double)
    float *Ch_lo = nullptr;   // [cap][3] mixed precision: low parts of the order-1 coefficients of Ch
    void *Cf = nullptr;       // [cap][num_c(p)] complete local expansion after the descent
    float *Cf_lo = nullptr;   // [cap][3] mixed precision: low parts of the order-1 coefficients of Cf
                              // (double-float: the field is the sum of the whole far field)
    int *leaves = nullptr;    // leaf cell ids
    int *bounds = nullptr;    // [cap][9] scratch of the build
    int *maker = nullptr;     // [cap] scratch of the build: block that made the cell
    int *before = nullptr;    // [cap] scratch of the build: children of its maker's earlier cells
    int *blocksum = nullptr;  // per-block scratch of cooperative kernels
    unsigned *done = nullptr; // [cap] descent: epoch in which the cell's complete expansion was written
    int *leaf_of = nullptr;   // [leaf_of_cap] leaf of each moonlet of the tree (tree order)
    double *rc_spec = nullptr;// [leaf_of_cap] fused walk: each moonlet's R + dt |v| bound the tree's collision
                              // geometry was computed with (tree order)
    int leaf_of_cap = 0;
};

struct WalkLists {
    int front_cap = 0, m2l_cap = 0, p2p_cap = 0, self_cap = 0, m2l_dir_cap = 0, p2p_dir_cap = 0;
    int2 *front[2] = {nullptr, nullptr};
    int *front_count = nullptr;   // [MAX_ITERS + 1]
    int2 *m2l = nullptr;          // well-separated cell pairs
    int2 *p2p = nullptr;          // leaf-leaf direct pairs
    int *self = nullptr;          // leaves interacting with themselves
    int *cnt = nullptr, *offs = nullptr, *cursor = nullptr;     // per-cell counting sort scratch [cap+1]
    int2 *m2l_dir = nullptr;      // (target, source) grouped by target
    int *p2p_off = nullptr;       // [cap+1] offsets of each target leaf's sources
    int2 *p2p_src = nullptr;      // each directed entry's source leaf as (first moonlet, moonlet count)
    int2 *cp2p = nullptr;         // collision walk: leaf pairs to test [p2p_cap]
    int *cself = nullptr;         // collision walk: leaves to test within [self_cap]
};

// One tree with everything a walk over it produces: cells, walk lists and
// the control block (tree description, counters, error word).  A context
// holds two, so that the collision search on the tree of x_n can run while
// the tree of x_{n+1} is built and walked.
struct TreeSet {
    Cells cells;
    WalkLists wl;
    Ctrl *ctl = nullptr;      // device
    Ctrl *ctl_h = nullptr;    // pinned host mirror
};

constexpr int WALK_MAX_ITERS = 96;

// Grid of a cooperative launch: the given blocks per SM, capped by the
// context's limit so that the cooperative grids of contexts driven on
// concurrent streams fit on the device together.
inline int coop_blocks(const ncorp_ctx *c, int per_sm);

// Every device (re)allocation of the library bumps this counter; a captured
// step graph is valid only for the value it was captured under.
unsigned long long alloc_generation();
void bump_alloc_generation();
void ensure_radix_scratch(ncorp_ctx *c, int n);
unsigned radix_epoch_limit();
void sort_near_sorted(ncorp_ctx *c, uint64_t *keys, uint32_t *idx, uint64_t *keys_alt, uint32_t *idx_alt, int n,
                      int bits);
constexpr int RESORT_MOVERS_CAP = 65536;  // movers of the nearly-sorted key sort (RS_MOVERS_MAX)
constexpr int RESORT_BLOCKS_CAP = 4096;

}  // namespace ncorp

// A captured CUDA graph of one resident step (see ncorp_step) and the host
// state it was captured for.
struct StepGraph {
    cudaGraphExec_t exec = nullptr;
    const void *key[6] = {};
    long long nums[10] = {};
    int launches = 0;
};

struct ncorp_ctx {
    ncorp_config cfg;
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    int coop_max = 0;               // cap on cooperative grid sizes (0: none); set when contexts run concurrently
    int side_blocks = 64;           // cap on the cooperative grids of a step's collision search (side stream)
    char err[512] = {0};

    int64_t n_cap = 0;
    int n = 0;
    // a forest (nd > 1): independent disks in the same arrays, disk d = moonlets [doff[d], doff[d + 1])
    int nd = 1;
    int forest_n = 0;                    // moonlets of all disks (nd > 1)
    int disk_of_cap = 0, nd_cap = 0;     // room in disk_of / doff, fbox, froot (kept across layouts)
    unsigned short *disk_of = nullptr;   // device [forest_n]
    int *doff = nullptr;                 // device [nd + 1]
    unsigned long long *fbox[2] = {nullptr, nullptr};   // device [nd][6] per tree set
    double *froot[2] = {nullptr, nullptr};              // device [nd][4] per tree set
    int cur_n = 0;                  // moonlets of the tree being built or walked
    int p = 0;
    double theta = 0.5;
    int s = 0;
    int s_tuned = 0;                // leaf size chosen by a batch's autotuner (0: none)
    long long g_cs = 0, g_pre = 0, g_post = 0;
    long long c_cs = 12, c_pre = 0, c_post = 16;

    ncorp::ParticleSet A, B, Cset;   // A: resident state; B: scratch (half-kicked v, drifted x); Cset: next order
    double *amx = nullptr, *amy = nullptr, *amz = nullptr;   // mutual acceleration (tree order)
    float4 *cv4 = nullptr;           // collision search, per moonlet: velocity rounded to FP32 (xyz) and
                                     // R + dt |v| rounded up (w)
    uint64_t *key_alt = nullptr;
    uint64_t *resort_mkey = nullptr;   // nearly-sorted key sort: movers and per-block counts
    uint32_t *resort_midx = nullptr;
    int *resort_bcount = nullptr;
    uint32_t *idx = nullptr, *idx_alt = nullptr;
    int *work_counter = nullptr;     // dynamic work distribution of persistent kernels
    int *tile_hist = nullptr;        // radix sort: digit histograms, epoch, status words
    int tile_hist_cap = 0;
    unsigned radix_epoch_limit = 0;  // radix tag epochs before the status words are cleared
    bool radix_dirty = false;        // a call timed out: the next sort clears its scratch first
    double *stage = nullptr;         // [n][3] AoS staging
    double *stage2 = nullptr;

    ncorp::Cells cells;
    ncorp::WalkLists wl;
    int pair_cap = 0;
    uint64_t *pairs = nullptr, *pairs_alt = nullptr;
    uint32_t *pair_idx = nullptr, *pair_idx_alt = nullptr;
    int64_t *pairs_out = nullptr;
    // collision resolution (allocated when resolve_f > 0)
    int2 *pair_where = nullptr;      // per pair: both moonlets' positions in the search tree's order
    double *res_tc = nullptr;        // per pair: impact time
    int *res_state = nullptr;        // per pair: undecided, resolved or skipped
    unsigned long long *node_tc = nullptr, *node_ij = nullptr;   // per moonlet: minima of a matching round
    int *node_owner = nullptr;       // per moonlet: 1 + the resolved pair holding it, else 0

    ncorp::Ctrl *ctl = nullptr;      // device
    ncorp::Ctrl *ctl_h = nullptr;    // pinned host mirror
    ncorp::TreeSet alt;              // the other tree set (cells, wl, ctl above are the current one)
    cudaStream_t side = nullptr;     // stream of the collision search while the next tree is built
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaStream_t side2 = nullptr;    // stream of the multipoles and the near field inside a gravity evaluation
    cudaEvent_t ev_geo = nullptr, ev_p2m = nullptr, ev_lists = nullptr, ev_near = nullptr;
    cudaEvent_t ev_spec0 = nullptr, ev_spec = nullptr;   // fused walk: the bounded collision climb beside the geometry
    int *err_acc = nullptr;          // device: error words of tree sets recycled during a call
    int *err_acc_h = nullptr;        // pinned host mirror

    // resident-state bookkeeping
    bool have_state = false;         // A holds a state
    bool tree_valid = false;         // cells describe A's positions, A.a valid
    bool pairs_sorted = false;
    int n_found = 0;
    const void *last_pos = nullptr, *last_vel = nullptr, *last_m = nullptr, *last_R = nullptr;
    int last_p = -1;
    double last_theta = -1.0;
    double time = 0.0;
    int64_t stats[NCORP_NSTATS] = {0};
    int tree_kind = 0;               // 1: gravity geometry valid, 2: collision geometry valid (bit mask)
    int grav_p = 0;                  // p of the last gravity evaluation (0: none)
    bool grav_local = false;         // the last gravity evaluation made local expansions (falcON)
    int launches = 0;                // kernels launched by the current call
    StepGraph graphs[2];             // resident steps alternate between two buffer rotations
    int graph_next = 0;
    bool graphs_on = true;           // ncorp_set_graphs
    bool graph_used = false;         // the last call ran a step graph
    cudaStream_t gstream = nullptr;  // stream the step graphs are captured on
    bool profile = false;
    // failure-path test knobs, read from the environment at ncorp_init (all off by default):
    // list/pair capacities capped until they first overflow, and the ncorp_step call (1-based) whose
    // grid barriers wait for an arrival that never comes (each gives up after the wait limit)
    int test_list_cap = 0, test_pair_cap = 0;
    // capacities an overflow has shown to be needed, applied to both tree sets (so that a tree set grown
    // after an overflow does not leave the other one to overflow on the next step)
    int floor_cells = 0, floor_front = 0, floor_m2l = 0, floor_p2p = 0, floor_self = 0;
    long long stall_call = 0, step_calls = 0;
    cudaEvent_t ev[NCORP_NSTAGES][8][2] = {};   // up to 8 intervals per stage per call
    int ev_used[NCORP_NSTAGES] = {0};
    double stage_ms[NCORP_NSTAGES] = {0};
    bool grav_mixed = false;
};

namespace ncorp {

// ---- launchers (sort.cu) ----
// gate (nullable): a device counter read by every launched kernel, which does nothing while it is 0
// (a step's tree is rebuilt only when its collision resolution moved a moonlet)
void launch_bbox_keys(ncorp_ctx *c, const double *x, const double *y, const double *z, int n, uint64_t *key,
                      uint32_t *qx, uint32_t *qy, uint32_t *qz, bool bbox_done = false, const int *gate = nullptr);
// by_disk: the keys are a forest's moonlet keys (every disk's own root cube); they are sorted by (disk, key)
void radix_sort_u64(ncorp_ctx *c, uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, int n,
                    int bits, bool bar_zeroed = false, const int *gate = nullptr, bool by_disk = false);
// spec_dt > 0 (fused walk): also the bounds on next step's R + dt |v| of the current tree set's moonlets,
// from src_xv's velocities and src_rest's accelerations
void launch_gather(ncorp_ctx *c, const ParticleSet &src_xv, const ParticleSet &src_rest, ParticleSet &dst, int n,
                   const uint32_t *idx, double G, const int *gate = nullptr, double spec_dt = 0.0);
void launch_iota(ncorp_ctx *c, uint32_t *idx, int n);

// ---- tree.cu ----
void launch_build(ncorp_ctx *c, const ParticleSet &P, int n, int s, const int *gate = nullptr);
void launch_climb_geometry(ncorp_ctx *c, const ParticleSet &P, double G, double theta);
void launch_multipoles(ncorp_ctx *c, const ParticleSet &P, int p, bool mixed, double G);
// rc_given (nullable): each moonlet's R + dt |v| given (the velocities are then not read and the pair
// test's per-moonlet values are not written); gate (nullable): nothing is done while *gate is 0
void launch_climb_collision(ncorp_ctx *c, const ParticleSet &P, const double *vx, const double *vy,
                            const double *vz, double dt, const double *rc_given = nullptr,
                            const int *gate = nullptr);

// ---- walk.cu ----
// gravity / collisions: the criteria walked (both: one traversal for both; the collision pairs go to
// the cp2p / cself lists); gate (nullable): the walk does nothing while *gate is 0
void launch_walk(ncorp_ctx *c, bool gravity, bool collisions, const int *gate = nullptr);

// ---- m2l.cu / eval.cu ----
void launch_m2l(ncorp_ctx *c, int p, bool mixed);
// complete local expansions of every cell (after launch_m2l, which opens the descent's epoch)
void launch_descend(ncorp_ctx *c, int p, bool mixed);
struct ExtForce {
    double GMc;            // G * central mass
    double star_k;         // G M_star / r_star^3 (0: off)
    double sx, sy, sz;     // star position
    double inv_rs2;        // 1 / r_star^2
    double bulge;          // G M_c R_c^2 J2 of the equatorial bulge (0: off)
};
void launch_near(ncorp_ctx *c, const ParticleSet &P, int p, bool mixed, double G);
// Algorithm StandardTree for the moonlets of S (tree order) on the current tree, whose geometry and
// multipoles are computed: S.ax = mutual + external, amx = mutual (want_mutual)
void launch_standard(ncorp_ctx *c, const ParticleSet &S, int n, int p, bool mixed, double G, ExtForce ext,
                     bool want_mutual, int pre, int post);
void launch_far(ncorp_ctx *c, const ParticleSet &P, int p, bool mixed, double G, ExtForce ext, bool want_mutual,
                double kick_h = 0.0);

// ---- collide.cu ----
// the box of (x, y, z) emptied and folded again into ctl when *gate != 0 (decided on the device)
void launch_bbox_gated(ncorp_ctx *c, const double *x, const double *y, const double *z, int n, Ctrl *ctl,
                       const int *gate);
void launch_resolve(ncorp_ctx *c, const ParticleSet &S, ParticleSet &D, int n, double dt);
void launch_collide(ncorp_ctx *c, const ParticleSet &P, const double *vx, const double *vy, const double *vz,
                    double dt, bool wide);
void launch_sort_pairs(ncorp_ctx *c, int count);
// collision search of the moonlets of P (tree order, velocities P.v*) by the standard tree code, on the
// current tree with its collision geometry
void launch_standard_collide(ncorp_ctx *c, const ParticleSet &P, double dt, int n, int pre, int post);

// ---- kdk.cu ----
void launch_aos_to_soa(ncorp_ctx *c, const double *aos, double *x, double *y, double *z, int n);
// abort_a / abort_b (nullable): error words; the scatter writes nothing when either holds an abort flag
// (a step that timed out or overflowed leaves the caller's arrays as they were)
void launch_scatter_aos(ncorp_ctx *c, const double *x, const double *y, const double *z, const int *perm,
                        double *aos, int n, const int *abort_a = nullptr, const int *abort_b = nullptr);
// v' = v + h a, x' = x + dt v' and the bounding box of x' into ctl (which
// must hold an empty box).
struct KickDriftArgs {
    const double *x, *y, *z, *vx, *vy, *vz, *ax, *ay, *az;
    double h, dt;
    double *ox, *oy, *oz, *ovx, *ovy, *ovz;
    int n;
    Ctrl *ctl;
    // fused walk (nullable rc_spec): every moonlet's R + dt |v'| is checked against rc_spec (set *stale
    // if one exceeds it) and written, with v' in FP32, into cv4 for the pair test
    const double *R, *rc_spec;
    int *stale;
    float4 *cv4;
};
void launch_kick_drift(ncorp_ctx *c, const KickDriftArgs &A);
void launch_scatter_state(ncorp_ctx *c, const ParticleSet &S, double *pos, double *vel, int n,
                          const int *abort_a = nullptr, const int *abort_b = nullptr);
void launch_unpack_pairs(ncorp_ctx *c, const uint64_t *packed, int64_t *out, int count);

// host-side error helper used by every launcher
#define NCORP_CUDA_CHECK(expr)                                                       \
    do {                                                                             \
        cudaError_t _e = (expr);                                                     \
        if (_e != cudaSuccess) throw ::ncorp::CudaError(_e, #expr, __FILE__, __LINE__); \
    } while (0)

struct CudaError {
    cudaError_t code;
    const char *expr, *file;
    int line;
    CudaError(cudaError_t c, const char *e, const char *f, int l) : code(c), expr(e), file(f), line(l) {}
};

inline int grid_for(int n, int block, int max_blocks = 1 << 20) {
    long long g = (static_cast<long long>(n) + block - 1) / block;
    if (g < 1) g = 1;
    if (g > max_blocks) g = max_blocks;
    return static_cast<int>(g);
}

}  // namespace ncorp

inline int ncorp::coop_blocks(const ncorp_ctx *c, int per_sm) {
    int g = per_sm * c->num_sms;
    if (c->coop_max > 0 && g > c->coop_max) g = c->coop_max;
    return g < 1 ? 1 : g;
}
