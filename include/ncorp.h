/*
 * ncorp.h -- C ABI of the GB300 falcON step library (libncorp.so).
 *
 * The library computes one O(N) falcON step for a disk of N moonlets orbiting
 * a central mass, as described by Couturier, Quillen & Nakajima (arXiv
 * 2310.20374): Hilbert-key sort and octree build (Sect. 3.4.1, 3.4.6), tree
 * climbing with P2M/M2M multipoles (Sect. 3.4.2, Eq. multipole_moment,
 * App. C), the symmetric dual-tree walk of Algorithm TreeWalk (Sect. 3.4.5)
 * with M2L (Eq. phi_expanded), near-field direct gravity and a tree-based
 * collision search (Sect. 3.1), and the tree descent L2L/L2P (Eq. shifting),
 * inside an SBAB1 kick-drift-kick leapfrog with merged kicks (Sect. 4.1) and
 * the central-body / distant-star forces of App. B.1 and B.3.
 *
 * Conventions shared by every entry point:
 *   - Every function returns an int status: NCORP_OK (0) or a negative
 *     NCORP_E* code.  ncorp_last_error() gives a message for the last failure
 *     on that context.  No C++ exception crosses this interface.
 *   - Array arguments may point to host memory or to device memory on the
 *     context's device; the library tells them apart with
 *     cudaPointerGetAttributes.  Host arrays are copied in and out inside the
 *     call.  The library never frees or retains caller memory.
 *   - Vectors are laid out [n][3] (x, y, z interleaved), doubles, row-major.
 *   - All device work is enqueued on the context's CUDA stream; every call
 *     synchronises that stream before it returns (to read the status word),
 *     so outputs are ready when the call returns.
 *   - Units are the caller's; the configuration fixes G and the central mass.
 *   - Invalid arguments (n < 1, p outside 1..6, theta outside (0,1), dt <= 0
 *     where a time step is needed, null pointers, non-finite inputs) return
 *     NCORP_EINVAL before any device work.
 */
#ifndef NCORP_H
#define NCORP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NCORP_OK         0
#define NCORP_EINVAL    -1   /* bad argument */
#define NCORP_ENOMEM    -2   /* device or host allocation failed */
#define NCORP_ECUDA     -3   /* a CUDA call failed; see ncorp_last_error */
#define NCORP_EOVERFLOW -4   /* an output did not fit the caller's capacity */
#define NCORP_ETIMEOUT  -5   /* a bounded device-side wait gave up */
#define NCORP_ESTATE    -6   /* call out of sequence (e.g. no state yet) */

#define NCORP_FP64  0        /* every stage in FP64 */
#define NCORP_MIXED 1        /* multipoles, M2L, P2P, L2L/L2P in FP32 with per-cell scaling;
                                positions, velocities, kicks/drifts, external forces, keys,
                                tree geometry and the collision test in FP64 */

typedef struct ncorp_ctx ncorp_ctx;

typedef struct {
    double G;                 /* gravitational constant */
    double central_mass;      /* M_c (App. B.1) */
    double central_radius;    /* R_c: radius of the equatorial bulge term (collisions with the central body
                                 are not searched) */
    int leaf_size;            /* s: cells with more than s moonlets are split (Sect. 3.4.1); 0 = default for p */
    int n_cs, n_cc_pre, n_cc_post;  /* gravity TreeWalk thresholds (Sect. 3.4.5); all 0 = defaults for p */
    int c_cs, c_cc_pre, c_cc_post;  /* collision TreeWalk thresholds; all 0 = 12, 0, 16 (Sect. 4.2) */
    int precision;            /* NCORP_FP64 or NCORP_MIXED */
    int collisions;           /* 1: search colliding pairs in every step's drift (Sect. 4.1) */
    double star_mass;         /* distant star (App. B.3); 0 disables the tidal term */
    double star_a;            /* star orbital radius */
    double star_obliquity;    /* obliquity epsilon of the central body (radians) */
    double t0;                /* initial time (sets the star's longitude n t) */
    double central_J2;        /* J2 of the central body's equatorial bulge (App. B.2): adds
                                 G M_c R_c^2 J2 / r^5 [(15 z^2 - 3 r^2) / (2 r^2) r - 3 z k] to every
                                 moonlet's acceleration, k = the frame's z axis (the body's rotation
                                 axis); 0 disables.  For a fluid body rotating at Omega,
                                 J2 = Omega^2 / (2 G M_c / R_c^3). */
    double resolve_f;         /* collision resolution in ncorp_step (Sect. 5.1, 5.2): 0 = colliding pairs are
                                 only reported; 1 <= f <= 2 = each is resolved at its impact time by the
                                 impulse J = alpha (dr.dv) dr, alpha = f m1 m2 / ((m1 + m2)(R1 + R2)^2)
                                 (f = 2 elastic, f = 1 the most inelastic), and the moonlets travel the rest
                                 of the step at their new velocities.  A moonlet takes at most one impact
                                 per step: pairs are resolved in increasing (impact time, i, j) and a pair
                                 with a moonlet already resolved in the step is reported but not resolved.
                                 The search still runs beside the new tree's build; a step that resolved an
                                 impact builds that tree again from the resolved drift.  Resolved moonlets
                                 need positive masses (v' = v -+ J/m): a massless one makes the step fail
                                 with NCORP_EINVAL (non-finite position).  Other values of resolve_f:
                                 NCORP_EINVAL at ncorp_init. */
    int n_cb_pre, n_cb_post;  /* thresholds N_cb,pre and N_cb,post of the standard tree code
                                 (ncorp_accel_standard, Algorithm StandardTree, Sect. 3.4.4); >= 0 */
    int c_cb_pre, c_cb_post;  /* the same thresholds for the standard tree code's collision search
                                 (ncorp_collide_standard); >= 0 */
    int fused_walk;           /* 1: one tree walk per ncorp_step for gravity and collisions (Algorithm
                                 TreeWalk with both criteria; Sect. 3.4.1: one tree per step).  The walk
                                 of the new tree x_{n+1} also collects the leaf pairs that the next
                                 step's collision search (at x_{n+1}, v_{n+3/2}) tests, with the collision
                                 geometry of a bound on each moonlet's R + dt |v_{n+3/2}| made from
                                 v_{n+1/2} + dt a_n and a margin of dt^2 |a_n| / 2.  The next step checks
                                 every bound against the true velocity; if one is exceeded it searches
                                 with its own collision walk as usual.  The pair set is the same either
                                 way (the brute-force one).  Applies to ncorp_step without collision
                                 resolution; 0 = separate walks (default). */
} ncorp_config;

/* Fills *cfg with G = 1, M_c = 1, R_c = 1, automatic leaf size and thresholds,
 * NCORP_MIXED, collisions on (reported, not resolved), no star, no bulge (J2 = 0),
 * standard tree thresholds N_cb,pre = 6 and N_cb,post = 16 for gravity and 0 and
 * 16 for collisions (Sect. 4.2). */
void ncorp_config_default(ncorp_config *cfg);

/* Creates a context for disks of up to n_max moonlets on CUDA device `device`.
 * cuda_stream is a cudaStream_t (NULL = the legacy default stream); the
 * context allocates its own device workspace (it grows on demand).
 * Environment variables read here (all optional):
 *   NCORP_RADIX_EPOCH_LIMIT (>= 1) lowers the number of radix sorts after
 *     which the context's sort scratch is cleared (default 2^28);
 *   NCORP_SIDE_BLOCKS (8..1024, default 64) caps the cooperative grids of
 *     a step's collision search, which runs beside the new tree's build and
 *     walk (their blocks must find room on the SMs together);
 *   NCORP_WAIT_LIMIT_MS (1..60000, default 1000) bounds every device-side
 *     grid-barrier wait of the context: a wait that runs longer makes the
 *     call fail with NCORP_ETIMEOUT instead of hanging;
 *   NCORP_TEST_STALL_STEP=k makes the k-th ncorp_step of the context wait at
 *     its grid barriers for an arrival that never comes, so that the step
 *     fails with NCORP_ETIMEOUT after the wait limit;
 *   NCORP_TEST_LIST_CAP / NCORP_TEST_PAIR_CAP start the walk lists / the
 *     colliding-pair buffer at that many entries, so that the first step
 *     that needs more overflows and is rerun with grown buffers.
 * The last three exist to test the failure paths and are off by default.
 * Errors: NCORP_EINVAL (null out/cfg, n_max < 1, bad config), NCORP_ECUDA,
 * NCORP_ENOMEM. */
int ncorp_init(ncorp_ctx **out, const ncorp_config *cfg, int64_t n_max, int device, void *cuda_stream);

/* Changes the stream later calls enqueue their work on.  Waits first for the
 * work already enqueued on the old stream.  Errors: NCORP_EINVAL (null ctx),
 * NCORP_ECUDA (the old stream reported an error). */
int ncorp_set_stream(ncorp_ctx *ctx, void *cuda_stream);

/* One SBAB1 step (Sect. 4.1): v += dt/2 a(x); collision search on (x, v)
 * during the drift (Sect. 3.1, Algorithm TreeWalk); x += dt v; rebuild the
 * tree and compute a(x) = falcON mutual gravity + central (+ star); v += dt/2 a.
 * positions/velocities [n][3] are read and overwritten with the new state in
 * the caller's order; masses/radii [n] are read.
 * Kicks are merged across calls: the acceleration and tree of the previous
 * call's final positions are kept on the device and reused when the next call
 * passes the same position/velocity/mass/radius pointers, the same n, p and
 * theta and the context was not used by ncorp_accel/ncorp_collide in between;
 * call ncorp_reset() after changing the arrays' contents yourself.
 * The pairs found are kept for ncorp_collisions().
 * A step whose internal lists overflow is rerun from the resident state with
 * grown buffers (invisible to the caller).  A step that fails with
 * NCORP_ETIMEOUT writes nothing to positions/velocities and drops the
 * resident state, so the next call re-reads the caller's arrays.
 * Errors: NCORP_EINVAL, NCORP_ECUDA, NCORP_ENOMEM, NCORP_ETIMEOUT. */
int ncorp_step(ncorp_ctx *ctx, double *positions, double *velocities, const double *masses,
               const double *radii, int64_t n, int p, double theta, double dt);

/* Enables (enable != 0, the default) or disables CUDA graphs for resident
 * steps.  A resident ncorp_step (same arrays, n, p, theta as the previous
 * call) makes the same launches every other call, so it is captured once per
 * buffer rotation into a CUDA graph (at most two kept per context) and
 * replayed; results are identical to the directly launched step.  Steps with
 * a distant star, steps timed by ncorp_profile and retries after a buffer
 * overflow are always launched directly.  Disabling waits for the context's
 * stream and frees the cached graphs.  Errors: NCORP_EINVAL, NCORP_ECUDA. */
int ncorp_set_graphs(ncorp_ctx *ctx, int enable);

/* Forgets the resident state, so the next ncorp_step re-reads its inputs. */
int ncorp_reset(ncorp_ctx *ctx);

/* Most disks one context can hold side by side (ncorp_set_disks). */
#define NCORP_MAX_DISKS 256

/* Lays the context's moonlets out as n_disks independent disks (a forest):
 * disk d is the sizes[d] (>= 1) moonlets that follow the earlier disks' in
 * every array a later call passes, whose n must then be the sum of sizes.
 * Every disk is a separate system: it has its own root cell and root cube
 * (Sect. 3.4.1 applied per disk), its own total mass in theta(M) (Dehnen
 * 2002, Eq. 13), and neither gravity nor the collision search (Algorithm
 * TreeWalk) ever pairs cells or moonlets of two disks; the central body,
 * bulge and star act on every disk alike.  Each stage of ncorp_step,
 * ncorp_accel and ncorp_collide then runs once over all disks (one launch
 * per stage, not one per disk), and the results of disk d equal those of the
 * same disk in a context of its own up to the rounding order of sums
 * (bit-equal colliding pairs; accelerations within the precision's
 * tolerance).  ncorp_collisions reports the pairs with indices into the
 * concatenated arrays (a pair never spans two disks).  The standard-tree
 * entry points (ncorp_accel_standard, ncorp_collide_standard) take one disk
 * only.  n_disks = 1 returns to one disk (sizes may then be NULL; if given,
 * its one entry is checked like the others).  The resident
 * state is dropped.  sizes: host memory [n_disks].  Synchronous.
 * Errors: NCORP_EINVAL (n_disks outside 1..NCORP_MAX_DISKS, a size < 1, more
 * than 2^30 moonlets in all), NCORP_ECUDA, NCORP_ENOMEM. */
int ncorp_set_disks(ncorp_ctx *ctx, int n_disks, const int64_t *sizes);

/* Colliding pairs found by the last ncorp_step or ncorp_collide: rows (i, j)
 * of caller indices with i < j, sorted lexicographically, no duplicates.
 * pairs: [cap][2] int64 (host or device); *n_pairs receives the total found.
 * If the total exceeds cap, the first cap rows are written and
 * NCORP_EOVERFLOW is returned (nothing is lost: call again with more room). */
int ncorp_collisions(ncorp_ctx *ctx, int64_t *pairs, int64_t cap, int64_t *n_pairs);

/* Accelerations at the given positions (one tree build, climb, walk, M2L,
 * near field and descent): acc [n][3] = mutual + central (+ star at the
 * context's time); acc_mutual [n][3] (nullable) = falcON mutual part only.
 * Invalidates the resident step state.  Errors as ncorp_step. */
int ncorp_accel(ncorp_ctx *ctx, const double *positions, const double *masses, int64_t n, int p,
                double theta, double *acc, double *acc_mutual);

/* Accelerations by the standard tree code (Algorithm StandardTree, Sect.
 * 3.4.4) on the same tree, geometry (r_crit = r_max / theta(M)) and
 * multipoles as ncorp_accel: every moonlet a is walked from the root; a cell
 * B with fewer than n_cb_pre moonlets is summed directly, a cell well
 * separated from a (r_crit,B^2 <= |x_a - s_B|^2, zero distance excluded)
 * contributes its order-p expansion at a, a cell with fewer than n_cb_post
 * moonlets or a leaf is summed directly, any other is opened.  acc / acc_mutual
 * as for ncorp_accel.  Counters: NCORP_STAT_M2L = moonlet-cell expansions,
 * NCORP_STAT_P2P_PAIRS = direct moonlet-cell sums, NCORP_STAT_P2P_INTER =
 * their moonlet pairs.  ncorp_expansions then exports multipoles only
 * (local != NULL: NCORP_ESTATE).  Errors as ncorp_accel. */
int ncorp_accel_standard(ncorp_ctx *ctx, const double *positions, const double *masses, int64_t n, int p,
                         double theta, double *acc, double *acc_mutual);

/* Collision search alone (Sect. 3.1, tree climb for collisions of Sect.
 * 3.4.2, Algorithm TreeWalk) on the given positions and velocities over a
 * step dt, with the tree of those positions.  Results via ncorp_collisions.
 * Invalidates the resident step state.  Errors as ncorp_step. */
int ncorp_collide(ncorp_ctx *ctx, const double *positions, const double *velocities,
                  const double *radii, int64_t n, double dt);

/* Collision search alone by the standard tree code (Algorithm StandardTree,
 * Sect. 3.4.4, its instructions for collisions) on the tree of the given
 * positions with the collision geometry of Sect. 3.4.2 (Eqs. center, rmax,
 * rcrit): every moonlet a is walked from the root with r_crit,a = R_a + dt |v_a|;
 * a cell B with fewer than c_cb_pre moonlets is searched directly; B is
 * skipped when ((r_crit,a + r_crit,B)(1 + 2^-40))^2 < |x_a - sbar_B|^2; a cell
 * with fewer than c_cb_post moonlets, or a leaf, is searched directly; any
 * other is opened.  Searching B directly tests a against the moonlets of B with
 * a larger caller index with the pairwise test of Sect. 3.1, so the pairs
 * found are exactly those of ncorp_collide.  Results via ncorp_collisions;
 * counters: NCORP_STAT_COL_PAIRS = cells searched directly, NCORP_STAT_COL_TESTS
 * = moonlet pairs tested.  Invalidates the resident step state.  Errors as
 * ncorp_collide. */
int ncorp_collide_standard(ncorp_ctx *ctx, const double *positions, const double *velocities,
                           const double *radii, int64_t n, double dt);

/* Copies the resident state (caller order) into positions/velocities [n][3].
 * NCORP_ESTATE if no step has run since init/reset. */
int ncorp_get_state(ncorp_ctx *ctx, double *positions, double *velocities);

/* Counters of the last call (int64 slots, see NCORP_STAT_*); writes
 * min(n_stats, NCORP_NSTATS) values to host memory. */
#define NCORP_STAT_CELLS        0
#define NCORP_STAT_LEAVES       1
#define NCORP_STAT_DEPTH        2
#define NCORP_STAT_M2L          3   /* well-separated cell pairs (gravity walk); moonlet-cell expansions
                                       after ncorp_accel_standard */
#define NCORP_STAT_P2P_PAIRS    4   /* cell pairs treated directly (gravity walk decisions); direct
                                       moonlet-cell sums after ncorp_accel_standard */
#define NCORP_STAT_P2P_SELF     5   /* cells treated directly with themselves (gravity) */
#define NCORP_STAT_P2P_INTER    6   /* particle pairs summed directly (gravity, unordered) */
#define NCORP_STAT_COL_PAIRS    7   /* cell pairs searched directly (collision walk decisions) */
#define NCORP_STAT_COL_SELF     8
#define NCORP_STAT_COL_TESTS    9   /* moonlet pairs examined by the collision test */
#define NCORP_STAT_COL_FOUND   10
#define NCORP_STAT_WALK_ITERS  11   /* frontier iterations of the last walk */
#define NCORP_STAT_M2L_DIRECTED 12  /* directed M2L entries evaluated */
#define NCORP_STAT_P2P_DIRECTED 13  /* directed leaf-source entries evaluated */
#define NCORP_STAT_LAUNCHES    14   /* CUDA kernels the last call launched */
#define NCORP_STAT_COL_ITERS   15   /* frontier iterations of the collision walk */
#define NCORP_STAT_GRAPH       16   /* 1 if the last ncorp_step ran as a replayed (or just captured) CUDA graph */
#define NCORP_STAT_SORT_PATH   17   /* key sort of the last tree: 1 nearly-sorted merge (steps) with the
                                       out-of-place keys ranked (at most 4096 of them), 2 the same with
                                       them radix-sorted (at most 65536), 0 radix sort of all keys, -1 radix
                                       sort after the merge found the kept keys out of order */
#define NCORP_STAT_RESOLVED    18   /* impacts resolved by the last ncorp_step (resolve_f > 0) */
#define NCORP_STAT_FUSED       19   /* 1 if the last ncorp_step's collision search tested the pairs listed by
                                       the previous step's fused walk (fused_walk = 1, no bound exceeded) */
#define NCORP_NSTATS           20

/* Writes min(n_stats, NCORP_NSTATS) counters of the last call (slots above)
 * to host memory stats[].  NCORP_EINVAL if ctx or stats is NULL. */
int ncorp_stats(ncorp_ctx *ctx, int64_t *stats, int n_stats);

/* Stage timers.  With profiling on, every call records CUDA events on the
 * context's stream around its stages and ncorp_stage_times() returns the
 * device milliseconds each stage took in the last call (summed when a stage
 * runs more than once).  Off by default; on costs a few event records. */
#define NCORP_STAGE_SORT     0   /* bounding box, keys, radix sort, gather */
#define NCORP_STAGE_BUILD    1   /* octree build, leaf list */
#define NCORP_STAGE_CLIMB    2   /* gravity climb: geometry, theta(M), r_crit; multipoles beside them */
#define NCORP_STAGE_WALK     3   /* gravity walk and per-target lists */
#define NCORP_STAGE_M2L      4
#define NCORP_STAGE_DESCEND  5   /* complete local expansions (Eq. shifting from the ancestors) */
#define NCORP_STAGE_EVAL     6   /* L2P of the local expansions, external forces */
#define NCORP_STAGE_COLLIDE  7   /* collision climb, walk and pair test */
#define NCORP_STAGE_KDK      8   /* kicks, drift, host/device copies of the state */
#define NCORP_STAGE_NEAR     9   /* near-field direct sums (beside M2L and the descent) */
#define NCORP_NSTAGES       10

/* Turns the stage timers on (enable != 0) or off.  NCORP_EINVAL if ctx is NULL. */
int ncorp_profile(ncorp_ctx *ctx, int enable);

/* Writes min(n, NCORP_NSTAGES) stage times of the last call, in milliseconds,
 * to host memory ms[] (zeros while profiling is off).  NCORP_EINVAL if ctx or
 * ms is NULL or n < 0. */
int ncorp_stage_times(ncorp_ctx *ctx, double *ms, int n);

/* Diagnostic export of the tree of the last ncorp_accel/ncorp_collide/ncorp_step
 * (level-major cells, Hilbert order within a level), for parity checks.
 * Any output may be NULL; all are host or device arrays:
 *   order [n] int64: caller index of the i-th moonlet in tree order
 *   keys  [n] uint64: 63-bit Hilbert key of the i-th moonlet in tree order
 *   root  [4] double: x_lo, y_lo, z_lo, L of the root cube (a forest of
 *         n_disks disks: [n_disks][4], every disk's root cube)
 *   cells [cap][7] int64: level, cx, cy, cz, first, count, n_children
 *   ggeo  [cap][6] double: M, s_x, s_y, s_z, r_max, r_crit (gravity climb)
 *   cgeo  [cap][5] double: sbar_x, sbar_y, sbar_z, r_max, r_crit (collision climb)
 * *n_cells receives the number of cells; NCORP_EOVERFLOW if it exceeds cap. */
int ncorp_tree_export(ncorp_ctx *ctx, int64_t *order, uint64_t *keys, double *root, int64_t *cells,
                      double *ggeo, double *cgeo, int64_t cap, int64_t *n_cells);

/* Diagnostic export of the expansions of the last gravity evaluation
 * (ncorp_accel or ncorp_step), cells in the order of ncorp_tree_export, all
 * unscaled and in FP64 (host or device arrays, any may be NULL):
 *   mult  [cap][nm]: multipole moments M_beta = sum_i mu_i (x_i - s)^beta of
 *         Eq. multipole_moment in symmetric multi-index form, orders 0 and
 *         2..p-1 (nm = 1 for p = 1, else p(p+1)(p+2)/6 - 3)
 *   local [cap][nc]: the complete local expansion C_alpha of each cell: the
 *         M2L sums of Eq. phi_expanded the walk gave the cell, plus its
 *         ancestors' translated to its centre by the descent (Eq. shifting),
 *         orders 1..p (nc = (p+1)(p+2)(p+3)/6 - 1)
 *   rho   [cap]: the cell's power-of-two scale
 * Within order n the components run over k = 0..n, c = 0..k with
 * (a, b, c) = (n-k, k-c, c) the powers of (x, y, z).  *p receives p.
 * NCORP_ESTATE if no gravity evaluation has run; NCORP_EOVERFLOW if the
 * cell count exceeds cap (the first cap cells are written). */
int ncorp_expansions(ncorp_ctx *ctx, double *mult, double *local, double *rho, int64_t cap, int64_t *n_cells,
                     int *p);

/* Releases the context and its device workspace (NULL is ignored). */
void ncorp_free(ncorp_ctx *ctx);

/* Message of the last failure on ctx (static storage owned by ctx; never NULL). */
const char *ncorp_last_error(const ncorp_ctx *ctx);

/* ---- Batches: many independent disks on one GPU ----------------------------
 * A batch keeps every disk's state on the device and advances all of them
 * together.  The disks that share (p, theta, dt) form one forest: a context
 * laid out by ncorp_set_disks, so that each stage of a step is one launch over
 * all of them however many there are.  ncorp_batch_run advances every forest
 * by n_steps steps through one CUDA graph per forest (captured on the first
 * run of that length and buffer rotation, replayed afterwards); the forests
 * run one after another, each filling the GPU.  Each disk is integrated as by ncorp_step
 * in a context of its own (the same SBAB1 step of Sect. 4.1 with the falcON
 * forces and the collision search of Sect. 3.1), up to the rounding order of
 * sums.  A batch is not thread-safe: call it from one host thread at a time.
 * Batches take no distant star (its position depends on each disk's time).
 * With leaf_size = 0 in the configuration, an autotuner chooses each large
 * forest's leaf size s: at the forest's first run (and when its size has
 * changed more than fourfold) it lays the forest out with each of a few
 * candidates around the default for p and times two steps from the same
 * state, keeping the fastest (NCORP_BATCH_TUNED, NCORP_BATCH_LEAF).
 * Environment variables read by ncorp_batch_create: NCORP_AUTOTUNE=0 turns
 * the tuner off; NCORP_VALIDATE=1 runs every forest one step at a time and
 * checks the invariants of its resident state (permutation, disk map, cell
 * ranges, leaf map) around each step, failing with NCORP_ESTATE on the first
 * violation (a diagnostic mode, slow). */
typedef struct ncorp_batch ncorp_batch;

/* Creates an empty batch on the current CUDA device; every disk uses cfg
 * (copied).  hbm_budget_bytes caps the device memory the batch may hold (0:
 * no cap); cuda_stream is the caller's stream: ncorp_batch_run starts after
 * the work already enqueued on it and the caller's later work waits for the
 * run.  Errors: NCORP_EINVAL (bad config, star_mass != 0), NCORP_ECUDA,
 * NCORP_ENOMEM. */
int ncorp_batch_create(ncorp_batch **out, const ncorp_config *cfg, size_t hbm_budget_bytes, void *cuda_stream);

/* Adds a disk of n moonlets: positions/velocities [n][3], masses/radii [n],
 * host or device arrays (copied; the caller keeps ownership); p, theta and
 * dt as for ncorp_step, fixed for the disk.  The disk joins a forest of its
 * (p, theta, dt) (another one is started when those have NCORP_MAX_DISKS
 * disks); that forest's tree and acceleration are computed at the start of
 * the next ncorp_batch_run (one force evaluation for all the disks added or
 * removed since the last run).  Admission by device memory: the disk is
 * refused when the bytes the batch holds plus 1.5 n times the largest
 * footprint per moonlet measured so far (4096 bytes before any measurement;
 * measured on forests of at least 65536 moonlets whose layout succeeded)
 * exceed the budget, or exceed the device memory still free.  *disk_id
 * receives the disk's id (unique within the batch).  Errors: NCORP_EINVAL
 * (arguments, non-finite positions or velocities), NCORP_ENOMEM (allocation
 * failed, or over the budget), NCORP_ECUDA; on error no disk is added. */
int ncorp_batch_add_disk(ncorp_batch *b, const double *positions, const double *velocities, const double *masses,
                         const double *radii, int64_t n, int p, double theta, double dt, int32_t *disk_id);

/* Advances every disk by n_steps SBAB1 steps (Sect. 4.1) and waits for them
 * (n_steps = 0 only lays out the forests that changed).  If an internal
 * buffer of a forest overflowed during the run, that forest is rerun from
 * its state at the start of the run one synchronous step at a time with
 * grown buffers (counted in NCORP_BATCH_FALLBACKS).  The colliding pairs of
 * each disk's last step are kept for ncorp_batch_collisions.  Errors:
 * NCORP_EINVAL (n_steps < 0, non-finite state), NCORP_ECUDA, NCORP_ENOMEM
 * (a forest could not be laid out in device memory: no disk was stepped, and
 * the run can be retried after removing disks), NCORP_ETIMEOUT,
 * NCORP_EOVERFLOW (also when the rerun of an overflowed forest could not
 * grow its buffers; the other forests have then taken their steps). */
int ncorp_batch_run(ncorp_batch *b, int n_steps);

/* Copies a disk's current state, in the order it was given, into
 * positions/velocities [n][3] (host or device).  NCORP_EINVAL for an unknown id. */
int ncorp_batch_get_state(ncorp_batch *b, int32_t disk_id, double *positions, double *velocities);

/* Colliding pairs of a disk's last step, as ncorp_collisions gives them
 * (indices into the disk's own arrays). */
int ncorp_batch_collisions(ncorp_batch *b, int32_t disk_id, int64_t *pairs, int64_t cap, int64_t *n_pairs);

/* Removes a disk and releases its share of device memory (a forest whose
 * last disk leaves is released; one that shrinks below half its capacity is
 * reallocated at its next layout); if positions and velocities are given
 * (both or neither), the disk's final state is copied there first, as by
 * ncorp_batch_get_state.  NCORP_EINVAL for an unknown id. */
int ncorp_batch_remove_disk(ncorp_batch *b, int32_t disk_id, double *positions, double *velocities);

/* Batch counters (int64 slots): */
#define NCORP_BATCH_DISKS      0   /* disks in the batch */
#define NCORP_BATCH_MOONLETS   1   /* moonlets over all disks */
#define NCORP_BATCH_BYTES      2   /* device bytes the batch holds (measured) */
#define NCORP_BATCH_FORESTS    3   /* forests: groups of disks with the same (p, theta, dt) */
#define NCORP_BATCH_FALLBACKS  4   /* forest reruns after a buffer overflow, since creation */
#define NCORP_BATCH_LAUNCHES   5   /* kernels launched by the last run */
#define NCORP_BATCH_TUNED      6   /* forests whose leaf size the autotuner chose, since creation */
#define NCORP_BATCH_LEAF       7   /* leaf size s of the batch's largest forest */
#define NCORP_BATCH_NINFO      8

/* Writes min(n_info, NCORP_BATCH_NINFO) batch counters to host memory info[]. */
int ncorp_batch_info(const ncorp_batch *b, int64_t *info, int n_info);

/* Releases the batch and all its disks (NULL is ignored). */
void ncorp_batch_free(ncorp_batch *b);

/* Message of the last failure of a batch call (never NULL). */
const char *ncorp_batch_last_error(const ncorp_batch *b);

/* Measured fused multiply-add throughput of device `device`, the peak the
 * ALU-bound stages are compared with: FP32 (precision = NCORP_MIXED) or FP64
 * (NCORP_FP64).  Runs independent FMA chains on every SM for about 5 ms, six
 * times on cuda_stream (the first a warm-up), and writes the best rate in
 * FLOP/s (2 per FMA) to *flop_per_s.  Allocates and frees a small output
 * buffer (grid x block elements; every thread writes only its own element).
 * Errors: NCORP_EINVAL (NULL output, other precision), NCORP_ENOMEM,
 * NCORP_ECUDA. */
int ncorp_fma_peak(int device, int precision, void *cuda_stream, double *flop_per_s);

/* Largest n accepted by ncorp_hilbert_sort_static. */
#define NCORP_STATIC_MAX_N 65536

/* Hilbert keys of n moonlets and their stable sort, without allocating any
 * memory: the key and sort stages of a step (the root cube around the
 * bounding box, 21-bit quantisation per axis and a 63-bit 3-D Hilbert key,
 * then the stable radix sort by (key, index)).  The paper has no
 * counterpart: this entry point exists for
 * callers that must not allocate device memory once they are set up (a fixed
 * device-memory budget, or a loop in which the implicit synchronisation of
 * cudaMalloc/cudaFree is not acceptable), and needs no context.
 *   positions [n][3] double, device memory of the current device (read)
 *   keys      [n] uint64, device (written): sorted keys, ascending
 *   order     [n] int64, device (written): order[i] = the index (row of
 *             positions) of the moonlet with the i-th smallest key; equal keys
 *             keep increasing index order
 *   cuda_stream: the stream the work is enqueued on (NULL: legacy default);
 *             the call synchronises it before returning, to read the status.
 * Results are bit-identical to the keys and order that ncorp_tree_export
 * reports after ncorp_accel on the same positions.
 * Scratch: one file-scope device array per device, sized for
 * NCORP_STATIC_MAX_N moonlets (about 3.4 MB); nothing is allocated or freed.
 * The call synchronises its stream to read the status word, so it cannot be
 * part of a CUDA graph capture.  The first call on a device looks up the
 * array's address (cudaGetSymbolAddress) with that device current.
 * The array keeps the contents of the last call; each call first resets the
 * parts that must start at zero (bounding-box accumulators, status word,
 * barrier counter) and overwrites everything else before reading it.
 * Calls whose device work overlaps (from several streams or host threads on
 * the same device) share that array and race: serialise them.
 * Errors: NCORP_EINVAL if n < 1, n > NCORP_STATIC_MAX_N, a pointer is NULL or
 * not device memory of the current device (all before any device work), or a
 * position is not finite; NCORP_ETIMEOUT if the sort's grid barrier timed
 * out; NCORP_ECUDA if a CUDA call failed. */
int ncorp_hilbert_sort_static(const double *positions, int64_t n, uint64_t *keys, int64_t *order,
                              void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* NCORP_H */
