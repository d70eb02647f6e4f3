// eval.cu -- tree descent and evaluation at the moonlets: the complete local
// expansion of every cell (Sect. 3.4.3, Eq. shifting), L2P at the moonlets,
// the direct ("brute force") gravity of each leaf's near-field list, and the
// central-body / distant-star forces (App. B.1, B.3).
//
// Evaluation in two kernels, so that the near field (which needs only the
// direct lists) can run while M2L and the descent produce the local
// expansions.  k_eval: every moonlet gets
//   sum_j mu_j (x_j - x)/|x_j - x|^3 over the moonlets of its leaf's direct list
// (mu_j = G m_j; coincident pairs, the moonlet itself included, are skipped).
// k_far: it adds
//   a = (1/rho) sum_{|beta| <= p-1} C-hat_{e_k+beta} (d/rho)^beta / beta!,  d = x - s_leaf,
// from its leaf's complete local expansion, and the external forces in FP64.
//
// Mixed precision: the direct sum reads every position as an FP32 pair
// (hi, lo) with x = hi + lo; (hi_j - hi_i) + (lo_j - lo_i) gives the
// separation to ~1e-7 relative at any distance, so no FP64 work is done per
// pair.
#include <type_traits>

#include "ctx.h"
#include "fields.cuh"

namespace ncorp {

struct ExpTable2 {
    unsigned char e[off(MAXP + 2)][3];
};
constexpr ExpTable2 make_exp_table2() {
    ExpTable2 t{};
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
__constant__ ExpTable2 c_exp2 = make_exp_table2();

struct EvalArgs {
    int n;                     // moonlets of the tree
    const int *leaves, *level, *parent, *first, *count, *leaf_of;
    const double *sx, *sy, *sz, *rho;
    const float4 *gh, *gl;
    const void *Cf;   // complete local expansions
    const float *Cf_lo;   // mixed: low parts of their order-1 coefficients
    const int *p2p_off;
    const int2 *p2p_src;      // per directed entry: the source leaf's (first, count)
    int p2p_dir_cap;
    const double *x, *y, *z, *m;
    const float4 *hi4, *lo4;
    double G;
    ExtForce ext;
    double *ax, *ay, *az;
    double *amx, *amy, *amz;
    double *nx, *ny, *nz;     // near-field sums per moonlet (tree order)
    double kick_h;            // k_far: v += kick_h a after the evaluation (0: no kick)
    double *vx, *vy, *vz;
    int *work;
    const Ctrl *ctl;
};

template <int P, typename real>
__device__ __forceinline__ void l2p(const real *C, real hx, real hy, real hz, real &ax, real &ay, real &az) {
    real wx[P], wy[P], wz[P];
    wx[0] = wy[0] = wz[0] = real(1);
#pragma unroll
    for (int k = 1; k < P; k++) {
        wx[k] = wx[k - 1] * hx;
        wy[k] = wy[k - 1] * hy;
        wz[k] = wz[k - 1] * hz;
    }
#pragma unroll
    for (int nb = 0; nb < P; nb++)
#pragma unroll
        for (int kb = 0; kb <= nb; kb++)
#pragma unroll
            for (int cb = 0; cb <= kb; cb++) {
                const int ab = nb - kb, bb = kb - cb;
                const real w = wx[ab] * wy[bb] * wz[cb] * static_cast<real>(inv_mfact(ab, bb, cb));
                ax += C[cidx(ab + 1, bb, cb)] * w;
                ay += C[cidx(ab, bb + 1, cb)] * w;
                az += C[cidx(ab, bb, cb + 1)] * w;
            }
}

// l2p without the terms of the order-1 coefficients (the field at the centre)
template <int P, typename real>
__device__ __forceinline__ void l2p_high(const real *C, real hx, real hy, real hz, real &ax, real &ay, real &az) {
    real wx[P], wy[P], wz[P];
    wx[0] = wy[0] = wz[0] = real(1);
#pragma unroll
    for (int k = 1; k < P; k++) {
        wx[k] = wx[k - 1] * hx;
        wy[k] = wy[k - 1] * hy;
        wz[k] = wz[k - 1] * hz;
    }
#pragma unroll
    for (int nb = 1; nb < P; nb++)
#pragma unroll
        for (int kb = 0; kb <= nb; kb++)
#pragma unroll
            for (int cb = 0; cb <= kb; cb++) {
                const int ab = nb - kb, bb = kb - cb;
                const real w = wx[ab] * wy[bb] * wz[cb] * static_cast<real>(inv_mfact(ab, bb, cb));
                ax += C[cidx(ab + 1, bb, cb)] * w;
                ay += C[cidx(ab, bb + 1, cb)] * w;
                az += C[cidx(ab, bb, cb + 1)] * w;
            }
}

// ---------------------------------------------------------------------------
// Tree descent (Sect. 3.4.3, Eq. shifting): every cell's complete local
// expansion is its own M2L sum plus its parent's complete expansion
// translated to the cell's centre,
//   C-hat_alpha(c) = C-hat_alpha(c, own)
//       + (rho_c/rho_a)^|alpha| sum_beta C-hat_{alpha+beta}(a) (h)^beta / beta!,
//   h = (s_c - s_a)/rho_a,  a = parent(c),
// from the root down: one translation per cell.  The result goes to Cf (Ch
// keeps the own M2L sums).
//
// One pass, no level barriers: warps claim cells in increasing index order
// (cells are level-major, so a parent always precedes its children) and a
// warp waits only for its cell's parent, whose warp claimed it earlier and is
// therefore running; the earliest unfinished cell always has its parent done,
// so the pass always advances.  A cell is published by its `done` word (the
// epoch of this descent, advanced by the M2L launch that precedes it), with
// release/acquire ordering; the wait is bounded (ERR_TIMEOUT) and gives up as
// soon as the call has aborted.
//
// A translation is done as three one-dimensional shifts, along x, y, z in
// turn (beta! = bx! by! bz!): D_gamma = sum_k C_{gamma + k e_axis} h_axis^k / k!,
// with coefficients beyond order p taken as zero.
//
// Mixed precision: the order-1 coefficients (the field at the centre) carry
// the whole far field of the disk and are passed down every level, so they
// are kept as double-float pairs (hi in Cf, lo in Cf_lo): the translation of
// the higher orders into them is formed in FP32 with the parent's order-1
// terms left out, and it and the cell's own M2L sum are added to the parent's
// pair exactly (two-sum), so that rounding does not build up with depth.
// ---------------------------------------------------------------------------
struct DescendArgs {
    const int *parent;
    const float4 *gh, *gl;
    const double *sx, *sy, *sz, *rho;
    const void *Ch;
    const float *Ch_lo;        // [cells][3] mixed: low parts of the own order-1 sums
    void *Cf;
    float *Cf_lo;              // [cells][3] mixed: low parts of the order-1 coefficients
    unsigned *done;            // [cells]: epoch of the descent that completed the cell
    int *work;                 // claim counter, zeroed by the M2L launch
    Ctrl *ctl;                 // desc_epoch: this descent's epoch (advanced by the M2L launch)
};

constexpr int DESC_WARPS = 8;

// Index of (a, b, c) + k e_axis in the order-1.. storage, for an output of
// order n with kk = b + c.
template <int AXIS>
__device__ __forceinline__ int shifted_index(int n, int kk, int c, int k) {
    const int m = n + k;
    const int t = AXIS == 0 ? kk : kk + k;
    return m * (m + 1) * (m + 2) / 6 + t * (t + 1) / 2 + c + (AXIS == 2 ? k : 0) - 1;
}

template <int P, int AXIS, typename real>
__device__ __forceinline__ real shift_axis(const real *src, const real (&w)[P + 1], int n, int kk, int c) {
    real s = src[shifted_index<AXIS>(n, kk, c, 0)];
#pragma unroll
    for (int k = 1; k <= P - 1; k++)
        if (k <= P - n) s += src[shifted_index<AXIS>(n, kk, c, k)] * w[k];
    return s;
}

__device__ __forceinline__ unsigned ld_acquire_u32_any(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <int P, typename real>
__global__ void __launch_bounds__(32 * DESC_WARPS) k_descend(DescendArgs A) {
    constexpr int NC = num_c(P);
    constexpr int PER = (NC + 31) / 32;
    constexpr bool f32 = std::is_same<real, float>::value;
    __shared__ real s_A[DESC_WARPS][NC];
    __shared__ real s_B[DESC_WARPS][NC];
    if (aborted(A.ctl)) return;
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const real *Ch = static_cast<const real *>(A.Ch);
    real *Cf = static_cast<real *>(A.Cf);
    real *sa = s_A[wl], *sb = s_B[wl];
    const unsigned ep = *reinterpret_cast<const volatile unsigned *>(&A.ctl->desc_epoch);
    const unsigned long long limit = A.ctl->wait_ns ? A.ctl->wait_ns : 1000000000ull;
    const int ncells = A.ctl->n_cells;
    int on[PER], okk[PER], oc[PER];
#pragma unroll
    for (int k = 0; k < PER; k++) {
        const int i = lane + 32 * k;
        const int e = i < NC ? i + 1 : 1;
        const int a0 = c_exp2.e[e][0], b0 = c_exp2.e[e][1], c0 = c_exp2.e[e][2];
        on[k] = a0 + b0 + c0;
        okk[k] = b0 + c0;
        oc[k] = c0;
    }
    while (true) {
        int c = 0;
        if (lane == 0) c = atomicAdd(A.work, 1);
        c = __shfl_sync(0xffffffffu, c, 0);
        if (c >= ncells) break;
        real acc[PER];
#pragma unroll
        for (int k = 0; k < PER; k++) {
            const int i = lane + 32 * k;
            acc[k] = i < NC ? Ch[(size_t)c * NC + i] : real(0);
        }
        // mixed: the order-1 pair of this cell (lanes 0..2); the root's is its own M2L sum
        float hi1 = f32 ? static_cast<float>(acc[0]) : 0.0f, lo1 = 0.0f, phi = 0.0f, plo = 0.0f;
        const float own_lo = (f32 && lane < 3) ? __ldg(&A.Ch_lo[3 * c + lane]) : 0.0f;
        lo1 = own_lo;
        const int a = A.parent[c];
        if (a >= 0) {
            int ok = 1;
            if (lane == 0) {
                const unsigned long long t0 = global_ns();
                for (unsigned spins = 0; ld_acquire_u32_any(&A.done[a]) != ep; spins++) {
                    if ((spins & 63u) == 63u && (aborted(A.ctl) || global_ns() - t0 > limit)) {
                        atomicOr(&A.ctl->err, ERR_TIMEOUT);
                        ok = 0;
                        break;
                    }
                }
            }
            if (!__shfl_sync(0xffffffffu, ok, 0)) return;
            __syncwarp();   // orders lane 0's acquire before every lane's reads of the parent
            for (int i = lane; i < NC; i += 32) sa[i] = __ldcg(&Cf[(size_t)a * NC + i]);
            if constexpr (f32) {   // the parent's order-1 pair is added exactly below, not shifted
                if (lane < 3) {
                    phi = sa[lane];
                    plo = __ldcg(&A.Cf_lo[3 * a + lane]);
                    sa[lane] = 0.0f;
                }
            }
            real hx, hy, hz, ratio;
            if constexpr (f32) {
                const float4 ch = A.gh[c], cl = A.gl[c], ah = A.gh[a], al = A.gl[a];
                const float ir = 1.0f / al.w;   // exact: rho is a power of two
                ratio = cl.w * ir;
                hx = ((ch.x - ah.x) + (cl.x - al.x)) * ir;
                hy = ((ch.y - ah.y) + (cl.y - al.y)) * ir;
                hz = ((ch.z - ah.z) + (cl.z - al.z)) * ir;
            } else {
                const double iar = 1.0 / A.rho[a];
                ratio = A.rho[c] * iar;
                hx = (A.sx[c] - A.sx[a]) * iar;
                hy = (A.sy[c] - A.sy[a]) * iar;
                hz = (A.sz[c] - A.sz[a]) * iar;
            }
            real wx[P + 1], wy[P + 1], wz[P + 1];
            wx[0] = wy[0] = wz[0] = real(1);
#pragma unroll
            for (int k = 1; k <= P; k++) {
                wx[k] = wx[k - 1] * hx;
                wy[k] = wy[k - 1] * hy;
                wz[k] = wz[k - 1] * hz;
            }
#pragma unroll
            for (int k = 2; k <= P; k++) {
                const real f = static_cast<real>(ifact(k));   // compile-time constant (k unrolled)
                wx[k] *= f; wy[k] *= f; wz[k] *= f;
            }
            __syncwarp();
#pragma unroll
            for (int k = 0; k < PER; k++)
                if (lane + 32 * k < NC) sb[lane + 32 * k] = shift_axis<P, 0>(sa, wx, on[k], okk[k], oc[k]);
            __syncwarp();
#pragma unroll
            for (int k = 0; k < PER; k++)
                if (lane + 32 * k < NC) sa[lane + 32 * k] = shift_axis<P, 1>(sb, wy, on[k], okk[k], oc[k]);
            __syncwarp();
#pragma unroll
            for (int k = 0; k < PER; k++) {
                if (lane + 32 * k >= NC) continue;
                real s = shift_axis<P, 2>(sa, wz, on[k], okk[k], oc[k]);
                for (int q = 0; q < on[k]; q++) s *= ratio;   // (rho_c/rho_a)^n, exact powers of two
                if (f32 && k == 0 && lane < 3) {
                    // order 1: (parent pair) * ratio + higher orders + own sum, in double-float
                    hi1 = phi * static_cast<float>(ratio);
                    lo1 = plo * static_cast<float>(ratio);
                    df_add(hi1, lo1, static_cast<float>(s));
                    df_add(hi1, lo1, static_cast<float>(acc[0]));
                    lo1 += own_lo;
                    acc[0] = static_cast<real>(hi1);
                } else {
                    acc[k] += s;
                }
            }
            __syncwarp();
        }
#pragma unroll
        for (int k = 0; k < PER; k++) {
            const int i = lane + 32 * k;
            if (i < NC) Cf[(size_t)c * NC + i] = acc[k];
        }
        if (f32 && lane < 3) A.Cf_lo[3 * c + lane] = lo1;
        __syncwarp();
        if (lane == 0) {
            fence_acq_rel_gpu();
            st_release_u32(&A.done[c], ep);
        }
    }
}

// ---------------------------------------------------------------------------
// Evaluation kernel: one block of EV_THREADS threads per leaf, leaves handed
// out dynamically.  The leaf's m targets (taken EV_THREADS at a time if the
// leaf is larger) are taken by G = floor(EV_THREADS / m) groups of m threads:
// thread (g, t) sums the staged sources k = g, g + G, g + 2G, ... for target
// t, so a leaf of a few moonlets keeps the lanes busy.  The direct list is
// staged EV_BUF moonlets at a time, cutting source leaves where the buffer
// ends.  Mixed precision: every thread adds its FP32 partial sum to a
// double-float total every 32 sources (two-sum), and the groups' totals are
// added in group order, so that the rounding of a long FP32 running sum
// (dominated by the nearest pull) does not grow with the direct list.
// ---------------------------------------------------------------------------
constexpr int EV_THREADS = 128;
constexpr int EV_BUF = 512;

template <int P, typename real>
struct EvShared {
    __align__(16) unsigned char buf[EV_BUF * 32];   // FP32: float4 hi[EV_BUF] (xyz, mu), lo[EV_BUF]
                                                    // FP64: double x, y, z, mu [EV_BUF]
    real red[6][EV_THREADS];
    int lfirst[32], lpre[32];
    int leaf, total, next_si, next_soff;
};

template <int P, typename real>
__global__ void __launch_bounds__(EV_THREADS, 6) k_eval(EvalArgs A) {
    constexpr bool f32 = std::is_same<real, float>::value;
    __shared__ EvShared<P, real> S;
    if (aborted(A.ctl)) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nl = A.ctl->n_leaves;
    float4 *sh = reinterpret_cast<float4 *>(S.buf), *sl = sh + EV_BUF;
    double *bx = reinterpret_cast<double *>(S.buf), *by = bx + EV_BUF, *bz = by + EV_BUF, *bm = bz + EV_BUF;
    while (true) {
        __syncthreads();
        if (tid == 0) S.leaf = atomicAdd(A.work, 1);
        __syncthreads();
        const int li = S.leaf;
        if (li >= nl) break;
        const int leaf = A.leaves[li];
        const int f = A.first[leaf], cnt = A.count[leaf];
        const int s0 = min(A.p2p_off[leaf], A.p2p_dir_cap), s1 = min(A.p2p_off[leaf + 1], A.p2p_dir_cap);
        for (int t0 = 0; t0 < cnt; t0 += EV_THREADS) {
            const int m = min(EV_THREADS, cnt - t0);
            const int G = EV_THREADS / m, g = tid / m, tt = tid - g * m;
            const bool act = g < G;   // the last EV_THREADS - G m threads only help with staging
            const int i = f + t0 + (act ? tt : 0);
            const float4 th = A.hi4[i], tl = A.lo4[i];
            const double X = A.x[i], Y = A.y[i], Z = A.z[i];
            real ax = real(0), ay = real(0), az = real(0);
            // mixed: double-float totals, to which the FP32 partial sums are added every 32 sources
            float h3[3] = {0.f, 0.f, 0.f}, l3[3] = {0.f, 0.f, 0.f};
            int si = s0, soff = 0;
            while (si < s1) {
                __syncthreads();
                if (warp == 0) {
                    const int idx = si + lane;
                    int fst = 0, c = 0;
                    if (idx < s1) {
                        const int2 e = A.p2p_src[idx];
                        fst = e.x;
                        c = e.y;
                    }
                    if (lane == 0) { fst += soff; c -= soff; }
                    int inc = c;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int v = __shfl_up_sync(0xffffffffu, inc, o);
                        if (lane >= o) inc += v;
                    }
                    const int exc = inc - c;
                    const int total = min(EV_BUF, __shfl_sync(0xffffffffu, inc, 31));
                    S.lfirst[lane] = fst;
                    S.lpre[lane] = exc;
                    // source leaves consumed completely; the next one may be cut
                    const unsigned done = __ballot_sync(0xffffffffu, idx < s1 && inc <= total);
                    const int L = __popc(done);
                    const int excL = __shfl_sync(0xffffffffu, exc, L & 31);
                    if (lane == 0) {
                        S.total = total;
                        S.next_si = si + L;
                        S.next_soff = (L < 32 && si + L < s1) ? (L == 0 ? soff : 0) + (total - excL) : 0;
                    }
                }
                __syncthreads();
                const int total = S.total;
                for (int t = tid; t < total; t += EV_THREADS) {
                    int q = 0;
#pragma unroll
                    for (int st = 16; st > 0; st >>= 1)
                        if (S.lpre[q + st] <= t) q += st;
                    const int jj = S.lfirst[q] + t - S.lpre[q];
                    if constexpr (f32) {
                        sh[t] = A.hi4[jj];
                        sl[t] = A.lo4[jj];
                    } else {
                        bx[t] = A.x[jj];
                        by[t] = A.y[jj];
                        bz[t] = A.z[jj];
                        bm[t] = A.G * A.m[jj];
                    }
                }
                si = S.next_si;
                soff = S.next_soff;
                __syncthreads();
                if (act) {
                    if constexpr (f32) {
                        for (int k0 = g; k0 < total; k0 += 32 * G) {
                            const int k1 = min(total, k0 + 32 * G);
#pragma unroll 4
                            for (int k = k0; k < k1; k += G) p2p_f32(sh[k], sl[k], th, tl, ax, ay, az);
                            df_add(h3[0], l3[0], ax); df_add(h3[1], l3[1], ay); df_add(h3[2], l3[2], az);
                            ax = ay = az = 0.f;
                        }
                    } else {
#pragma unroll 2
                        for (int k = g; k < total; k += G) p2p_f64(bx[k], by[k], bz[k], bm[k], X, Y, Z, ax, ay, az);
                    }
                }
            }
            if constexpr (f32) {   // the groups' double-float totals, added in group order
                if (G > 1) {
                    __syncthreads();
#pragma unroll
                    for (int d = 0; d < 3; d++) {
                        S.red[d][tid] = h3[d];
                        S.red[3 + d][tid] = l3[d];
                    }
                    __syncthreads();
                    if (g == 0) {
#pragma unroll
                        for (int d = 0; d < 3; d++) {
                            h3[d] = l3[d] = 0.f;
                            for (int q = 0; q < G; q++) {
                                df_add(h3[d], l3[d], S.red[d][q * m + tt]);
                                l3[d] += S.red[3 + d][q * m + tt];
                            }
                        }
                    }
                }
                if (g == 0 && act) {
                    A.nx[i] = static_cast<double>(h3[0]) + static_cast<double>(l3[0]);
                    A.ny[i] = static_cast<double>(h3[1]) + static_cast<double>(l3[1]);
                    A.nz[i] = static_cast<double>(h3[2]) + static_cast<double>(l3[2]);
                }
            } else {
                if (G > 1) {
                    __syncthreads();
                    S.red[0][tid] = ax;
                    S.red[1][tid] = ay;
                    S.red[2][tid] = az;
                    __syncthreads();
                    if (g == 0) {
                        ax = ay = az = real(0);
                        for (int q = 0; q < G; q++) {
                            ax += S.red[0][q * m + tt];
                            ay += S.red[1][q * m + tt];
                            az += S.red[2][q * m + tt];
                        }
                    }
                }
                if (g == 0 && act) {
                    A.nx[i] = static_cast<double>(ax);
                    A.ny[i] = static_cast<double>(ay);
                    A.nz[i] = static_cast<double>(az);
                }
            }
        }
    }
}

// L2P of each leaf's complete local expansion (Eq. shifting at the moonlet),
// plus the near-field sums and the external forces: one thread per moonlet
// in tree order (the moonlets of a leaf are consecutive, so the threads of a
// warp read the same few expansions: broadcast loads).
constexpr int FAR_THREADS = 256;

template <int P, typename real>
__global__ void __launch_bounds__(FAR_THREADS) k_far(EvalArgs A) {
    constexpr int NC = num_c(P);
    constexpr bool f32 = std::is_same<real, float>::value;
    if (aborted(A.ctl)) return;
    const real *Cf = static_cast<const real *>(A.Cf);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += gridDim.x * blockDim.x) {
        const int leaf = __ldg(&A.leaf_of[i]);
        const real *C = Cf + (size_t)leaf * NC;
        const double X = A.x[i], Y = A.y[i], Z = A.z[i];
        double fx, fy, fz;   // the far field at the moonlet
        if constexpr (f32) {
            // the order-1 pair (hi in Cf, lo in Cf_lo) and the higher orders, added in FP64
            const float4 lgh = __ldg(&A.gh[leaf]), lgl = __ldg(&A.gl[leaf]);
            const float4 th = A.hi4[i], tl = A.lo4[i];
            const float irf = 1.0f / lgl.w;   // exact: rho is a power of two
            float lx = 0.f, ly = 0.f, lz = 0.f;
            l2p_high<P, real>(C, ((th.x - lgh.x) + (tl.x - lgl.x)) * irf, ((th.y - lgh.y) + (tl.y - lgl.y)) * irf,
                              ((th.z - lgh.z) + (tl.z - lgl.z)) * irf, lx, ly, lz);
            const double ir = static_cast<double>(irf);
            fx = ((static_cast<double>(C[0]) + static_cast<double>(__ldg(&A.Cf_lo[3 * leaf]))) + static_cast<double>(lx)) * ir;
            fy = ((static_cast<double>(C[1]) + static_cast<double>(__ldg(&A.Cf_lo[3 * leaf + 1]))) + static_cast<double>(ly)) * ir;
            fz = ((static_cast<double>(C[2]) + static_cast<double>(__ldg(&A.Cf_lo[3 * leaf + 2]))) + static_cast<double>(lz)) * ir;
        } else {
            const double irho = 1.0 / A.rho[leaf];
            real lx = real(0), ly = real(0), lz = real(0);
            l2p<P, real>(C, (X - A.sx[leaf]) * irho, (Y - A.sy[leaf]) * irho, (Z - A.sz[leaf]) * irho, lx, ly, lz);
            fx = lx * irho; fy = ly * irho; fz = lz * irho;
        }
        double ex, ey, ez;
        external_force(A.ext, X, Y, Z, ex, ey, ez);
        // far part + near sums, added in FP64 (the near sums arrive as double-float totals)
        const double mx = fx + A.nx[i];
        const double my = fy + A.ny[i];
        const double mz = fz + A.nz[i];
        const double gx = mx + ex, gy = my + ey, gz = mz + ez;
        A.ax[i] = gx;
        A.ay[i] = gy;
        A.az[i] = gz;
        if (A.amx) { A.amx[i] = mx; A.amy[i] = my; A.amz[i] = mz; }
        if (A.kick_h != 0.0) {   // the step's closing half kick, as k_kick computes it
            A.vx[i] = dadd(A.vx[i], dmul(A.kick_h, gx));
            A.vy[i] = dadd(A.vy[i], dmul(A.kick_h, gy));
            A.vz[i] = dadd(A.vz[i], dmul(A.kick_h, gz));
        }
    }
}

template <int P, typename real>
static void descend_t(ncorp_ctx *c, DescendArgs D) {
    int per_sm = 0;
    NCORP_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, reinterpret_cast<const void *>(k_descend<P, real>), 32 * DESC_WARPS, 0));
    if (per_sm < 1) per_sm = 1;
    k_descend<P, real><<<per_sm * c->num_sms, 32 * DESC_WARPS, 0, c->stream>>>(D);
    c->launches++;
    NCORP_CUDA_CHECK(cudaGetLastError());
}

template <int P, typename real>
static void eval_t(ncorp_ctx *c, const EvalArgs &A) {
    int per_sm = 0;
    NCORP_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, reinterpret_cast<const void *>(k_eval<P, real>), EV_THREADS, 0));
    if (per_sm < 1) per_sm = 1;
    k_eval<P, real><<<per_sm * c->num_sms, EV_THREADS, 0, c->stream>>>(A);
    c->launches++;
}

template <int P, typename real>
static void far_t(ncorp_ctx *c, const EvalArgs &A) {
    k_far<P, real><<<grid_for(A.n, FAR_THREADS, 8 * c->num_sms), FAR_THREADS, 0, c->stream>>>(A);
    c->launches++;
}

void launch_descend(ncorp_ctx *c, int p, bool mixed) {
    Cells &C = c->cells;
    DescendArgs D;
    D.parent = C.parent;
    D.gh = C.gh; D.gl = C.gl; D.sx = C.sx; D.sy = C.sy; D.sz = C.sz; D.rho = C.rho;
    D.Ch = C.Ch; D.Ch_lo = C.Ch_lo; D.Cf = C.Cf; D.Cf_lo = C.Cf_lo; D.done = C.done; D.work = c->work_counter + 1; D.ctl = c->ctl;
#define NCORP_DESC_CASE(PP)                      \
    case PP:                                     \
        if (mixed) descend_t<PP, float>(c, D);   \
        else descend_t<PP, double>(c, D);        \
        break;
    switch (p) {
        NCORP_DESC_CASE(1)
        NCORP_DESC_CASE(2)
        NCORP_DESC_CASE(3)
        NCORP_DESC_CASE(4)
        NCORP_DESC_CASE(5)
        NCORP_DESC_CASE(6)
        default: break;
    }
#undef NCORP_DESC_CASE
}

static EvalArgs eval_args(ncorp_ctx *c, const ParticleSet &P, double G, ExtForce ext, bool want_mutual) {
    Cells &C = c->cells;
    EvalArgs A;
    A.n = c->cur_n;
    A.leaves = C.leaves; A.level = C.level; A.parent = C.parent; A.first = C.first; A.count = C.count;
    A.leaf_of = C.leaf_of;
    A.sx = C.sx; A.sy = C.sy; A.sz = C.sz; A.rho = C.rho;
    A.gh = C.gh; A.gl = C.gl;
    A.Cf = C.Cf;
    A.Cf_lo = C.Cf_lo;
    A.p2p_off = c->wl.p2p_off; A.p2p_src = c->wl.p2p_src; A.p2p_dir_cap = c->wl.p2p_dir_cap;
    A.x = P.x; A.y = P.y; A.z = P.z; A.m = P.m;
    A.hi4 = P.hi4; A.lo4 = P.lo4;
    A.G = G;
    A.ext = ext;
    A.ax = P.ax; A.ay = P.ay; A.az = P.az;
    A.amx = want_mutual ? c->amx : nullptr;
    A.amy = want_mutual ? c->amy : nullptr;
    A.amz = want_mutual ? c->amz : nullptr;
    A.nx = c->amx; A.ny = c->amy; A.nz = c->amz;   // the far kernel overwrites them in place
    A.work = c->work_counter;
    A.ctl = c->ctl;
    A.kick_h = 0.0;
    A.vx = A.vy = A.vz = nullptr;
    return A;
}

// The work counter was zeroed by the gravity walk's k_walk_init.
void launch_near(ncorp_ctx *c, const ParticleSet &P, int p, bool mixed, double G) {
    const EvalArgs A = eval_args(c, P, G, ExtForce{}, false);
#define NCORP_EVAL_CASE(PP)                      \
    case PP:                                     \
        if (mixed) eval_t<PP, float>(c, A);      \
        else eval_t<PP, double>(c, A);           \
        break;
    switch (p) {
        NCORP_EVAL_CASE(1)
        NCORP_EVAL_CASE(2)
        NCORP_EVAL_CASE(3)
        NCORP_EVAL_CASE(4)
        NCORP_EVAL_CASE(5)
        NCORP_EVAL_CASE(6)
        default: break;
    }
#undef NCORP_EVAL_CASE
    NCORP_CUDA_CHECK(cudaGetLastError());
}

void launch_far(ncorp_ctx *c, const ParticleSet &P, int p, bool mixed, double G, ExtForce ext, bool want_mutual,
                double kick_h) {
    EvalArgs A = eval_args(c, P, G, ext, want_mutual);
    A.kick_h = kick_h;
    A.vx = P.vx; A.vy = P.vy; A.vz = P.vz;
#define NCORP_FAR_CASE(PP)                       \
    case PP:                                     \
        if (mixed) far_t<PP, float>(c, A);       \
        else far_t<PP, double>(c, A);            \
        break;
    switch (p) {
        NCORP_FAR_CASE(1)
        NCORP_FAR_CASE(2)
        NCORP_FAR_CASE(3)
        NCORP_FAR_CASE(4)
        NCORP_FAR_CASE(5)
        NCORP_FAR_CASE(6)
        default: break;
    }
#undef NCORP_FAR_CASE
    NCORP_CUDA_CHECK(cudaGetLastError());
}

}  // namespace ncorp
