// eval.cu -- tree descent and evaluation at the moonlets: L2L from the root
// to each leaf and L2P (Eq. shifting), the direct ("brute force") gravity of
// the leaf's near-field list, and the central-body / distant-star forces
// (App. B.1, B.3).
//
// One warp per leaf, leaves handed out dynamically.  The descent of Sect.
// 3.4.3 (a cell adds its parent's C translated to its own centre, from the
// root down) is followed along the leaf's ancestor chain:
//   C-hat_alpha(child) = C-hat_alpha(child, own M2L)
//       + (rho_c/rho_p)^|alpha| sum_beta C-hat_{alpha+beta}(parent) (delta/rho_p)^beta / beta!,
//   delta = s_child - s_parent,
// which is Eq. shifting over symmetric multi-indices in scaled form.  Then
// every moonlet of the leaf gets
//   a = (1/rho) sum_{|beta| <= p-1} C-hat_{e_k+beta} (d/rho)^beta / beta!,  d = x - s_leaf,
// plus sum_j mu_j (x_j - x)/|x_j - x|^3 over the moonlets of its direct list
// (mu_j = G m_j; coincident pairs, the moonlet itself included, are skipped),
// plus the external forces in FP64.  Each lane owns two moonlets and builds
// their sums in registers; they are written once.
//
// Mixed precision: the direct sum reads every position as an FP32 pair
// (hi, lo) with x = hi + lo; (hi_j - hi_i) + (lo_j - lo_i) gives the
// separation to ~1e-7 relative at any distance, so no FP64 work is done per
// pair.
#include <type_traits>

#include "ctx.h"

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
    const int *leaves, *level, *parent, *first, *count;
    const double *sx, *sy, *sz, *rho;
    const float4 *gh, *gl, *shift;
    const void *Ch;
    const int *p2p_off, *p2p_src;
    int p2p_dir_cap;
    const double *x, *y, *z, *m;
    const float4 *hi4, *lo4;
    double G;
    ExtForce ext;
    double *ax, *ay, *az;
    double *amx, *amy, *amz;
    int *work;
    const Ctrl *ctl;
};

constexpr int EVAL_WARPS = 4;   // warps per block

constexpr int EVAL_BUF = 128;   // staged source moonlets per warp

template <int P, typename real>
struct EvalShared {
    static constexpr int NC = num_c(P);
    real C[1][NC];
    float4 h[EVAL_BUF], l[EVAL_BUF];         // FP32 path: staged sources (hi + mu, lo)
    double dx[32], dy[32], dz[32], dm[32];   // FP64 path
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

__device__ __forceinline__ void external_force(const ExtForce &E, double X, double Y, double Z, double &ex, double &ey,
                                               double &ez) {
    const double r2 = X * X + Y * Y + Z * Z;
    const double fc = -E.GMc / (r2 * sqrt(r2));
    ex = fc * X;
    ey = fc * Y;
    ez = fc * Z;
    if (E.star_k != 0.0) {
        const double c3 = 3.0 * (X * E.sx + Y * E.sy + Z * E.sz) * E.inv_rs2;
        ex -= E.star_k * (X - c3 * E.sx);
        ey -= E.star_k * (Y - c3 * E.sy);
        ez -= E.star_k * (Z - c3 * E.sz);
    }
}

__device__ __forceinline__ void p2p_f32(const float4 &h, const float4 &l, const float4 &th, const float4 &tl, float &ax,
                                        float &ay, float &az) {
    const float dx = (h.x - th.x) + (l.x - tl.x);
    const float dy = (h.y - th.y) + (l.y - tl.y);
    const float dz = (h.z - th.z) + (l.z - tl.z);
    const float r2 = dx * dx + dy * dy + dz * dz;
    if (r2 > 1e-30f) {
        const float inv = rsqrtf(r2);
        const float f3 = h.w * inv * inv * inv;
        ax += dx * f3;
        ay += dy * f3;
        az += dz * f3;
    }
}

__device__ __forceinline__ void p2p_f64(double jx, double jy, double jz, double mu, double X, double Y, double Z,
                                        double &ax, double &ay, double &az) {
    const double dx = jx - X, dy = jy - Y, dz = jz - Z;
    const double r2 = dx * dx + dy * dy + dz * dz;
    if (r2 > 0.0) {
        const double inv = 1.0 / sqrt(r2);
        const double f3 = mu * inv * inv * inv;
        ax += dx * f3;
        ay += dy * f3;
        az += dz * f3;
    }
}

// ---------------------------------------------------------------------------
// Tree descent (Sect. 3.4.3): level by level from the root, every cell adds
// its parent's (already complete) local expansion translated to its own
// centre.  One cooperative launch; a warp per cell, lanes over the output
// coefficients; the cell's C-hat is overwritten with the complete expansion.
// ---------------------------------------------------------------------------
struct DescendArgs {
    const int *parent;
    const float4 *shift;
    const double *sx, *sy, *sz, *rho;
    void *Ch;
    Ctrl *ctl;
};

template <int P, typename real>
__global__ void __launch_bounds__(256) k_descend(DescendArgs A) {
    constexpr int NC = num_c(P);
    constexpr bool f32 = std::is_same<real, float>::value;
    __shared__ real s_C[8][NC];
    __shared__ real s_pw[8][3][P + 1];
    if (aborted(A.ctl)) return;
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
    real *Ch = static_cast<real *>(A.Ch);
    volatile Ctrl *vc = A.ctl;
    const int maxl = vc->max_level;
    for (int lev = 1; lev <= maxl; lev++) {
        const int ls = vc->level_start[lev], le = vc->level_start[lev + 1];
        for (int c = ls + gw; c < le; c += nwarps) {
            const int pc = A.parent[c];
            for (int i = lane; i < NC; i += 32) s_C[wl][i] = __ldcg(&Ch[(size_t)pc * NC + i]);
            real ratio;
            if constexpr (f32) {
                const float4 sh = A.shift[c];
                ratio = sh.w;
                if (lane < 3) {
                    const float h = lane == 0 ? sh.x : (lane == 1 ? sh.y : sh.z);
                    float pw = 1.0f;
                    for (int k = 0; k <= P; k++) {
                        s_pw[wl][lane][k] = pw;
                        pw *= h;
                    }
                }
            } else {
                const double iprho = 1.0 / A.rho[pc];
                ratio = A.rho[c] * iprho;
                if (lane < 3) {
                    const double dv = lane == 0 ? A.sx[c] - A.sx[pc] : (lane == 1 ? A.sy[c] - A.sy[pc] : A.sz[c] - A.sz[pc]);
                    const real h = dv * iprho;
                    real pw = real(1);
                    for (int k = 0; k <= P; k++) {
                        s_pw[wl][lane][k] = pw;
                        pw *= h;
                    }
                }
            }
            __syncwarp();
            for (int i = lane; i < NC; i += 32) {
                const int a = c_exp2.e[i + 1][0], b = c_exp2.e[i + 1][1], cc = c_exp2.e[i + 1][2];
                const int n = a + b + cc;
                real acc = real(0);
                for (int nb = 0; nb <= P - n; nb++)
                    for (int kb = 0; kb <= nb; kb++)
                        for (int c2 = 0; c2 <= kb; c2++) {
                            const int ab = nb - kb, bb = kb - c2;
                            const real w = s_pw[wl][0][ab] * s_pw[wl][1][bb] * s_pw[wl][2][c2] *
                                           static_cast<real>(c_ifact[ab] * c_ifact[bb] * c_ifact[c2]);
                            acc += s_C[wl][cidx(a + ab, b + bb, cc + c2)] * w;
                        }
                for (int k = 0; k < n; k++) acc *= ratio;   // (rho_c/rho_p)^n applied to the small factor first
                Ch[(size_t)c * NC + i] += acc;
            }
            __syncwarp();
        }
        if (!grid_sync(A.ctl)) return;
    }
}

// Near field of one group of targets (NT per lane) from the leaf's direct
// list: source leaves are taken four at a time, their moonlets staged into
// the warp's buffer, and every lane sums over the whole buffer.
template <int NT>
__device__ __forceinline__ void p2p_list_f32(const EvalArgs &A, float4 *bh, float4 *bl, int s0, int s1, int lane,
                                             const float4 *th, const float4 *tl, float *ax, float *ay, float *az) {
    for (int si = s0; si < s1; si += 4) {
        const int nc = min(4, s1 - si);
        int fst = 0, cn = 0;
        if (lane < nc) {
            const int src = A.p2p_src[si + lane];
            fst = A.first[src];
            cn = A.count[src];
        }
        int f[4], o[4], total = 0;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            f[q] = __shfl_sync(0xffffffffu, fst, q);
            o[q] = total;
            total += __shfl_sync(0xffffffffu, cn, q);
        }
        for (int w0 = 0; w0 < total; w0 += EVAL_BUF) {
            const int lim = min(EVAL_BUF, total - w0);
            __syncwarp();
            for (int t = lane; t < EVAL_BUF; t += 32) {
                const int g = w0 + t;
                if (t < lim) {
                    const int q = g >= o[3] ? 3 : (g >= o[2] ? 2 : (g >= o[1] ? 1 : 0));
                    const int jj = f[q] + g - o[q];
                    bh[t] = A.hi4[jj];
                    bl[t] = A.lo4[jj];
                } else if (t < ((lim + 7) & ~7)) {   // pad to a multiple of 8 with mu = 0 far away
                    bh[t] = make_float4(1e18f, 0.f, 0.f, 0.f);
                    bl[t] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            __syncwarp();
            const int lim8 = (lim + 7) & ~7;
            for (int k = 0; k < lim8; k += 8) {
#pragma unroll
                for (int u = 0; u < 8; u++) {
                    const float4 h = bh[k + u], l = bl[k + u];
#pragma unroll
                    for (int t = 0; t < NT; t++) p2p_f32(h, l, th[t], tl[t], ax[t], ay[t], az[t]);
                }
            }
        }
    }
}

template <int NT>
__device__ __forceinline__ void p2p_list_f64(const EvalArgs &A, double *bx, double *by, double *bz, double *bm,
                                             int s0, int s1, int lane, const double *X, const double *Y,
                                             const double *Z, double *ax, double *ay, double *az) {
    for (int si = s0; si < s1; si++) {
        const int src = A.p2p_src[si];
        const int sf = A.first[src], sc = A.count[src];
        for (int j0 = 0; j0 < sc; j0 += 32) {
            const int lim = min(32, sc - j0);
            __syncwarp();
            if (lane < lim) {
                const int j = sf + j0 + lane;
                bx[lane] = A.x[j];
                by[lane] = A.y[j];
                bz[lane] = A.z[j];
                bm[lane] = A.G * A.m[j];
            }
            __syncwarp();
            for (int k = 0; k < lim; k++)
#pragma unroll
                for (int t = 0; t < NT; t++) p2p_f64(bx[k], by[k], bz[k], bm[k], X[t], Y[t], Z[t], ax[t], ay[t], az[t]);
        }
    }
}

// L2P + near field + external forces for the targets f + t0 + lane + 32 t, t < NT
template <int P, typename real, int NT>
__device__ __forceinline__ void eval_targets(const EvalArgs &A, EvalShared<P, real> &S, const real *C, int leaf, int f,
                                             int cnt, int t0, int lane, int s0, int s1) {
    constexpr bool f32 = std::is_same<real, float>::value;
    const float4 lgh = A.gh[leaf], lgl = A.gl[leaf];
    const float irf = 1.0f / lgl.w;   // exact: rho is a power of two
    real ax[NT], ay[NT], az[NT];
    double X[NT], Y[NT], Z[NT];
    float4 th[NT], tl[NT];
    bool act[NT];
#pragma unroll
    for (int t = 0; t < NT; t++) {
        const int ti = t0 + lane + 32 * t;
        act[t] = ti < cnt;
        const int i = f + (act[t] ? ti : 0);
        ax[t] = ay[t] = az[t] = real(0);
        X[t] = A.x[i]; Y[t] = A.y[i]; Z[t] = A.z[i];
        th[t] = A.hi4[i];
        tl[t] = A.lo4[i];
        if constexpr (f32) {
            l2p<P, real>(C, ((th[t].x - lgh.x) + (tl[t].x - lgl.x)) * irf, ((th[t].y - lgh.y) + (tl[t].y - lgl.y)) * irf,
                         ((th[t].z - lgh.z) + (tl[t].z - lgl.z)) * irf, ax[t], ay[t], az[t]);
            ax[t] *= irf; ay[t] *= irf; az[t] *= irf;
        } else {
            const double irho = 1.0 / A.rho[leaf];
            l2p<P, real>(C, (X[t] - A.sx[leaf]) * irho, (Y[t] - A.sy[leaf]) * irho, (Z[t] - A.sz[leaf]) * irho, ax[t],
                         ay[t], az[t]);
            ax[t] *= irho; ay[t] *= irho; az[t] *= irho;
        }
    }
    if constexpr (f32) p2p_list_f32<NT>(A, S.h, S.l, s0, s1, lane, th, tl, ax, ay, az);
    else p2p_list_f64<NT>(A, S.dx, S.dy, S.dz, S.dm, s0, s1, lane, X, Y, Z, ax, ay, az);
#pragma unroll
    for (int t = 0; t < NT; t++) {
        if (!act[t]) continue;
        const int i = f + t0 + lane + 32 * t;
        double ex, ey, ez;
        external_force(A.ext, X[t], Y[t], Z[t], ex, ey, ez);
        const double mx = ax[t], my = ay[t], mz = az[t];
        A.ax[i] = mx + ex;
        A.ay[i] = my + ey;
        A.az[i] = mz + ez;
        if (A.amx) { A.amx[i] = mx; A.amy[i] = my; A.amz[i] = mz; }
    }
}

template <int P, typename real>
__global__ void __launch_bounds__(32 * EVAL_WARPS, 4) k_eval(EvalArgs A) {
    constexpr int NC = num_c(P);
    __shared__ EvalShared<P, real> sh_all[EVAL_WARPS];
    if (aborted(A.ctl)) return;
    EvalShared<P, real> &S = sh_all[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const real *Ch = static_cast<const real *>(A.Ch);
    const int nl = A.ctl->n_leaves;
    while (true) {
        int li = 0;
        if (lane == 0) li = atomicAdd(A.work, 1);
        li = __shfl_sync(0xffffffffu, li, 0);
        if (li >= nl) break;
        const int leaf = A.leaves[li];
        __syncwarp();
        for (int i = lane; i < NC; i += 32) S.C[0][i] = Ch[(size_t)leaf * NC + i];   // complete after the descent
        __syncwarp();
        const int f = A.first[leaf], cnt = A.count[leaf];
        const int s0 = min(A.p2p_off[leaf], A.p2p_dir_cap), s1 = min(A.p2p_off[leaf + 1], A.p2p_dir_cap);
        if (cnt <= 32) {
            eval_targets<P, real, 1>(A, S, S.C[0], leaf, f, cnt, 0, lane, s0, s1);
        } else {
            for (int t0 = 0; t0 < cnt; t0 += 64) eval_targets<P, real, 2>(A, S, S.C[0], leaf, f, cnt, t0, lane, s0, s1);
        }
        __syncwarp();
    }
}

template <int P, typename real>
static void descend_t(ncorp_ctx *c, DescendArgs D) {
    int per_sm = 0;
    NCORP_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, reinterpret_cast<const void *>(k_descend<P, real>), 256, 0));
    if (per_sm < 1) per_sm = 1;
    if (per_sm > 2) per_sm = 2;
    void *args[] = {&D};
    NCORP_CUDA_CHECK(cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(k_descend<P, real>),
                                                 dim3(per_sm * c->num_sms), dim3(256), args, 0, c->stream));
    c->launches++;
}

template <int P, typename real>
static void eval_t(ncorp_ctx *c, const EvalArgs &A) {
    k_eval<P, real><<<8 * c->num_sms, 32 * EVAL_WARPS, 0, c->stream>>>(A);
    c->launches++;
}

void launch_descend(ncorp_ctx *c, int p, bool mixed) {
    Cells &C = c->cells;
    DescendArgs D;
    D.parent = C.parent; D.shift = C.shift; D.sx = C.sx; D.sy = C.sy; D.sz = C.sz; D.rho = C.rho;
    D.Ch = C.Ch; D.ctl = c->ctl;
    NCORP_CUDA_CHECK(cudaMemsetAsync(&c->ctl->bar_count, 0, sizeof(unsigned), c->stream));
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

void launch_eval(ncorp_ctx *c, const ParticleSet &P, int p, bool mixed, double G, ExtForce ext, bool want_mutual) {
    Cells &C = c->cells;
    EvalArgs A;
    A.leaves = C.leaves; A.level = C.level; A.parent = C.parent; A.first = C.first; A.count = C.count;
    A.sx = C.sx; A.sy = C.sy; A.sz = C.sz; A.rho = C.rho;
    A.gh = C.gh; A.gl = C.gl; A.shift = C.shift;
    A.Ch = C.Ch;
    A.p2p_off = c->wl.p2p_off; A.p2p_src = c->wl.p2p_src; A.p2p_dir_cap = c->wl.p2p_dir_cap;
    A.x = P.x; A.y = P.y; A.z = P.z; A.m = P.m;
    A.hi4 = P.hi4; A.lo4 = P.lo4;
    A.G = G;
    A.ext = ext;
    A.ax = P.ax; A.ay = P.ay; A.az = P.az;
    A.amx = want_mutual ? c->amx : nullptr;
    A.amy = want_mutual ? c->amy : nullptr;
    A.amz = want_mutual ? c->amz : nullptr;
    A.work = c->work_counter;
    A.ctl = c->ctl;
    NCORP_CUDA_CHECK(cudaMemsetAsync(c->work_counter, 0, sizeof(int), c->stream));
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

}  // namespace ncorp
