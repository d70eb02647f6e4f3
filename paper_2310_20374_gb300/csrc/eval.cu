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

template <int P, typename real>
struct EvalShared {
    static constexpr int NC = num_c(P);
    real C[2][NC];
    real pw[3][P + 1];
    int path[MAX_LEVEL + 2];
    float4 h[32], l[32];                     // FP32 path: staged sources (hi + mu, lo)
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

template <int P, typename real>
__global__ void __launch_bounds__(32 * EVAL_WARPS) k_eval(EvalArgs A) {
    constexpr int NC = num_c(P);
    constexpr bool f32 = std::is_same<real, float>::value;
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
        // ---- ancestor chain and descent
        if (lane == 0) {
            int c = leaf;
            for (int d = A.level[leaf]; d >= 0; d--) {
                S.path[d] = c;
                c = A.parent[c];
            }
        }
        __syncwarp();
        const int depth = A.level[leaf];
        for (int i = lane; i < NC; i += 32) S.C[0][i] = Ch[(size_t)S.path[0] * NC + i];
        int cb = 0;
        __syncwarp();
        for (int d = 1; d <= depth; d++) {
            const int pc = S.path[d - 1], cc = S.path[d];
            const double iprho = 1.0 / A.rho[pc];
            if (lane < 3) {
                const double dv = lane == 0 ? A.sx[cc] - A.sx[pc] : (lane == 1 ? A.sy[cc] - A.sy[pc] : A.sz[cc] - A.sz[pc]);
                const real h = static_cast<real>(dv * iprho);
                real pw = real(1);
                for (int k = 0; k <= P; k++) {
                    S.pw[lane][k] = pw;
                    pw *= h;
                }
            }
            __syncwarp();
            const real ratio = static_cast<real>(A.rho[cc] * iprho);
            for (int i = lane; i < NC; i += 32) {
                const int a = c_exp2.e[i + 1][0], b = c_exp2.e[i + 1][1], c = c_exp2.e[i + 1][2];
                const int n = a + b + c;
                real acc = real(0);
                for (int nb = 0; nb <= P - n; nb++)
                    for (int kb = 0; kb <= nb; kb++)
                        for (int c2 = 0; c2 <= kb; c2++) {
                            const int ab = nb - kb, bb = kb - c2;
                            const real w = S.pw[0][ab] * S.pw[1][bb] * S.pw[2][c2] *
                                           static_cast<real>(c_ifact[ab] * c_ifact[bb] * c_ifact[c2]);
                            acc += S.C[cb][cidx(a + ab, b + bb, c + c2)] * w;
                        }
                for (int k = 0; k < n; k++) acc *= ratio;   // (rho_c/rho_p)^n applied to the small factor first
                S.C[cb ^ 1][i] = Ch[(size_t)cc * NC + i] + acc;
            }
            cb ^= 1;
            __syncwarp();
        }
        const real *C = S.C[cb];
        // ---- moonlets of the leaf, two per lane
        const int f = A.first[leaf], cnt = A.count[leaf];
        const double lsx = A.sx[leaf], lsy = A.sy[leaf], lsz = A.sz[leaf];
        const double irho = 1.0 / A.rho[leaf];
        const int s0 = min(A.p2p_off[leaf], A.p2p_dir_cap), s1 = min(A.p2p_off[leaf + 1], A.p2p_dir_cap);
        for (int t0 = 0; t0 < cnt; t0 += 64) {
            const int i0 = f + t0 + lane, i1 = i0 + 32;
            const bool act0 = t0 + lane < cnt, act1 = t0 + lane + 32 < cnt;
            real ax0 = 0, ay0 = 0, az0 = 0, ax1 = 0, ay1 = 0, az1 = 0;
            float4 th0 = make_float4(0, 0, 0, 0), tl0 = th0, th1 = th0, tl1 = th0;
            double X0 = 0, Y0 = 0, Z0 = 0, X1 = 0, Y1 = 0, Z1 = 0;
            if (act0) {
                X0 = A.x[i0]; Y0 = A.y[i0]; Z0 = A.z[i0];
                l2p<P, real>(C, static_cast<real>((X0 - lsx) * irho), static_cast<real>((Y0 - lsy) * irho),
                             static_cast<real>((Z0 - lsz) * irho), ax0, ay0, az0);
                if (f32) { th0 = A.hi4[i0]; tl0 = A.lo4[i0]; }
            }
            if (act1) {
                X1 = A.x[i1]; Y1 = A.y[i1]; Z1 = A.z[i1];
                l2p<P, real>(C, static_cast<real>((X1 - lsx) * irho), static_cast<real>((Y1 - lsy) * irho),
                             static_cast<real>((Z1 - lsz) * irho), ax1, ay1, az1);
                if (f32) { th1 = A.hi4[i1]; tl1 = A.lo4[i1]; }
            }
            {
                const real ir = static_cast<real>(irho);
                ax0 *= ir; ay0 *= ir; az0 *= ir;
                ax1 *= ir; ay1 *= ir; az1 *= ir;
            }
            for (int si = s0; si < s1; si++) {
                const int src = A.p2p_src[si];
                const int sf = A.first[src], sc = A.count[src];
                for (int j0 = 0; j0 < sc; j0 += 32) {
                    const int lim = min(32, sc - j0);
                    __syncwarp();
                    if (lane < lim) {
                        const int j = sf + j0 + lane;
                        if (f32) {
                            S.h[lane] = A.hi4[j];
                            S.l[lane] = A.lo4[j];
                        } else {
                            S.dx[lane] = A.x[j];
                            S.dy[lane] = A.y[j];
                            S.dz[lane] = A.z[j];
                            S.dm[lane] = A.G * A.m[j];
                        }
                    }
                    __syncwarp();
                    if constexpr (f32) {
                        for (int k = 0; k < lim; k++) {
                            const float4 h = S.h[k], l = S.l[k];
                            p2p_f32(h, l, th0, tl0, ax0, ay0, az0);
                            p2p_f32(h, l, th1, tl1, ax1, ay1, az1);
                        }
                    } else {
                        for (int k = 0; k < lim; k++) {
                            const double jx = S.dx[k], jy = S.dy[k], jz = S.dz[k], mu = S.dm[k];
                            p2p_f64(jx, jy, jz, mu, X0, Y0, Z0, ax0, ay0, az0);
                            p2p_f64(jx, jy, jz, mu, X1, Y1, Z1, ax1, ay1, az1);
                        }
                    }
                }
            }
            if (act0) {
                double ex, ey, ez;
                external_force(A.ext, X0, Y0, Z0, ex, ey, ez);
                const double mx = ax0, my = ay0, mz = az0;
                A.ax[i0] = mx + ex;
                A.ay[i0] = my + ey;
                A.az[i0] = mz + ez;
                if (A.amx) { A.amx[i0] = mx; A.amy[i0] = my; A.amz[i0] = mz; }
            }
            if (act1) {
                double ex, ey, ez;
                external_force(A.ext, X1, Y1, Z1, ex, ey, ez);
                const double mx = ax1, my = ay1, mz = az1;
                A.ax[i1] = mx + ex;
                A.ay[i1] = my + ey;
                A.az[i1] = mz + ez;
                if (A.amx) { A.amx[i1] = mx; A.amy[i1] = my; A.amz[i1] = mz; }
            }
        }
        __syncwarp();
    }
}

template <int P, typename real>
static void eval_t(ncorp_ctx *c, const EvalArgs &A) {
    k_eval<P, real><<<8 * c->num_sms, 32 * EVAL_WARPS, 0, c->stream>>>(A);
}

void launch_eval(ncorp_ctx *c, const ParticleSet &P, int p, bool mixed, double G, ExtForce ext, bool want_mutual) {
    Cells &C = c->cells;
    EvalArgs A;
    A.leaves = C.leaves; A.level = C.level; A.parent = C.parent; A.first = C.first; A.count = C.count;
    A.sx = C.sx; A.sy = C.sy; A.sz = C.sz; A.rho = C.rho;
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
