// eval.cu -- tree descent and evaluation at the moonlets: L2L from the root
// to each leaf and L2P (Eq. shifting), the direct ("brute force") gravity of
// the leaf's near-field list, and the central-body / distant-star forces
// (App. B.1, B.3).
//
// One CTA per leaf.  The descent of Sect. 3.4.3 (a cell adds its parent's
// C translated to its own centre, from the root down) is followed along the
// leaf's ancestor chain:
//   C-hat_alpha(child) = C-hat_alpha(child, own M2L)
//       + (rho_c/rho_p)^|alpha| sum_beta C-hat_{alpha+beta}(parent) (delta/rho_p)^beta / beta!,
//   delta = s_child - s_parent,
// which is Eq. shifting over symmetric multi-indices in scaled form.  Then
// every moonlet of the leaf gets
//   a = (1/rho) sum_{|beta| <= p-1} C-hat_{e_k+beta} (d/rho)^beta / beta!,  d = x - s_leaf,
// plus sum_j mu_j (x_j - x)/|x_j - x|^3 over the moonlets of its direct list
// (mu_j = G m_j; j = i skipped), plus the external forces in FP64.  The sum of
// every moonlet is built in registers by one thread and written once.
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
    double G;
    ExtForce ext;
    double *ax, *ay, *az;
    double *amx, *amy, *amz;
    const Ctrl *ctl;
};

__device__ __forceinline__ float rsqrt_real(float v) { return rsqrtf(v); }
__device__ __forceinline__ double rsqrt_real(double v) { return 1.0 / sqrt(v); }

template <int P, typename real, int BS>
__global__ void __launch_bounds__(BS) k_eval(EvalArgs A) {
    constexpr int NC = num_c(P);
    __shared__ int s_path[MAX_LEVEL + 2];
    __shared__ int s_depth;
    __shared__ real s_C[2][NC];
    __shared__ real s_pw[3][P + 1];
    __shared__ real s_x[BS], s_y[BS], s_z[BS], s_mu[BS];
    // low parts of the staged positions (FP32 only): x - s_leaf = hi + lo
    __shared__ real s_xl[sizeof(real) == 4 ? BS : 1], s_yl[sizeof(real) == 4 ? BS : 1], s_zl[sizeof(real) == 4 ? BS : 1];
    constexpr bool split = sizeof(real) == 4;
    __shared__ int s_j[BS];
    const real *Ch = static_cast<const real *>(A.Ch);
    const int tid = threadIdx.x;
    if (aborted(A.ctl)) return;
    const int nl = A.ctl->n_leaves;
    for (int li = blockIdx.x; li < nl; li += gridDim.x) {
        const int leaf = A.leaves[li];
        if (tid == 0) {
            const int lev = A.level[leaf];
            int c = leaf;
            for (int d = lev; d >= 0; d--) {
                s_path[d] = c;
                c = A.parent[c];
            }
            s_depth = lev;
        }
        __syncthreads();
        const int depth = s_depth;
        for (int i = tid; i < NC; i += BS) s_C[0][i] = Ch[(size_t)s_path[0] * NC + i];
        int cb = 0;
        __syncthreads();
        for (int d = 1; d <= depth; d++) {
            const int pc = s_path[d - 1], cc = s_path[d];
            const double iprho = 1.0 / A.rho[pc];
            if (tid < 3) {
                const double dv = tid == 0 ? A.sx[cc] - A.sx[pc] : (tid == 1 ? A.sy[cc] - A.sy[pc] : A.sz[cc] - A.sz[pc]);
                const real h = static_cast<real>(dv * iprho);
                real pw = real(1);
                for (int k = 0; k <= P; k++) {
                    s_pw[tid][k] = pw;
                    pw *= h;
                }
            }
            __syncthreads();
            const real ratio = static_cast<real>(A.rho[cc] * iprho);
            for (int i = tid; i < NC; i += BS) {
                const int a = c_exp2.e[i + 1][0], b = c_exp2.e[i + 1][1], c = c_exp2.e[i + 1][2];
                const int n = a + b + c;
                real acc = real(0);
                for (int nb = 0; nb <= P - n; nb++)
                    for (int kb = 0; kb <= nb; kb++)
                        for (int cb2 = 0; cb2 <= kb; cb2++) {
                            const int ab = nb - kb, bb = kb - cb2;
                            const real w = s_pw[0][ab] * s_pw[1][bb] * s_pw[2][cb2] *
                                           static_cast<real>(c_ifact[ab] * c_ifact[bb] * c_ifact[cb2]);
                            acc += s_C[cb][cidx(a + ab, b + bb, c + cb2)] * w;
                        }
                for (int k = 0; k < n; k++) acc *= ratio;   // (rho_c/rho_p)^n applied to the small factor first
                s_C[cb ^ 1][i] = Ch[(size_t)cc * NC + i] + acc;
            }
            cb ^= 1;
            __syncthreads();
        }
        const int f = A.first[leaf], cnt = A.count[leaf];
        const double lsx = A.sx[leaf], lsy = A.sy[leaf], lsz = A.sz[leaf];
        const double irho = 1.0 / A.rho[leaf];
        const int s0 = min(A.p2p_off[leaf], A.p2p_dir_cap), s1 = min(A.p2p_off[leaf + 1], A.p2p_dir_cap);
        for (int t0 = 0; t0 < cnt; t0 += BS) {
            const int ti = t0 + tid;
            const bool act = ti < cnt;
            const int i = f + ti;
            real px = 0, py = 0, pz = 0, pxl = 0, pyl = 0, pzl = 0, ax = 0, ay = 0, az = 0;
            if (act) {
                const double dx = A.x[i] - lsx, dy = A.y[i] - lsy, dz = A.z[i] - lsz;
                px = static_cast<real>(dx);
                py = static_cast<real>(dy);
                pz = static_cast<real>(dz);
                if (split) {
                    pxl = static_cast<real>(dx - static_cast<double>(px));
                    pyl = static_cast<real>(dy - static_cast<double>(py));
                    pzl = static_cast<real>(dz - static_cast<double>(pz));
                }
                const real hx = static_cast<real>(dx * irho), hy = static_cast<real>(dy * irho),
                           hz = static_cast<real>(dz * irho);
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
                        for (int cb2 = 0; cb2 <= kb; cb2++) {
                            const int ab = nb - kb, bb = kb - cb2;
                            const real w = wx[ab] * wy[bb] * wz[cb2] * static_cast<real>(inv_mfact(ab, bb, cb2));
                            ax += s_C[cb][cidx(ab + 1, bb, cb2)] * w;
                            ay += s_C[cb][cidx(ab, bb + 1, cb2)] * w;
                            az += s_C[cb][cidx(ab, bb, cb2 + 1)] * w;
                        }
                const real ir = static_cast<real>(irho);
                ax *= ir;
                ay *= ir;
                az *= ir;
            }
            for (int si = s0; si < s1; si++) {
                const int src = A.p2p_src[si];
                const int sf = A.first[src], sc = A.count[src];
                for (int j0 = 0; j0 < sc; j0 += BS) {
                    __syncthreads();
                    if (tid < sc - j0) {
                        const int j = sf + j0 + tid;
                        const double qx = A.x[j] - lsx, qy = A.y[j] - lsy, qz = A.z[j] - lsz;
                        const real hx = static_cast<real>(qx), hy = static_cast<real>(qy), hz = static_cast<real>(qz);
                        s_x[tid] = hx;
                        s_y[tid] = hy;
                        s_z[tid] = hz;
                        if (split) {
                            s_xl[tid] = static_cast<real>(qx - static_cast<double>(hx));
                            s_yl[tid] = static_cast<real>(qy - static_cast<double>(hy));
                            s_zl[tid] = static_cast<real>(qz - static_cast<double>(hz));
                        }
                        s_mu[tid] = static_cast<real>(A.G * A.m[j]);
                        s_j[tid] = j;
                    }
                    __syncthreads();
                    if (act) {
                        const int lim = min(BS, sc - j0);
                        for (int k = 0; k < lim; k++) {
                            real dx = s_x[k] - px, dy = s_y[k] - py, dz = s_z[k] - pz;
                            if (split) {   // (hi_j - hi_i) + (lo_j - lo_i): separation to ~1e-7 relative
                                dx += s_xl[k] - pxl;
                                dy += s_yl[k] - pyl;
                                dz += s_zl[k] - pzl;
                            }
                            const real r2 = dx * dx + dy * dy + dz * dz;
                            if (s_j[k] != i && r2 > (split ? real(1e-30) : real(0))) {
                                const real inv = rsqrt_real(r2);
                                const real f3 = s_mu[k] * inv * inv * inv;
                                ax += dx * f3;
                                ay += dy * f3;
                                az += dz * f3;
                            }
                        }
                    }
                }
            }
            if (act) {
                const double X = A.x[i], Y = A.y[i], Z = A.z[i];
                const double r2 = X * X + Y * Y + Z * Z;
                const double fc = -A.ext.GMc / (r2 * sqrt(r2));
                double ex = fc * X, ey = fc * Y, ez = fc * Z;
                if (A.ext.star_k != 0.0) {
                    const double c3 = 3.0 * (X * A.ext.sx + Y * A.ext.sy + Z * A.ext.sz) * A.ext.inv_rs2;
                    ex -= A.ext.star_k * (X - c3 * A.ext.sx);
                    ey -= A.ext.star_k * (Y - c3 * A.ext.sy);
                    ez -= A.ext.star_k * (Z - c3 * A.ext.sz);
                }
                const double mx = static_cast<double>(ax), my = static_cast<double>(ay), mz = static_cast<double>(az);
                A.ax[i] = mx + ex;
                A.ay[i] = my + ey;
                A.az[i] = mz + ez;
                if (A.amx) {
                    A.amx[i] = mx;
                    A.amy[i] = my;
                    A.amz[i] = mz;
                }
            }
        }
        __syncthreads();
    }
}

template <int P, typename real>
static void eval_t(ncorp_ctx *c, const EvalArgs &A) {
    if (c->s <= 64) k_eval<P, real, 64><<<16 * c->num_sms, 64, 0, c->stream>>>(A);
    else k_eval<P, real, 128><<<8 * c->num_sms, 128, 0, c->stream>>>(A);
}

void launch_eval(ncorp_ctx *c, const ParticleSet &P, int p, bool mixed, double G, ExtForce ext, bool want_mutual) {
    Cells &C = c->cells;
    EvalArgs A;
    A.leaves = C.leaves; A.level = C.level; A.parent = C.parent; A.first = C.first; A.count = C.count;
    A.sx = C.sx; A.sy = C.sy; A.sz = C.sz; A.rho = C.rho;
    A.Ch = C.Ch;
    A.p2p_off = c->wl.p2p_off; A.p2p_src = c->wl.p2p_src; A.p2p_dir_cap = c->wl.p2p_dir_cap;
    A.x = P.x; A.y = P.y; A.z = P.z; A.m = P.m;
    A.G = G;
    A.ext = ext;
    A.ax = P.ax; A.ay = P.ay; A.az = P.az;
    A.amx = want_mutual ? c->amx : nullptr;
    A.amy = want_mutual ? c->amy : nullptr;
    A.amz = want_mutual ? c->amz : nullptr;
    A.ctl = c->ctl;
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
