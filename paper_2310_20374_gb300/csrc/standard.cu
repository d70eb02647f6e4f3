// standard.cu -- the standard tree code (Algorithm StandardTree, Sect. 3.4.4)
// for mutual gravity, on the falcON tree with its geometry and multipoles.
// Every moonlet a is walked from the root: a cell B with fewer than N_cb,pre
// moonlets is summed directly; a well-separated one contributes its
// expansion at a (M2P, the m = 1 term of Eq. phi_expanded for a point
// target); one with fewer than N_cb,post moonlets, or a leaf, is summed
// directly; any other is opened, its children taken in order.  A moonlet is
// a point (r_crit = 0): B is well separated from a when
// r_crit,B^2 <= |x_a - s_B|^2 and the distance is not zero (the expansion is
// singular at its own centre).
//
// Work layout: a warp takes 32 consecutive moonlets of the key order (close
// in space) and walks the tree once for all of them with a stack of
// (cell, lanes) entries.  At a cell every lane still concerned decides for
// its own moonlet; the lanes that sum directly do so together (the cell's
// moonlets are read once for the warp), the lanes that expand evaluate the
// expansion at their moonlet, and the children are pushed with the lanes
// that open the cell.  A lane thus visits exactly the cells its moonlet's own
// walk visits, in the same order.
//
// Decisions: first in FP32 (double-float separation against r_crit rounded
// to FP32, with a 2^-16 relative margin either way), in FP64 in the oracle's
// order of operations inside the margin and at separations too small for
// the double-float positions to resolve (|d| below ~2^-26 |x|), so they are
// those of the FP64 criterion.
//
// M2P with the cells' power-of-two scaled multipoles
// M-hat_beta = sum mu (d/rho_B)^beta / beta!, u = (x - s_B)/rho_B:
//   a_i = (1/rho_B^2) sum_beta (-1)^|beta| D_{e_i+beta}(u) M-hat_beta,
// beta over order 0 and orders 2..p-1 (the dipole about s_B vanishes).
#include <type_traits>

#include "ctx.h"
#include "fields.cuh"

namespace ncorp {

constexpr int ST_WARPS = 4;
constexpr int ST_STACK = 8 * (MAX_LEVEL + 3);   // a walk holds at most 7 entries per level, plus one

struct StandardArgs {
    const int *first, *count, *child0, *nchild;
    const double *sx, *sy, *sz, *rcrit, *rho;
    const float4 *gh, *gl;    // centre hi (xyz), r_crit in FP32 (w); centre lo (xyz), rho (w)
    const void *Mh;
    const double *x, *y, *z, *m;
    const float4 *hi4, *lo4;
    double G;
    int pre, post, n;
    ExtForce ext;
    double *ax, *ay, *az;     // mutual + external
    double *amx, *amy, *amz;  // mutual only (nullable)
    Ctrl *ctl;
};

template <int P, typename real>
__global__ void __launch_bounds__(32 * ST_WARPS) k_standard(StandardArgs A) {
    constexpr int NM = num_m(P), ND = num_d(P);
    constexpr bool f32 = std::is_same<real, float>::value;
    constexpr unsigned FULL = 0xffffffffu;
    __shared__ int s_cell[ST_WARPS][ST_STACK];
    __shared__ unsigned s_mask[ST_WARPS][ST_STACK];
    if (aborted(A.ctl)) return;
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const real *Mh = static_cast<const real *>(A.Mh);
    long long n_exp = 0, n_dir = 0, n_pairs = 0;
    bool overflow = false;
    for (int base = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < A.n; base += nwarps * 32) {
        const int i = base + lane;
        const bool valid = i < A.n;
        const int ii = valid ? i : base;
        const double X = A.x[ii], Y = A.y[ii], Z = A.z[ii];
        const float4 th = A.hi4[ii], tl = A.lo4[ii];
        real mx = real(0), my = real(0), mz = real(0);
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
            const bool leaf = A.nchild[c] == 0;
            int d = -1;   // 0: direct, 1: expansion, 2: open
            if (mine) {
                if (nb < A.pre) {
                    d = 0;
                } else {
                    const float4 ch = A.gh[c], cl = A.gl[c];
                    const float dx = (th.x - ch.x) + (tl.x - cl.x);
                    const float dy = (th.y - ch.y) + (tl.y - cl.y);
                    const float dz = (th.z - ch.z) + (tl.z - cl.z);
                    const float d2f = dx * dx + dy * dy + dz * dz, t2f = ch.w * ch.w;
                    // below |d| ~ 2^-26 |x| the double-float representation error (~2^-47 |x|) is no
                    // longer small against d (a moonlet and its own small leaf): FP64 decides there
                    const float fl = (fabsf(th.x) + fabsf(th.y) + fabsf(th.z)) * 0x1p-26f;
                    bool sep;
                    if (d2f > fl * fl && d2f > t2f * (1.0f + 0x1p-16f)) {
                        sep = true;
                    } else if (d2f > fl * fl && d2f < t2f * (1.0f - 0x1p-16f)) {
                        sep = false;
                    } else {
                        const double ex = dsub(X, A.sx[c]), ey = dsub(Y, A.sy[c]), ez = dsub(Z, A.sz[c]);
                        const double d2 = dsq3(ex, ey, ez), rc = A.rcrit[c];
                        sep = d2 > 0.0 && dmul(rc, rc) <= d2;
                    }
                    d = sep ? 1 : ((nb < A.post || leaf) ? 0 : 2);
                }
            }
            const unsigned m_dir = __ballot_sync(FULL, d == 0);
            const unsigned m_open = __ballot_sync(FULL, d == 2);
            if (m_dir) {   // the cell's moonlets, read once for the warp
                if (d == 0) {
                    n_dir++;
                    n_pairs += nb;
                }
                for (int k = f; k < f + nb; k++) {
                    if constexpr (f32) {
                        const float4 h = A.hi4[k], l = A.lo4[k];
                        if (d == 0) p2p_f32(h, l, th, tl, mx, my, mz);
                    } else {
                        const double jx = A.x[k], jy = A.y[k], jz = A.z[k], mu = A.G * A.m[k];
                        if (d == 0) p2p_f64(jx, jy, jz, mu, X, Y, Z, mx, my, mz);
                    }
                }
            }
            if (d == 1) {
                n_exp++;
                real ux, uy, uz, s2;
                if constexpr (f32) {
                    const float4 ch = A.gh[c], cl = A.gl[c];
                    const float irf = 1.0f / cl.w;   // exact: rho is a power of two
                    ux = ((th.x - ch.x) + (tl.x - cl.x)) * irf;
                    uy = ((th.y - ch.y) + (tl.y - cl.y)) * irf;
                    uz = ((th.z - ch.z) + (tl.z - cl.z)) * irf;
                    s2 = irf * irf;
                } else {
                    const double ir = 1.0 / A.rho[c];
                    ux = (X - A.sx[c]) * ir;
                    uy = (Y - A.sy[c]) * ir;
                    uz = (Z - A.sz[c]) * ir;
                    s2 = ir * ir;
                }
                real D[ND];
                green_derivatives<P, real>(ux, uy, uz, D);
                const real *Ms = Mh + (size_t)c * NM;
                real gx = real(0), gy = real(0), gz = real(0);
#pragma unroll
                for (int nbm = 0; nbm < P; nbm++) {
                    if (nbm == 1) continue;
#pragma unroll
                    for (int kb = 0; kb <= nbm; kb++) {
#pragma unroll
                        for (int cb = 0; cb <= kb; cb++) {
                            const int ab = nbm - kb, bb = kb - cb;
                            const real w = (nbm & 1) ? -__ldg(&Ms[midx(ab, bb, cb)]) : __ldg(&Ms[midx(ab, bb, cb)]);
                            gx += D[sidx(ab + 1, bb, cb)] * w;
                            gy += D[sidx(ab, bb + 1, cb)] * w;
                            gz += D[sidx(ab, bb, cb + 1)] * w;
                        }
                    }
                }
                mx += gx * s2;
                my += gy * s2;
                mz += gz * s2;
            }
            if (m_open) {
                const int c0 = A.child0[c], nch = A.nchild[c];
                if (sp + nch > ST_STACK) {   // cannot happen within MAX_LEVEL levels; never write past the stack
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
        if (valid) {
            double ex, ey, ez;
            external_force(A.ext, X, Y, Z, ex, ey, ez);
            const double gx = static_cast<double>(mx), gy = static_cast<double>(my), gz = static_cast<double>(mz);
            A.ax[i] = gx + ex;
            A.ay[i] = gy + ey;
            A.az[i] = gz + ez;
            if (A.amx) {
                A.amx[i] = gx;
                A.amy[i] = gy;
                A.amz[i] = gz;
            }
        }
    }
    if (__any_sync(FULL, overflow) && lane == 0) atomicOr(&A.ctl->err, ERR_LEVEL);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        n_exp += __shfl_xor_sync(FULL, n_exp, o);
        n_dir += __shfl_xor_sync(FULL, n_dir, o);
        n_pairs += __shfl_xor_sync(FULL, n_pairs, o);
    }
    if (lane == 0) {
        atomicAdd(reinterpret_cast<unsigned long long *>(&A.ctl->n_m2p), static_cast<unsigned long long>(n_exp));
        atomicAdd(reinterpret_cast<unsigned long long *>(&A.ctl->dec_pairs), static_cast<unsigned long long>(n_dir));
        atomicAdd(reinterpret_cast<unsigned long long *>(&A.ctl->n_inter), static_cast<unsigned long long>(n_pairs));
    }
}

template <int P, typename real>
static void standard_t(ncorp_ctx *c, const StandardArgs &A) {
    const int warps = (A.n + 31) / 32;
    const int grid = std::max(1, std::min((warps + ST_WARPS - 1) / ST_WARPS, 16 * c->num_sms));
    k_standard<P, real><<<grid, 32 * ST_WARPS, 0, c->stream>>>(A);
    c->launches++;
}

void launch_standard(ncorp_ctx *c, const ParticleSet &S, int n, int p, bool mixed, double G, ExtForce ext,
                     bool want_mutual, int pre, int post) {
    const Cells &C = c->cells;
    StandardArgs A;
    A.first = C.first; A.count = C.count; A.child0 = C.child0; A.nchild = C.nchild;
    A.sx = C.sx; A.sy = C.sy; A.sz = C.sz; A.rcrit = C.rcrit; A.rho = C.rho;
    A.gh = C.gh; A.gl = C.gl;
    A.Mh = C.Mh;
    A.x = S.x; A.y = S.y; A.z = S.z; A.m = S.m;
    A.hi4 = S.hi4; A.lo4 = S.lo4;
    A.G = G;
    A.pre = pre; A.post = post; A.n = n;
    A.ext = ext;
    A.ax = S.ax; A.ay = S.ay; A.az = S.az;
    A.amx = want_mutual ? c->amx : nullptr;
    A.amy = want_mutual ? c->amy : nullptr;
    A.amz = want_mutual ? c->amz : nullptr;
    A.ctl = c->ctl;
#define NCORP_STD_CASE(PP)                          \
    case PP:                                        \
        if (mixed) standard_t<PP, float>(c, A);     \
        else standard_t<PP, double>(c, A);          \
        break;
    switch (p) {
        NCORP_STD_CASE(1)
        NCORP_STD_CASE(2)
        NCORP_STD_CASE(3)
        NCORP_STD_CASE(4)
        NCORP_STD_CASE(5)
        NCORP_STD_CASE(6)
        default: break;
    }
#undef NCORP_STD_CASE
    NCORP_CUDA_CHECK(cudaGetLastError());
}

}  // namespace ncorp
