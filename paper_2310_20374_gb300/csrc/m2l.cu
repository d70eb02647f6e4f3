// m2l.cu -- cell-cell interactions of well-separated pairs (Eq. phi_expanded).
//
// For a target cell A and a source cell B, R = s_A - s_B:
//   C_alpha(s_A) = sum_beta (-1)^|beta| D_{alpha+beta}(R) M_beta(s_B) / beta!,
//   1 <= |alpha| <= p, |alpha| + |beta| <= p, beta in {0} U {|beta| >= 2},
// which is Eq. phi_expanded with the full-index contraction written over
// symmetric multi-indices (the multinomial count of equal index tuples turns
// 1/n! into 1/beta!).  D_gamma = d^gamma (1/|R|) follows from the identity
// r^2 d_i(1/r) + x_i (1/r) = 0 differentiated gamma times, which gives
//   n r^2 D_gamma = -(2n-1) sum_j gamma_j x_j D_{gamma-e_j}
//                   - (n-1) sum_j gamma_j (gamma_j - 1) D_{gamma-2e_j},  n = |gamma|.
//
// Scaling: with rho_A, rho_B the cells' power-of-two scales and u = R/rho_A,
//   C-hat_alpha(A) = C_alpha rho_A^|alpha|
//                  = (1/rho_A) sum_beta D_{alpha+beta}(u) (-rho_B/rho_A)^|beta| M-hat_beta(B),
// so that the per-entry sum needs no alpha-dependent factor and the 1/rho_A is
// applied once per target.
//
// Mixed precision: the order-1 coefficients (the field) of every source's
// contribution are formed in FP32 and added to double-float totals (two-sum),
// and the lanes' totals are combined the same way, so that the field of a
// target cell, summed over many sources whose pulls largely cancel, keeps the
// accuracy of the single contributions; the low parts go to Ch_lo.
//
// Work layout: the directed entries (target, source) are grouped by target.
// One warp per target cell: the lanes take the target's sources in turn, each
// accumulating the target's coefficients in registers; a butterfly reduction
// then leaves the sums on every lane, and each lane stores its share of the
// coefficients (the warp owns the target, so no atomics are needed; targets
// without entries get zeros).  Both directions of a pair are evaluated
// (A <- B and B <- A), which is the symmetric treatment of Sect. 3.4.3 split
// into its two halves.
#include "ctx.h"
#include "fields.cuh"

namespace ncorp {

struct M2LArgs {
    const int2 *dir;
    const int *offs;    // [n_cells + 1]: entries of target c are dir[offs[c], offs[c + 1])
    int dir_cap;
    const double *sx, *sy, *sz, *rho;
    const float4 *gh, *gl;
    const void *Mh;
    void *Ch;
    float *Ch_lo;       // mixed: low parts of the order-1 sums
    Ctrl *ctl;
    int *desc_work;     // the descent's claim counter, zeroed here
};

constexpr int M2L_WARPS = 4;
// Three blocks per SM (at most 170 registers per thread, a few spilled): the
// kernel is latency-bound at two blocks (measured 61 -> 53 us on the 1e5 disk).

template <int P, typename real>
__global__ void __launch_bounds__(32 * M2L_WARPS, 3) k_m2l(M2LArgs A) {
    constexpr int NM = num_m(P), NC = num_c(P), ND = num_d(P);
    constexpr bool f32 = sizeof(real) == 4;
    const real *__restrict__ Mh = static_cast<const real *>(A.Mh);
    real *Ch = static_cast<real *>(A.Ch);
    if (aborted(A.ctl)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {   // opens the following descent: fresh epoch, claims from 0
        A.ctl->desc_epoch += 1u;
        *A.desc_work = 0;
    }
    const int lane = threadIdx.x & 31;
    // warps numbered across the blocks first, so that neighbouring targets land on different SMs
    const int gw0 = (threadIdx.x >> 5) * gridDim.x + blockIdx.x, nwarps = (gridDim.x * blockDim.x) >> 5;
    const int ncells = A.ctl->n_cells;
    for (int c = gw0; c < ncells; c += nwarps) {
        const int e0 = min(__ldg(&A.offs[c]), A.dir_cap), e1 = min(__ldg(&A.offs[c + 1]), A.dir_cap);
        real acc[NC];
#pragma unroll
        for (int i = 0; i < NC; i++) acc[i] = real(0);
        double irho = 1.0, tx = 0.0, ty = 0.0, tz = 0.0;
        float4 th = make_float4(0.f, 0.f, 0.f, 1.f), tl = th;
        float irf = 1.0f;
        if (e1 > e0) {
            if constexpr (f32) {
                th = A.gh[c];
                tl = A.gl[c];
                irf = 1.0f / tl.w;   // exact: rho is a power of two
            } else {
                irho = 1.0 / A.rho[c];
                tx = A.sx[c];
                ty = A.sy[c];
                tz = A.sz[c];
            }
        }
        float lo1[3] = {0.f, 0.f, 0.f};   // mixed: low parts of acc[0..2]
        for (int e = e0 + lane; e < e1; e += 32) {
            const int src = A.dir[e].y;
            real t1[3] = {real(0), real(0), real(0)};   // this source's order-1 contribution
            real ux, uy, uz, q;
            if constexpr (f32) {   // separation from double-float centres, no FP64 work
                const float4 sh = A.gh[src], sl = A.gl[src];
                ux = ((th.x - sh.x) + (tl.x - sl.x)) * irf;
                uy = ((th.y - sh.y) + (tl.y - sl.y)) * irf;
                uz = ((th.z - sh.z) + (tl.z - sl.z)) * irf;
                q = -sl.w * irf;   // -rho_B / rho_A
            } else {
                ux = (tx - A.sx[src]) * irho;
                uy = (ty - A.sy[src]) * irho;
                uz = (tz - A.sz[src]) * irho;
                q = -A.rho[src] * irho;
            }
            real D[ND];
            green_derivatives<P, real>(ux, uy, uz, D);
            const real *Ms = Mh + (size_t)src * NM;
            real qn = real(1);
#pragma unroll
            for (int nb = 0; nb < P; nb++) {
                if (nb == 1) {
                    qn *= q;
                    continue;
                }
#pragma unroll
                for (int kb = 0; kb <= nb; kb++) {
#pragma unroll
                    for (int cb = 0; cb <= kb; cb++) {
                        const int ab = nb - kb, bb = kb - cb;
                        const real w = qn * __ldg(&Ms[midx(ab, bb, cb)]);
#pragma unroll
                        for (int na = 1; na <= P - nb; na++) {
#pragma unroll
                            for (int ka = 0; ka <= na; ka++) {
#pragma unroll
                                for (int ca = 0; ca <= ka; ca++) {
                                    const int aa = na - ka, ba = ka - ca;
                                    if (na == 1) t1[cidx(aa, ba, ca)] += D[sidx(aa + ab, ba + bb, ca + cb)] * w;
                                    else acc[cidx(aa, ba, ca)] += D[sidx(aa + ab, ba + bb, ca + cb)] * w;
                                }
                            }
                        }
                    }
                }
                qn *= q;
            }
#pragma unroll
            for (int d = 0; d < 3; d++) {
                if constexpr (f32) df_add(acc[d], lo1[d], t1[d]);
                else acc[d] += t1[d];
            }
        }
        // sums over the lanes (the same on every lane), scaled by 1/rho_A; lane l stores l, l + 32, ...
        const real f = f32 ? static_cast<real>(irf) : static_cast<real>(irho);
#pragma unroll
        for (int i = 0; i < NC; i++) {
            real v = acc[i];
            if (f32 && i < 3) {   // order 1: double-float butterfly
                float hv = static_cast<float>(v), lv = lo1[i];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float oh = __shfl_xor_sync(0xffffffffu, hv, o), ol = __shfl_xor_sync(0xffffffffu, lv, o);
                    df_add(hv, lv, oh);
                    lv += ol;
                }
                if (i == lane) {
                    Ch[(size_t)c * NC + i] = static_cast<real>(hv) * f;
                    A.Ch_lo[3 * c + i] = lv * static_cast<float>(f);   // f: a power of two
                }
                continue;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if ((i & 31) == lane) Ch[(size_t)c * NC + i] = v * f;
        }
    }
}

template <int P, typename real>
static void m2l_t(ncorp_ctx *c, const M2LArgs &A) {
    k_m2l<P, real><<<8 * c->num_sms, 32 * M2L_WARPS, 0, c->stream>>>(A); c->launches++;
}

void launch_m2l(ncorp_ctx *c, int p, bool mixed) {
    Cells &C = c->cells;
    M2LArgs A;
    A.dir = c->wl.m2l_dir;
    A.offs = c->wl.offs;
    A.dir_cap = c->wl.m2l_dir_cap;
    A.sx = C.sx; A.sy = C.sy; A.sz = C.sz; A.rho = C.rho;
    A.gh = C.gh; A.gl = C.gl;
    A.Mh = C.Mh;
    A.Ch = C.Ch;
    A.Ch_lo = C.Ch_lo;
    A.ctl = c->ctl;
    A.desc_work = c->work_counter + 1;
#define NCORP_M2L_CASE(PP)                       \
    case PP:                                     \
        if (mixed) m2l_t<PP, float>(c, A);       \
        else m2l_t<PP, double>(c, A);            \
        break;
    switch (p) {
        NCORP_M2L_CASE(1)
        NCORP_M2L_CASE(2)
        NCORP_M2L_CASE(3)
        NCORP_M2L_CASE(4)
        NCORP_M2L_CASE(5)
        NCORP_M2L_CASE(6)
        default: break;
    }
#undef NCORP_M2L_CASE
    NCORP_CUDA_CHECK(cudaGetLastError());
}

}  // namespace ncorp
