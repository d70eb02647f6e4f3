// fields.cuh -- device functions shared by the evaluation kernels: the
// derivatives of the Green function 1/|R| (Eq. gradient), the direct pull of
// one moonlet on another (FP32 double-float separation or FP64), and the
// external forces of the central body, its bulge and the distant star.
#pragma once

#include "ctx.h"

namespace ncorp {

// D_gamma(u) = d^gamma (1/|u|) for |gamma| <= P, packed by sidx: from the
// identity r^2 d_i(1/r) + x_i (1/r) = 0 differentiated gamma times,
//   n r^2 D_gamma = -(2n-1) sum_j gamma_j x_j D_{gamma-e_j}
//                   - (n-1) sum_j gamma_j (gamma_j - 1) D_{gamma-2e_j},  n = |gamma|.
template <int P, typename real>
__device__ __forceinline__ void green_derivatives(real ux, real uy, real uz, real *D) {
    const real r2 = ux * ux + uy * uy + uz * uz;
    const real ir2 = real(1) / r2;
    D[0] = sqrt(ir2);
#pragma unroll
    for (int n = 1; n <= P; n++) {
#pragma unroll
        for (int k = 0; k <= n; k++) {
#pragma unroll
            for (int c = 0; c <= k; c++) {
                const int a = n - k, b = k - c;
                real s1 = real(0), s2 = real(0);
                if (a >= 1) s1 += real(a) * ux * D[sidx(a - 1, b, c)];
                if (b >= 1) s1 += real(b) * uy * D[sidx(a, b - 1, c)];
                if (c >= 1) s1 += real(c) * uz * D[sidx(a, b, c - 1)];
                if (a >= 2) s2 += real(a * (a - 1)) * D[sidx(a - 2, b, c)];
                if (b >= 2) s2 += real(b * (b - 1)) * D[sidx(a, b - 2, c)];
                if (c >= 2) s2 += real(c * (c - 1)) * D[sidx(a, b, c - 2)];
                D[sidx(a, b, c)] = -(real(2 * n - 1) * s1 + real(n - 1) * s2) * (ir2 * real(1.0 / n));
            }
        }
    }
}

// 1/r from r^2: an FP32 reciprocal square root refined by two Newton steps
// in FP64 (the seed's relative error ~2^-22 squares twice, to the FP64
// rounding level): with 1/r^3 = y^3 and 1/r^5 = y^5 about a third of the FP64
// instructions of correctly rounded square roots and divisions; outside the
// FP32 range the direct form.
__device__ __forceinline__ double inv_r(double r2) {
    if (!(r2 > 1e-30 && r2 < 1e30)) return 1.0 / sqrt(r2);
    double y = static_cast<double>(rsqrtf(static_cast<float>(r2)));
    const double hr2 = -0.5 * r2;
    y = y * fma(hr2, y * y, 1.5);
    y = y * fma(hr2, y * y, 1.5);
    return y;
}

// Central body (App. B.1), its equatorial bulge (App. B.2, k = z axis) and the
// distant star's tide (App. B.3), in FP64.
__device__ __forceinline__ void external_force(const ExtForce &E, double X, double Y, double Z, double &ex, double &ey,
                                               double &ez) {
    const double r2 = X * X + Y * Y + Z * Z;
    const double y = inv_r(r2), y2 = y * y, y3 = y2 * y;
    const double fc = -E.GMc * y3;
    ex = fc * X;
    ey = fc * Y;
    ez = fc * Z;
    if (E.bulge != 0.0) {
        const double q = E.bulge * y3 * y2;   // G M_c R_c^2 J2 / r^5
        const double radial = q * (15.0 * Z * Z - 3.0 * r2) * (0.5 * y2);
        ex += radial * X;
        ey += radial * Y;
        ez += radial * Z - 3.0 * q * Z;
    }
    if (E.star_k != 0.0) {
        const double c3 = 3.0 * (X * E.sx + Y * E.sy + Z * E.sz) * E.inv_rs2;
        ex -= E.star_k * (X - c3 * E.sx);
        ey -= E.star_k * (Y - c3 * E.sy);
        ez -= E.star_k * (Z - c3 * E.sz);
    }
}

// One near-field pair, FP32: the separation from the (hi, lo) pairs, then
// mu_j d / |d|^3; a coincident pair (d = 0, the moonlet itself) adds 0.
// The hardware reciprocal square root y carries a relative error d of a few
// 1e-8 that y^3 triples; with the residual e = 1 - r^2 y^2 = -2d (one FMA),
// y^3 (1 + 3e/2) = r^-3 (1 + O(d^2)) removes it, so that a term is accurate
// to the rounding of its few products (a moonlet whose neighbours' pulls
// nearly cancel sees every term's error against a small total).
__device__ __forceinline__ void p2p_f32(const float4 &h, const float4 &l, const float4 &th, const float4 &tl, float &ax,
                                        float &ay, float &az) {
    const float dx = (h.x - th.x) + (l.x - tl.x);
    const float dy = (h.y - th.y) + (l.y - tl.y);
    const float dz = (h.z - th.z) + (l.z - tl.z);
    // r^2 below 1e-20 (coincident pairs, the moonlet itself) is raised to 1e-20: y^3 stays finite and
    // d = 0 makes the term 0 (pairs closer than 1e-10 do not occur in a disk of moonlets)
    const float r2 = fmaxf(dx * dx + dy * dy + dz * dz, 1e-20f);
    const float y = rsqrtf(r2);
    const float y2 = y * y;
    const float e = fmaf(-r2, y2, 1.0f);
    const float f = h.w * (y2 * y);
    const float f3 = fmaf(f, 1.5f * e, f);
    ax += dx * f3;
    ay += dy * f3;
    az += dz * f3;
}

// (hi, lo) + b, renormalised (Knuth's two-sum of hi and b, its error added to lo)
__device__ __forceinline__ void df_add(float &hi, float &lo, float b) {
    const float s = hi + b;
    const float bv = s - hi;
    const float e = (hi - (s - bv)) + (b - bv);
    const float l = lo + e;
    hi = s + l;
    lo = l - (hi - s);
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

}  // namespace ncorp
