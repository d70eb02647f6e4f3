// collide.cu -- the pairwise collision test of Sect. 3.1 over the direct lists
// of the collision walk, and the sorting of the colliding pairs.
//
// Straight-line trajectories over the step: with dr = r1 - r2, dv = v1 - v2,
//   Delta = (dr.dv)^2 + dv^2 ((R1 + R2)^2 - dr^2),
//   dt_c  = -(dr.dv + sqrt(Delta)) / dv^2,
// the pair collides within the step iff Delta >= 0 and 0 <= dt_c <= dt
// (dv = 0: no collision).  Evaluated in FP64 with exactly rounded operations
// in a fixed order, (1, 2) being the pair in increasing caller index, so that
// the set of pairs is reproducible bit for bit.
#include "ctx.h"

namespace ncorp {

__device__ __forceinline__ bool collide_test(double x1, double y1, double z1, double u1, double v1, double w1,
                                             double R1, double x2, double y2, double z2, double u2, double v2,
                                             double w2, double R2, double dt) {
    const double dx = dsub(x1, x2), dy = dsub(y1, y2), dz = dsub(z1, z2);
    const double ux = dsub(u1, u2), uy = dsub(v1, v2), uz = dsub(w1, w2);
    const double b = dadd(dadd(dmul(dx, ux), dmul(dy, uy)), dmul(dz, uz));
    const double dr2 = dsq3(dx, dy, dz);
    const double dv2 = dsq3(ux, uy, uz);
    if (dv2 == 0.0) return false;
    const double Rs = dadd(R1, R2);
    const double Delta = dadd(dmul(b, b), dmul(dv2, dsub(dmul(Rs, Rs), dr2)));
    if (Delta < 0.0) return false;
    const double tc = ddiv(-dadd(b, dsqrt(Delta)), dv2);
    return tc >= 0.0 && tc <= dt;
}

struct CollideArgs {
    const int2 *p2p;
    const int *self;
    const int *first, *count;
    const double *x, *y, *z, *vx, *vy, *vz, *R;
    const float4 *hi4, *lo4;
    const float *rc;           // R + dt |v| rounded up to FP32
    const int *perm;
    double dt;
    uint64_t *pairs;
    int cap, self_cap, p2p_cap;
    Ctrl *ctl;
};

__device__ __forceinline__ void test_and_emit(const CollideArgs &A, int u, int v) {
    int a = u, b = v;
    if (A.perm[a] > A.perm[b]) {
        a = v;
        b = u;
    }
    if (collide_test(A.x[a], A.y[a], A.z[a], A.vx[a], A.vy[a], A.vz[a], A.R[a], A.x[b], A.y[b], A.z[b], A.vx[b],
                     A.vy[b], A.vz[b], A.R[b], A.dt)) {
        const int slot = atomicAdd(&A.ctl->n_found, 1);
        if (slot < A.cap)
            A.pairs[slot] = (static_cast<unsigned long long>(A.perm[a]) << 32) | static_cast<unsigned>(A.perm[b]);
        else
            atomicOr(&A.ctl->err, ERR_PAIRS);
    }
}

// A pair can only collide within the step if |dr| <= R1 + R2 + dt |dv| <= rc1 + rc2
// (rc = R + dt |v|).  The separation is evaluated from the double-float
// positions (relative error ~1e-7) and compared with (rc1 + rc2)^2 (1 + 2^-10);
// only pairs inside that bound reach the exact FP64 test, so the pair set is
// the one the FP64 test alone gives.
__device__ __forceinline__ bool may_touch(const float4 &h, const float4 &l, float r, const float4 &th,
                                          const float4 &tl, float tr) {
    const float dx = (h.x - th.x) + (l.x - tl.x);
    const float dy = (h.y - th.y) + (l.y - tl.y);
    const float dz = (h.z - th.z) + (l.z - tl.z);
    const float s = r + tr;
    return dx * dx + dy * dy + dz * dz <= s * s * (1.0f + 0x1p-10f);
}

constexpr int COL_WARPS = 8;

// Warp per direct item (a leaf with itself, or a pair of leaves).  The
// source leaf is staged COL_STAGE moonlets at a time; the item's targets are
// taken 32 at a time, m of them occupying T = pow2ceil(m) lanes, and the
// warp's lanes form G = 32 / T groups: lane (g, t) tests target t against the
// staged sources k = g, g + G, ...  so small leaves keep the lanes busy.
constexpr int COL_STAGE = 64;

__global__ void __launch_bounds__(32 * COL_WARPS) k_collide(CollideArgs A) {
    __shared__ float4 s_h[COL_WARPS][COL_STAGE], s_l[COL_WARPS][COL_STAGE];
    __shared__ float s_r[COL_WARPS][COL_STAGE];
    if (aborted(A.ctl)) return;
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int ns = min(A.ctl->n_self, A.self_cap), np = min(A.ctl->n_p2p, A.p2p_cap);
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    long long tests = 0;
    for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < ns + np; w += nwarps) {
        int ct, cs;
        if (w < ns) {
            ct = cs = A.self[w];
        } else {
            const int2 e = A.p2p[w - ns];
            ct = e.x;
            cs = e.y;
        }
        const bool self = ct == cs;
        const int ft = A.first[ct], nt = A.count[ct], fs = A.first[cs], nsrc = A.count[cs];
        if (lane == 0) tests += self ? static_cast<long long>(nt) * (nt - 1) / 2 : static_cast<long long>(nt) * nsrc;
        for (int t0 = 0; t0 < nt; t0 += 32) {
            const int m = min(32, nt - t0);
            int lg = 0;
            while ((1 << lg) < m) lg++;
            const int T = 1 << lg, G = 32 >> lg, tt = lane & (T - 1), g = lane >> lg;
            const int u = t0 + tt;
            const bool act = tt < m;
            float4 th = make_float4(0.f, 0.f, 0.f, 0.f), tl = th;
            float tr = 0.f;
            if (act) { th = A.hi4[ft + u]; tl = A.lo4[ft + u]; tr = A.rc[ft + u]; }
            for (int j0 = 0; j0 < nsrc; j0 += COL_STAGE) {
                const int lim = min(COL_STAGE, nsrc - j0);
                __syncwarp();
                for (int k = lane; k < lim; k += 32) {
                    s_h[wl][k] = A.hi4[fs + j0 + k];
                    s_l[wl][k] = A.lo4[fs + j0 + k];
                    s_r[wl][k] = A.rc[fs + j0 + k];
                }
                __syncwarp();
                if (act) {
                    for (int k = g; k < lim; k += G) {
                        const int v = j0 + k;
                        if ((!self || v > u) && may_touch(s_h[wl][k], s_l[wl][k], s_r[wl][k], th, tl, tr))
                            test_and_emit(A, ft + u, fs + v);
                    }
                }
            }
        }
    }
    if (lane == 0 && tests)
        atomicAdd(reinterpret_cast<unsigned long long *>(&A.ctl->n_tests), static_cast<unsigned long long>(tests));
}

void launch_collide(ncorp_ctx *c, const ParticleSet &P, const double *vx, const double *vy, const double *vz,
                    double dt) {
    CollideArgs A;
    A.p2p = c->wl.p2p; A.self = c->wl.self;
    A.first = c->cells.first; A.count = c->cells.count;
    A.x = P.x; A.y = P.y; A.z = P.z; A.vx = vx; A.vy = vy; A.vz = vz; A.R = P.R;
    A.hi4 = P.hi4; A.lo4 = P.lo4; A.rc = c->rcf;
    A.perm = P.perm;
    A.dt = dt;
    A.pairs = c->pairs;
    A.cap = c->pair_cap;
    A.self_cap = c->wl.self_cap;
    A.p2p_cap = c->wl.p2p_cap;
    A.ctl = c->ctl;
    // two blocks per SM: the search runs beside the main chain's cooperative kernels, which must find
    // room on every SM while it runs
    k_collide<<<2 * c->num_sms, 32 * COL_WARPS, 0, c->stream>>>(A); c->launches++;
    NCORP_CUDA_CHECK(cudaGetLastError());
}

__global__ void k_unpack_pairs(const uint64_t *__restrict__ packed, int64_t *__restrict__ out, int count) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const uint64_t v = packed[i];
        out[2 * i] = static_cast<int64_t>(v >> 32);
        out[2 * i + 1] = static_cast<int64_t>(v & 0xffffffffull);
    }
}

void launch_sort_pairs(ncorp_ctx *c, int count) {
    if (count <= 0) return;
    launch_iota(c, c->pair_idx, count);
    radix_sort_u64(c, c->pairs, c->pair_idx, c->pairs_alt, c->pair_idx_alt, count, 64);
}

void launch_unpack_pairs(ncorp_ctx *c, const uint64_t *packed, int64_t *out, int count) {
    if (count <= 0) return;
    k_unpack_pairs<<<grid_for(count, 256, 4 * c->num_sms), 256, 0, c->stream>>>(packed, out, count); c->launches++;
    NCORP_CUDA_CHECK(cudaGetLastError());
}

}  // namespace ncorp
