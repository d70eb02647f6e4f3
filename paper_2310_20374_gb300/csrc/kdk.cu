// kdk.cu -- the SBAB1 leapfrog pieces (Sect. 4.1: half kick, drift, half
// kick; consecutive half kicks merged between outputs) and the conversions
// between the caller's [n][3] arrays and the library's tree-ordered SoA.  The
// opening half kick and the drift are one kernel (with the bounding box of
// the drifted positions); the closing half kick is applied by the far-field
// kernel (eval.cu) right after the acceleration.
//
// Kicks and drifts use exactly rounded FP64 (v + (dt/2) a, x + dt v), so a
// step is reproducible bit for bit given the same accelerations.
#include "ctx.h"

namespace ncorp {

__global__ void k_aos_to_soa(const double *__restrict__ aos, double *x, double *y, double *z, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        x[i] = aos[3 * i];
        y[i] = aos[3 * i + 1];
        z[i] = aos[3 * i + 2];
    }
}

__device__ __forceinline__ bool scatter_gated(const int *a, const int *b) {
    return (a && (*reinterpret_cast<const volatile int *>(a) & ERR_ABORT_MASK)) ||
           (b && (*reinterpret_cast<const volatile int *>(b) & ERR_ABORT_MASK));
}

__global__ void k_scatter_aos(const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z,
                              const int *__restrict__ perm, double *__restrict__ aos, int n, const int *abort_a,
                              const int *abort_b) {
    if (scatter_gated(abort_a, abort_b)) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int u = perm[i];
        aos[3 * u] = x[i];
        aos[3 * u + 1] = y[i];
        aos[3 * u + 2] = z[i];
    }
}

// Half kick, drift and the bounding box of the drifted positions in one
// pass (the step's opening): v' = v + h a, x' = x + dt v', and the box of x'
// folded as in k_bbox (integer images, one atomic per bound per block).
__global__ void __launch_bounds__(256) k_kick_drift(KickDriftArgs A) {
    __shared__ unsigned long long s_b[6][8];
    __shared__ int s_bad;
    if (aborted(A.ctl)) return;   // the run aborted in an earlier step: nothing is computed from it
    unsigned long long lo[3] = {~0ull, ~0ull, ~0ull}, hi[3] = {0ull, 0ull, 0ull};
    bool bad = false;
    if (A.ctl->disk_of) {   // a forest: the same step, every disk's own box
        const int lane = threadIdx.x & 31;
        for (int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < A.n; base += gridDim.x * blockDim.x) {
            const int i = base + lane;
            const bool valid = i < A.n;
            unsigned long long l[3] = {~0ull, ~0ull, ~0ull}, h[3] = {0ull, 0ull, 0ull};
            if (valid) {
                const double vx = dadd(A.vx[i], dmul(A.h, A.ax[i]));
                const double vy = dadd(A.vy[i], dmul(A.h, A.ay[i]));
                const double vz = dadd(A.vz[i], dmul(A.h, A.az[i]));
                A.ovx[i] = vx;
                A.ovy[i] = vy;
                A.ovz[i] = vz;
                const double v[3] = {dadd(A.x[i], dmul(A.dt, vx)), dadd(A.y[i], dmul(A.dt, vy)),
                                     dadd(A.z[i], dmul(A.dt, vz))};
                A.ox[i] = v[0];
                A.oy[i] = v[1];
                A.oz[i] = v[2];
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(v[k]));
                    bad |= (u & 0x7ff0000000000000ull) == 0x7ff0000000000000ull;
                    l[k] = h[k] = ord_encode(v[k]);
                }
            }
            fold_disk_box(A.ctl, valid ? A.ctl->disk_of[i] : 0, valid, l, h);
        }
        if (bad) atomicOr(&A.ctl->err, ERR_NONFINITE);
        return;
    }
    if (threadIdx.x == 0) s_bad = 0;
    bool over = false;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += gridDim.x * blockDim.x) {
        const double vx = dadd(A.vx[i], dmul(A.h, A.ax[i]));
        const double vy = dadd(A.vy[i], dmul(A.h, A.ay[i]));
        const double vz = dadd(A.vz[i], dmul(A.h, A.az[i]));
        A.ovx[i] = vx;
        A.ovy[i] = vy;
        A.ovz[i] = vz;
        if (A.rc_spec) {   // fused walk: this step's R + dt |v| against the bound the tree was walked with
            const double e = dadd(A.R[i], dmul(A.dt, dnorm3(vx, vy, vz)));
            over |= !(e <= A.rc_spec[i]);
            A.cv4[i] = make_float4(static_cast<float>(vx), static_cast<float>(vy), static_cast<float>(vz),
                                   __double2float_ru(e));
        }
        const double v[3] = {dadd(A.x[i], dmul(A.dt, vx)), dadd(A.y[i], dmul(A.dt, vy)), dadd(A.z[i], dmul(A.dt, vz))};
        A.ox[i] = v[0];
        A.oy[i] = v[1];
        A.oz[i] = v[2];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(v[k]));
            bad |= (u & 0x7ff0000000000000ull) == 0x7ff0000000000000ull;
            const unsigned long long e = ord_encode(v[k]);
            lo[k] = e < lo[k] ? e : lo[k];
            hi[k] = e > hi[k] ? e : hi[k];
        }
    }
    if (over) atomicOr(A.stale, 1);
#pragma unroll
    for (int k = 0; k < 3; k++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long a = __shfl_xor_sync(0xffffffffu, lo[k], o);
            const unsigned long long b = __shfl_xor_sync(0xffffffffu, hi[k], o);
            lo[k] = a < lo[k] ? a : lo[k];
            hi[k] = b > hi[k] ? b : hi[k];
        }
    __syncthreads();
    if (__any_sync(0xffffffffu, bad) && lane_id() == 0) s_bad = 1;
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane_id() == 0)
#pragma unroll
        for (int k = 0; k < 3; k++) {
            s_b[k][w] = lo[k];
            s_b[3 + k][w] = hi[k];
        }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int k = threadIdx.x;
        unsigned long long r = s_b[k][0];
        for (int j = 1; j < nw; j++) {
            const unsigned long long v = s_b[k][j];
            r = k < 3 ? (v < r ? v : r) : (v > r ? v : r);
        }
        if (k < 3) atomicMin(&A.ctl->bbox[k], r);
        else atomicMax(&A.ctl->bbox[k], r);
    }
    if (threadIdx.x == 0 && s_bad) atomicOr(&A.ctl->err, ERR_NONFINITE);
}

// Positions and velocities to the caller's order in one pass.
__global__ void k_scatter_state(const double *__restrict__ x, const double *__restrict__ y,
                                const double *__restrict__ z, const double *__restrict__ vx,
                                const double *__restrict__ vy, const double *__restrict__ vz,
                                const int *__restrict__ perm, double *__restrict__ pos, double *__restrict__ vel, int n,
                                const int *abort_a, const int *abort_b) {
    if (scatter_gated(abort_a, abort_b)) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int u = perm[i];
        pos[3 * u] = x[i];
        pos[3 * u + 1] = y[i];
        pos[3 * u + 2] = z[i];
        vel[3 * u] = vx[i];
        vel[3 * u + 1] = vy[i];
        vel[3 * u + 2] = vz[i];
    }
}

static int eg(ncorp_ctx *c, int n) { return grid_for(n, 256, 16 * c->num_sms); }

void launch_aos_to_soa(ncorp_ctx *c, const double *aos, double *x, double *y, double *z, int n) {
    k_aos_to_soa<<<eg(c, n), 256, 0, c->stream>>>(aos, x, y, z, n); c->launches++;
    NCORP_CUDA_CHECK(cudaGetLastError());
}

void launch_scatter_aos(ncorp_ctx *c, const double *x, const double *y, const double *z, const int *perm,
                        double *aos, int n, const int *abort_a, const int *abort_b) {
    k_scatter_aos<<<eg(c, n), 256, 0, c->stream>>>(x, y, z, perm, aos, n, abort_a, abort_b); c->launches++;
    NCORP_CUDA_CHECK(cudaGetLastError());
}

void launch_kick_drift(ncorp_ctx *c, const KickDriftArgs &A) {
    k_kick_drift<<<grid_for(A.n, 256, c->num_sms), 256, 0, c->stream>>>(A); c->launches++;
    NCORP_CUDA_CHECK(cudaGetLastError());
}

void launch_scatter_state(ncorp_ctx *c, const ParticleSet &S, double *pos, double *vel, int n, const int *abort_a,
                          const int *abort_b) {
    k_scatter_state<<<eg(c, n), 256, 0, c->stream>>>(S.x, S.y, S.z, S.vx, S.vy, S.vz, S.perm, pos, vel, n, abort_a,
                                                     abort_b);
    c->launches++;
    NCORP_CUDA_CHECK(cudaGetLastError());
}


}  // namespace ncorp
