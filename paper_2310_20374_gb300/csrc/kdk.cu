// kdk.cu -- the SBAB1 leapfrog pieces (Sect. 4.1: half kick, drift, half
// kick; consecutive half kicks merged between outputs) and the conversions
// between the caller's [n][3] arrays and the library's tree-ordered SoA.
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

__global__ void k_scatter_aos(const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z,
                              const int *__restrict__ perm, double *__restrict__ aos, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int u = perm[i];
        aos[3 * u] = x[i];
        aos[3 * u + 1] = y[i];
        aos[3 * u + 2] = z[i];
    }
}

__global__ void k_scatter_scalar(const double *__restrict__ v, const int *__restrict__ perm, double *__restrict__ out,
                                 int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[perm[i]] = v[i];
}

__global__ void k_kick(const double *__restrict__ vx, const double *__restrict__ vy, const double *__restrict__ vz,
                       const double *__restrict__ ax, const double *__restrict__ ay, const double *__restrict__ az,
                       double h, double *ox, double *oy, double *oz, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        ox[i] = dadd(vx[i], dmul(h, ax[i]));
        oy[i] = dadd(vy[i], dmul(h, ay[i]));
        oz[i] = dadd(vz[i], dmul(h, az[i]));
    }
}

__global__ void k_drift(const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z,
                        const double *__restrict__ vx, const double *__restrict__ vy, const double *__restrict__ vz,
                        double dt, double *ox, double *oy, double *oz, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        ox[i] = dadd(x[i], dmul(dt, vx[i]));
        oy[i] = dadd(y[i], dmul(dt, vy[i]));
        oz[i] = dadd(z[i], dmul(dt, vz[i]));
    }
}

static int eg(ncorp_ctx *c, int n) { return grid_for(n, 256, 16 * c->num_sms); }

void launch_aos_to_soa(ncorp_ctx *c, const double *aos, double *x, double *y, double *z, int n) {
    k_aos_to_soa<<<eg(c, n), 256, 0, c->stream>>>(aos, x, y, z, n); c->launches++;
    NCORP_CUDA_CHECK(cudaGetLastError());
}

void launch_scatter_aos(ncorp_ctx *c, const double *x, const double *y, const double *z, const int *perm,
                        double *aos, int n) {
    k_scatter_aos<<<eg(c, n), 256, 0, c->stream>>>(x, y, z, perm, aos, n); c->launches++;
    NCORP_CUDA_CHECK(cudaGetLastError());
}

void launch_scatter_scalar(ncorp_ctx *c, const double *v, const int *perm, double *out, int n) {
    k_scatter_scalar<<<eg(c, n), 256, 0, c->stream>>>(v, perm, out, n); c->launches++;
    NCORP_CUDA_CHECK(cudaGetLastError());
}

void launch_kick(ncorp_ctx *c, const double *vx, const double *vy, const double *vz, const double *ax,
                 const double *ay, const double *az, double h, double *ox, double *oy, double *oz, int n) {
    k_kick<<<eg(c, n), 256, 0, c->stream>>>(vx, vy, vz, ax, ay, az, h, ox, oy, oz, n); c->launches++;
    NCORP_CUDA_CHECK(cudaGetLastError());
}

void launch_drift(ncorp_ctx *c, const double *x, const double *y, const double *z, const double *vx,
                  const double *vy, const double *vz, double dt, double *ox, double *oy, double *oz, int n) {
    k_drift<<<eg(c, n), 256, 0, c->stream>>>(x, y, z, vx, vy, vz, dt, ox, oy, oz, n); c->launches++;
    NCORP_CUDA_CHECK(cudaGetLastError());
}

}  // namespace ncorp
