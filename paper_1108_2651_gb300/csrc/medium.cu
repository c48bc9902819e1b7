// Medium upload and small reductions.
//
// Medium (paper, Eq. 3 and Sec. "Lattice BGK formulation"): from relative
// eps_r, mu_r per site, c_eff^2 = c_ref^2/(eps_r mu_r) (c = 1/sqrt(mu0 eps0)),
// c_L^2 = (D-1) c_eff^2, rest weight w0 = 1 - D c_L^2, which must lie in
// [0, 1); grad ln mu by periodic central differences.  Validation is done in
// FP64 in a first pass that writes nothing, so a rejected medium leaves the
// handle's previous medium in place.
#include "lbem_internal.cuh"

namespace lbk {

__global__ void medium_check(const float *eps, const float *mu, long long n, int D, double c_ref2, double fsum,
                             double mubar, unsigned *bad) {
    unsigned local = 0;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        const double e = eps[s], m = mu ? (double)mu[s] : 1.0;
        if (!(e > 0.0) || !(m > 0.0) || !isfinite(e) || !isfinite(m)) {
            local++;
            continue;
        }
        const double cl = (D - 1) * c_ref2 / (e * m * mubar);
        const double w0 = 1.0 - fsum * cl;  // 1 - D c_L^2; anisotropic: 1 - (c_x^2 + c_y^2)
        if (!(w0 >= 0.0 && w0 < 1.0)) local++;
    }
    if (local) atomicAdd(bad, local);
}

__global__ void medium_write(Grid G, int D, double c_ref2, double mubar, const float *eps, const float *mu, float *cL2,
                             float *mu_out) {
    const long long n = (long long)G.nx * G.nrows;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        const long long row = s / G.nx;
        const int x = (int)(s - row * G.nx);
        const double m = mu ? (double)mu[s] : 1.0;
        const double cl = (D - 1) * c_ref2 / ((double)eps[s] * m * mubar);
        cL2[row * G.pitch + x] = (float)cl;
        if (mu_out) mu_out[row * G.pitch + x] = (float)m;
    }
}

__global__ void medium_grad(Grid G, int D, const float *mu_p, float *dlnmu) {
    const long long n = (long long)G.nx * G.nrows;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        const long long row = s / G.nx;
        const int x = (int)(s - row * G.nx);
        const int z = (int)(row / G.ny), y = (int)(row - (long long)z * G.ny);
        auto at = [&](int xx, int yy, int zz) {
            return log((double)mu_p[((long long)zz * G.ny + yy) * G.pitch + xx]);
        };
        const double gx = 0.5 * (at((x + 1) % G.nx, y, z) - at((x - 1 + G.nx) % G.nx, y, z));
        const double gy = 0.5 * (at(x, (y + 1) % G.ny, z) - at(x, (y - 1 + G.ny) % G.ny, z));
        dlnmu[row * G.pitch + x] = (float)gx;
        dlnmu[G.plane + row * G.pitch + x] = (float)gy;
        if (D == 3) {
            const double gz = 0.5 * (at(x, y, (z + 1) % G.nz) - at(x, y, (z - 1 + G.nz) % G.nz));
            dlnmu[2 * G.plane + row * G.pitch + x] = (float)gz;
        }
    }
}

static unsigned grid_for(long long n) {
    long long b = (n + 255) / 256;
    return (unsigned)(b < 4096 ? (b < 1 ? 1 : b) : 4096);
}

cudaError_t launch_medium(lbem_t *h, const float *eps, const float *mu, double fsum, double mubar, unsigned *bad,
                          cudaStream_t s) {
    // pass 1: validation only (caller reads *bad and decides)
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    medium_check<<<grid_for(h->nsite), 256, 0, s>>>(eps, mu, h->nsite, h->dim, h->c_ref2, fsum, mubar, bad);
    return cudaGetLastError();
}

cudaError_t launch_medium_write(lbem_t *h, const float *eps, const float *mu, double mubar, cudaStream_t s) {
    medium_write<<<grid_for(h->nsite), 256, 0, s>>>(h->grid, h->dim, h->c_ref2, mubar, eps, mu, h->cL2,
                                                     mu ? h->mu : nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !mu) return e;
    medium_grad<<<grid_for(h->nsite), 256, 0, s>>>(h->grid, h->dim, h->mu, h->dlnmu);
    return cudaGetLastError();
}

__global__ void maxabs_kernel(const float *a, long long n, unsigned *out) {
    float m = 0.f;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        const float v = fabsf(a[s]);
        if (v > m || v != v) m = (v != v) ? __int_as_float(0x7f800000) : v;
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(FULL, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));  // non-negative floats order as uints
}

cudaError_t launch_maxabs(const float *a, long long n, unsigned *out, cudaStream_t s) {
    maxabs_kernel<<<grid_for(n), 256, 0, s>>>(a, n, out);
    return cudaGetLastError();
}

// Fixed-order reduction of [n][3] partial sums (deterministic for a given n).
__global__ void reduce_partials_kernel(const double *p, int n, double *out) {
    __shared__ double sh[3][256];
    double a[3] = {0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < n; i += 256)
        for (int k = 0; k < 3; k++) a[k] += p[3 * i + k];
    for (int k = 0; k < 3; k++) sh[k][threadIdx.x] = a[k];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int k = 0; k < 3; k++) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; k++) out[k] = sh[k][0];
}

cudaError_t launch_reduce_partials(const double *partials, int n, double *out, cudaStream_t s) {
    reduce_partials_kernel<<<1, 256, 0, s>>>(partials, n, out);
    return cudaGetLastError();
}

// Energy density and Poynting vector per site from dense E, B (paper, Sec. "Heterogeneous media"):
//   u = sum_a (B_a^2 + E_a^2 / c_eff^2),   P_a = eps_abc E_b B_c,   c_eff^2 = c_L^2 / (D - 1)
__global__ void energy_flux_kernel(Grid G, int D, const float *E, const float *B, const float *cL2, float *u, float *P) {
    const long long n = (long long)G.nx * G.nrows;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        const long long row = s / G.nx;
        const int x = (int)(s - row * G.nx);
        const float ce2 = cL2[row * G.pitch + x] / (float)(D - 1);
        const float ex = E[s], ey = E[n + s], ez = E[2 * n + s];
        const float bx = B[s], by = B[n + s], bz = B[2 * n + s];
        if (u) u[s] = (bx * bx + by * by + bz * bz) + (ex * ex + ey * ey + ez * ez) / ce2;
        if (P) {
            P[s] = ey * bz - ez * by;
            P[n + s] = ez * bx - ex * bz;
            P[2 * n + s] = ex * by - ey * bx;
        }
    }
}

cudaError_t launch_energy_flux(const lbem_t *h, const float *E, const float *B, float *u, float *P, cudaStream_t s) {
    energy_flux_kernel<<<grid_for(h->nsite), 256, 0, s>>>(h->grid, h->dim, E, B, h->cL2, u, P);
    return cudaGetLastError();
}

int diag_blocks(long long nsite) {
    long long b = (nsite + BLOCK - 1) / BLOCK;
    return (int)(b < 1216 ? (b < 1 ? 1 : b) : 1216);  // 152 SMs x 8
}

}  // namespace lbk
