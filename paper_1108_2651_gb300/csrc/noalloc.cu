// lbem_diagnostics_static: the FP64 diagnostics of lbem_diagnostics for a state
// held entirely in caller memory, for callers that must not allocate device
// memory.  Examples: a program that reserves all device memory for its own
// pool at start-up and hands out only its own buffers, or a long-running
// loop whose memory budget is fixed after initialisation, where any
// cudaMalloc (by us or by a library on our behalf) could fail or is forbidden.
//
// The only scratch is the per-block partial sums.  They live in the
// file-scope static device array below (every GPU that loads the library
// holds it until the process exits): 3 doubles per block for at most
// kStaticBlocks blocks, i.e. 192 KiB.  Each block reduces at most
// kSitesPerBlock sites, so grids of more than kStaticBlocks * kSitesPerBlock
// sites are rejected (LBEM_ERR_ARG).
//
// Scope: the state of a periodic, isotropic, non-dispersive handle (lbem_set_medium, no walls, no pole, no
// anisotropic tensor); for such a state the three sums are those of lbem_diagnostics.  Before anything is
// launched, each caller buffer is checked against the extent of the device allocation that holds it
// (cuMemGetAddressRange, fetched through the runtime's driver entry point), so an undersized or unpadded
// state is an argument error and not an out-of-bounds read.
//
// Set-up: the first call on each device, with that device current, looks up
// the array's device address with cudaGetSymbolAddress (the host-side name of
// a __device__ array is only a stand-in and must not be passed to a kernel).
// That first call should therefore come before any stream capture on that
// device.  Every call shares the one array; a call overwrites every slot it
// later reads, so nothing needs clearing, but calls that overlap on the GPU
// (on different streams without ordering) race on it.
#include <cuda.h>
#include <math.h>

#include <mutex>

#include "lbem_internal.cuh"

namespace lbk {

constexpr int kStaticBlocks = 8192;
constexpr int kSitesPerBlock = 16 * BLOCK;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_diag_scratch[3 * kStaticBlocks];

static void *g_scratch_addr[kMaxDevices];
static std::mutex g_scratch_mu;

static lbem_status scratch_address(double **out) {
    int dev = 0;
    LBEM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(LBEM_ERR_ARG, "lbem_diagnostics_static: device index too large");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_diag_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e, "lbem_diagnostics_static: cudaGetSymbolAddress");
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<double *>(g_scratch_addr[dev]);
    return LBEM_OK;
}

static bool on_device(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

using AddressRange = CUresult (*)(CUdeviceptr *, size_t *, CUdeviceptr);

static AddressRange address_range_fn() {
    static AddressRange fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<AddressRange>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// Whether `bytes` bytes from p lie inside the device allocation that holds p.
static lbem_status check_extent(const void *p, size_t bytes, const char *what) {
    AddressRange fn = address_range_fn();
    if (!fn) return fail(LBEM_ERR_CUDA, "lbem_diagnostics_static: cuMemGetAddressRange is unavailable");
    CUdeviceptr base = 0;
    size_t size = 0;
    if (fn(&base, &size, (CUdeviceptr)p) != CUDA_SUCCESS)
        return fail(LBEM_ERR_ARG, std::string("lbem_diagnostics_static: the extent of ") + what +
                                      " cannot be determined (not a device allocation)");
    const size_t avail = (size_t)(base + size - (CUdeviceptr)p);
    if (avail < bytes)
        return fail(LBEM_ERR_ARG, std::string("lbem_diagnostics_static: ") + what + " needs " + std::to_string(bytes) +
                                      " bytes but its allocation ends after " + std::to_string(avail));
    return LBEM_OK;
}

struct StaticGeom {
    int D, nx, ny, nz, pitch;
    long long plane, nsite;
    double c_ref2;
};

// c_L^2 at a site from the caller's eps_r (and mu_r), as lbem_set_medium computes it.
__device__ __forceinline__ double cl_at(const StaticGeom &g, const float *eps, const float *mu, long long s) {
    const double m = mu ? (double)mu[s] : 1.0;
    return (double)(float)((g.D - 1) * g.c_ref2 / ((double)eps[s] * m));
}

// pre-collision value of plane p at (x, y, z): stored at the writing site x - c_i
__device__ __forceinline__ double pulled(const StaticGeom &g, const float *st, int p, int x, int y, int z) {
    int i, cx = 0, cy = 0, cz = 0;
    if (g.D == 2) {
        i = p;
        const int tx[5] = {0, 1, 0, -1, 0}, ty[5] = {0, 0, 1, 0, -1};
        cx = tx[i];
        cy = ty[i];
    } else {
        i = p / 3;
        const int tc[7][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {-1, 0, 0}, {0, -1, 0}, {0, 0, -1}};
        cx = tc[i][0];
        cy = tc[i][1];
        cz = tc[i][2];
    }
    const int xs = (x - cx + g.nx) % g.nx, ys = (y - cy + g.ny) % g.ny, zs = (z - cz + g.nz) % g.nz;
    return (double)st[p * g.plane + ((long long)zs * g.ny + ys) * g.pitch + xs];
}

__device__ double b_at(const StaticGeom &g, const float *st, int comp, int x, int y, int z) {
    if (g.D == 2) {  // B_x = g_4 - g_2, B_y = g_1 - g_3
        return comp == 0 ? pulled(g, st, 4, x, y, z) - pulled(g, st, 2, x, y, z)
                         : pulled(g, st, 1, x, y, z) - pulled(g, st, 3, x, y, z);
    }
    auto R = [&](int gm, int k) { return pulled(g, st, (1 + k) * 3 + gm, x, y, z) - pulled(g, st, (4 + k) * 3 + gm, x, y, z); };
    if (comp == 0) return R(1, 2) - R(2, 1);
    if (comp == 1) return R(2, 0) - R(0, 2);
    return R(0, 1) - R(1, 0);
}

__global__ void __launch_bounds__(BLOCK) diag_static_kernel(StaticGeom g, const float *st, const float *eps,
                                                            const float *mu, double *partials) {
    __shared__ double sh[3][BLOCK / 32];
    double acc[3] = {0.0, 0.0, 0.0};
    const int npop = g.D == 2 ? 5 : 21;
    for (long long s = (long long)blockIdx.x * BLOCK + threadIdx.x; s < g.nsite; s += (long long)gridDim.x * BLOCK) {
        const int x = (int)(s % g.nx);
        const long long rr = s / g.nx;
        const int y = (int)(rr % g.ny), z = (int)(rr / g.ny);
        const double cl = cl_at(g, eps, mu, s);
        const double ce2 = cl / (g.D - 1), w0 = 1.0 - g.D * cl, wm = 0.5 * cl;
        double sg[3] = {0.0, 0.0, 0.0}, q = 0.0;
        for (int p = 0; p < npop; p++) {
            const double v = pulled(g, st, p, x, y, z);
            const int comp = g.D == 2 ? 2 : p % 3;
            sg[comp] += v;
            const bool rest = g.D == 2 ? p == 0 : p < 3;
            if (!rest) q += v * v / wm;
            else if (w0 != 0.0) q += v * v / w0;
        }
        acc[1] += 2.0 * q;
        const int nb = g.D == 2 ? 2 : 3;
        double div = 0.0;
        for (int k = 0; k < 3; k++) {
            const double e = -cl * sg[k];
            acc[0] += e * e / ce2;
        }
        for (int k = 0; k < nb; k++) {
            const double b = b_at(g, st, k, x, y, z);
            acc[0] += b * b;
            const int xp = k == 0 ? (x + 1) % g.nx : x, xm = k == 0 ? (x - 1 + g.nx) % g.nx : x;
            const int yp = k == 1 ? (y + 1) % g.ny : y, ym = k == 1 ? (y - 1 + g.ny) % g.ny : y;
            const int zp = k == 2 ? (z + 1) % g.nz : z, zm = k == 2 ? (z - 1 + g.nz) % g.nz : z;
            div += 0.5 * (b_at(g, st, k, xp, yp, zp) - b_at(g, st, k, xm, ym, zm));
        }
        acc[2] += div * div;
    }
    for (int k = 0; k < 3; k++) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
        if ((threadIdx.x & 31) == 0) sh[k][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double r = 0.0;
        for (int w = 0; w < BLOCK / 32; w++) r += sh[threadIdx.x][w];
        partials[3 * blockIdx.x + threadIdx.x] = r;
    }
}

// Fixed-order sum of the nblocks partials; out[2] becomes the L2 norm of div B.
__global__ void diag_static_finish(const double *partials, int nblocks, double *out) {
    __shared__ double sh[3][256];
    double a[3] = {0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < nblocks; i += 256)
        for (int k = 0; k < 3; k++) a[k] += partials[3 * i + k];
    for (int k = 0; k < 3; k++) sh[k][threadIdx.x] = a[k];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int k = 0; k < 3; k++) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sh[0][0];
        out[1] = sh[1][0];
        out[2] = sqrt(sh[2][0]);
    }
}

}  // namespace lbk

using namespace lbk;

extern "C" lbem_status lbem_diagnostics_static(int dim, int nx, int ny, int nz, const void *state, const float *eps_r,
                                               const float *mu_r, double c_ref2, double *out, void *stream) {
    if (dim != 2 && dim != 3) return fail(LBEM_ERR_ARG, "lbem_diagnostics_static: dim must be 2 or 3");
    if (dim == 2) nz = 1;
    if (nx < 1 || ny < 1 || nz < 1) return fail(LBEM_ERR_ARG, "lbem_diagnostics_static: grid sizes must be >= 1");
    // each factor bounded by division first, so the product below cannot overflow
    const long long limit = (long long)kStaticBlocks * kSitesPerBlock;
    if (nx > limit || ny > limit / nx || nz > limit / ((long long)nx * ny))
        return fail(LBEM_ERR_ARG, "lbem_diagnostics_static: grid of " + std::to_string(nx) + " x " +
                                      std::to_string(ny) + " x " + std::to_string(nz) +
                                      " sites exceeds the static scratch limit of " + std::to_string(limit) +
                                      " sites");
    const long long nsite = (long long)nx * ny * nz;
    const long long nblocks = (nsite + kSitesPerBlock - 1) / kSitesPerBlock;
    if (!state || !eps_r || !out) return fail(LBEM_ERR_ARG, "lbem_diagnostics_static: null pointer");
    if (!on_device(state) || !on_device(eps_r) || !on_device(out) || (mu_r && !on_device(mu_r)))
        return fail(LBEM_ERR_ARG, "lbem_diagnostics_static: state, eps_r, mu_r and out must be device memory");
    const int npop = dim == 2 ? 5 : 21;
    const size_t state_bytes = sizeof(float) * (size_t)npop * (size_t)round_up(nx, 32) * (size_t)ny * (size_t)nz;
    lbem_status st = check_extent(state, state_bytes, "state");
    if (st == LBEM_OK) st = check_extent(eps_r, sizeof(float) * (size_t)nsite, "eps_r");
    if (st == LBEM_OK && mu_r) st = check_extent(mu_r, sizeof(float) * (size_t)nsite, "mu_r");
    if (st == LBEM_OK) st = check_extent(out, 3 * sizeof(double), "out");
    if (st != LBEM_OK) return st;
    double *scratch = nullptr;
    st = scratch_address(&scratch);
    if (st != LBEM_OK) return st;
    StaticGeom g;
    g.D = dim;
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.pitch = round_up(nx, 32);  // the row pitch of lbem_create's layout
    g.plane = (long long)g.pitch * ny * nz;
    g.nsite = nsite;
    g.c_ref2 = c_ref2 > 0 ? c_ref2 : (dim == 2 ? 0.5 : 1.0 / 6.0);
    cudaStream_t s = (cudaStream_t)stream;
    diag_static_kernel<<<(unsigned)nblocks, BLOCK, 0, s>>>(g, static_cast<const float *>(state), eps_r, mu_r, scratch);
    LBEM_CUDA(cudaGetLastError());
    diag_static_finish<<<1, 256, 0, s>>>(scratch, (int)nblocks, out);
    LBEM_CUDA(cudaGetLastError());
    return LBEM_OK;
}
