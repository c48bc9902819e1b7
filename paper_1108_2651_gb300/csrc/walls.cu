// Walls and absorbing layers (FP32 storage): the 2D edge kernel and the wall-aware grad ln mu (2D and 3D).  In
// 3D the one-site-per-thread stream-collide kernel applies walls and layers itself (kernels3d.cu).
//
// The paper treats periodic domains only and leaves other boundaries open.
// Here a wall sits half a site beyond the first / last site of an axis: a
// population that would be pulled across it is the opposite population of
// the same site, collided one step earlier, times -1 (PEC: E_z and the normal
// B vanish on the wall) or +1 (PMC: the tangential B vanishes).  An absorbing
// layer of L sites inside each wall multiplies the post-collision populations
// of a site at distance i from the wall-adjacent site by
// 1 - gamma_max ((L - i)/L)^2 (both axes' factors at corners), damping E and
// B alike so the layer keeps the wave impedance of the medium.
//
// The stream-collide kernels stay periodic and unchanged.  After each launch
// of k steps, edge2d recomputes those k steps on the bands whose result the
// walls or layers change -- the sites within max(L, 1) + k - 1 of a wall --
// from the launch's input state, and overwrites them (and their receiver
// samples).  Each edge tile stages its output rectangle plus a k-site halo in
// shared memory and performs the k steps there with the same per-site
// arithmetic as the stream-collide kernels (collide2d, mu_source,
// site_events), so interior and band sites, and every steps-per-launch
// setting, give the same bits.  The bands are O(nx + ny) sites: a few percent
// of a large grid.
#include <algorithm>
#include <vector>

#include "lbem_internal.cuh"

namespace lbk {

constexpr int EDGE_THREADS = 512;
constexpr int EDGE_MAX_WINDOW = 1536;  // staged sites per tile (output rectangle plus halo)
constexpr int EDGE_PER_THREAD = EDGE_MAX_WINDOW / EDGE_THREADS;

// Per staged site: current and next populations (10 floats), c_L^2, the layer factor; with mu, grad ln mu.
// Then per window column its global x and per window row its global y (-1 beyond a wall) and whether the row
// holds sources or receivers.
__host__ __device__ constexpr int edge_floats_per_site(bool mu) { return 12 + (mu ? 2 : 0); }

// AN: an anisotropic medium (a uniform in-plane tensor, a.med.ar, a.med.amu, no pole): collide2d_an and the events
// scaled as site_events scales them, as the general single-step kernel and step2d_ss2<AN> / step2d_tb2<AN> do.
template <bool MU, bool AN = false>
__global__ void __launch_bounds__(EDGE_THREADS, 3) edge2d(StepArgs a, Walls w, const EdgeTile *tiles, int k) {
    extern __shared__ __align__(16) float sm[];
    const Grid &G = a.g;
    const EdgeTile T = tiles[blockIdx.x];
    const int WW = T.w + 2 * k, WH = T.h + 2 * k, NW = WW * WH;
    const int wx0 = T.x0 - k, wy0 = T.y0 - k;  // unwrapped coordinates of window site (0, 0)
    float *cur = sm, *nxt = sm + 5 * NW, *cl = sm + 10 * NW, *fac = sm + 11 * NW;
    float *dxm = sm + 12 * NW, *dym = sm + 13 * NW;  // MU only
    int *colg = reinterpret_cast<int *>(sm + edge_floats_per_site(MU) * NW), *rowg = colg + WW, *rowev = rowg + WH;
    const float *in = static_cast<const float *>(a.in.data);
    const float sx = w.kind[0] == 1 ? -1.f : 1.f, sy = w.kind[1] == 1 ? -1.f : 1.f;

    // global coordinate of an unwrapped one along an axis, or -1 beyond a wall
    auto gcoord = [](int v, int n, int kind) { return kind ? ((unsigned)v < (unsigned)n ? v : -1) : wrapi(v, n); };
    for (int i = threadIdx.x; i < WW; i += EDGE_THREADS) colg[i] = gcoord(wx0 + i, G.nx, w.kind[0]);
    for (int j = threadIdx.x; j < WH; j += EDGE_THREADS) {
        const int gy = gcoord(wy0 + j, G.ny, w.kind[1]);
        rowg[j] = gy;
        rowev[j] = (gy >= 0 && a.evt.rowptr) ? (__ldg(a.evt.rowptr + gy + 1) > __ldg(a.evt.rowptr + gy)) : 0;
    }
    // this thread's window sites s = threadIdx.x + u * EDGE_THREADS, as (column, row); row WH marks none
    int ci[EDGE_PER_THREAD], rj[EDGE_PER_THREAD];
#pragma unroll
    for (int u = 0; u < EDGE_PER_THREAD; u++) {
        const int s = threadIdx.x + u * EDGE_THREADS;
        rj[u] = s < NW ? s / WW : WH;
        ci[u] = s - rj[u] * WW;
    }
    __syncthreads();

    // window load: a thread's sites are loaded together (the loads of all of them in flight at once)
    {
        float v[EDGE_PER_THREAD][5], c[EDGE_PER_THREAD], f[EDGE_PER_THREAD], dx[EDGE_PER_THREAD],
            dy[EDGE_PER_THREAD];
        bool ok[EDGE_PER_THREAD];
#pragma unroll
        for (int u = 0; u < EDGE_PER_THREAD; u++) {
            const int gx = rj[u] < WH ? colg[ci[u]] : -1, gy = rj[u] < WH ? rowg[rj[u]] : -1;
            ok[u] = gx >= 0 && gy >= 0;
            if (ok[u]) {
                const long long o = (long long)gy * G.pitch + gx;
                const long long oi = (long long)gy * a.in.pitch + gx;
#pragma unroll
                for (int p = 0; p < 5; p++) v[u][p] = __ldg(in + p * a.in.plane + oi);
                c[u] = __ldg(a.med.cL2 + o);
                f[u] = __fmul_rn(w.fx ? __ldg(w.fx + gx) : 1.f, w.fy ? __ldg(w.fy + gy) : 1.f);
                if (MU) {
                    dx[u] = __ldg(a.med.dlnmu + o);
                    dy[u] = __ldg(a.med.dlnmu + G.plane + o);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < EDGE_PER_THREAD; u++) {
            const int s = threadIdx.x + u * EDGE_THREADS;
            if (ok[u]) {
#pragma unroll
                for (int p = 0; p < 5; p++) cur[p * NW + s] = v[u][p];
                cl[s] = c[u];
                fac[s] = f[u];
                if (MU) {
                    dxm[s] = dx[u];
                    dym[s] = dy[u];
                }
            }
        }
    }
    __syncthreads();

    const float ar = AN ? a.med.ar : 1.f, ri = AN ? __fdiv_rn(1.f, ar) : 1.f, fs = __fadd_rn(ar, ri);
    for (int step = 0; step < k; step++) {
        const long long t = a.t + step;
#pragma unroll
        for (int u = 0; u < EDGE_PER_THREAD; u++) {
            const int i = ci[u], j = rj[u];
            if (j >= WH) continue;
            const int gx = colg[i], gy = rowg[j];
            if (gx < 0 || gy < 0) continue;
            const int s = threadIdx.x + u * EDGE_THREADS;
            // pulls g_i(x) = g'_i(x - c_i): across a wall the opposite population of this site times the wall
            // sign; beyond the window's open edges the value is never used by an output site (0 here)
            const float g0 = cur[s];
            float g1 = 0.f, g2 = 0.f, g3 = 0.f, g4 = 0.f;
            if (w.kind[0] && gx == 0) g1 = sx * cur[3 * NW + s];
            else if (i > 0) g1 = cur[NW + s - 1];
            if (w.kind[0] && gx == G.nx - 1) g3 = sx * cur[NW + s];
            else if (i + 1 < WW) g3 = cur[3 * NW + s + 1];
            if (w.kind[1] && gy == 0) g2 = sy * cur[4 * NW + s];
            else if (j > 0) g2 = cur[2 * NW + s - WW];
            if (w.kind[1] && gy == G.ny - 1) g4 = sy * cur[2 * NW + s];
            else if (j + 1 < WH) g4 = cur[4 * NW + s + WW];
            const float c = cl[s];
            float shat = 0.f;
            if (MU) shat = mu_source(g4 - g2, g1 - g3, dxm[s], dym[s]);
            if (rowev[j]) {
                const bool owned = i >= k && i < k + T.w && j >= k && j < k + T.h;
                shat = AN ? site_events(a, gx, gy, t, owned, g0, g1, g2, g3, g4, c, 0.f, 0.f, ar, ri, a.med.amu)
                          : site_events(a, gx, gy, t, owned, g0, g1, g2, g3, g4, c, shat);
            }
            const Out5 r = AN ? collide2d_an(g0, g1, g2, g3, g4, c, shat, ar, ri, fs, 0.f)
                              : collide2d(g0, g1, g2, g3, g4, c, shat);
            const float f = fac[s];
            nxt[s] = __fmul_rn(r.o0, f);
            nxt[NW + s] = __fmul_rn(r.o1, f);
            nxt[2 * NW + s] = __fmul_rn(r.o2, f);
            nxt[3 * NW + s] = __fmul_rn(r.o3, f);
            nxt[4 * NW + s] = __fmul_rn(r.o4, f);
        }
        __syncthreads();
        float *tmp = cur;
        cur = nxt;
        nxt = tmp;
    }

    // the output rectangle (window columns and rows k .. k + w - 1, k .. k + h - 1)
    float *out = static_cast<float *>(a.out.data);
#pragma unroll
    for (int u = 0; u < EDGE_PER_THREAD; u++) {
        const int i = ci[u], j = rj[u];
        if (j < k || j >= k + T.h || i < k || i >= k + T.w) continue;
        const int s = threadIdx.x + u * EDGE_THREADS;
        const long long o = (long long)(T.y0 + j - k) * a.out.pitch + (T.x0 + i - k);
#pragma unroll
        for (int p = 0; p < 5; p++) out[p * a.out.plane + o] = cur[p * NW + s];
    }
}

// Tiles covering the bands of a k-step launch: per walled axis the sites within max(L, 1) + k - 1 of either
// wall (the whole axis when the two bands meet); the y bands skip columns the x bands already cover.  Each
// tile's output rectangle plus its k-site halo holds at most EDGE_MAX_WINDOW sites.
std::vector<EdgeTile> edge_tiles(const Grid &G, const int kind[2], int layer, int k) {
    std::vector<EdgeTile> t;
    const int bw = std::max(layer, 1) + k - 1;
    auto cover = [&](int x0, int x1, int y0, int y1, bool across_x) {
        // rectangle [x0, x1) x [y0, y1); tiles are at most 64 sites across the band
        if (x0 >= x1 || y0 >= y1) return;
        int tw, th;
        if (across_x) {
            tw = std::min(x1 - x0, 64);
            th = std::max(1, EDGE_MAX_WINDOW / (tw + 2 * k) - 2 * k);
        } else {
            th = std::min(y1 - y0, 64);
            tw = std::max(1, EDGE_MAX_WINDOW / (th + 2 * k) - 2 * k);
        }
        for (int y = y0; y < y1; y += th)
            for (int x = x0; x < x1; x += tw) t.push_back({x, y, std::min(tw, x1 - x), std::min(th, y1 - y)});
    };
    // column ranges of the x bands
    std::vector<std::pair<int, int>> xr;
    if (kind[0]) {
        if (2 * bw >= G.nx) xr.push_back({0, G.nx});
        else {
            xr.push_back({0, bw});
            xr.push_back({G.nx - bw, G.nx});
        }
        for (auto &r : xr) cover(r.first, r.second, 0, G.ny, true);
    }
    if (kind[1]) {
        // the columns left to the y bands
        std::vector<std::pair<int, int>> cols;
        if (xr.empty()) cols.push_back({0, G.nx});
        else if (xr.size() == 2) cols.push_back({bw, G.nx - bw});
        std::vector<std::pair<int, int>> yr;
        if (2 * bw >= G.ny) yr.push_back({0, G.ny});
        else {
            yr.push_back({0, bw});
            yr.push_back({G.ny - bw, G.ny});
        }
        for (auto &c : cols)
            for (auto &r : yr) cover(c.first, c.second, r.first, r.second, false);
    }
    return t;
}

size_t edge_smem_bytes(int k, const std::vector<EdgeTile> &tiles, bool mu) {
    int nw = 0, wh = 0;
    for (auto &e : tiles) {
        nw = std::max(nw, (e.w + 2 * k) * (e.h + 2 * k));
        wh = std::max(wh, e.h + 2 * k);
    }
    int ww = 0;
    for (auto &e : tiles) ww = std::max(ww, e.w + 2 * k);
    return sizeof(float) * (size_t)edge_floats_per_site(mu) * nw + sizeof(int) * (size_t)(ww + 2 * wh);
}

cudaError_t launch_edge_2d(const StepArgs &a, const Walls &w, const EdgeTile *d_tiles, int ntiles, size_t smem, int k,
                           bool aniso, cudaStream_t s) {
    if (ntiles == 0) return cudaSuccess;
    static bool attr[3] = {false, false, false};
    const bool mu = a.med.dlnmu != nullptr;
    if (aniso && mu) return cudaErrorInvalidValue;  // an anisotropic medium has a uniform permeability
    const int v = aniso ? 2 : mu ? 1 : 0;
    if (!attr[v]) {
        const int max_bytes = (int)((sizeof(float) * edge_floats_per_site(true) + 3 * sizeof(int)) * EDGE_MAX_WINDOW);
        cudaError_t e = v == 2   ? cudaFuncSetAttribute(edge2d<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                        max_bytes)
                        : v == 1 ? cudaFuncSetAttribute(edge2d<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                        max_bytes)
                                 : cudaFuncSetAttribute(edge2d<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                        max_bytes);
        if (e != cudaSuccess) return e;
        attr[v] = true;
    }
    if (v == 2) edge2d<false, true><<<ntiles, EDGE_THREADS, smem, s>>>(a, w, d_tiles, k);
    else if (v == 1) edge2d<true><<<ntiles, EDGE_THREADS, smem, s>>>(a, w, d_tiles, k);
    else edge2d<false><<<ntiles, EDGE_THREADS, smem, s>>>(a, w, d_tiles, k);
    return cudaGetLastError();
}

// grad ln mu with walls: at the first / last site of a walled axis the missing neighbour is the mirror image
// (the site itself), as on the doubled periodic domain the walls stand for (2D and 3D).
__global__ void medium_grad_walls(Grid G, int D, int kx, int ky, int kz, const float *mu_p, float *dlnmu) {
    const long long n = (long long)G.nx * G.nrows;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        const long long row = s / G.nx;
        const int x = (int)(s - row * G.nx);
        const int z = (int)(row / G.ny), y = (int)(row - (long long)z * G.ny);
        auto nb = [](int v, int d, int len, int kind) {
            const int u = v + d;
            if (!kind) return (u + len) % len;
            return u < 0 ? 0 : (u >= len ? len - 1 : u);
        };
        auto at = [&](int xx, int yy, int zz) {
            return log((double)mu_p[((long long)zz * G.ny + yy) * G.pitch + xx]);
        };
        const double gx = 0.5 * (at(nb(x, 1, G.nx, kx), y, z) - at(nb(x, -1, G.nx, kx), y, z));
        const double gy = 0.5 * (at(x, nb(y, 1, G.ny, ky), z) - at(x, nb(y, -1, G.ny, ky), z));
        dlnmu[row * G.pitch + x] = (float)gx;
        dlnmu[G.plane + row * G.pitch + x] = (float)gy;
        if (D == 3) {
            const double gz = 0.5 * (at(x, y, nb(z, 1, G.nz, kz)) - at(x, y, nb(z, -1, G.nz, kz)));
            dlnmu[2 * G.plane + row * G.pitch + x] = (float)gz;
        }
    }
}

cudaError_t launch_medium_grad_walls(const lbem_t *h, cudaStream_t s) {
    const long long n = h->nsite;
    const unsigned blocks = (unsigned)std::min<long long>(4096, std::max<long long>(1, (n + 255) / 256));
    medium_grad_walls<<<blocks, 256, 0, s>>>(h->grid, h->dim, h->bc[0], h->bc[1], h->bc[2], h->mu, h->dlnmu);
    return cudaGetLastError();
}

}  // namespace lbk
