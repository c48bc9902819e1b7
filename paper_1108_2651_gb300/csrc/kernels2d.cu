// 2D (D2Q5) kernels of the lattice-Boltzmann Maxwell scheme of Hanasoge,
// Succi & Orszag (arXiv:1108.2651): fused pull-stream + moments + source +
// BGK collision (Eqs. 3, 8, 17, 18), initial state (Eq. 8), field extraction
// (Eqs. 9-10) and FP64 diagnostics.
//
// The single independent tensor component g_i = g_{i,xy} is stored per
// direction i (D2Q5 order c_0 = 0, c_1 = +x, c_2 = +y, c_3 = -x, c_4 = -y).
// With tau = dt/2 (Delta t / tau = 2) and the weights of moving particles
// equal to c_L^2/2, the collision of Eq. 17 with the equilibrium of Eq. 8
// reduces per site to (sigma = sum_i g_i, Lambda = c_L^2 sigma = -E_z,
// B_y = g_1 - g_3, B_x = g_4 - g_2):
//   g'_1 = Lambda - g_3 + T_m    g'_3 = Lambda - g_1 + T_m
//   g'_2 = Lambda - g_4 + T_m    g'_4 = Lambda - g_2 + T_m
//   g'_0 = 2 w0 sigma - g_0 + T_0,   w0 = 1 - 2 c_L^2,
// since 2 g^(0)_1 = Lambda + B_y etc.  The source of Eq. 3 is S_z = c_L^2 S^
// with S^ = B_x d_y ln mu - B_y d_x ln mu - mu j_z, and the tensor source
// T_i = -(w_i / c_L^2) S_z gives T_m = -c_L^2 S^/2, T_0 = -w0 S^.
//
// Thread mapping: one warp covers 128 consecutive sites of one row, 4 per
// lane, loaded as one 4-element vector per population.  The +x / -x pulls are
// shifted by one site: the neighbouring lane's element arrives by a warp
// shuffle; the first and last lane of a warp fetch one element each.
#include "lbem_internal.cuh"

namespace lbk {

template <int ST>
struct Pull2D {
    float4 g[5];
};

// Pre-collision populations of the 4 sites (row, 4c..4c+3): g_i(x) = buf_i(x - c_i).
// Must be called by all 32 lanes of a warp (shuffles); lanes with c >= nchunk
// load nothing and their results are discarded by the caller.
template <int ST>
__device__ __forceinline__ void pull2d(const PopBuf &in, const Grid &G, int row, int c, int lane, float4 g[5]) {
    using C = Codec<ST>;
    const int x0 = 4 * c;
    const bool active = c < G.nchunk;  // lanes past the row end load nothing
    const int ym = row == 0 ? G.ny - 1 : row - 1;
    const int yp = row == G.ny - 1 ? 0 : row + 1;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    g[0] = active ? C::load4(in, 0, row, c) : z4;
    float4 a1 = active ? C::load4(in, 1, row, c) : z4;
    g[2] = active ? C::load4(in, 2, ym, c) : z4;
    float4 a3 = active ? C::load4(in, 3, row, c) : z4;
    g[4] = active ? C::load4(in, 4, yp, c) : z4;
    float prev = __shfl_up_sync(FULL, a1.w, 1);
    float next = __shfl_down_sync(FULL, a3.x, 1);
    if (lane == 0 && active) prev = C::load1(in, 1, row, c == 0 ? G.nx - 1 : x0 - 1);
    if (lane == 31 && x0 + 4 < G.nx) next = C::load1(in, 3, row, x0 + 4);
    g[1] = make_float4(prev, a1.x, a1.y, a1.z);
    g[3] = make_float4(a3.y, a3.z, a3.w, next);
    if (c == G.nchunk - 1) set(g[3], G.nx - 1 - x0, C::load1(in, 3, row, 0));  // periodic wrap at x = nx-1
}

// Collision of one site (closed form above).  shat = S^ (zero without sources).
struct Out5 {
    float o0, o1, o2, o3, o4;
};
__device__ __forceinline__ Out5 collide2d(float g0, float g1, float g2, float g3, float g4, float cl, float shat) {
    const float s = ((g0 + g1) + (g2 + g3)) + g4;
    const float L = cl * s;
    const float w0 = 1.f - 2.f * cl;
    const float Tm = -0.5f * cl * shat;
    const float T0 = -w0 * shat;
    Out5 o;
    o.o1 = (L - g3) + Tm;
    o.o3 = (L - g1) + Tm;
    o.o2 = (L - g4) + Tm;
    o.o4 = (L - g2) + Tm;
    o.o0 = (2.f * w0 * s - g0) + T0;
    return o;
}

__device__ __forceinline__ float field2d(int comp, float cl, float s, float bx, float by) {
    switch (comp) {
        case 2: return -cl * s;  // E_z = -Lambda_xy
        case 3: return bx;
        case 4: return by;
        default: return 0.f;  // E_x, E_y, B_z are not representable in 2D
    }
}

template <int ST, bool MU, int R>
__global__ void __launch_bounds__(BLOCK) step2d(StepArgs a) {
    using C = Codec<ST>;
    const Grid &G = a.g;
    const int lane = threadIdx.x & 31;
    const long long wg = ((long long)blockIdx.x * BLOCK + threadIdx.x) >> 5;
    const int wpr = G.nchunk_pad >> 5;
    const int rg = (int)(wg / wpr);
    const int c = (int)(wg - (long long)rg * wpr) * 32 + lane;
    const int row0 = rg * R;
    if (row0 >= G.ny) return;  // warp-uniform
    const bool active = c < G.nchunk;

    float4 g[R][5];
    float4 cl[R];
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int row = min(row0 + r, G.ny - 1);
        pull2d<ST>(a.in, G, row, c, lane, g[r]);
        cl[r] = active ? __ldg(reinterpret_cast<const float4 *>(a.med.cL2 + (long long)row * G.pitch) + c)
                       : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int row = row0 + r;
        if (row >= G.ny) break;  // warp-uniform
        float4 shat = make_float4(0.f, 0.f, 0.f, 0.f);
        if (MU && active) {
            const float4 dx = __ldg(reinterpret_cast<const float4 *>(a.med.dlnmu + (long long)row * G.pitch) + c);
            const float4 dy =
                __ldg(reinterpret_cast<const float4 *>(a.med.dlnmu + G.plane + (long long)row * G.pitch) + c);
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const float bx = get(g[r][4], j) - get(g[r][2], j), by = get(g[r][1], j) - get(g[r][3], j);
                set(shat, j, bx * get(dy, j) - by * get(dx, j));
            }
        }
        if (a.evt.rowptr) {
            const int e0 = __ldg(a.evt.rowptr + row), e1 = __ldg(a.evt.rowptr + row + 1);
            for (int e = e0; e < e1; e++) {
                const Event ev = a.evt.ev[e];
                if ((ev.x >> 2) != c || !active) continue;
                const int j = ev.x & 3;
                if (ev.kind == 0) {
                    if (ev.comp == 2 && a.t < a.evt.nt) {
                        float jz = __ldg(a.evt.amp + (long long)ev.index * a.evt.nt + a.t);
                        if (MU) jz *= __ldg(a.med.mu + (long long)row * G.pitch + ev.x);
                        set(shat, j, get(shat, j) - jz);
                    }
                } else if (a.t < a.evt.cap) {
                    const float gj[5] = {get(g[r][0], j), get(g[r][1], j), get(g[r][2], j), get(g[r][3], j),
                                         get(g[r][4], j)};
                    const float s = ((gj[0] + gj[1]) + (gj[2] + gj[3])) + gj[4];
                    a.evt.traces[(long long)ev.index * a.evt.cap + a.t] =
                        field2d(ev.comp, get(cl[r], j), s, gj[4] - gj[2], gj[1] - gj[3]);
                }
            }
        }
        float4 o0, o1, o2, o3, o4;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            Out5 o = collide2d(get(g[r][0], j), get(g[r][1], j), get(g[r][2], j), get(g[r][3], j), get(g[r][4], j),
                               get(cl[r], j), get(shat, j));
            set(o0, j, o.o0);
            set(o1, j, o.o1);
            set(o2, j, o.o2);
            set(o3, j, o.o3);
            set(o4, j, o.o4);
        }
        if (active) {
            C::store4(a.out, 0, row, c, o0);
            C::store4(a.out, 1, row, c, o1);
            C::store4(a.out, 2, row, c, o2);
            C::store4(a.out, 3, row, c, o3);
            C::store4(a.out, 4, row, c, o4);
        }
    }
}

// ------------------------------------------------------------------ launchers
static const int kRows2d[] = {1, 2, 4};
int nvariants_2d() { return 3; }

template <int ST, bool MU>
static cudaError_t launch_st(const StepArgs &a, int variant, cudaStream_t s) {
    const int R = kRows2d[variant];
    const long long warps = (long long)((a.g.ny + R - 1) / R) * (a.g.nchunk_pad / 32);
    const long long blocks = (warps * 32 + BLOCK - 1) / BLOCK;
    switch (R) {
        case 1: step2d<ST, MU, 1><<<(unsigned)blocks, BLOCK, 0, s>>>(a); break;
        case 2: step2d<ST, MU, 2><<<(unsigned)blocks, BLOCK, 0, s>>>(a); break;
        default: step2d<ST, MU, 4><<<(unsigned)blocks, BLOCK, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_step_2d(const StepArgs &a, int storage, bool has_mu, int variant, cudaStream_t s) {
    if (variant < 0 || variant >= nvariants_2d()) variant = 0;
#define LBEM_CASE(ST)                                                                               \
    case ST: return has_mu ? launch_st<ST, true>(a, variant, s) : launch_st<ST, false>(a, variant, s);
    switch (storage) {
        LBEM_CASE(LBEM_F32)
        LBEM_CASE(LBEM_F16)
        LBEM_CASE(LBEM_BF16)
        LBEM_CASE(LBEM_I16B)
        default: return cudaErrorInvalidValue;
    }
#undef LBEM_CASE
}

// ------------------------------------------------------------------ initial state: buf_i(x) = g^(0)_i(x + c_i)
template <int ST>
__global__ void __launch_bounds__(BLOCK) init2d(Grid G, PopBuf out, const float *cL2, const float *E, const float *B,
                                                long long nsite) {
    using C = Codec<ST>;
    const long long tid = (long long)blockIdx.x * BLOCK + threadIdx.x;
    const int row = (int)(tid / G.nchunk_pad);
    const int c = (int)(tid - (long long)row * G.nchunk_pad);
    if (row >= G.ny || c >= G.nchunk) return;
    const int cx[5] = {0, 1, 0, -1, 0}, cy[5] = {0, 0, 1, 0, -1};
    for (int i = 0; i < 5; i++) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int j = 0; j < 4; j++) {
            const int x = 4 * c + j;
            if (x >= G.nx) break;
            const int xs = (x + cx[i] + G.nx) % G.nx, ys = (row + cy[i] + G.ny) % G.ny;
            const long long sd = (long long)ys * G.nx + xs;
            const float cl = cL2[(long long)ys * G.pitch + xs];
            const float Lam = E ? -E[2 * nsite + sd] : 0.f;
            const float bx = B ? B[sd] : 0.f, by = B ? B[nsite + sd] : 0.f;
            // Eq. 8: g^(0)_i = (w_i / c_L^2) [Lambda + c_ix B_y - c_iy B_x]
            const float wc = (i == 0) ? (1.f - 2.f * cl) / cl : 0.5f;
            set(v, j, wc * (Lam + cx[i] * by - cy[i] * bx));
        }
        C::store4(out, i, row, c, v);
    }
}

cudaError_t launch_init_2d(const lbem_t *h, const float *E, const float *B, cudaStream_t s) {
    const Grid &G = h->grid;
    const long long n = (long long)G.ny * G.nchunk_pad;
    const unsigned blocks = (unsigned)((n + BLOCK - 1) / BLOCK);
    const PopBuf &o = h->buf[h->cur];
    switch (h->storage) {
        case LBEM_F32: init2d<LBEM_F32><<<blocks, BLOCK, 0, s>>>(G, o, h->cL2, E, B, h->nsite); break;
        case LBEM_F16: init2d<LBEM_F16><<<blocks, BLOCK, 0, s>>>(G, o, h->cL2, E, B, h->nsite); break;
        case LBEM_BF16: init2d<LBEM_BF16><<<blocks, BLOCK, 0, s>>>(G, o, h->cL2, E, B, h->nsite); break;
        default: init2d<LBEM_I16B><<<blocks, BLOCK, 0, s>>>(G, o, h->cL2, E, B, h->nsite); break;
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------ field extraction (dense [3][nsite] outputs)
template <int ST>
__global__ void __launch_bounds__(BLOCK) fields2d(Grid G, PopBuf in, const float *cL2, float *E, float *B,
                                                  long long nsite) {
    const int lane = threadIdx.x & 31;
    const long long wg = ((long long)blockIdx.x * BLOCK + threadIdx.x) >> 5;
    const int wpr = G.nchunk_pad >> 5;
    const int row = (int)(wg / wpr);
    const int c = (int)(wg - (long long)row * wpr) * 32 + lane;
    if (row >= G.ny) return;
    float4 g[5];
    pull2d<ST>(in, G, row, c, lane, g);
    if (c >= G.nchunk) return;
    const float4 cl = __ldg(reinterpret_cast<const float4 *>(cL2 + (long long)row * G.pitch) + c);
    for (int j = 0; j < 4; j++) {
        const int x = 4 * c + j;
        if (x >= G.nx) break;
        const long long sd = (long long)row * G.nx + x;
        const float s = ((get(g[0], j) + get(g[1], j)) + (get(g[2], j) + get(g[3], j))) + get(g[4], j);
        if (E) {
            E[sd] = 0.f;
            E[nsite + sd] = 0.f;
            E[2 * nsite + sd] = -get(cl, j) * s;
        }
        if (B) {
            B[sd] = get(g[4], j) - get(g[2], j);
            B[nsite + sd] = get(g[1], j) - get(g[3], j);
            B[2 * nsite + sd] = 0.f;
        }
    }
}

cudaError_t launch_fields_2d(const lbem_t *h, float *E, float *B, cudaStream_t s) {
    const Grid &G = h->grid;
    const long long warps = (long long)G.ny * (G.nchunk_pad / 32);
    const unsigned blocks = (unsigned)((warps * 32 + BLOCK - 1) / BLOCK);
    const PopBuf &in = h->buf[h->cur];
    switch (h->storage) {
        case LBEM_F32: fields2d<LBEM_F32><<<blocks, BLOCK, 0, s>>>(G, in, h->cL2, E, B, h->nsite); break;
        case LBEM_F16: fields2d<LBEM_F16><<<blocks, BLOCK, 0, s>>>(G, in, h->cL2, E, B, h->nsite); break;
        case LBEM_BF16: fields2d<LBEM_BF16><<<blocks, BLOCK, 0, s>>>(G, in, h->cL2, E, B, h->nsite); break;
        default: fields2d<LBEM_I16B><<<blocks, BLOCK, 0, s>>>(G, in, h->cL2, E, B, h->nsite); break;
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------ FP64 diagnostics
template <int ST>
__device__ __forceinline__ double pop2d(const PopBuf &in, const Grid &G, int i, int x, int y) {
    // pre-collision g_i at (x, y): buf_i(x - c_i)
    const int cx[5] = {0, 1, 0, -1, 0}, cy[5] = {0, 0, 1, 0, -1};
    const int xs = (x - cx[i] + G.nx) % G.nx, ys = (y - cy[i] + G.ny) % G.ny;
    return (double)Codec<ST>::load1(in, i, ys, xs);
}

template <int ST>
__device__ __forceinline__ void bfield2d(const PopBuf &in, const Grid &G, int x, int y, double &bx, double &by) {
    bx = pop2d<ST>(in, G, 4, x, y) - pop2d<ST>(in, G, 2, x, y);
    by = pop2d<ST>(in, G, 1, x, y) - pop2d<ST>(in, G, 3, x, y);
}

__device__ __forceinline__ double block_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < BLOCK / 32; k++) r += sh[k];
    return r;  // valid in thread 0
}

template <int ST>
__global__ void __launch_bounds__(BLOCK) diag2d(Grid G, PopBuf in, const float *cL2, double *partials) {
    __shared__ double sh[BLOCK / 32];
    double en = 0.0, inv = 0.0, dv = 0.0;
    const long long nsite = (long long)G.nx * G.ny;
    for (long long s = (long long)blockIdx.x * BLOCK + threadIdx.x; s < nsite; s += (long long)gridDim.x * BLOCK) {
        const int y = (int)(s / G.nx), x = (int)(s - (long long)y * G.nx);
        double g[5], sum = 0.0;
        for (int i = 0; i < 5; i++) {
            g[i] = pop2d<ST>(in, G, i, x, y);
            sum += g[i];
        }
        const double cl = (double)cL2[(long long)y * G.pitch + x];
        const double Ez = -cl * sum, bx = g[4] - g[2], by = g[1] - g[3];
        en += bx * bx + by * by + Ez * Ez / cl;  // c_eff^2 = c_L^2 in 2D
        const double w0 = 1.0 - 2.0 * cl, wm = 0.5 * cl;
        double q = (g[1] * g[1] + g[2] * g[2] + g[3] * g[3] + g[4] * g[4]) / wm;
        if (w0 != 0.0) q += g[0] * g[0] / w0;
        inv += 2.0 * q;  // g_xy and g_yx = -g_xy both count
        double bxp, byp, bxm, bym, t1, t2;
        bfield2d<ST>(in, G, (x + 1) % G.nx, y, bxp, t1);
        bfield2d<ST>(in, G, (x - 1 + G.nx) % G.nx, y, bxm, t2);
        bfield2d<ST>(in, G, x, (y + 1) % G.ny, t1, byp);
        bfield2d<ST>(in, G, x, (y - 1 + G.ny) % G.ny, t2, bym);
        const double div = 0.5 * (bxp - bxm) + 0.5 * (byp - bym);
        dv += div * div;
    }
    const double a = block_sum(en, sh), b = block_sum(inv, sh), c = block_sum(dv, sh);
    if (threadIdx.x == 0) {
        partials[3 * blockIdx.x + 0] = a;
        partials[3 * blockIdx.x + 1] = b;
        partials[3 * blockIdx.x + 2] = c;
    }
}

cudaError_t launch_diag_2d(const lbem_t *h, double *partials, int nblocks, cudaStream_t s) {
    const PopBuf &in = h->buf[h->cur];
    switch (h->storage) {
        case LBEM_F32: diag2d<LBEM_F32><<<nblocks, BLOCK, 0, s>>>(h->grid, in, h->cL2, partials); break;
        case LBEM_F16: diag2d<LBEM_F16><<<nblocks, BLOCK, 0, s>>>(h->grid, in, h->cL2, partials); break;
        case LBEM_BF16: diag2d<LBEM_BF16><<<nblocks, BLOCK, 0, s>>>(h->grid, in, h->cL2, partials); break;
        default: diag2d<LBEM_I16B><<<nblocks, BLOCK, 0, s>>>(h->grid, in, h->cL2, partials); break;
    }
    return cudaGetLastError();
}

}  // namespace lbk
