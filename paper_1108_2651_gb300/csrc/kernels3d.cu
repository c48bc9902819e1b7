// 3D (D3Q7) kernels of the lattice-Boltzmann Maxwell scheme of Hanasoge,
// Succi & Orszag (arXiv:1108.2651).
//
// The antisymmetric tensor g_{i,ab} is stored as its pseudo-vector
// h_{i,gamma} (g_{i,ab} = eps_{gamma a b} h_{i,gamma}): plane p = 3 i + gamma,
// i = 0..6 with c_1..c_3 = +x,+y,+z and c_4..c_6 = -x,-y,-z.  In this form
// (with lambda_gamma = -E_gamma, sigma_gamma = sum_i h_{i,gamma}):
//   Eq. 9 :  lambda = c_L^2 sigma                    => E = -c_L^2 sigma
//   Eq. 10:  R_{gamma kappa} = sum_i c_{i kappa} h_{i gamma};  the magnetic
//            field is read as B_nu = eps_{gamma kappa nu} R_{gamma kappa}
//            (the sum of the two tensor components that carry B_nu)
//   Eq. 8 :  h^(0)_{i gamma} = (w_i / c_L^2) [lambda_gamma + (c_i x B/2)_gamma]
//            (equilibrium built with B/(D-1) = B/2, the stable reading; the
//            waves then travel at c_eff^2 = c_L^2/2)
//   Eq. 17 at tau = dt/2 with w_i/c_L^2 = 1/2 for moving particles:
//            h'_{i gamma} = lambda_gamma + (c_i x B)_gamma/2 - h_{i gamma} + T_m
//            h'_{0 gamma} = 2 w0 sigma_gamma - h_{0 gamma} + T_0,  w0 = 1 - 3 c_L^2
//   Eq. 3 :  S = c_eff^2 (B x grad ln mu - mu j) = (c_L^2/2) S^,
//            T_{i gamma} = -(w_i/c_L^2) S_gamma:  T_m = -(c_L^2/4) S^, T_0 = -(w0/2) S^.
#include "lbem_internal.cuh"

namespace lbk {

struct Rows3 {
    int r0, ym, zm, yp, zp;  // own row and the rows pulled from (y-1, z-1, y+1, z+1)
};

__device__ __forceinline__ Rows3 rows3(const Grid &G, int row) {
    const int z = row / G.ny, y = row - z * G.ny;
    Rows3 r;
    r.r0 = row;
    r.ym = z * G.ny + (y == 0 ? G.ny - 1 : y - 1);
    r.yp = z * G.ny + (y == G.ny - 1 ? 0 : y + 1);
    r.zm = (z == 0 ? G.nz - 1 : z - 1) * G.ny + y;
    r.zp = (z == G.nz - 1 ? 0 : z + 1) * G.ny + y;
    return r;
}

// Pre-collision h_{i gamma} of the 4 sites (row, 4c..4c+3); all 32 lanes must call.
__device__ __forceinline__ void pull3d(const PopBuf &in, const Grid &G, int row, int c, int lane, float4 v[21]) {
    using C = Codec<LBEM_F32>;
    const Rows3 R = rows3(G, row);
    const int x0 = 4 * c;
    const bool active = c < G.nchunk;  // lanes past the row end load nothing
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int gm = 0; gm < 3; gm++) {
        v[0 + gm] = active ? C::load4(in, 0 + gm, R.r0, c) : z4;
        float4 a1 = active ? C::load4(in, 3 + gm, R.r0, c) : z4;
        v[6 + gm] = active ? C::load4(in, 6 + gm, R.ym, c) : z4;
        v[9 + gm] = active ? C::load4(in, 9 + gm, R.zm, c) : z4;
        float4 a4 = active ? C::load4(in, 12 + gm, R.r0, c) : z4;
        v[15 + gm] = active ? C::load4(in, 15 + gm, R.yp, c) : z4;
        v[18 + gm] = active ? C::load4(in, 18 + gm, R.zp, c) : z4;
        float prev = __shfl_up_sync(FULL, a1.w, 1);
        float next = __shfl_down_sync(FULL, a4.x, 1);
        if (lane == 0 && active) prev = C::load1(in, 3 + gm, R.r0, c == 0 ? G.nx - 1 : x0 - 1);
        if (lane == 31 && x0 + 4 < G.nx) next = C::load1(in, 12 + gm, R.r0, x0 + 4);
        v[3 + gm] = make_float4(prev, a1.x, a1.y, a1.z);
        v[12 + gm] = make_float4(a4.y, a4.z, a4.w, next);
        if (c == G.nchunk - 1) set(v[12 + gm], G.nx - 1 - x0, C::load1(in, 12 + gm, R.r0, 0));
    }
}

struct Mom3 {
    float sx, sy, sz, bx, by, bz;
};

__device__ __forceinline__ Mom3 moments3(const float h[21]) {
    Mom3 m;
    m.sx = ((h[0] + h[3]) + (h[6] + h[9])) + ((h[12] + h[15]) + h[18]);
    m.sy = ((h[1] + h[4]) + (h[7] + h[10])) + ((h[13] + h[16]) + h[19]);
    m.sz = ((h[2] + h[5]) + (h[8] + h[11])) + ((h[14] + h[17]) + h[20]);
    // R_{gamma kappa} = h[(1+kappa)*3 + gamma] - h[(4+kappa)*3 + gamma]
    m.bx = (h[10] - h[19]) - (h[8] - h[17]);   // R_yz - R_zy
    m.by = (h[5] - h[14]) - (h[9] - h[18]);    // R_zx - R_xz
    m.bz = (h[6] - h[15]) - (h[4] - h[13]);    // R_xy - R_yx
    return m;
}

__device__ __forceinline__ float field3d(int comp, float cl, const Mom3 &m) {
    switch (comp) {
        case 0: return -cl * m.sx;
        case 1: return -cl * m.sy;
        case 2: return -cl * m.sz;
        case 3: return m.bx;
        case 4: return m.by;
        default: return m.bz;
    }
}

// In-place collision of one site: h[p] <- h'[p].
__device__ __forceinline__ void collide3d(float h[21], float cl, float shx, float shy, float shz) {
    const Mom3 m = moments3(h);
    const float w0 = 1.f - 3.f * cl;
    const float lx = cl * m.sx, ly = cl * m.sy, lz = cl * m.sz;
    const float tmx = -0.25f * cl * shx, tmy = -0.25f * cl * shy, tmz = -0.25f * cl * shz;
    const float hbx = 0.5f * m.bx, hby = 0.5f * m.by, hbz = 0.5f * m.bz;
    // rest
    h[0] = (2.f * w0 * m.sx - h[0]) - 0.5f * w0 * shx;
    h[1] = (2.f * w0 * m.sy - h[1]) - 0.5f * w0 * shy;
    h[2] = (2.f * w0 * m.sz - h[2]) - 0.5f * w0 * shz;
    // +x: c x B = (0, -Bz, By)
    h[3] = (lx - h[3]) + tmx;
    h[4] = ((ly - hbz) - h[4]) + tmy;
    h[5] = ((lz + hby) - h[5]) + tmz;
    // +y: c x B = (Bz, 0, -Bx)
    h[6] = ((lx + hbz) - h[6]) + tmx;
    h[7] = (ly - h[7]) + tmy;
    h[8] = ((lz - hbx) - h[8]) + tmz;
    // +z: c x B = (-By, Bx, 0)
    h[9] = ((lx - hby) - h[9]) + tmx;
    h[10] = ((ly + hbx) - h[10]) + tmy;
    h[11] = (lz - h[11]) + tmz;
    // -x
    h[12] = (lx - h[12]) + tmx;
    h[13] = ((ly + hbz) - h[13]) + tmy;
    h[14] = ((lz - hby) - h[14]) + tmz;
    // -y
    h[15] = ((lx - hbz) - h[15]) + tmx;
    h[16] = (ly - h[16]) + tmy;
    h[17] = ((lz + hbx) - h[17]) + tmz;
    // -z
    h[18] = ((lx + hby) - h[18]) + tmx;
    h[19] = ((ly - hbx) - h[19]) + tmy;
    h[20] = (lz - h[20]) + tmz;
}

template <bool MU>
__global__ void __launch_bounds__(BLOCK) step3d(StepArgs a) {
    using C = Codec<LBEM_F32>;
    const Grid &G = a.g;
    const int lane = threadIdx.x & 31;
    const long long wg = ((long long)blockIdx.x * BLOCK + threadIdx.x) >> 5;
    const int wpr = G.nchunk_pad >> 5;
    const int row = (int)(wg / wpr);
    const int c = (int)(wg - (long long)row * wpr) * 32 + lane;
    if (row >= G.nrows) return;  // warp-uniform
    const bool active = c < G.nchunk;
    float4 v[21];
    pull3d(a.in, G, row, c, lane, v);
    const float4 cl = active ? __ldg(reinterpret_cast<const float4 *>(a.med.cL2 + (long long)row * G.pitch) + c)
                             : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 shx = make_float4(0.f, 0.f, 0.f, 0.f), shy = shx, shz = shx;
    if (MU && active) {
        const float4 dx = __ldg(reinterpret_cast<const float4 *>(a.med.dlnmu + (long long)row * G.pitch) + c);
        const float4 dy = __ldg(reinterpret_cast<const float4 *>(a.med.dlnmu + G.plane + (long long)row * G.pitch) + c);
        const float4 dz =
            __ldg(reinterpret_cast<const float4 *>(a.med.dlnmu + 2 * G.plane + (long long)row * G.pitch) + c);
#pragma unroll
        for (int j = 0; j < 4; j++) {
            float h[21];
#pragma unroll
            for (int p = 0; p < 21; p++) h[p] = get(v[p], j);
            const Mom3 m = moments3(h);
            set(shx, j, m.by * get(dz, j) - m.bz * get(dy, j));
            set(shy, j, m.bz * get(dx, j) - m.bx * get(dz, j));
            set(shz, j, m.bx * get(dy, j) - m.by * get(dx, j));
        }
    }
    if (a.evt.rowptr) {
        const int e0 = __ldg(a.evt.rowptr + row), e1 = __ldg(a.evt.rowptr + row + 1);
        for (int e = e0; e < e1; e++) {
            const Event ev = a.evt.ev[e];
            if ((ev.x >> 2) != c || !active) continue;
            const int j = ev.x & 3;
            if (ev.kind == 0) {
                if (a.t < a.evt.nt) {
                    float jj = __ldg(a.evt.amp + (long long)ev.index * a.evt.nt + a.t);
                    if (MU) jj *= __ldg(a.med.mu + (long long)row * G.pitch + ev.x);
                    if (ev.comp == 0) set(shx, j, get(shx, j) - jj);
                    else if (ev.comp == 1) set(shy, j, get(shy, j) - jj);
                    else set(shz, j, get(shz, j) - jj);
                }
            } else if (a.t < a.evt.cap) {
                float h[21];
#pragma unroll
                for (int p = 0; p < 21; p++) h[p] = get(v[p], j);
                a.evt.traces[(long long)ev.index * a.evt.cap + a.t] = field3d(ev.comp, get(cl, j), moments3(h));
            }
        }
    }
#pragma unroll
    for (int j = 0; j < 4; j++) {
        float h[21];
#pragma unroll
        for (int p = 0; p < 21; p++) h[p] = get(v[p], j);
        collide3d(h, get(cl, j), get(shx, j), get(shy, j), get(shz, j));
#pragma unroll
        for (int p = 0; p < 21; p++) set(v[p], j, h[p]);
    }
    if (active) {
#pragma unroll
        for (int p = 0; p < 21; p++) C::store4(a.out, p, row, c, v[p]);
    }
}

// Walls (walls.cu, in 3D): a population h_{i gamma} pulled across a wall normal to axis a is the site's own
// h_{opp(i) gamma} times wall_sign3(kind, gamma, a): the geometric mirror of the tensor component it carries
// (+1 when gamma == a, -1 otherwise) times +1 for PEC and -1 for PMC.
__device__ __forceinline__ float wall_sign3(int kind, int gm, int ax) {
    return (kind == 1 ? 1.f : -1.f) * (gm == ax ? 1.f : -1.f);
}

// One site per thread: a warp covers 32 consecutive sites of a row; the +-x
// pulls are plain (unaligned, coalesced) loads whose overlap L1/L2 absorbs.
// Far fewer registers than the 4-sites-per-lane kernel, so more warps per SM.
// With WL, pulls across walls follow wall_sign3 and the absorbing layer's
// factor fx(x) fy(y) fz(z) scales the result.
template <bool MU, bool WL = false>
__global__ void __launch_bounds__(BLOCK, WL ? 5 : 1) step3d_site(StepArgs a, Walls w) {
    const Grid &G = a.g;
    const int tpr = G.pitch;  // threads per row (pitch is a multiple of 32)
    const long long tid = (long long)blockIdx.x * BLOCK + threadIdx.x;
    const int row = (int)(tid / tpr);
    const int x = (int)(tid - (long long)row * tpr);
    if (row >= G.nrows || x >= G.nx) return;
    const Rows3 R = rows3(G, row);
    const int xm = x == 0 ? G.nx - 1 : x - 1, xp = x == G.nx - 1 ? 0 : x + 1;
    const float *in = static_cast<const float *>(a.in.data);
    auto ld = [&](int p, int r, int xx) { return __ldg(in + p * G.plane + (long long)r * G.pitch + xx); };
    float h[21];
#pragma unroll
    for (int gm = 0; gm < 3; gm++) {
        h[0 + gm] = ld(0 + gm, R.r0, x);
        h[3 + gm] = ld(3 + gm, R.r0, xm);
        h[6 + gm] = ld(6 + gm, R.ym, x);
        h[9 + gm] = ld(9 + gm, R.zm, x);
        h[12 + gm] = ld(12 + gm, R.r0, xp);
        h[15 + gm] = ld(15 + gm, R.yp, x);
        h[18 + gm] = ld(18 + gm, R.zp, x);
    }
    int y = 0, z = 0;
    if (WL) {
        z = row / G.ny;
        y = row - z * G.ny;
        const int pos[3] = {x, y, z}, len[3] = {G.nx, G.ny, G.nz};
#pragma unroll
        for (int ax = 0; ax < 3; ax++) {
            if (!w.kind[ax]) continue;
            // +ax movers (direction 1 + ax) pulled from pos - 1, -ax movers (4 + ax) from pos + 1
            if (pos[ax] == 0)
#pragma unroll
                for (int gm = 0; gm < 3; gm++) h[3 * (1 + ax) + gm] = wall_sign3(w.kind[ax], gm, ax) * ld(3 * (4 + ax) + gm, R.r0, x);
            if (pos[ax] == len[ax] - 1)
#pragma unroll
                for (int gm = 0; gm < 3; gm++) h[3 * (4 + ax) + gm] = wall_sign3(w.kind[ax], gm, ax) * ld(3 * (1 + ax) + gm, R.r0, x);
        }
    }
    const long long o = (long long)row * G.pitch + x;
    const float cl = __ldg(a.med.cL2 + o);
    float shx = 0.f, shy = 0.f, shz = 0.f;
    if (MU) {
        const float dx = __ldg(a.med.dlnmu + o), dy = __ldg(a.med.dlnmu + G.plane + o),
                    dz = __ldg(a.med.dlnmu + 2 * G.plane + o);
        const Mom3 m = moments3(h);
        shx = m.by * dz - m.bz * dy;
        shy = m.bz * dx - m.bx * dz;
        shz = m.bx * dy - m.by * dx;
    }
    if (a.evt.rowptr) {
        const int e0 = __ldg(a.evt.rowptr + row), e1 = __ldg(a.evt.rowptr + row + 1);
        for (int e = e0; e < e1; e++) {
            const Event ev = a.evt.ev[e];
            if (ev.x != x) continue;
            if (ev.kind == 0) {
                if (a.t < a.evt.nt) {
                    float jj = __ldg(a.evt.amp + (long long)ev.index * a.evt.nt + a.t);
                    if (MU) jj *= __ldg(a.med.mu + o);
                    if (ev.comp == 0) shx -= jj;
                    else if (ev.comp == 1) shy -= jj;
                    else shz -= jj;
                }
            } else if (a.t < a.evt.cap) {
                a.evt.traces[(long long)ev.index * a.evt.cap + a.t] = field3d(ev.comp, cl, moments3(h));
            }
        }
    }
    collide3d(h, cl, shx, shy, shz);
    float *out = static_cast<float *>(a.out.data);
    if (WL && (w.fx || w.fy || w.fz)) {
        const float f = __fmul_rn(__fmul_rn(w.fx ? w.fx[x] : 1.f, w.fy ? w.fy[y] : 1.f), w.fz ? w.fz[z] : 1.f);
#pragma unroll
        for (int p = 0; p < 21; p++) h[p] = __fmul_rn(h[p], f);
    }
#pragma unroll
    for (int p = 0; p < 21; p++) __stcs(out + p * G.plane + o, h[p]);
}

// 0 = four sites per lane; 1 = one site per thread; 2 = as 1 (forward), with the adjoint kernel's
// registers capped for 5 resident blocks per SM
int nvariants_3d() { return 3; }

cudaError_t launch_step_3d(const StepArgs &a, bool has_mu, int variant, cudaStream_t s, const Walls *w) {
    const bool walls = w && (w->kind[0] || w->kind[1] || w->kind[2]);
    if (variant >= 1 || walls) {  // walls: the one-site-per-thread kernel, which applies them
        const long long threads = (long long)a.g.nrows * a.g.pitch;
        const unsigned blocks = (unsigned)((threads + BLOCK - 1) / BLOCK);
        const Walls wv = walls ? *w : Walls();
        if (walls) {
            if (has_mu) step3d_site<true, true><<<blocks, BLOCK, 0, s>>>(a, wv);
            else step3d_site<false, true><<<blocks, BLOCK, 0, s>>>(a, wv);
        } else {
            if (has_mu) step3d_site<true><<<blocks, BLOCK, 0, s>>>(a, wv);
            else step3d_site<false><<<blocks, BLOCK, 0, s>>>(a, wv);
        }
        return cudaGetLastError();
    }
    const long long warps = (long long)a.g.nrows * (a.g.nchunk_pad / 32);
    const unsigned blocks = (unsigned)((warps * 32 + BLOCK - 1) / BLOCK);
    if (has_mu) step3d<true><<<blocks, BLOCK, 0, s>>>(a);
    else step3d<false><<<blocks, BLOCK, 0, s>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ initial state: buf_{i gamma}(x) = h^(0)_{i gamma}(x + c_i)
// (with walls, where x + c_i lies beyond a wall normal to axis a, buf_{i gamma}(x) is what site x pulls back:
// wall_sign3 times h^(0)_{opp(i) gamma}(x))
__global__ void __launch_bounds__(BLOCK) init3d(Grid G, PopBuf out, const float *cL2, const float *E, const float *B,
                                                long long nsite, Walls w) {
    const long long tid = (long long)blockIdx.x * BLOCK + threadIdx.x;
    const int row = (int)(tid / G.nchunk_pad);
    const int c = (int)(tid - (long long)row * G.nchunk_pad);
    if (row >= G.nrows || c >= G.nchunk) return;
    const int z = row / G.ny, y = row - z * G.ny;
    const int cc[7][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {-1, 0, 0}, {0, -1, 0}, {0, 0, -1}};
    for (int i = 0; i < 7; i++) {
        float4 v[3] = {make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f),
                       make_float4(0.f, 0.f, 0.f, 0.f)};
        for (int j = 0; j < 4; j++) {
            const int x = 4 * c + j;
            if (x >= G.nx) break;
            int xs = x + cc[i][0], ys = y + cc[i][1], zs = z + cc[i][2], ie = i, wax = -1;
            const int pos[3] = {xs, ys, zs}, len[3] = {G.nx, G.ny, G.nz};
            for (int ax = 0; ax < 3; ax++)
                if (w.kind[ax] && (pos[ax] < 0 || pos[ax] >= len[ax])) wax = ax;
            if (wax >= 0) {  // beyond a wall: the site's own opposite population
                xs = x;
                ys = y;
                zs = z;
                ie = i == 0 ? 0 : (i <= 3 ? i + 3 : i - 3);
            }
            xs = (xs + G.nx) % G.nx;
            ys = (ys + G.ny) % G.ny;
            zs = (zs + G.nz) % G.nz;
            const long long sd = ((long long)zs * G.ny + ys) * G.nx + xs;
            const float cl = cL2[((long long)zs * G.ny + ys) * G.pitch + xs];
            float e[3], b[3];
            for (int k = 0; k < 3; k++) {
                e[k] = E ? E[k * nsite + sd] : 0.f;
                b[k] = B ? 0.5f * B[k * nsite + sd] : 0.f;  // equilibrium uses B/(D-1)
            }
            const float cxb[3] = {cc[ie][1] * b[2] - cc[ie][2] * b[1], cc[ie][2] * b[0] - cc[ie][0] * b[2],
                                  cc[ie][0] * b[1] - cc[ie][1] * b[0]};
            const float wc = (ie == 0) ? (1.f - 3.f * cl) / cl : 0.5f;
            for (int k = 0; k < 3; k++) {
                const float sg = wax >= 0 ? wall_sign3(w.kind[wax], k, wax) : 1.f;
                set(v[k], j, sg * (wc * (-e[k] + cxb[k])));
            }
        }
        for (int k = 0; k < 3; k++) Codec<LBEM_F32>::store4(out, 3 * i + k, row, c, v[k]);
    }
}

static Walls walls_of(const lbem_t *h) {
    Walls w;
    for (int a = 0; a < 3; a++) w.kind[a] = h->bc[a];
    return w;
}

cudaError_t launch_init_3d(const lbem_t *h, const float *E, const float *B, cudaStream_t s) {
    const Grid &G = h->grid;
    const long long n = (long long)G.nrows * G.nchunk_pad;
    init3d<<<(unsigned)((n + BLOCK - 1) / BLOCK), BLOCK, 0, s>>>(G, h->buf[h->cur], h->cL2, E, B, h->nsite,
                                                                 walls_of(h));
    return cudaGetLastError();
}

// ------------------------------------------------------------------ field extraction
__global__ void __launch_bounds__(BLOCK) fields3d(Grid G, PopBuf in, const float *cL2, float *E, float *B,
                                                  long long nsite, Walls w) {
    const int lane = threadIdx.x & 31;
    const long long wg = ((long long)blockIdx.x * BLOCK + threadIdx.x) >> 5;
    const int wpr = G.nchunk_pad >> 5;
    const int row = (int)(wg / wpr);
    const int c = (int)(wg - (long long)row * wpr) * 32 + lane;
    if (row >= G.nrows) return;
    float4 v[21];
    pull3d(in, G, row, c, lane, v);
    if (c >= G.nchunk) return;
    const float4 cl = __ldg(reinterpret_cast<const float4 *>(cL2 + (long long)row * G.pitch) + c);
    for (int j = 0; j < 4; j++) {
        const int x = 4 * c + j;
        if (x >= G.nx) break;
        float h[21];
        for (int p = 0; p < 21; p++) h[p] = get(v[p], j);
        {  // pulls across walls
            const int z = row / G.ny, y = row - z * G.ny;
            const int pos[3] = {x, y, z}, len[3] = {G.nx, G.ny, G.nz};
            for (int ax = 0; ax < 3; ax++) {
                if (!w.kind[ax]) continue;
                for (int gm = 0; gm < 3; gm++) {
                    if (pos[ax] == 0)
                        h[3 * (1 + ax) + gm] = wall_sign3(w.kind[ax], gm, ax) *
                                               Codec<LBEM_F32>::load1(in, 3 * (4 + ax) + gm, row, x);
                    if (pos[ax] == len[ax] - 1)
                        h[3 * (4 + ax) + gm] = wall_sign3(w.kind[ax], gm, ax) *
                                               Codec<LBEM_F32>::load1(in, 3 * (1 + ax) + gm, row, x);
                }
            }
        }
        const Mom3 m = moments3(h);
        const long long sd = (long long)row * G.nx + x;
        const float q = get(cl, j);
        if (E) {
            E[sd] = -q * m.sx;
            E[nsite + sd] = -q * m.sy;
            E[2 * nsite + sd] = -q * m.sz;
        }
        if (B) {
            B[sd] = m.bx;
            B[nsite + sd] = m.by;
            B[2 * nsite + sd] = m.bz;
        }
    }
}

cudaError_t launch_fields_3d(const lbem_t *h, float *E, float *B, cudaStream_t s) {
    const Grid &G = h->grid;
    const long long warps = (long long)G.nrows * (G.nchunk_pad / 32);
    fields3d<<<(unsigned)((warps * 32 + BLOCK - 1) / BLOCK), BLOCK, 0, s>>>(G, h->buf[h->cur], h->cL2, E, B, h->nsite,
                                                                          walls_of(h));
    return cudaGetLastError();
}

// ------------------------------------------------------------------ FP64 diagnostics
__device__ __forceinline__ double pop3d(const PopBuf &in, const Grid &G, const Walls &w, int p, int x, int y, int z) {
    const int i = p / 3, gm = p - 3 * i;
    const int cc[7][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {-1, 0, 0}, {0, -1, 0}, {0, 0, -1}};
    const int u[3] = {x - cc[i][0], y - cc[i][1], z - cc[i][2]}, len[3] = {G.nx, G.ny, G.nz};
    for (int ax = 0; ax < 3; ax++)  // across a wall: the site's own opposite population, signed
        if (w.kind[ax] && (u[ax] < 0 || u[ax] >= len[ax])) {
            const int io = i <= 3 ? i + 3 : i - 3;
            return (double)wall_sign3(w.kind[ax], gm, ax) *
                   (double)Codec<LBEM_F32>::load1(in, 3 * io + gm, z * G.ny + y, x);
        }
    const int xs = (u[0] + G.nx) % G.nx, ys = (u[1] + G.ny) % G.ny, zs = (u[2] + G.nz) % G.nz;
    return (double)Codec<LBEM_F32>::load1(in, p, zs * G.ny + ys, xs);
}

__device__ __forceinline__ double bcomp3d(const PopBuf &in, const Grid &G, const Walls &w, int comp, int x, int y,
                                          int z) {
    // B_x = R_yz - R_zy, B_y = R_zx - R_xz, B_z = R_xy - R_yx; R_{g k} = h[(1+k)*3+g] - h[(4+k)*3+g]
    auto Rgk = [&](int g, int k) {
        return pop3d(in, G, w, (1 + k) * 3 + g, x, y, z) - pop3d(in, G, w, (4 + k) * 3 + g, x, y, z);
    };
    if (comp == 0) return Rgk(1, 2) - Rgk(2, 1);
    if (comp == 1) return Rgk(2, 0) - Rgk(0, 2);
    return Rgk(0, 1) - Rgk(1, 0);
}

__device__ __forceinline__ double block_sum3(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < BLOCK / 32; k++) r += sh[k];
    return r;
}

__global__ void __launch_bounds__(BLOCK) diag3d(Grid G, PopBuf in, const float *cL2, double *partials, Walls w) {
    __shared__ double sh[BLOCK / 32];
    double en = 0.0, inv = 0.0, dv = 0.0;
    const long long nsite = (long long)G.nx * G.ny * G.nz;
    for (long long s = (long long)blockIdx.x * BLOCK + threadIdx.x; s < nsite; s += (long long)gridDim.x * BLOCK) {
        const int x = (int)(s % G.nx);
        const long long rr = s / G.nx;
        const int y = (int)(rr % G.ny), z = (int)(rr / G.ny);
        double h[21], sg[3] = {0.0, 0.0, 0.0};
        for (int p = 0; p < 21; p++) {
            h[p] = pop3d(in, G, w, p, x, y, z);
            sg[p % 3] += h[p];
        }
        const double cl = (double)cL2[rr * G.pitch + x];
        const double ce2 = 0.5 * cl;
        double b[3];
        for (int k = 0; k < 3; k++) b[k] = bcomp3d(in, G, w, k, x, y, z);
        for (int k = 0; k < 3; k++) {
            const double e = -cl * sg[k];
            en += b[k] * b[k] + e * e / ce2;
        }
        const double w0 = 1.0 - 3.0 * cl, wm = 0.5 * cl;
        double q = 0.0;
        for (int p = 3; p < 21; p++) q += h[p] * h[p] / wm;
        if (w0 != 0.0)
            for (int p = 0; p < 3; p++) q += h[p] * h[p] / w0;
        inv += 2.0 * q;  // g_ab and g_ba both count
        // (periodic central differences, also next to walls)
        const double div =
            0.5 * (bcomp3d(in, G, w, 0, (x + 1) % G.nx, y, z) - bcomp3d(in, G, w, 0, (x - 1 + G.nx) % G.nx, y, z)) +
            0.5 * (bcomp3d(in, G, w, 1, x, (y + 1) % G.ny, z) - bcomp3d(in, G, w, 1, x, (y - 1 + G.ny) % G.ny, z)) +
            0.5 * (bcomp3d(in, G, w, 2, x, y, (z + 1) % G.nz) - bcomp3d(in, G, w, 2, x, y, (z - 1 + G.nz) % G.nz));
        dv += div * div;
    }
    const double a = block_sum3(en, sh), b = block_sum3(inv, sh), c = block_sum3(dv, sh);
    if (threadIdx.x == 0) {
        partials[3 * blockIdx.x + 0] = a;
        partials[3 * blockIdx.x + 1] = b;
        partials[3 * blockIdx.x + 2] = c;
    }
}

cudaError_t launch_diag_3d(const lbem_t *h, double *partials, int nblocks, cudaStream_t s) {
    diag3d<<<nblocks, BLOCK, 0, s>>>(h->grid, h->buf[h->cur], h->cL2, partials, walls_of(h));
    return cudaGetLastError();
}

}  // namespace lbk
