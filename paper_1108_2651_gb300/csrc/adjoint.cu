// Reverse-time adjoint of the stream-collide step (not in the paper): the
// gradient of a function of the receiver traces with respect to the relative
// permittivity, for FP32 storage and uniform mu.
//
// Forward map of one step (Eqs. 17-18), site by site: the post-collision
// p^t(y) = M(y) g^t(y) + T^t(y) streams to g^{t+1}_i(y + c_i) = p^t_i(y).
// With lambda^t = dL/dg^t (pre-collision) and mu^t = dL/dp^t:
//   mu^t_i(y)   = lambda^{t+1}_i(y + c_i)                  (transpose of streaming)
//   lambda^t(y) = M(y)^T mu^t(y) + d l_t / d g^t(y)        (receivers at time t)
//   dL/dc_L^2(y) += mu^t(y) . [dM/dc_L^2 g^t(y) + dT^t/dc_L^2(y)] + d l_t/dc_L^2(y)
// M = 2P - I with P the equilibrium map of Eq. 8.  Written out (tau = dt/2,
// moving weights c_L^2/2, w0 = 1 - D c_L^2, nu = sum_i w_i mu_i):
//   2D:  lambda_0 = 2 nu - mu_0,  lambda_1 = 2 nu - mu_3,  lambda_3 = 2 nu - mu_1,
//        lambda_2 = 2 nu - mu_4,  lambda_4 = 2 nu - mu_2
//   3D:  lambda_{0a} = 2 nu_a - mu_{0a},
//        lambda_{ja} = 2 nu_a + (c_j x V)_a / 2 - mu_{ja},  V = sum_i mu_i x c_i
// and, with sigma = sum_i g_i (per component) and j the point current,
//   2D:  dM g/dc_L^2 = sigma (moving), -4 sigma (rest);  dT/dc_L^2 = j/2, -2 j
//   3D:  dM g/dc_L^2 = sigma (moving), -6 sigma (rest);  dT/dc_L^2 = j/4, -3 j/2
// Receivers: E = -c_L^2 sigma gives d/dg_i = -c_L^2 and d/dc_L^2 = -sigma;
// B components are differences of populations (2D: B_x = g_4 - g_2,
// B_y = g_1 - g_3; 3D: B = sum_i g_i x c_i).  Finally
//   dL/d eps_r = dL/dc_L^2 * dc_L^2/d eps_r = -dL/dc_L^2 * c_L^2 / eps_r.
//
// Checkpointing: lbem_forward_record keeps the state every K steps; the
// backward pass recomputes one segment of at most K states at a time (kept
// in device memory) and runs the adjoint kernel backwards through it.  The
// gradient is accumulated over time steps in FP64; each step's contribution at
// a site is formed in FP32, like the rest of the arithmetic (GB300's FP64 rate
// is a small fraction of its FP32 rate, and the per-site FP64 products had made
// the adjoint step compute-bound).
#include <math.h>

#include <algorithm>
#include <vector>

#include "lbem_internal.cuh"

namespace lbk {

struct AdjointState {
    int nsteps = 0, every = 0, ncp = 0;
    long long t0 = 0;
    size_t state_floats = 0;
    float *cps = nullptr;   // [ncp][state]
    float *seg = nullptr;   // [every][state]
    float *lam = nullptr;   // [2][state]
    double *gcl = nullptr;  // [plane]
    float *cot = nullptr;   // [nrec][nsteps]
    float *gout = nullptr;  // [nsite] staging for host outputs
    double *gcl_out = nullptr;
};

void adjoint_free(lbem_t *h) {
    if (!h || !h->adj) return;
    AdjointState *a = h->adj;
    cudaFree(a->cps);
    cudaFree(a->seg);
    cudaFree(a->lam);
    cudaFree(a->gcl);
    cudaFree(a->cot);
    cudaFree(a->gout);
    cudaFree(a->gcl_out);
    delete a;
    h->adj = nullptr;
}

struct AdjArgs {
    Grid g;
    const float *lam_in;  // lambda^{t+1}, site layout [npop][plane]
    float *lam_out;       // lambda^t
    PopBuf state;         // forward buffer at time t (g^t = pull)
    const float *cL2;
    double *gcl;
    Events evt;           // sources (j) and receivers (cotangent)
    const float *cot;     // [nrec][nsteps]
    int nsteps;
    long long t, t0;
};

__device__ __forceinline__ float4 f4(const float *base, long long plane, int p, int row, int pitch, int c) {
    return __ldg(reinterpret_cast<const float4 *>(base + p * plane + (long long)row * pitch) + c);
}
__device__ __forceinline__ float f1(const float *base, long long plane, int p, int row, int pitch, int x) {
    return __ldg(base + p * plane + (long long)row * pitch + x);
}

// Element x of plane p shifted by one site: want = +1 gives v(x+1), -1 gives v(x-1),
// for the 4 sites of this lane (all 32 lanes must call).
__device__ __forceinline__ float4 xshift(const float *base, long long plane, int p, int row, const Grid &G, int c,
                                         int lane, int want, bool active) {
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 a = active ? f4(base, plane, p, row, G.pitch, c) : z4;
    const int x0 = 4 * c;
    if (want < 0) {
        float prev = __shfl_up_sync(FULL, a.w, 1);
        if (lane == 0 && active) prev = f1(base, plane, p, row, G.pitch, c == 0 ? G.nx - 1 : x0 - 1);
        return make_float4(prev, a.x, a.y, a.z);
    }
    float next = __shfl_down_sync(FULL, a.x, 1);
    if (lane == 31 && x0 + 4 < G.nx) next = f1(base, plane, p, row, G.pitch, x0 + 4);
    float4 r = make_float4(a.y, a.z, a.w, next);
    if (c == G.nchunk - 1) set(r, G.nx - 1 - x0, f1(base, plane, p, row, G.pitch, 0));
    return r;
}

// ------------------------------------------------------------------ 2D
__global__ void __launch_bounds__(BLOCK) adjoint2d(AdjArgs a) {
    const Grid &G = a.g;
    const int lane = threadIdx.x & 31;
    const long long wg = ((long long)blockIdx.x * BLOCK + threadIdx.x) >> 5;
    const int wpr = G.nchunk_pad >> 5;
    const int row = (int)(wg / wpr);
    const int c = (int)(wg - (long long)row * wpr) * 32 + lane;
    if (row >= G.ny) return;
    const bool active = c < G.nchunk;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const int ym = row == 0 ? G.ny - 1 : row - 1, yp = row == G.ny - 1 ? 0 : row + 1;
    const float *L = a.lam_in;
    // mu_i(y) = lambda_i(y + c_i)
    float4 m[5];
    m[0] = active ? f4(L, G.plane, 0, row, G.pitch, c) : z4;
    m[1] = xshift(L, G.plane, 1, row, G, c, lane, +1, active);
    m[2] = active ? f4(L, G.plane, 2, yp, G.pitch, c) : z4;
    m[3] = xshift(L, G.plane, 3, row, G, c, lane, -1, active);
    m[4] = active ? f4(L, G.plane, 4, ym, G.pitch, c) : z4;
    // sigma of g^t(y): g_i(y) = P_i(y - c_i)
    const float *S = static_cast<const float *>(a.state.data);
    float4 sg = active ? f4(S, G.plane, 0, row, G.pitch, c) : z4;
    {
        const float4 s1 = xshift(S, G.plane, 1, row, G, c, lane, -1, active);
        const float4 s3 = xshift(S, G.plane, 3, row, G, c, lane, +1, active);
        const float4 s2 = active ? f4(S, G.plane, 2, ym, G.pitch, c) : z4;
        const float4 s4 = active ? f4(S, G.plane, 4, yp, G.pitch, c) : z4;
        sg = make_float4(((sg.x + s1.x) + (s2.x + s3.x)) + s4.x, ((sg.y + s1.y) + (s2.y + s3.y)) + s4.y,
                         ((sg.z + s1.z) + (s2.z + s3.z)) + s4.z, ((sg.w + s1.w) + (s2.w + s3.w)) + s4.w);
    }
    if (!active) return;
    const float4 cl = f4(a.cL2, 0, 0, row, G.pitch, c);
    float4 jz = z4;
    float4 o[5];
    float dg[4] = {0.f, 0.f, 0.f, 0.f};  // this step's contribution, FP32; accumulated over steps in FP64
    for (int j = 0; j < 4; j++) {
        const float q = get(cl, j), w0 = 1.f - 2.f * q;
        const float mm = ((get(m[1], j) + get(m[2], j)) + get(m[3], j)) + get(m[4], j);
        const float nu = w0 * get(m[0], j) + 0.5f * q * mm;
        set(o[0], j, 2.f * nu - get(m[0], j));
        set(o[1], j, 2.f * nu - get(m[3], j));
        set(o[3], j, 2.f * nu - get(m[1], j));
        set(o[2], j, 2.f * nu - get(m[4], j));
        set(o[4], j, 2.f * nu - get(m[2], j));
        const float s = get(sg, j);
        dg[j] = s * mm - 4.f * (s * get(m[0], j));
    }
    if (a.evt.rowptr) {
        const int e0 = __ldg(a.evt.rowptr + row), e1 = __ldg(a.evt.rowptr + row + 1);
        for (int e = e0; e < e1; e++) {
            const Event ev = a.evt.ev[e];
            if ((ev.x >> 2) != c) continue;
            const int j = ev.x & 3;
            if (ev.kind == 0) {
                if (ev.comp == 2 && a.t < a.evt.nt) set(jz, j, get(jz, j) + __ldg(a.evt.amp + (long long)ev.index * a.evt.nt + a.t));
            } else {
                const long long n = a.t - a.t0;
                if (n < 0 || n >= a.nsteps || a.t >= a.evt.cap) continue;
                const float r = __ldg(a.cot + (long long)ev.index * a.nsteps + n);
                if (ev.comp == 2) {  // E_z = -c_L^2 sigma
                    const float d = -get(cl, j) * r;
                    for (int i = 0; i < 5; i++) set(o[i], j, get(o[i], j) + d);
                    dg[j] -= get(sg, j) * r;
                } else if (ev.comp == 3) {  // B_x = g_4 - g_2
                    set(o[4], j, get(o[4], j) + r);
                    set(o[2], j, get(o[2], j) - r);
                } else if (ev.comp == 4) {  // B_y = g_1 - g_3
                    set(o[1], j, get(o[1], j) + r);
                    set(o[3], j, get(o[3], j) - r);
                }
            }
        }
    }
    for (int j = 0; j < 4; j++) {
        const float mm = ((get(m[1], j) + get(m[2], j)) + get(m[3], j)) + get(m[4], j);
        dg[j] += get(jz, j) * (0.5f * mm - 2.f * get(m[0], j));
        const int x = 4 * c + j;
        if (x < G.nx) a.gcl[(long long)row * G.pitch + x] += (double)dg[j];
    }
    for (int i = 0; i < 5; i++) Codec<LBEM_F32>::store4(PopBuf{a.lam_out, nullptr, G.plane, 0, G.pitch, 0}, i, row, c, o[i]);
}

// ------------------------------------------------------------------ 3D
__global__ void __launch_bounds__(BLOCK) adjoint3d(AdjArgs a) {
    const Grid &G = a.g;
    const int lane = threadIdx.x & 31;
    const long long wg = ((long long)blockIdx.x * BLOCK + threadIdx.x) >> 5;
    const int wpr = G.nchunk_pad >> 5;
    const int row = (int)(wg / wpr);
    const int c = (int)(wg - (long long)row * wpr) * 32 + lane;
    if (row >= G.nrows) return;
    const bool active = c < G.nchunk;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const int z = row / G.ny, y = row - z * G.ny;
    const int rym = z * G.ny + (y == 0 ? G.ny - 1 : y - 1), ryp = z * G.ny + (y == G.ny - 1 ? 0 : y + 1);
    const int rzm = (z == 0 ? G.nz - 1 : z - 1) * G.ny + y, rzp = (z == G.nz - 1 ? 0 : z + 1) * G.ny + y;
    const float *L = a.lam_in;
    const float *S = static_cast<const float *>(a.state.data);
    float4 m[21];
    float4 sg[3];
#pragma unroll
    for (int gm = 0; gm < 3; gm++) {
        // mu_{i gamma}(y) = lambda_{i gamma}(y + c_i)
        m[0 + gm] = active ? f4(L, G.plane, 0 + gm, row, G.pitch, c) : z4;
        m[3 + gm] = xshift(L, G.plane, 3 + gm, row, G, c, lane, +1, active);
        m[6 + gm] = active ? f4(L, G.plane, 6 + gm, ryp, G.pitch, c) : z4;
        m[9 + gm] = active ? f4(L, G.plane, 9 + gm, rzp, G.pitch, c) : z4;
        m[12 + gm] = xshift(L, G.plane, 12 + gm, row, G, c, lane, -1, active);
        m[15 + gm] = active ? f4(L, G.plane, 15 + gm, rym, G.pitch, c) : z4;
        m[18 + gm] = active ? f4(L, G.plane, 18 + gm, rzm, G.pitch, c) : z4;
        // sigma_gamma of g^t(y), g_i(y) = P_i(y - c_i)
        float4 acc = active ? f4(S, G.plane, 0 + gm, row, G.pitch, c) : z4;
        const float4 s1 = xshift(S, G.plane, 3 + gm, row, G, c, lane, -1, active);
        const float4 s4 = xshift(S, G.plane, 12 + gm, row, G, c, lane, +1, active);
        const float4 s2 = active ? f4(S, G.plane, 6 + gm, rym, G.pitch, c) : z4;
        const float4 s3 = active ? f4(S, G.plane, 9 + gm, rzm, G.pitch, c) : z4;
        const float4 s5 = active ? f4(S, G.plane, 15 + gm, ryp, G.pitch, c) : z4;
        const float4 s6 = active ? f4(S, G.plane, 18 + gm, rzp, G.pitch, c) : z4;
        for (int j = 0; j < 4; j++)
            set(acc, j, ((get(acc, j) + get(s1, j)) + (get(s2, j) + get(s3, j))) + ((get(s4, j) + get(s5, j)) + get(s6, j)));
        sg[gm] = acc;
    }
    if (!active) return;
    const float4 cl = f4(a.cL2, 0, 0, row, G.pitch, c);
    float4 jv[3] = {z4, z4, z4};
    float dg[4] = {0.f, 0.f, 0.f, 0.f};  // this step's contribution, FP32; accumulated over steps in FP64
    // receivers add to lambda after M^T; collect them first per site
    float4 recE[3] = {z4, z4, z4}, recB[3] = {z4, z4, z4};
    if (a.evt.rowptr) {
        const int e0 = __ldg(a.evt.rowptr + row), e1 = __ldg(a.evt.rowptr + row + 1);
        for (int e = e0; e < e1; e++) {
            const Event ev = a.evt.ev[e];
            if ((ev.x >> 2) != c) continue;
            const int j = ev.x & 3;
            if (ev.kind == 0) {
                if (a.t < a.evt.nt) set(jv[ev.comp], j, get(jv[ev.comp], j) + __ldg(a.evt.amp + (long long)ev.index * a.evt.nt + a.t));
            } else {
                const long long n = a.t - a.t0;
                if (n < 0 || n >= a.nsteps || a.t >= a.evt.cap) continue;
                const float r = __ldg(a.cot + (long long)ev.index * a.nsteps + n);
                if (ev.comp < 3) set(recE[ev.comp], j, get(recE[ev.comp], j) + r);
                else set(recB[ev.comp - 3], j, get(recB[ev.comp - 3], j) + r);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < 4; j++) {
        float h[21];
#pragma unroll
        for (int p = 0; p < 21; p++) h[p] = get(m[p], j);
        const float q = get(cl, j), w0 = 1.f - 3.f * q;
        float mv[3], nu[3];
        for (int gm = 0; gm < 3; gm++) {
            mv[gm] = ((h[3 + gm] + h[6 + gm]) + (h[9 + gm] + h[12 + gm])) + (h[15 + gm] + h[18 + gm]);
            nu[gm] = w0 * h[gm] + 0.5f * q * mv[gm];
        }
        // V = sum_i mu_i x c_i, the same contraction that reads B from h
        const float vx = (h[10] - h[19]) - (h[8] - h[17]);
        const float vy = (h[5] - h[14]) - (h[9] - h[18]);
        const float vz = (h[6] - h[15]) - (h[4] - h[13]);
        const float hx = 0.5f * vx, hy = 0.5f * vy, hz = 0.5f * vz;
        const float Lx = 2.f * nu[0], Ly = 2.f * nu[1], Lz = 2.f * nu[2];
        float o[21];
        o[0] = Lx - h[0];
        o[1] = Ly - h[1];
        o[2] = Lz - h[2];
        o[3] = Lx - h[3];             // +x: c x V = (0, -Vz, Vy)
        o[4] = (Ly - hz) - h[4];
        o[5] = (Lz + hy) - h[5];
        o[6] = (Lx + hz) - h[6];      // +y: (Vz, 0, -Vx)
        o[7] = Ly - h[7];
        o[8] = (Lz - hx) - h[8];
        o[9] = (Lx - hy) - h[9];      // +z: (-Vy, Vx, 0)
        o[10] = (Ly + hx) - h[10];
        o[11] = Lz - h[11];
        o[12] = Lx - h[12];           // -x
        o[13] = (Ly + hz) - h[13];
        o[14] = (Lz - hy) - h[14];
        o[15] = (Lx - hz) - h[15];    // -y
        o[16] = Ly - h[16];
        o[17] = (Lz + hx) - h[17];
        o[18] = (Lx + hy) - h[18];    // -z
        o[19] = (Ly - hx) - h[19];
        o[20] = Lz - h[20];
        float d = 0.f;
        for (int gm = 0; gm < 3; gm++) {
            const float s = get(sg[gm], j);
            d += s * mv[gm] - 6.f * (s * h[gm]);
            d += get(jv[gm], j) * (0.25f * mv[gm] - 1.5f * h[gm]);
            // E_gamma = -c_L^2 sigma_gamma receivers
            const float rE = get(recE[gm], j);
            if (rE != 0.f) {
                for (int i = 0; i < 7; i++) o[3 * i + gm] -= q * rE;
                d -= s * rE;
            }
        }
        // B receivers: B_nu = sum_i (g_i x c_i)_nu = eps_{gamma kappa nu} c_{i kappa} g_{i gamma}
        const float bx = get(recB[0], j), by = get(recB[1], j), bz = get(recB[2], j);
        if (bx != 0.f || by != 0.f || bz != 0.f) {
            // d B_x/d h: +h[10](+z,y) -h[19](-z,y) -h[8](+y,z) +h[17](-y,z)
            o[10] += bx; o[19] -= bx; o[8] -= bx; o[17] += bx;
            o[5] += by; o[14] -= by; o[9] -= by; o[18] += by;
            o[6] += bz; o[15] -= bz; o[4] -= bz; o[13] += bz;
        }
#pragma unroll
        for (int p = 0; p < 21; p++) set(m[p], j, o[p]);
        dg[j] = d;
    }
    for (int j = 0; j < 4; j++) {
        const int x = 4 * c + j;
        if (x < G.nx) a.gcl[(long long)row * G.pitch + x] += (double)dg[j];
    }
    PopBuf ob{a.lam_out, nullptr, G.plane, 0, G.pitch, 0};
#pragma unroll
    for (int p = 0; p < 21; p++) Codec<LBEM_F32>::store4(ob, p, row, c, m[p]);
}

// One site per thread (48-64 registers instead of 170): the same update as adjoint3d.  The FP64
// gradient accumulator is loaded with the other operands, at the top, so its latency overlaps theirs.
template <int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) adjoint3d_site(AdjArgs a) {
    const Grid &G = a.g;
    const long long tid = (long long)blockIdx.x * BLOCK + threadIdx.x;
    const int row = (int)(tid / G.pitch);
    const int x = (int)(tid - (long long)row * G.pitch);
    if (row >= G.nrows || x >= G.nx) return;
    const int z = row / G.ny, y = row - z * G.ny;
    const int rym = z * G.ny + (y == 0 ? G.ny - 1 : y - 1), ryp = z * G.ny + (y == G.ny - 1 ? 0 : y + 1);
    const int rzm = (z == 0 ? G.nz - 1 : z - 1) * G.ny + y, rzp = (z == G.nz - 1 ? 0 : z + 1) * G.ny + y;
    const int xm = x == 0 ? G.nx - 1 : x - 1, xp = x == G.nx - 1 ? 0 : x + 1;
    const float *L = a.lam_in;
    const float *S = static_cast<const float *>(a.state.data);
    auto at = [&](const float *b, int p, int r, int xx) { return __ldg(b + p * G.plane + (long long)r * G.pitch + xx); };
    const long long o = (long long)row * G.pitch + x;
    const double gacc = a.gcl[o];
    float h[21], sg[3];
#pragma unroll
    for (int gm = 0; gm < 3; gm++) {
        // mu_{i gamma}(y) = lambda_{i gamma}(y + c_i)
        h[0 + gm] = at(L, 0 + gm, row, x);
        h[3 + gm] = at(L, 3 + gm, row, xp);
        h[6 + gm] = at(L, 6 + gm, ryp, x);
        h[9 + gm] = at(L, 9 + gm, rzp, x);
        h[12 + gm] = at(L, 12 + gm, row, xm);
        h[15 + gm] = at(L, 15 + gm, rym, x);
        h[18 + gm] = at(L, 18 + gm, rzm, x);
        // sigma_gamma of g^t(y), g_i(y) = P_i(y - c_i)
        sg[gm] = ((at(S, 0 + gm, row, x) + at(S, 3 + gm, row, xm)) + (at(S, 6 + gm, rym, x) + at(S, 9 + gm, rzm, x))) +
                 ((at(S, 12 + gm, row, xp) + at(S, 15 + gm, ryp, x)) + at(S, 18 + gm, rzp, x));
    }
    const float q = __ldg(a.cL2 + o), w0 = 1.f - 3.f * q;
    float jv[3] = {0.f, 0.f, 0.f}, rE[3] = {0.f, 0.f, 0.f}, rB[3] = {0.f, 0.f, 0.f};
    if (a.evt.rowptr) {
        const int e0 = __ldg(a.evt.rowptr + row), e1 = __ldg(a.evt.rowptr + row + 1);
        for (int e = e0; e < e1; e++) {
            const Event ev = a.evt.ev[e];
            if (ev.x != x) continue;
            if (ev.kind == 0) {
                if (a.t < a.evt.nt) {
                    const float jj = __ldg(a.evt.amp + (long long)ev.index * a.evt.nt + a.t);
                    if (ev.comp == 0) jv[0] += jj;
                    else if (ev.comp == 1) jv[1] += jj;
                    else jv[2] += jj;
                }
            } else {
                const long long n = a.t - a.t0;
                if (n < 0 || n >= a.nsteps || a.t >= a.evt.cap) continue;
                const float r = __ldg(a.cot + (long long)ev.index * a.nsteps + n);
                switch (ev.comp) {
                    case 0: rE[0] += r; break;
                    case 1: rE[1] += r; break;
                    case 2: rE[2] += r; break;
                    case 3: rB[0] += r; break;
                    case 4: rB[1] += r; break;
                    default: rB[2] += r; break;
                }
            }
        }
    }
    float mv[3], nu[3];
#pragma unroll
    for (int gm = 0; gm < 3; gm++) {
        mv[gm] = ((h[3 + gm] + h[6 + gm]) + (h[9 + gm] + h[12 + gm])) + (h[15 + gm] + h[18 + gm]);
        nu[gm] = w0 * h[gm] + 0.5f * q * mv[gm];
    }
    const float vx = (h[10] - h[19]) - (h[8] - h[17]);
    const float vy = (h[5] - h[14]) - (h[9] - h[18]);
    const float vz = (h[6] - h[15]) - (h[4] - h[13]);
    const float hx = 0.5f * vx, hy = 0.5f * vy, hz = 0.5f * vz;
    const float Lx = 2.f * nu[0], Ly = 2.f * nu[1], Lz = 2.f * nu[2];
    float d = 0.f;  // this step's contribution, FP32; accumulated over steps in FP64
#pragma unroll
    for (int gm = 0; gm < 3; gm++) {
        d += sg[gm] * mv[gm] - 6.f * (sg[gm] * h[gm]);
        d += jv[gm] * (0.25f * mv[gm] - 1.5f * h[gm]);
    }
    float out[21];
    out[0] = Lx - h[0];
    out[1] = Ly - h[1];
    out[2] = Lz - h[2];
    out[3] = Lx - h[3];
    out[4] = (Ly - hz) - h[4];
    out[5] = (Lz + hy) - h[5];
    out[6] = (Lx + hz) - h[6];
    out[7] = Ly - h[7];
    out[8] = (Lz - hx) - h[8];
    out[9] = (Lx - hy) - h[9];
    out[10] = (Ly + hx) - h[10];
    out[11] = Lz - h[11];
    out[12] = Lx - h[12];
    out[13] = (Ly + hz) - h[13];
    out[14] = (Lz - hy) - h[14];
    out[15] = (Lx - hz) - h[15];
    out[16] = Ly - h[16];
    out[17] = (Lz + hx) - h[17];
    out[18] = (Lx + hy) - h[18];
    out[19] = (Ly - hx) - h[19];
    out[20] = Lz - h[20];
#pragma unroll
    for (int gm = 0; gm < 3; gm++)
        if (rE[gm] != 0.f) {
            for (int i = 0; i < 7; i++) out[3 * i + gm] -= q * rE[gm];
            d -= sg[gm] * rE[gm];
        }
    if (rB[0] != 0.f || rB[1] != 0.f || rB[2] != 0.f) {
        out[10] += rB[0]; out[19] -= rB[0]; out[8] -= rB[0]; out[17] += rB[0];
        out[5] += rB[1]; out[14] -= rB[1]; out[9] -= rB[1]; out[18] += rB[1];
        out[6] += rB[2]; out[15] -= rB[2]; out[4] -= rB[2]; out[13] += rB[2];
    }
    a.gcl[o] = gacc + (double)d;
#pragma unroll
    for (int p = 0; p < 21; p++) __stcs(a.lam_out + p * G.plane + o, out[p]);
}

// dL/d eps_r = -dL/dc_L^2 * c_L^2 / eps_r with eps_r = (D-1) c_ref^2 / c_L^2 (mu = 1), dense output.
__global__ void adjoint_finish(Grid G, const double *gcl, const float *cL2, int D, double c_ref2, float *geps,
                               double *gcl_dense) {
    const long long n = (long long)G.nx * G.nrows;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        const long long row = s / G.nx;
        const int x = (int)(s - row * G.nx);
        const double g = gcl[row * G.pitch + x];
        const double q = cL2[row * G.pitch + x];
        if (geps) geps[s] = (float)(-g * q * q / ((D - 1) * c_ref2));
        if (gcl_dense) gcl_dense[s] = g;
    }
}

static cudaError_t launch_adjoint(const lbem_t *h, const AdjArgs &a) {
    if (h->dim == 3 && h->variant >= 1) {  // the one-site-per-thread shapes, as the forward kernel
        const long long threads = (long long)a.g.nrows * a.g.pitch;
        const unsigned blocks = (unsigned)((threads + BLOCK - 1) / BLOCK);
        if (h->variant == 2) adjoint3d_site<5><<<blocks, BLOCK, 0, h->stream>>>(a);  // registers capped
        else adjoint3d_site<1><<<blocks, BLOCK, 0, h->stream>>>(a);
        return cudaGetLastError();
    }
    const long long warps = (long long)a.g.nrows * (a.g.nchunk_pad / 32);
    const unsigned blocks = (unsigned)((warps * 32 + BLOCK - 1) / BLOCK);
    if (h->dim == 2) adjoint2d<<<blocks, BLOCK, 0, h->stream>>>(a);
    else adjoint3d<<<blocks, BLOCK, 0, h->stream>>>(a);
    return cudaGetLastError();
}

static cudaError_t launch_fwd(const lbem_t *h, const StepArgs &a) {
    if (h->dim == 2) return launch_step_2d(a, h->storage, false, h->variant, h->stream);
    return launch_step_3d(a, false, h->variant, h->stream);
}

bool is_device_ptr(const void *p);
lbem_status device_input(lbem_t *h, const float *p, size_t count, size_t off, const float **out);

}  // namespace lbk

using namespace lbk;

extern "C" {

lbem_status lbem_forward_record(lbem_t *h, int nsteps, int every) {
    if (!h) return fail(LBEM_ERR_ARG, "null handle");
    if (nsteps < 1 || every < 1) return fail(LBEM_ERR_ARG, "lbem_forward_record: nsteps >= 1 and checkpoint_every >= 1");
    if (!h->has_medium) return fail(LBEM_ERR_STATE, "lbem_forward_record: set a medium first");
    if (h->storage != LBEM_F32) return fail(LBEM_ERR_STATE, "lbem_forward_record: the adjoint needs LBEM_F32 storage");
    if (h->has_mu) return fail(LBEM_ERR_STATE, "lbem_forward_record: the adjoint supports uniform mu only (mu_r = NULL)");
    if (h->walls()) return fail(LBEM_ERR_STATE, "lbem_forward_record: the adjoint supports periodic boundaries only");
    if (h->disp || h->aniso)
        return fail(LBEM_ERR_STATE, "lbem_forward_record: the adjoint supports non-dispersive isotropic media only");
    adjoint_free(h);
    AdjointState *A = new AdjointState();
    h->adj = A;
    A->nsteps = nsteps;
    A->every = std::min(every, nsteps);
    A->ncp = (nsteps + A->every - 1) / A->every;
    A->t0 = h->t;
    A->state_floats = (size_t)h->npop * h->grid.plane;
    const size_t sb = A->state_floats * sizeof(float);
    if (cudaMalloc((void **)&A->cps, sb * A->ncp) != cudaSuccess) {
        cudaGetLastError();
        adjoint_free(h);
        return fail(LBEM_ERR_NOMEM, "lbem_forward_record: no room for the checkpoints");
    }
    for (int n = 0; n < nsteps; n++) {
        if (n % A->every == 0)
            LBEM_CUDA(cudaMemcpyAsync(A->cps + (size_t)(n / A->every) * A->state_floats, h->buf[h->cur].data, sb,
                                      cudaMemcpyDeviceToDevice, h->stream));
        StepArgs a = step_args(h, h->cur);
        LBEM_CUDA(launch_fwd(h, a));
        h->cur ^= 1;
        h->t++;
    }
    return LBEM_OK;
}

lbem_status lbem_adjoint(lbem_t *h, const float *trace_cot, float *grad_eps, double *grad_cL2) {
    if (!h) return fail(LBEM_ERR_ARG, "null handle");
    AdjointState *A = h->adj;
    if (!A) return fail(LBEM_ERR_STATE, "lbem_adjoint: call lbem_forward_record first");
    if (h->nrec > 0 && h->cap < A->t0 + A->nsteps)
        return fail(LBEM_ERR_STATE, "lbem_adjoint: receiver capacity shorter than the recorded run");
    const size_t sb = A->state_floats * sizeof(float);
    const Grid &G = h->grid;
    if (!A->seg) {
        cudaError_t e = cudaMalloc((void **)&A->seg, sb * A->every);
        if (e == cudaSuccess) e = cudaMalloc((void **)&A->lam, 2 * sb);
        if (e == cudaSuccess) e = cudaMalloc((void **)&A->gcl, sizeof(double) * G.plane);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(LBEM_ERR_NOMEM, "lbem_adjoint: no room for the segment and adjoint buffers");
        }
    }
    const size_t ncot = (size_t)h->nrec * A->nsteps;
    cudaFree(A->cot);
    A->cot = nullptr;
    if (ncot) {
        if (!trace_cot) return fail(LBEM_ERR_ARG, "lbem_adjoint: trace_cot is NULL but receivers are set");
        LBEM_CUDA(cudaMalloc((void **)&A->cot, ncot * sizeof(float)));
        LBEM_CUDA(cudaMemcpyAsync(A->cot, trace_cot, ncot * sizeof(float), cudaMemcpyDefault, h->stream));
    }
    LBEM_CUDA(cudaMemsetAsync(A->lam, 0, 2 * sb, h->stream));
    LBEM_CUDA(cudaMemsetAsync(A->gcl, 0, sizeof(double) * G.plane, h->stream));
    int lc = 0;  // lam[lc] holds lambda^{t+1}
    StepArgs base = step_args(h, 0);
    for (int k = A->ncp - 1; k >= 0; k--) {
        const int n0 = k * A->every;
        const int len = std::min(A->every, A->nsteps - n0);
        LBEM_CUDA(cudaMemcpyAsync(A->seg, A->cps + (size_t)k * A->state_floats, sb, cudaMemcpyDeviceToDevice, h->stream));
        for (int j = 1; j < len; j++) {  // recompute the segment's states (sources on, no trace writes)
            StepArgs a = base;
            a.in.data = A->seg + (size_t)(j - 1) * A->state_floats;
            a.out.data = A->seg + (size_t)j * A->state_floats;
            a.evt.cap = 0;
            a.t = A->t0 + n0 + j - 1;
            LBEM_CUDA(launch_fwd(h, a));
        }
        for (int j = len - 1; j >= 0; j--) {
            AdjArgs a;
            a.g = G;
            a.lam_in = A->lam + (size_t)lc * A->state_floats;
            a.lam_out = A->lam + (size_t)(lc ^ 1) * A->state_floats;
            a.state = base.in;
            a.state.data = A->seg + (size_t)j * A->state_floats;
            a.cL2 = h->cL2;
            a.gcl = A->gcl;
            a.evt = base.evt;
            a.cot = A->cot;
            a.nsteps = A->nsteps;
            a.t = A->t0 + n0 + j;
            a.t0 = A->t0;
            LBEM_CUDA(launch_adjoint(h, a));
            lc ^= 1;
        }
    }
    const bool eh = grad_eps && !is_device_ptr(grad_eps);
    const bool ch = grad_cL2 && !is_device_ptr(grad_cL2);
    if (eh && !A->gout) LBEM_CUDA(cudaMalloc((void **)&A->gout, sizeof(float) * h->nsite));
    if (ch && !A->gcl_out) LBEM_CUDA(cudaMalloc((void **)&A->gcl_out, sizeof(double) * h->nsite));
    float *ge = eh ? A->gout : grad_eps;
    double *gc = ch ? A->gcl_out : grad_cL2;
    adjoint_finish<<<1024, 256, 0, h->stream>>>(G, A->gcl, h->cL2, h->dim, h->c_ref2, ge, gc);
    LBEM_CUDA(cudaGetLastError());
    if (eh) LBEM_CUDA(cudaMemcpyAsync(grad_eps, ge, sizeof(float) * h->nsite, cudaMemcpyDeviceToHost, h->stream));
    if (ch) LBEM_CUDA(cudaMemcpyAsync(grad_cL2, gc, sizeof(double) * h->nsite, cudaMemcpyDeviceToHost, h->stream));
    if (eh || ch) LBEM_CUDA(cudaStreamSynchronize(h->stream));
    return LBEM_OK;
}

}  // extern "C"
