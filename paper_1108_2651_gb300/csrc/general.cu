// The general single-step kernel (2D, FP32 storage): frequency-dispersive
// permittivity (one Drude-Lorentz pole per site) and anisotropic media.
//
// Eq. 3 carries a polarization term, a convolution with the time derivative of
// the permittivity, which the paper leaves to auxiliary differential
// equations.  Here it is one pole per site,
//     d_t J + gamma J + wr^2 P = wp^2 E,   J = d_t P   (P in units of E),
// i.e. eps(omega) = eps_inf (1 + wp^2 / (wr^2 - omega^2 - i gamma omega)).  It
// enters in displacement form: the lattice's zeroth moment carries D/eps_inf
// (no source: d_t D = curl H), the field is E = D/eps_inf - P, and P enters the
// equilibrium's second moment only (+P on every moving population's Lambda,
// -4P on the rest population, so the zeroth and first moments are unchanged):
//     g'_1 = (Lambda + P) - g_3 + T_m  (and likewise 2, 3, 4)
//     g'_0 = 2 w0 sigma - g_0 - 4P + T_0
// (entering -d_t P through the source T of Eq. 17 instead is unstable: the
// source's (c^2/2) Lap S part acts on the accumulated current).  J lives at
// half steps, P at whole ones; from the pre-collision E(t):
//     J(t+1/2) = [(1 - gamma/2) J(t-1/2) + wp^2 E(t) - wr^2 P(t)] / (1 + gamma/2)
//     P(t+1)   = P(t) + J(t+1/2)
// and the collision at t uses P(t).  Stable where wp^2 + wr^2 <= 4 w0.
//
// Anisotropic media (the paper: different weights for particles moving along
// different axes), read as a uniform in-plane relative permeability tensor
// diag(mu_xx, mu_yy) with eps_r per site: axis x moves at c_x^2 = r cbar^2 and
// axis y at c_y^2 = cbar^2 / r, r = sqrt(mu_xx / mu_yy), where cbar^2 =
// c_ref^2 / (eps_r sqrt(mu_xx mu_yy)) is the stored c_L^2 (so c_x^2 =
// c_ref^2 / (eps_r mu_yy), the speed of a wave moving along x).  Moving particles
// of axis a weigh c_a^2 / 2 and w0 = 1 - cbar^2 (r + 1/r); the closed form of
// the collision keeps its shape with Lambda read per axis and the source split
// by weight:
//     g'_1 = r (Lambda + P) - g_3 + r T_m,   g'_2 = (Lambda + P) / r - g_4 + T_m / r
//     g'_0 = 2 w0 sigma - g_0 - 2 (r + 1/r) P + T_0
// (likewise 3, 4), with S^ = -sqrt(mu_xx mu_yy) j_z; fields E_z = -cbar^2 sigma
// - P, B_x = r (g_4 - g_2), B_y = (g_1 - g_3) / r.  r = 1 with no pole is the
// plain scheme.
//
// step2d_gen is the single-step kernel for these media (a pole, an anisotropic
// tensor), with walls and layers too.  Without walls the two-step tile kernel
// (tblock.cu) also steps them, with the same site update (collide2d_an,
// pole_update).  Thread mapping as the plain single-step kernel: one warp
// covers 128 consecutive sites of a row, 4 per lane, with 16-byte loads and
// the +-x pulls by warp shuffle (pull2d); pulls across a wall are then replaced
// by the wall rule of walls.cu.  Per site: the B x grad ln mu source, sources
// and receivers, the pole, the collision, the absorbing layer's factor.  The
// pole's arrays are planes like c_L^2; J is read and written at the site only
// (in place), P is read from the plane of the input's parity and written to
// the other (a two-step launch reads P at sites of neighbouring tiles).
#include <algorithm>

#include "lbem_internal.cuh"

namespace lbk {

template <bool MU>
__global__ void __launch_bounds__(BLOCK, 4) step2d_gen(StepArgs a, Walls w, General q) {
    using C = Codec<LBEM_F32>;
    const Grid &G = a.g;
    const int lane = threadIdx.x & 31;
    const long long wg = ((long long)blockIdx.x * BLOCK + threadIdx.x) >> 5;
    const int wpr = G.nchunk_pad >> 5;
    const int row = (int)(wg / wpr);
    const int c = (int)(wg - (long long)row * wpr) * 32 + lane;
    if (row >= G.ny) return;  // warp-uniform
    const bool active = c < G.nchunk;
    const int x0 = 4 * c;
    float4 g[5];
    pull2d<LBEM_F32>(a.in, G, row, c, lane, g);
    if (!active) return;
    // pulls across a wall: the site's own opposite population times the wall sign
    const float sx = w.kind[0] == 1 ? -1.f : 1.f, sy = w.kind[1] == 1 ? -1.f : 1.f;
    if (w.kind[1] && row == 0) {
        const float4 v = C::load4(a.in, 4, row, c);
        g[2] = make_float4(sy * v.x, sy * v.y, sy * v.z, sy * v.w);
    }
    if (w.kind[1] && row == G.ny - 1) {
        const float4 v = C::load4(a.in, 2, row, c);
        g[4] = make_float4(sy * v.x, sy * v.y, sy * v.z, sy * v.w);
    }
    if (w.kind[0] && x0 == 0) set(g[1], 0, sx * C::load1(a.in, 3, row, 0));
    if (w.kind[0] && x0 + 4 >= G.nx) set(g[3], G.nx - 1 - x0, sx * C::load1(a.in, 1, row, G.nx - 1));
    const long long o4 = (long long)row * G.pitch + x0;  // first of the lane's 4 sites in a medium plane
    const float4 cl = *reinterpret_cast<const float4 *>(a.med.cL2 + o4);
    float4 dlx = make_float4(0.f, 0.f, 0.f, 0.f), dly = dlx;
    if (MU) {
        dlx = *reinterpret_cast<const float4 *>(a.med.dlnmu + o4);
        dly = *reinterpret_cast<const float4 *>(a.med.dlnmu + G.plane + o4);
    }
    float4 sig4;  // sigma = sum_i g_i per site (the order of collide2d)
#pragma unroll
    for (int j = 0; j < 4; j++)
        set(sig4, j, __fadd_rn(__fadd_rn(__fadd_rn(get(g[0], j), get(g[1], j)), __fadd_rn(get(g[2], j), get(g[3], j))),
                               get(g[4], j)));
    float4 P4 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (q.wp2) {
        // the pole, from the pre-collision field E = D/eps_inf - P; the collision below uses P(t)
        P4 = *reinterpret_cast<const float4 *>(q.P + o4);
        const float4 J4 = *reinterpret_cast<const float4 *>(q.J + o4);
        const float4 wp4 = *reinterpret_cast<const float4 *>(q.pc + o4);
        const float4 wr4 = *reinterpret_cast<const float4 *>(q.pb + o4);
        const float4 gm4 = *reinterpret_cast<const float4 *>(q.pa + o4);
        float4 Jn4, Pn4;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            float J = get(J4, j), P = get(P4, j);
            pole_update(get(cl, j), get(sig4, j), get(wp4, j), get(wr4, j), get(gm4, j), J, P);
            set(Jn4, j, J);
            set(Pn4, j, P);
        }
        *reinterpret_cast<float4 *>(q.J + o4) = Jn4;
        *reinterpret_cast<float4 *>(q.Pn + o4) = Pn4;
    }
    const float4 one4 = make_float4(1.f, 1.f, 1.f, 1.f);
    const float4 fx4 = w.fx ? *reinterpret_cast<const float4 *>(w.fx + x0) : one4;
    const float fy = w.fy ? w.fy[row] : 1.f;
    const bool ev = a.evt.rowptr && __ldg(a.evt.rowptr + row) != __ldg(a.evt.rowptr + row + 1);
    const float r = q.r, ri = __fdiv_rn(1.f, q.r), fs = __fadd_rn(r, ri);  // fs = 2 when isotropic
    float4 o[5];
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const float g0 = get(g[0], j), g1 = get(g[1], j), g2 = get(g[2], j), g3 = get(g[3], j), g4 = get(g[4], j);
        const float ck = get(cl, j);
        float shat = MU ? mu_source(g4 - g2, g1 - g3, get(dlx, j), get(dly, j)) : 0.f;
        const float sig = get(sig4, j);
        const float P = get(P4, j);
        if (ev && x0 + j < G.nx)
            shat = site_events(a, x0 + j, row, a.t, true, g0, g1, g2, g3, g4, ck, shat, P, r, ri, q.mubar);
        // collision with the second moment Lambda + P read per axis
        const float Lam = __fadd_rn(__fmul_rn(ck, sig), P);
        const float Lx = __fmul_rn(r, Lam), Ly = __fmul_rn(ri, Lam);
        const float w0 = __fsub_rn(1.f, __fmul_rn(fs, ck));
        const float Tm = __fmul_rn(-0.5f * ck, shat), T0 = __fmul_rn(-w0, shat);
        const float Tx = __fmul_rn(r, Tm), Ty = __fmul_rn(ri, Tm);
        const float f = __fmul_rn(get(fx4, j), fy);
        set(o[0], j, __fmul_rn(__fadd_rn(__fsub_rn(__fsub_rn(__fmul_rn(2.f * w0, sig), g0), __fmul_rn(2.f * fs, P)), T0),
                               f));
        set(o[1], j, __fmul_rn(__fadd_rn(__fsub_rn(Lx, g3), Tx), f));
        set(o[2], j, __fmul_rn(__fadd_rn(__fsub_rn(Ly, g4), Ty), f));
        set(o[3], j, __fmul_rn(__fadd_rn(__fsub_rn(Lx, g1), Tx), f));
        set(o[4], j, __fmul_rn(__fadd_rn(__fsub_rn(Ly, g2), Ty), f));
    }
#pragma unroll
    for (int p = 0; p < 5; p++) C::store4(a.out, p, row, c, o[p]);
}

cudaError_t launch_step_2d_gen(const StepArgs &a, const Walls &w, const General &q, cudaStream_t s) {
    const long long warps = (long long)a.g.ny * (a.g.nchunk_pad / 32);
    const unsigned blocks = (unsigned)((warps * 32 + BLOCK - 1) / BLOCK);
    if (a.med.dlnmu) step2d_gen<true><<<blocks, BLOCK, 0, s>>>(a, w, q);
    else step2d_gen<false><<<blocks, BLOCK, 0, s>>>(a, w, q);
    return cudaGetLastError();
}

// Validation of a pole (dense [nsite] arrays, or planes with the grid's pitch; wr2, gam may be null) against a medium: finite, non-negative,
// wp^2 + wr^2 <= 4 w0 with w0 = 1 - fsum c_L^2 in FP64 (fsum = 2, or r + 1/r for an anisotropic medium).  The
// medium is either the stored c_L^2 (pitched; eps null) or a new eps_r, mu_r (dense; mu may be null) with
// c_L^2 = c_ref^2 / (eps_r mu_r mubar).
__global__ void disp_check(Grid G, const float *cL2, const float *eps, const float *mu, double c_ref2, double fsum,
                           double mubar, const float *wp2, const float *wr2, const float *gam, bool pitched,
                           unsigned *bad) {
    unsigned local = 0;
    const long long n = (long long)G.nx * G.ny;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(s / G.nx), x = (int)(s - (long long)y * G.nx);
        const long long k = pitched ? (long long)y * G.pitch + x : s;
        const double p = wp2[k], r = wr2 ? (double)wr2[k] : 0.0, g = gam ? (double)gam[k] : 0.0;
        const double cl = eps ? c_ref2 / ((double)eps[s] * (mu ? (double)mu[s] : 1.0) * mubar)
                              : (double)cL2[(long long)y * G.pitch + x];
        const double w0 = 1.0 - fsum * cl;
        if (!(p >= 0.0 && r >= 0.0 && g >= 0.0 && isfinite(p) && isfinite(r) && isfinite(g)) || p + r > 4.0 * w0)
            local++;
    }
    if (local) atomicAdd(bad, local);
}

static unsigned blocks_for(long long n) {
    return (unsigned)std::min<long long>(4096, std::max<long long>(1, (n + 255) / 256));
}

cudaError_t launch_disp_check(const lbem_t *h, const float *eps, const float *mu, double fsum, double mubar,
                              const float *wp2, const float *wr2, const float *gam, bool pitched, unsigned *bad,
                              cudaStream_t s) {
    disp_check<<<blocks_for(h->nsite), 256, 0, s>>>(h->grid, h->cL2, eps, mu, h->c_ref2, fsum, mubar, wp2, wr2, gam,
                                                     pitched, bad);
    return cudaGetLastError();
}

// dense [nsite] (null: zeros) -> plane with the grid's pitch (padding columns zero)
__global__ void to_plane(Grid G, const float *src, float *dst) {
    const long long n = (long long)G.pitch * G.ny;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(k / G.pitch), x = (int)(k - (long long)y * G.pitch);
        dst[k] = (src && x < G.nx) ? src[(long long)y * G.nx + x] : 0.f;
    }
}

cudaError_t launch_to_plane(const lbem_t *h, const float *src, float *dst, cudaStream_t s) {
    to_plane<<<blocks_for((long long)h->grid.pitch * h->grid.ny), 256, 0, s>>>(h->grid, src, dst);
    return cudaGetLastError();
}

// pole_update's per-site coefficients from the pole's parameter planes, formed in FP64 and rounded once:
// pa = (1 - gam/2)/(1 + gam/2), pb = wr^2/(1 + gam/2), pc = wp^2/(1 + gam/2) (padding: zero parameters, pa = 1).
__global__ void pole_coefficients(long long n, const float *wp2, const float *wr2, const float *gam, float *pc,
                                  float *pb, float *pa) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const double d = 1.0 + 0.5 * (double)gam[k];
        pa[k] = (float)((1.0 - 0.5 * (double)gam[k]) / d);
        pb[k] = (float)((double)wr2[k] / d);
        pc[k] = (float)((double)wp2[k] / d);
    }
}

cudaError_t launch_pole_coefficients(const lbem_t *h, cudaStream_t s) {
    const long long n = h->grid.plane;
    pole_coefficients<<<blocks_for(n), 256, 0, s>>>(n, h->d_wp2, h->d_wr2, h->d_gam, h->d_pc, h->d_pb, h->d_pa);
    return cudaGetLastError();
}

}  // namespace lbk
