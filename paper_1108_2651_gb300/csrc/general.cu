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
// step2d_gen is the single-step kernel for the media the fast kernels do not
// cover (a pole, an anisotropic tensor), one site per thread: pulls with
// periodic wrap or across walls (the wall rule of walls.cu), the B x grad ln mu
// source, sources and receivers, the pole, the collision, the absorbing layer's
// factor.  J and P are read and written at the site only, so they are updated
// in place.
#include <algorithm>

#include "lbem_internal.cuh"

namespace lbk {

template <bool MU>
__global__ void __launch_bounds__(256) step2d_gen(StepArgs a, Walls w, General q) {
    const Grid &G = a.g;
    const long long n = (long long)G.nx * G.ny;
    const float *in = static_cast<const float *>(a.in.data);
    float *out = static_cast<float *>(a.out.data);
    const long long PL = a.in.plane, PO = a.out.plane;
    const float sx = w.kind[0] == 1 ? -1.f : 1.f, sy = w.kind[1] == 1 ? -1.f : 1.f;
    const float r = q.r, ri = __fdiv_rn(1.f, q.r), fs = __fadd_rn(r, ri);  // fs = 2 when isotropic
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(s / G.nx), x = (int)(s - (long long)y * G.nx);
        const long long rw = (long long)y * a.in.pitch;
        const int ym = y == 0 ? G.ny - 1 : y - 1, yp = y == G.ny - 1 ? 0 : y + 1;
        const int xm = x == 0 ? G.nx - 1 : x - 1, xp = x == G.nx - 1 ? 0 : x + 1;
        // pulls g_i(x) = g'_i(x - c_i); across a wall the site's own opposite population times the wall sign
        const float g0 = in[rw + x];
        const float g1 = (w.kind[0] && x == 0) ? sx * in[3 * PL + rw + x] : in[PL + rw + xm];
        const float g3 = (w.kind[0] && x == G.nx - 1) ? sx * in[PL + rw + x] : in[3 * PL + rw + xp];
        const float g2 = (w.kind[1] && y == 0) ? sy * in[4 * PL + rw + x] : in[2 * PL + (long long)ym * a.in.pitch + x];
        const float g4 = (w.kind[1] && y == G.ny - 1) ? sy * in[2 * PL + rw + x]
                                                        : in[4 * PL + (long long)yp * a.in.pitch + x];
        const long long o = (long long)y * G.pitch + x;
        const float cl = a.med.cL2[o];
        float shat = MU ? mu_source(g4 - g2, g1 - g3, a.med.dlnmu[o], a.med.dlnmu[G.plane + o]) : 0.f;
        const float sig = __fadd_rn(__fadd_rn(__fadd_rn(g0, g1), __fadd_rn(g2, g3)), g4);
        float P = 0.f;
        if (q.wp2) {
            // the pole, from the pre-collision field E = D/eps_inf - P
            P = q.P[s];
            const float J = q.J[s], gm = q.gam[s];
            const float E = __fsub_rn(__fmul_rn(-cl, sig), P);
            const float num = __fadd_rn(__fsub_rn(__fmul_rn(__fsub_rn(1.f, 0.5f * gm), J), __fmul_rn(q.wr2[s], P)),
                                        __fmul_rn(q.wp2[s], E));
            const float Jn = __fdiv_rn(num, __fadd_rn(1.f, 0.5f * gm));
            q.J[s] = Jn;
            q.P[s] = __fadd_rn(P, Jn);
        }
        if (a.evt.rowptr && __ldg(a.evt.rowptr + y) != __ldg(a.evt.rowptr + y + 1))
            shat = site_events(a, x, y, a.t, true, g0, g1, g2, g3, g4, cl, shat, P, r, ri, q.mubar);
        // collision with the second moment Lambda + P read per axis
        const float Lam = __fadd_rn(__fmul_rn(cl, sig), P);
        const float Lx = __fmul_rn(r, Lam), Ly = __fmul_rn(ri, Lam);
        const float w0 = __fsub_rn(1.f, __fmul_rn(fs, cl));
        const float Tm = __fmul_rn(-0.5f * cl, shat), T0 = __fmul_rn(-w0, shat);
        const float Tx = __fmul_rn(r, Tm), Ty = __fmul_rn(ri, Tm);
        const float f = __fmul_rn(w.fx ? w.fx[x] : 1.f, w.fy ? w.fy[y] : 1.f);
        const long long ro = (long long)y * a.out.pitch + x;
        out[ro] = __fmul_rn(
            __fadd_rn(__fsub_rn(__fsub_rn(__fmul_rn(2.f * w0, sig), g0), __fmul_rn(2.f * fs, P)), T0), f);
        out[PO + ro] = __fmul_rn(__fadd_rn(__fsub_rn(Lx, g3), Tx), f);
        out[2 * PO + ro] = __fmul_rn(__fadd_rn(__fsub_rn(Ly, g4), Ty), f);
        out[3 * PO + ro] = __fmul_rn(__fadd_rn(__fsub_rn(Lx, g1), Tx), f);
        out[4 * PO + ro] = __fmul_rn(__fadd_rn(__fsub_rn(Ly, g2), Ty), f);
    }
}

cudaError_t launch_step_2d_gen(const StepArgs &a, const Walls &w, const General &q, cudaStream_t s) {
    static int per_sm[2] = {0, 0}, nsm = 0;
    const bool mu = a.med.dlnmu != nullptr;
    if (!per_sm[mu]) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (mu) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[1], step2d_gen<true>, 256, 0);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[0], step2d_gen<false>, 256, 0);
        if (per_sm[mu] < 1) per_sm[mu] = 1;
    }
    const long long n = (long long)a.g.nx * a.g.ny;
    const long long blocks = std::min<long long>((n + 255) / 256, (long long)per_sm[mu] * nsm);
    if (mu) step2d_gen<true><<<(unsigned)blocks, 256, 0, s>>>(a, w, q);
    else step2d_gen<false><<<(unsigned)blocks, 256, 0, s>>>(a, w, q);
    return cudaGetLastError();
}

// Validation of a pole (dense [nsite] arrays; wr2, gam may be null) against a medium: finite, non-negative,
// wp^2 + wr^2 <= 4 w0 with w0 = 1 - fsum c_L^2 in FP64 (fsum = 2, or r + 1/r for an anisotropic medium).  The
// medium is either the stored c_L^2 (pitched; eps null) or a new eps_r, mu_r (dense; mu may be null) with
// c_L^2 = c_ref^2 / (eps_r mu_r mubar).
__global__ void disp_check(Grid G, const float *cL2, const float *eps, const float *mu, double c_ref2, double fsum,
                           double mubar, const float *wp2, const float *wr2, const float *gam, unsigned *bad) {
    unsigned local = 0;
    const long long n = (long long)G.nx * G.ny;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(s / G.nx), x = (int)(s - (long long)y * G.nx);
        const double p = wp2[s], r = wr2 ? (double)wr2[s] : 0.0, g = gam ? (double)gam[s] : 0.0;
        const double cl = eps ? c_ref2 / ((double)eps[s] * (mu ? (double)mu[s] : 1.0) * mubar)
                              : (double)cL2[(long long)y * G.pitch + x];
        const double w0 = 1.0 - fsum * cl;
        if (!(p >= 0.0 && r >= 0.0 && g >= 0.0 && isfinite(p) && isfinite(r) && isfinite(g)) || p + r > 4.0 * w0)
            local++;
    }
    if (local) atomicAdd(bad, local);
}

cudaError_t launch_disp_check(const lbem_t *h, const float *eps, const float *mu, double fsum, double mubar,
                              const float *wp2, const float *wr2, const float *gam, unsigned *bad, cudaStream_t s) {
    const unsigned blocks = (unsigned)std::min<long long>(4096, std::max<long long>(1, (h->nsite + 255) / 256));
    disp_check<<<blocks, 256, 0, s>>>(h->grid, h->cL2, eps, mu, h->c_ref2, fsum, mubar, wp2, wr2, gam, bad);
    return cudaGetLastError();
}

}  // namespace lbk
