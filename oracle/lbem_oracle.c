/*
 * lbem_oracle.c -- plain FP64 CPU oracle of the lattice-Boltzmann scheme for
 * electromagnetic waves of Hanasoge, Succi & Orszag, "Lattice Boltzmann Method
 * for Electromagnetic Wave Propagation" (EPL; arXiv:1108.2651).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * statement of what the GPU library computes.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it; the product path
 * never does.  It shares no code, header, table or helper with the CUDA
 * library.
 *
 * What is stored: the FULL D x D tensor g_{i,alpha,beta} for every lattice
 * direction i (paper, Sec. "Lattice BGK formulation": the distribution is a
 * tensor with built-in antisymmetry g_{ab} = -g_{ba}).  Nothing here exploits
 * that antisymmetry, so a test can check it bit for bit.
 *
 * Layout: site s = x + nx*(y + ny*z); g[((s*Q + i)*D + a)*D + b].
 * Lattice (Sec. "Lattice BGK formulation", the 4+1 and 6+1 speed lattices):
 *   c_0 = 0; c_1..c_D = +e_1..+e_D; c_{D+1}..c_{2D} = -e_1..-e_D.
 *   In 2D this is the paper's counter-clockwise order (1,0),(0,1),(-1,0),(0,-1).
 *   The 3D order is not given by the paper; any order gives the same fields.
 *
 * Readings of the paper taken here (each is also listed in the design notes):
 *  R1  c_L^2 = sum_i w_i c_ix^2 = (1-w0)/D, the per-axis second moment of the
 *      weights (the paper's "sum_i w_i c_i^2" read per axis, which is what
 *      makes Eqs. 9-11 hold and gives its (1-w0)/3 for the 6+1 lattice).
 *  R2  B_beta is read from the first moment R_{a b k} = sum_i c_ik g_iab as
 *      B_beta = sum_{alpha != beta} R_{alpha beta alpha} (Eq. 10 with
 *      gamma = alpha, summed over the D-1 tensor components that carry it),
 *      and the equilibrium of Eq. 8 is built with B/(D-1).  In 2D this is
 *      literally Eq. 8; in 3D it is the reading that is stable.  The wave
 *      speed is then c_eff^2 = c_L^2/(D-1).
 *  R3  The source of Eq. 3 uses the physical wave speed c_eff^2 and
 *      1/eps0 = mu0 c_eff^2; the frequency-dispersive (convolution) part of
 *      Eq. 3 is not modelled (the paper defers it).
 *  R4  Order within a step: moments from the pre-collision g; fields are
 *      reported from those moments; T is added once, post-collision, with the
 *      source at time t (Eq. 17); then streaming (Eq. 18).
 *  R5  grad(ln mu) by second-order central differences, periodic.
 *  R6  Periodic boundaries in every direction, unless walls are asked for.
 *  R7  Walls (the paper treats periodic domains only and leaves reflecting
 *      and absorbing boundaries open): a wall sits half a site beyond the
 *      first and last site of an axis.  A particle that streams across it
 *      comes back to the site it left, in the opposite direction, times
 *      s = +1 (halfway bounce-back) or s = -1 (anti-bounce-back).  In 2D the
 *      state then evolves exactly as the periodic state on a domain twice as
 *      long with the mirror image of the medium, fields and currents
 *      (populations i <-> opposite(i) times s): s = -1 makes E_z and B_normal
 *      odd about the wall (a perfect electric conductor, PEC); s = +1 makes
 *      the tangential B odd (a perfect magnetic conductor, PMC).  grad ln mu
 *      at the first / last site uses the mirror image of mu (the one-sided
 *      difference halved), as the doubled domain would.  In 3D (and
 *      consistently in 2D) the factor is per tensor component: a wall across
 *      axis a reflects g_bc with (b == a ? -1 : 1) (c == a ? -1 : 1), the
 *      geometric mirror of the tensor, times +1 (PEC) or -1 (PMC); in 2D the
 *      component xy then gets -1 (PEC) or +1 (PMC) at either wall, as above.
 *  R8  Absorbing layer of L sites inside each wall: after the collision the
 *      populations of a site at distance i = 0 .. L-1 from the wall-adjacent
 *      site are multiplied by 1 - gamma_i, gamma_i = gamma_max ((L - i)/L)^2,
 *      the factors of two axes multiplied at corners.  Scaling E and B by the
 *      same factor damps them equally (matched electric and magnetic
 *      conductivity), so the layer keeps the wave impedance of the medium.
 *  R9  Frequency-dispersive permittivity (the convolution term of Eq. 3,
 *      which the paper defers to auxiliary differential equations): one
 *      Drude-Lorentz pole per site, d_t J + gamma J + wr^2 P = wp^2 E with
 *      J = d_t P (P in units of E: eps(omega) = eps_inf (1 + wp^2 / (wr^2 -
 *      omega^2 - i gamma omega))).  Entering P as the source S = -d_t P of
 *      Eq. 3 makes the scheme unstable (the source's (c^2/2) Lap S part acts
 *      on the accumulated current); it enters instead as the displacement
 *      form of the same equations: the lattice's zeroth moment carries
 *      D/eps_inf (no source: d_t D = curl H), the field is E = D/eps_inf - P,
 *      and the equilibrium keeps its zeroth and first moments while its
 *      second moment Lambda_ab takes E (Lambda_ab += eps_gab P_g: +1/2 of
 *      that on every moving population, -D times it on the rest one).  J
 *      lives at half steps, P at whole ones; at time t, from the pre-collision
 *      E(t) = D(t)/eps_inf - P(t):
 *        J(t+1/2) = [(1 - gamma/2) J(t-1/2) + wp^2 E(t) - wr^2 P(t)] / (1 + gamma/2)
 *        P(t+1)   = P(t) + J(t+1/2)
 *      and the collision at t uses P(t).  A uniform medium then has the plane
 *      waves 4 sin^2(omega/2) = 4 c^2 (sin^2(kx/2) + sin^2(ky/2)) + wp^2
 *      (wr = gamma = 0), and stays stable where wp^2 + wr^2 <= 4 w0.
 *  R10 Anisotropic media (the paper: different weights for particles moving
 *      along different axes): a uniform in-plane relative permeability
 *      tensor diag(mu_xx, mu_yy) in 2D, eps_r per site.  The lattice speed of
 *      axis a is c_a^2 = f_a cbar^2 with cbar^2 = c_ref^2 / (eps_r sqrt(mu_xx
 *      mu_yy)) (stored as c_L^2), f_x = r, f_y = 1/r, r = sqrt(mu_xx / mu_yy):
 *      c_x^2 = c_ref^2 / (eps_r mu_yy) is the speed of a wave moving along x.
 *      Moving particles of axis a carry w = c_a^2/2, so w0 = 1 - sum_a c_a^2;
 *      Lambda = cbar^2 sum_i g_i gives E (E_z = -cbar^2 sigma); the first
 *      moments carry H up to a uniform factor, so B_x = s_x (g_4 - g_2), B_y =
 *      s_y (g_1 - g_3) with s_x = r, s_y = 1/r; the equilibrium has the same
 *      moments as Eq. 8 with c^2 read per axis.  The source S of Eq. 3 uses
 *      mu = sqrt(mu_xx mu_yy) (so 1/eps0 = c_ref^2/eps_r).  The update is then
 *      exactly 2D TM Maxwell with that tensor and a heterogeneous eps_r, and
 *      r = 1 is the isotropic scheme with mu_r = mu_xx.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Floating-point type of every quantity.  The oracle is FP64 (the default); building with -DOR_REAL=float
 * gives an FP32 build of the same source, used only to time a like-for-like CPU figure, never as a reference. */
#ifndef OR_REAL
#define OR_REAL double
#endif
typedef OR_REAL real;

#define MAXQ 7
#define MAXD 3

typedef struct {
    int D, Q, nx, ny, nz;
    long nsite;
    int c[MAXQ][3]; /* lattice velocities, unused axes 0 */
    real fa[3];   /* per-axis lattice speeds c_a^2 = fa[a] c_L^2 (reading R10; 1 when isotropic) */
    real bs[3];   /* B_b = bs[b] x its first moment (reading R10; 1 when isotropic) */
} lattice_t;

/* Lattice of Sec. "Lattice BGK formulation": 2D rest particles plus +/- unit
 * speeds along each axis. */
static void make_lattice(lattice_t *L, int D, int nx, int ny, int nz) {
    L->D = D;
    L->Q = 2 * D + 1;
    L->nx = nx;
    L->ny = ny;
    L->nz = (D == 3) ? nz : 1;
    L->nsite = (long)L->nx * L->ny * L->nz;
    memset(L->c, 0, sizeof(L->c));
    for (int a = 0; a < 3; a++) L->fa[a] = L->bs[a] = 1.0;
    for (int a = 0; a < D; a++) {
        L->c[1 + a][a] = +1;
        L->c[1 + D + a][a] = -1;
    }
}

/* Levi-Civita symbol epsilon_{abc}, indices 0..2: +1 on even permutations of
 * (0,1,2), -1 on odd ones, 0 when an index repeats. */
static const real LEVI[3][3][3] = {
    {{0, 0, 0}, {0, 0, 1}, {0, -1, 0}},
    {{0, 0, -1}, {0, 0, 0}, {1, 0, 0}},
    {{0, 1, 0}, {-1, 0, 0}, {0, 0, 0}},
};
static inline real levi(int a, int b, int c) { return LEVI[a][b][c]; }

/* Periodic wrap of coordinate v + d into [0, n), for |d| <= n. */
static inline long wrap(long v, int d, long n) {
    v += d;
    if (v >= n) v -= n;
    if (v < 0) v += n;
    return v;
}

/* Site index of (x + dx, y + dy, z + dz) with periodic wrap, |d| <= 1. */
static long shifted(const lattice_t *L, long s, int dx, int dy, int dz) {
    long x = s % L->nx;
    long y = (s / L->nx) % L->ny;
    long z = s / ((long)L->nx * L->ny);
    return wrap(x, dx, L->nx) + L->nx * (wrap(y, dy, L->ny) + L->ny * wrap(z, dz, L->nz));
}

/* Coordinate v + d along an axis of length n with boundary kind `bc` (0 = periodic, else walls): the periodic
 * wrap, or the mirror image inside the wall (-1 -> 0, n -> n-1), for |d| <= 1. */
static inline long mirror_or_wrap(long v, int d, long n, int bc) {
    if (!bc) return wrap(v, d, n);
    v += d;
    if (v < 0) return -1 - v;
    if (v >= n) return 2 * n - 1 - v;
    return v;
}

/* Damping factor 1 - gamma of reading R8 at coordinate v of an axis of length n (1 outside the layer). */
static real layer_factor(long v, long n, int layer, real gamma_max) {
    long i = v < n - 1 - v ? v : n - 1 - v; /* distance from the nearer wall-adjacent site */
    if (layer <= 0 || i >= layer) return 1.0;
    real r = (real)(layer - i) / layer;
    return 1.0 - gamma_max * r * r;
}

static inline real *G(const lattice_t *L, real *g, long s, int i) {
    return g + ((s * L->Q + i) * L->D) * L->D;
}

/* Anisotropy ratio r = sqrt(mu_xx / mu_yy) of reading R10 (2D; r = 1: isotropic). */
static void set_axes(lattice_t *L, real r) {
    if (L->D != 2 || !(r > 0.0) || r == 1.0) return;
    L->fa[0] = r;
    L->fa[1] = 1.0 / r;
    L->bs[0] = r;
    L->bs[1] = 1.0 / r;
}

/* axis along which direction i moves (-1 for the rest particle) */
static int axis_of(const lattice_t *L, int i) {
    for (int a = 0; a < L->D; a++)
        if (L->c[i][a]) return a;
    return -1;
}

/* Lattice weights (Sec. "Lattice BGK formulation"): moving particles all get
 * w_i = (1 - w0)/(2D); the rest particle gets w0.  With per-axis speeds
 * (reading R10) a moving particle of axis a gets (1 - w0) fa[a] / (2 sum_b fa[b])
 * = c_a^2 / 2. */
static real weight(const lattice_t *L, int i, real w0) {
    if (i == 0) return w0;
    real sum = 0.0;
    for (int b = 0; b < L->D; b++) sum += L->fa[b];
    return (1.0 - w0) * L->fa[axis_of(L, i)] / (2.0 * sum);
}

/* ------------------------------------------------------------------------ */
/* Medium: Eq. 3's heterogeneity and c = 1/sqrt(mu0 eps0).                   */
/* ------------------------------------------------------------------------ */

/*
 * From relative permittivity eps_r and permeability mu_r per site:
 *   c_eff^2 = c_ref^2 / (eps_r mu_r)             (c = 1/sqrt(mu0 eps0))
 *   c_L^2   = (D-1) c_eff^2                       (reading R2)
 *   w0      = 1 - D c_L^2                         (reading R1)
 *   dlnmu_k = (ln mu(x+e_k) - ln mu(x-e_k)) / 2   (reading R5)
 * mu_r may be NULL (mu = 1).  Returns the number of sites whose w0 falls
 * outside [0, 1) or whose inputs are not finite and positive.
 */
long or_medium(int D, int nx, int ny, int nz, real c_ref2, const real *eps_r, const real *mu_r, const int *bc,
               real aniso_r, real *ceff2, real *cL2, real *w0, real *mu, real *dlnmu) {
    lattice_t L;
    make_lattice(&L, D, nx, ny, nz);
    set_axes(&L, aniso_r);
    real fsum = 0.0;
    for (int a = 0; a < D; a++) fsum += L.fa[a];
    long bad = 0;
    for (long s = 0; s < L.nsite; s++) {
        real e = eps_r[s];
        real m = mu_r ? mu_r[s] : 1.0;
        if (!(e > 0.0) || !(m > 0.0) || !isfinite(e) || !isfinite(m)) {
            bad++;
            e = 1.0;
            m = 1.0;
        }
        ceff2[s] = c_ref2 / (e * m);
        cL2[s] = (D - 1) * ceff2[s];
        w0[s] = 1.0 - fsum * cL2[s]; /* 1 - D c_L^2, or 1 - sum_a c_a^2 (reading R10) */
        mu[s] = m;
        if (!(w0[s] >= 0.0 && w0[s] < 1.0)) bad++;
    }
    for (long s = 0; s < L.nsite; s++) {
        const long xyz[3] = {s % L.nx, (s / L.nx) % L.ny, s / ((long)L.nx * L.ny)};
        const long n[3] = {L.nx, L.ny, L.nz};
        for (int k = 0; k < 3; k++) dlnmu[3 * s + k] = 0.0;
        for (int k = 0; k < D; k++) {
            long p[3] = {xyz[0], xyz[1], xyz[2]}, m[3] = {xyz[0], xyz[1], xyz[2]};
            p[k] = mirror_or_wrap(xyz[k], +1, n[k], bc ? bc[k] : 0);
            m[k] = mirror_or_wrap(xyz[k], -1, n[k], bc ? bc[k] : 0);
            long sp = p[0] + L.nx * (p[1] + L.ny * p[2]);
            long sm = m[0] + L.nx * (m[1] + L.ny * m[2]);
            dlnmu[3 * s + k] = 0.5 * (log(mu[sp]) - log(mu[sm]));
        }
    }
    return bad;
}

/* ------------------------------------------------------------------------ */
/* Moments (Eqs. 9, 10 and the field recovery after Eq. 6).                  */
/* ------------------------------------------------------------------------ */

/*
 * Moments of the pre-collision tensor distribution at one site:
 *   Lambda_ab = c_L^2 sum_i g_iab                        (Eq. 9)
 *   E_g       = -1/2 eps_{g a b} Lambda_ab               (recovery of E from Lambda)
 *   R_abk     = sum_i c_ik g_iab                         (Eq. 10)
 *   B_b       = sum_{a != b} R_{a b a}                    (reading R2)
 * E and B are 3-vectors; in 2D only E_z, B_x, B_y can be non-zero.
 */
static void site_moments(const lattice_t *L, const real *gs, real cL2, real Lam[MAXD][MAXD], real E[3],
                         real B[3]) {
    const int D = L->D, Q = L->Q;
    real R[MAXD][MAXD][MAXD];
    for (int a = 0; a < D; a++)
        for (int b = 0; b < D; b++) {
            real sum = 0.0;
            for (int i = 0; i < Q; i++) sum += gs[(i * D + a) * D + b];
            Lam[a][b] = cL2 * sum;
            for (int k = 0; k < D; k++) {
                real r = 0.0;
                for (int i = 0; i < Q; i++) r += L->c[i][k] * gs[(i * D + a) * D + b];
                R[a][b][k] = r;
            }
        }
    for (int g = 0; g < 3; g++) {
        real e = 0.0;
        for (int a = 0; a < D; a++)
            for (int b = 0; b < D; b++) e += levi(g, a, b) * Lam[a][b];
        E[g] = -0.5 * e;
    }
    for (int b = 0; b < 3; b++) {
        real v = 0.0;
        if (b < D)
            for (int a = 0; a < D; a++)
                if (a != b) v += R[a][b][a];
        B[b] = L->bs[b] * v;
    }
}

/* Local equilibrium, Eq. 8:
 *   g^(0)_iab = (w_i / c_L^2) [ Lambda_ab + c_ia Bq_b - c_ib Bq_a ]
 * with Bq = B/(D-1) (reading R2).  With per-axis speeds (reading R10) the c^2
 * of the B term is that of the particle's axis, c_a^2 = fa[a] c_L^2, and Bq is
 * the first moment B/bs. */
static void equilibrium(const lattice_t *L, real cL2, real w0, real Lam[MAXD][MAXD], const real B[3],
                        real *geq) {
    const int D = L->D, Q = L->Q;
    real Bq[3];
    for (int k = 0; k < 3; k++) Bq[k] = B[k] / (D - 1) / L->bs[k];
    for (int i = 0; i < Q; i++) {
        const real w = weight(L, i, w0), ax = i == 0 ? 1.0 : L->fa[axis_of(L, i)];
        for (int a = 0; a < D; a++)
            for (int b = 0; b < D; b++)
                geq[(i * D + a) * D + b] =
                    (w / cL2) * Lam[a][b] + (w / (ax * cL2)) * (L->c[i][a] * Bq[b] - L->c[i][b] * Bq[a]);
    }
}

/* Initial state g = g^(0)(E, B): Lambda_ab = -eps_{g a b} E_g (Sec. "The
 * Maxwell Equations", conservative form) and B as given.  E, B are
 * [nsite][3]; either may be NULL (zero). */
void or_init(int D, int nx, int ny, int nz, const real *cL2, const real *w0, const real *E, const real *B,
             real *g, real aniso_r) {
    lattice_t L;
    make_lattice(&L, D, nx, ny, nz);
    set_axes(&L, aniso_r);
    for (long s = 0; s < L.nsite; s++) {
        real Lam[MAXD][MAXD], Bs[3] = {0, 0, 0};
        for (int a = 0; a < D; a++)
            for (int b = 0; b < D; b++) {
                real v = 0.0;
                if (E)
                    for (int k = 0; k < 3; k++) v -= levi(k, a, b) * E[3 * s + k];
                Lam[a][b] = v;
            }
        if (B)
            for (int k = 0; k < 3; k++) Bs[k] = B[3 * s + k];
        equilibrium(&L, cL2[s], w0[s], Lam, Bs, G(&L, g, s, 0));
    }
}

/* E and B ([nsite][3]) of a pre-collision state. */
void or_fields(int D, int nx, int ny, int nz, const real *cL2, const real *g, real *E, real *B,
               real aniso_r) {
    lattice_t L;
    make_lattice(&L, D, nx, ny, nz);
    set_axes(&L, aniso_r);
#pragma omp parallel for schedule(static)
    for (long s = 0; s < L.nsite; s++) {
        real Lam[MAXD][MAXD];
        site_moments(&L, g + s * L.Q * D * D, cL2[s], Lam, E + 3 * s, B + 3 * s);
    }
}

/* ------------------------------------------------------------------------ */
/* Collision (Eq. 17) with the tensor source T of Sec. "Lattice BGK          */
/* formulation" and the source S of Eq. 3.                                   */
/* ------------------------------------------------------------------------ */

/*
 * One site's post-collision state, Eq. 17 with Delta t = 1, tau = 1/2 (the
 * non-dissipative choice of Sec. "Lattice BGK formulation"):
 *   g'_iab = (1 - dt/tau) g_iab + (dt/tau) g^(0)_iab + T_iab dt
 *   T_iab  = -(w_i/c_L^2) eps_{g a b} S_g
 *   S_g    = c_eff^2 eps_{g b k} B_b d_k ln(mu) - mu c_eff^2 j_g     (Eq. 3, R3)
 * j is the current density at this site and time (3-vector).
 */
static void collide_site(const lattice_t *L, real cL2, real w0, real ceff2, real mus, const real dlnmu[3],
                         const real j[3], const real *ppol, const real *gin, real *gout, real E[3],
                         real B[3]) {
    const int D = L->D, Q = L->Q;
    const real dt = 1.0, tau = 0.5;
    real Lam[MAXD][MAXD], S[3], geq[MAXQ * MAXD * MAXD];
    site_moments(L, gin, cL2, Lam, E, B);
    if (ppol) /* reading R9: the field is D/eps_inf - P */
        for (int g = 0; g < 3; g++) E[g] -= ppol[g];
    for (int g = 0; g < 3; g++) {
        real curl = 0.0;
        for (int b = 0; b < 3; b++)
            for (int k = 0; k < 3; k++) curl += levi(g, b, k) * B[b] * dlnmu[k];
        S[g] = ceff2 * curl - mus * ceff2 * j[g];
    }
    equilibrium(L, cL2, w0, Lam, B, geq);
    if (ppol) {
        /* reading R9: second moment Lambda_ab + eps_gab P_g, zeroth and first moments unchanged */
        for (int a = 0; a < D; a++)
            for (int b = 0; b < D; b++) {
                real dl = 0.0;
                for (int g = 0; g < 3; g++) dl += levi(g, a, b) * ppol[g];
                real fsum = 0.0; /* sum_a c_a^2 / c_L^2: D when isotropic */
                for (int k = 0; k < D; k++) fsum += L->fa[k];
                for (int i = 0; i < Q; i++)
                    geq[(i * D + a) * D + b] += (i == 0 ? -fsum : 0.5 * L->fa[axis_of(L, i)]) * dl;
            }
    }
    for (int i = 0; i < Q; i++) {
        real wc = weight(L, i, w0) / cL2;
        for (int a = 0; a < D; a++)
            for (int b = 0; b < D; b++) {
                real T = 0.0;
                for (int g = 0; g < 3; g++) T -= wc * levi(g, a, b) * S[g];
                int n = (i * D + a) * D + b;
                gout[n] = (1.0 - dt / tau) * gin[n] + (dt / tau) * geq[n] + T * dt;
            }
    }
}

/* Field sample of a receiver: comp 0..2 = E_x..E_z, 3..5 = B_x..B_z. */
static real pick(const real E[3], const real B[3], int comp) { return comp < 3 ? E[comp] : B[comp - 3]; }

typedef struct {
    int nsrc;
    const long *site;
    const int *comp;    /* 0..2: component of j */
    const real *amp;  /* [nsrc][nt]: j(t) */
    int nt;
} sources_t;

/* j at a site and time, summed over the point sources there. */
static void current_at(const sources_t *src, long s, int t, real j[3]) {
    j[0] = j[1] = j[2] = 0.0;
    if (!src) return;
    for (int k = 0; k < src->nsrc; k++)
        if (src->site[k] == s && t >= 0 && t < src->nt) j[src->comp[k]] += src->amp[(long)k * src->nt + t];
}

/*
 * Advance nsteps time steps, Eqs. 17 then 18.  g holds the pre-collision
 * state at time t0 on entry and at t0 + nsteps on exit.  j(t) is taken from
 * amp[k][t] for t in [0, nt).  Receivers record (before each collision) the
 * field at time t0 + n into traces[r][n], n = 0..nsteps-1.  bc[a] (NULL = all
 * periodic) is the boundary of axis a: 0 periodic, 1 PEC wall, 2 PMC wall
 * (readings R6-R7); `layer` > 0 adds the absorbing layer of reading R8 inside
 * every wall.  Returns 0.
 */
int or_run(int D, int nx, int ny, int nz, const real *cL2, const real *w0, const real *ceff2, const real *mu,
           const real *dlnmu, real *g, int t0, int nsteps, int nsrc, const long *src_site, const int *src_comp,
           const real *src_amp, int nt, int nrec, const long *rec_site, const int *rec_comp, real *traces,
           const int *bc, int layer, real gamma_max, const real *wp2, const real *wr2, const real *gam,
           real *Jpol, real *Ppol, real aniso_r) {
    lattice_t L;
    make_lattice(&L, D, nx, ny, nz);
    set_axes(&L, aniso_r);
    int kind[3] = {0, 0, 0};
    for (int a = 0; bc && a < 3; a++) kind[a] = a < D ? bc[a] : 0;
    const long len[3] = {L.nx, L.ny, L.nz};
    const long per = (long)L.Q * D * D;
    real *gpost = malloc(sizeof(real) * per * L.nsite);
    real *E = malloc(sizeof(real) * 3 * L.nsite);
    real *B = malloc(sizeof(real) * 3 * L.nsite);
    sources_t src = {nsrc, src_site, src_comp, src_amp, nt};
    for (int n = 0; n < nsteps; n++) {
        int t = t0 + n;
        /* collision at every site (Eq. 17) */
#pragma omp parallel for schedule(static)
        for (long s = 0; s < L.nsite; s++) {
            real j[3];
            current_at(&src, s, t, j);
            real pt[3];
            const real *ppol = NULL;
            if (wp2) {
                /* the pole's update from the pre-collision E(t) = D/eps_inf - P(t) (reading R9) */
                real Lam[MAXD][MAXD], Et[3], Bt[3];
                site_moments(&L, g + s * per, cL2[s], Lam, Et, Bt);
                const real gm = gam ? gam[s] : 0.0, om = wr2 ? wr2[s] : 0.0;
                for (int a = 0; a < 3; a++) {
                    pt[a] = Ppol[3 * s + a];
                    const real ea = Et[a] - pt[a];
                    const real jn = ((1.0 - 0.5 * gm) * Jpol[3 * s + a] + wp2[s] * ea - om * pt[a]) / (1.0 + 0.5 * gm);
                    Jpol[3 * s + a] = jn;
                    Ppol[3 * s + a] = pt[a] + jn;
                }
                ppol = pt; /* the collision at t uses P(t) */
            }
            collide_site(&L, cL2[s], w0[s], ceff2[s], mu[s], dlnmu + 3 * s, j, ppol, g + s * per, gpost + s * per,
                         E + 3 * s, B + 3 * s);
            /* absorbing layer (reading R8): scale the post-collision populations */
            const long xyz[3] = {s % L.nx, (s / L.nx) % L.ny, s / ((long)L.nx * L.ny)};
            real f = 1.0;
            for (int a = 0; a < D; a++)
                if (kind[a]) f *= layer_factor(xyz[a], len[a], layer, gamma_max);
            if (f != 1.0)
                for (long k = 0; k < per; k++) gpost[s * per + k] *= f;
        }
        for (int r = 0; r < nrec; r++) traces[(long)r * nsteps + n] = pick(E + 3 * rec_site[r], B + 3 * rec_site[r], rec_comp[r]);
        /* streaming (Eq. 18): g_i(x + c_i, t+1) = g'_i(x, t) */
#pragma omp parallel for schedule(static)
        for (long s = 0; s < L.nsite; s++) {
            const long x = s % L.nx, y = (s / L.nx) % L.ny, z = s / ((long)L.nx * L.ny);
            for (int i = 0; i < L.Q; i++) {
                /* a particle that would cross a wall (reading R7) returns to s in the opposite direction, times
                 * -1 at a PEC wall and +1 at a PMC wall */
                const long xyz[3] = {x + L.c[i][0], y + L.c[i][1], z + L.c[i][2]};
                int crossed = -1;
                for (int a = 0; a < D; a++)
                    if (kind[a] && (xyz[a] < 0 || xyz[a] >= len[a])) crossed = a;
                if (crossed >= 0) {
                    const int io = i == 0 ? 0 : (i <= D ? i + D : i - D); /* opposite direction */
                    const real wall = kind[crossed] == 1 ? 1.0 : -1.0;   /* PEC: the geometric mirror */
                    const real *src = G(&L, gpost, s, i);
                    real *dst = G(&L, g, s, io);
                    for (int b = 0; b < D; b++)
                        for (int c = 0; c < D; c++)
                            dst[b * D + c] = wall * (b == crossed ? -1.0 : 1.0) * (c == crossed ? -1.0 : 1.0) *
                                             src[b * D + c];
                    continue;
                }
                long d = wrap(x, L.c[i][0], L.nx) + L.nx * (wrap(y, L.c[i][1], L.ny) + L.ny * wrap(z, L.c[i][2], L.nz));
                memcpy(G(&L, g, d, i), G(&L, gpost, s, i), sizeof(real) * D * D);
            }
        }
    }
    free(gpost);
    free(E);
    free(B);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Diagnostics (Sec. "Heterogeneous media"; Eq. 19's concern with div B).    */
/* ------------------------------------------------------------------------ */

/*
 * out[0] = field energy  sum_x sum_a (B_a^2 + E_a^2 / c_eff^2)   (Sec. "Heterogeneous media")
 * out[1] = sum_x sum_i sum_ab g_iab^2 / w_i  (terms with w_i = 0 skipped)
 * out[2] = sqrt( sum_x (div B)^2 ), div B by periodic central differences
 * Sums run over sites in order, serially.
 */
void or_diagnostics(int D, int nx, int ny, int nz, const real *cL2, const real *w0, const real *ceff2,
                    const real *g, real *out, real aniso_r) {
    lattice_t L;
    make_lattice(&L, D, nx, ny, nz);
    set_axes(&L, aniso_r);
    real *E = malloc(sizeof(real) * 3 * L.nsite), *B = malloc(sizeof(real) * 3 * L.nsite);
    or_fields(D, nx, ny, nz, cL2, g, E, B, aniso_r);
    real en = 0.0, inv = 0.0, dv = 0.0;
    for (long s = 0; s < L.nsite; s++) {
        for (int a = 0; a < 3; a++) en += B[3 * s + a] * B[3 * s + a] + E[3 * s + a] * E[3 * s + a] / ceff2[s];
        for (int i = 0; i < L.Q; i++) {
            real w = weight(&L, i, w0[s]);
            if (w == 0.0) continue;
            const real *gi = g + (s * L.Q + i) * D * D;
            for (int n = 0; n < D * D; n++) inv += gi[n] * gi[n] / w;
        }
        real div = 0.0;
        for (int k = 0; k < D; k++) {
            int dp[3] = {0, 0, 0};
            dp[k] = 1;
            long sp = shifted(&L, s, dp[0], dp[1], dp[2]);
            long sm = shifted(&L, s, -dp[0], -dp[1], -dp[2]);
            div += 0.5 * (B[3 * sp + k] - B[3 * sm + k]);
        }
        dv += div * div;
    }
    out[0] = en;
    out[1] = inv;
    out[2] = sqrt(dv);
    free(E);
    free(B);
}

/* ------------------------------------------------------------------------ */
/* Adjoint of the time stepping (not in the paper: gradient of a receiver    */
/* misfit with respect to the permittivity).                                 */
/* ------------------------------------------------------------------------ */

/*
 * Post-collision state of one site as a function of c_L^2 alone, with
 * w0 = 1 - D c_L^2 and c_eff^2 = c_L^2/(D-1) (readings R1, R2).  Written out,
 * every term of Eq. 17 is affine in c_L^2 for fixed g, mu and j:
 *   moving i: (w_i/c_L^2) = 1/(2D) * D = 1/2 and Lambda = c_L^2 sum g,
 *   rest i  : w0 = 1 - D c_L^2,
 *   S       : proportional to c_eff^2, multiplied by w_i/c_L^2 in T.
 * The adjoint below uses that: d g'/d c_L^2 = (g'(2c) - g'(c)) / c exactly.
 */
static void collide_c(const lattice_t *L, real c, real mus, const real dlnmu[3], const real j[3],
                      const real *gin, real *gout) {
    real E[3], B[3];
    collide_site(L, c, 1.0 - L->D * c, c / (L->D - 1), mus, dlnmu, j, NULL, gin, gout, E, B);
}

/*
 * Gradient of the misfit
 *   Lmis = 1/2 sum_{n<nsteps} sum_r ( F_r(t0+n) - obs[r][n] )^2,
 * F_r the receiver fields recorded by or_run, with respect to eps_r at every
 * site, for a run that starts from g0 (pre-collision state at t0, held fixed).
 * Backward recursion over stored states: with  g^{n+1} = S (M_n g^n + T_n),
 *   lam^{N} = 0,  lam^n = M_n^T S^T lam^{n+1} + dl_n/dg^n,
 *   dL/dc_L^2(x) += (S^T lam^{n+1})(x) . d(M_n g^n + T_n)(x)/dc_L^2 + dl_n/dc_L^2(x)
 * and  dL/deps_r = dL/dc_L^2 * dc_L^2/deps_r = -dL/dc_L^2 * c_L^2 / eps_r.
 * M_n^T is applied as the transpose of the explicit local matrix of
 * collide_c (built column by column from unit vectors).
 * Returns the misfit; grad_eps is [nsite].
 */
real or_adjoint(int D, int nx, int ny, int nz, const real *eps_r, const real *cL2, const real *mu,
                  const real *dlnmu, const real *g0, int t0, int nsteps, int nsrc, const long *src_site,
                  const int *src_comp, const real *src_amp, int nt, int nrec, const long *rec_site,
                  const int *rec_comp, const real *obs, real *grad_eps) {
    lattice_t L;
    make_lattice(&L, D, nx, ny, nz);
    const long per = (long)L.Q * D * D;
    const long ns = L.nsite;
    real *w0 = malloc(sizeof(real) * ns), *ceff2 = malloc(sizeof(real) * ns);
    for (long s = 0; s < ns; s++) {
        w0[s] = 1.0 - D * cL2[s];
        ceff2[s] = cL2[s] / (D - 1);
    }
    /* forward pass, keeping every pre-collision state */
    real *states = malloc(sizeof(real) * per * ns * (nsteps + 1));
    real *traces = malloc(sizeof(real) * (nrec > 0 ? nrec : 1) * (nsteps > 0 ? nsteps : 1));
    memcpy(states, g0, sizeof(real) * per * ns);
    for (int n = 0; n < nsteps; n++) {
        memcpy(states + (long)(n + 1) * per * ns, states + (long)n * per * ns, sizeof(real) * per * ns);
        real *tr_n = malloc(sizeof(real) * (nrec > 0 ? nrec : 1));
        or_run(D, nx, ny, nz, cL2, w0, ceff2, mu, dlnmu, states + (long)(n + 1) * per * ns, t0 + n, 1, nsrc, src_site,
               src_comp, src_amp, nt, nrec, rec_site, rec_comp, tr_n, NULL, 0, 0.0, NULL, NULL, NULL, NULL, NULL, 1.0);
        for (int r = 0; r < nrec; r++) traces[(long)r * nsteps + n] = tr_n[r];
        free(tr_n);
    }
    real misfit = 0.0;
    for (int r = 0; r < nrec; r++)
        for (int n = 0; n < nsteps; n++) {
            real d = traces[(long)r * nsteps + n] - obs[(long)r * nsteps + n];
            misfit += 0.5 * d * d;
        }
    /* backward pass */
    real *lam = calloc(per * ns, sizeof(real));   /* lam^{n+1} */
    real *lpost = malloc(sizeof(real) * per * ns); /* S^T lam^{n+1} */
    real *gcl = calloc(ns, sizeof(real));          /* dL/dc_L^2 */
    for (int n = nsteps - 1; n >= 0; n--) {
        const real *gn = states + (long)n * per * ns;
        /* S^T: streaming moved g'_i(x) to x + c_i, so its transpose pulls back */
        for (long s = 0; s < ns; s++)
            for (int i = 0; i < L.Q; i++) {
                long d = shifted(&L, s, L.c[i][0], L.c[i][1], L.c[i][2]);
                memcpy(G(&L, lpost, s, i), G(&L, lam, d, i), sizeof(real) * D * D);
            }
#pragma omp parallel for schedule(static)
        for (long s = 0; s < ns; s++) {
            real j[3], zero[3] = {0, 0, 0};
            sources_t src = {nsrc, src_site, src_comp, src_amp, nt};
            current_at(&src, s, t0 + n, j);
            const real *gs = gn + s * per;
            const real *ls = lpost + s * per;
            real *out = lam + s * per;
            /* lam^n(x) = M^T lpost(x): column m of M is collide_c(unit e_m) with j = 0 */
            real unit[MAXQ * MAXD * MAXD], col[MAXQ * MAXD * MAXD];
            for (long m = 0; m < per; m++) {
                memset(unit, 0, sizeof(unit));
                unit[m] = 1.0;
                collide_c(&L, cL2[s], mu[s], dlnmu + 3 * s, zero, unit, col);
                real v = 0.0;
                for (long q = 0; q < per; q++) v += col[q] * ls[q];
                out[m] = v;
            }
            /* dL/dc_L^2 through the collision and source (affine in c_L^2) */
            real ga[MAXQ * MAXD * MAXD], gb[MAXQ * MAXD * MAXD];
            collide_c(&L, 2.0 * cL2[s], mu[s], dlnmu + 3 * s, j, gs, ga);
            collide_c(&L, cL2[s], mu[s], dlnmu + 3 * s, j, gs, gb);
            real v = 0.0;
            for (long q = 0; q < per; q++) v += ls[q] * (ga[q] - gb[q]) / cL2[s];
            gcl[s] += v;
        }
        /* receivers: dl_n/dg^n and dl_n/dc_L^2 (E = -1/2 eps Lambda, Lambda = c_L^2 sum g) */
        for (int r = 0; r < nrec; r++) {
            long s = rec_site[r];
            int comp = rec_comp[r];
            real d = traces[(long)r * nsteps + n] - obs[(long)r * nsteps + n];
            const real *gs = gn + s * per;
            real *out = lam + s * per;
            for (int i = 0; i < L.Q; i++)
                for (int a = 0; a < D; a++)
                    for (int b = 0; b < D; b++) {
                        int m = (i * D + a) * D + b;
                        if (comp < 3) {
                            real e = -0.5 * levi(comp, a, b);
                            out[m] += d * e * cL2[s];
                            gcl[s] += d * e * gs[m];
                        } else {
                            int bc = comp - 3; /* B_bc = sum_{a != bc} sum_i c_ia g_{i a bc} */
                            if (b == bc && a != bc) out[m] += d * L.c[i][a];
                        }
                    }
        }
    }
    for (long s = 0; s < ns; s++) grad_eps[s] = -gcl[s] * cL2[s] / eps_r[s];
    free(lam);
    free(lpost);
    free(gcl);
    free(states);
    free(traces);
    free(w0);
    free(ceff2);
    return misfit;
}

/* Number of OpenMP threads the oracle runs with (1 without OpenMP). */
/* Set the number of OpenMP threads (timing on one core); returns the number in effect. */
int or_set_threads(int n) {
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    extern int omp_get_max_threads(void);
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

int or_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
