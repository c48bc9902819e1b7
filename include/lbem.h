/*
 * lbem.h -- C ABI of the GB300 (sm_103a) lattice-Boltzmann Maxwell solver.
 *
 * The method is that of Hanasoge, Succi & Orszag, "Lattice Boltzmann Method
 * for Electromagnetic Wave Propagation" (EPL; arXiv:1108.2651): an
 * antisymmetric tensor ("pseudo-vector") distribution g_{i,alpha,beta} on the
 * D2Q5 ("4+1") or D3Q7 ("6+1") lattice, BGK collision at tau = dt/2 with the
 * local equilibrium of Eq. 8 and the tensor source T_i built from Eq. 3's
 * heterogeneity source S, followed by streaming (Eqs. 17-18); E and B are
 * recovered from the zeroth and first moments (Eqs. 9-10).
 *
 * Conventions (every entry point):
 *  - Every call returns an lbem_status; on failure a thread-local message is
 *    available from lbem_last_error().  A handle stays usable after any
 *    LBEM_ERR_ARG / LBEM_ERR_MEDIUM / LBEM_ERR_STATE failure.
 *  - Grids are dense, C order: site s = x + nx*(y + ny*z) (nz = 1 in 2D).
 *    Vector fields are component-major: F[c*nsite + s], c = 0,1,2 for x,y,z.
 *  - Pointer arguments to grid-sized arrays may be host or device memory
 *    (unified addressing); inputs are copied before the call returns or are
 *    read by work enqueued on the handle's stream, outputs are written by
 *    work enqueued on the stream.  Caller-owned memory is never freed or
 *    retained past the call.  Host output buffers are complete when the call
 *    returns; device outputs are complete when the stream reaches the call.
 *  - Work runs asynchronously on the handle's stream (lbem_desc.stream);
 *    errors raised by device work surface at the next synchronising call
 *    (lbem_diagnostics, lbem_traces to host, lbem_sync) as LBEM_ERR_CUDA.
 *  - Handles are not thread-safe: one thread drives one handle at a time.
 *  - The state is 32-bit float arithmetic; the storage of the distribution is
 *    FP32, or one of three 16-bit formats (lbem_storage).
 */
#ifndef LBEM_H
#define LBEM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbem lbem_t;
typedef struct lbem_batch lbem_batch_t;

typedef enum {
    LBEM_OK = 0,
    LBEM_ERR_ARG = 1,      /* invalid argument (null handle, bad size, index out of range) */
    LBEM_ERR_CUDA = 2,     /* a CUDA runtime call or a kernel failed */
    LBEM_ERR_MEDIUM = 3,   /* medium rejected: eps, mu not finite and > 0, or rest weight w0 outside [0, 1) */
    LBEM_ERR_UNSTABLE = 4, /* non-finite values found in the state */
    LBEM_ERR_TIMEOUT = 5,  /* a bounded device-side wait gave up */
    LBEM_ERR_STATE = 6,    /* call not valid in the handle's current state (e.g. no medium yet) */
    LBEM_ERR_NOMEM = 7     /* device allocation failed */
} lbem_status;

/* Storage format of the distribution (arithmetic is always FP32). */
typedef enum {
    LBEM_F32 = 0,  /* 4 bytes per value */
    LBEM_F16 = 1,  /* IEEE binary16 of s*g, s a power of two chosen from the inputs (2 bytes) */
    LBEM_BF16 = 2, /* bfloat16 of g (2 bytes) */
    LBEM_I16B = 3  /* int16 mantissas sharing one exponent byte per 4 consecutive sites along x (2.25 bytes) */
} lbem_storage;

/* Boundary of one axis (lbem_set_boundaries). */
typedef enum {
    LBEM_BC_PERIODIC = 0, /* the default */
    LBEM_BC_PEC = 1,      /* perfect electric conductor: tangential E and normal B vanish on the wall */
    LBEM_BC_PMC = 2       /* perfect magnetic conductor: tangential B vanishes on the wall */
} lbem_bc;

typedef struct {
    int dim;        /* 2 (D2Q5, fields E_z, B_x, B_y) or 3 (D3Q7, all six components) */
    int nx, ny, nz; /* grid size, periodic in every direction unless lbem_set_boundaries puts walls;
                       nz ignored in 2D; each >= 1 */
    int storage;    /* lbem_storage; LBEM_F32 in 3D */
    double c_ref2;  /* wave speed squared (lattice units) at eps = mu = 1; <= 0 selects the largest the
                       lattice carries with a non-negative rest weight: 1/2 in 2D, 1/6 in 3D */
    void *stream;   /* cudaStream_t the handle enqueues on; NULL = legacy default stream */
} lbem_desc;

/* ---------------------------------------------------------------- lifecycle */

/* Create a solver on the current CUDA device: allocates the two population
 * buffers (ping-pong), the medium arrays and small scratch.  The state starts
 * at t = 0 with all fields zero.  *out receives the handle (owned by the
 * caller, released with lbem_destroy).  LBEM_ERR_ARG for invalid sizes,
 * LBEM_ERR_NOMEM if the device memory does not fit. */
lbem_status lbem_create(const lbem_desc *desc, lbem_t **out);

/* Release every device allocation of the handle (synchronises its stream). */
void lbem_destroy(lbem_t *h);

/* Replace the stream the handle enqueues on (cudaStream_t as void*). */
lbem_status lbem_set_stream(lbem_t *h, void *stream);

/* Wait for all work enqueued on the handle's stream; reports deferred device errors, and LBEM_ERR_TIMEOUT
 * if a shared-memory tile or chunk load of a two-step kernel (lbem_set_temporal_blocking) gave up waiting. */
lbem_status lbem_sync(lbem_t *h);

/* Limit of the bounded device-side waits on the current device (all handles on it): a CTA of the two- and
 * three-step kernels that has waited this long for its tile's TMA window gives up, lets the copies in flight
 * land (bounded again, 2 s, independent of this limit), records the failure and exits, and the next lbem_sync or
 * lbem_check_guards returns LBEM_ERR_TIMEOUT; the launch's output state is then invalid (reload or re-initialise
 * it).  Not in the paper: a failure-detection knob.  seconds in [0, 3600] (LBEM_ERR_ARG otherwise); the default
 * is 2.  0 gives up at every wait without polling, which exercises the give-up path with ordinary, in-bounds
 * loads.  Takes effect for launches enqueued after the call. */
lbem_status lbem_set_wait_limit(double seconds);

/* Message of the last failed call on this thread ("" if none). */
const char *lbem_last_error(void);

/* Grid geometry: number of sites and the bytes of one saved state (lbem_save_state). */
lbem_status lbem_info(const lbem_t *h, long long *nsite, size_t *state_bytes);

/* ---------------------------------------------------------------- problem set-up */

/* Medium upload (paper, Eq. 3 and Sec. "Lattice BGK formulation").  eps_r and
 * mu_r are relative permittivity and permeability per site ([nsite] floats,
 * host or device); mu_r may be NULL (mu = 1 everywhere).  Per site:
 *   c_eff^2 = c_ref2 / (eps_r mu_r)      (c = 1/sqrt(mu0 eps0))
 *   c_L^2   = (D-1) c_eff^2              (equilibrium's lattice speed parameter)
 *   w0      = 1 - D c_L^2                (rest weight; moving weights (1-w0)/(2D))
 *   grad ln mu by periodic central differences (only kept when mu_r is given)
 * Validated in FP64 on the device: LBEM_ERR_MEDIUM (handle's previous medium
 * kept) if any site has eps_r or mu_r not finite and > 0, or w0 outside
 * [0, 1).  Synchronises the stream (to read the validation count). */
lbem_status lbem_set_medium(lbem_t *h, const float *eps_r, const float *mu_r);

/* Anisotropic medium (the paper: different weights for particles moving along
 * different axes): eps_r per site ([nsite] floats, host or device) and a
 * uniform in-plane relative permeability tensor diag(mu_xx, mu_yy), 2D TM.  The
 * lattice speed of axis x is c_x^2 = c_ref2 / (eps_r mu_yy) (a wave moving
 * along x), of axis y c_y^2 = c_ref2 / (eps_r mu_xx); moving particles of an
 * axis weigh c_a^2 / 2, w0 = 1 - c_x^2 - c_y^2 must lie in [0, 1)
 * (LBEM_ERR_MEDIUM otherwise, previous medium kept).  Fields: E_z =
 * -cbar^2 sigma with cbar^2 = sqrt(c_x^2 c_y^2), B_x = r (g_4 - g_2), B_y =
 * (g_1 - g_3) / r, r = sqrt(mu_xx / mu_yy); a current j_z enters with
 * mu = sqrt(mu_xx mu_yy).  mu_xx = mu_yy = mu is the isotropic scheme with a
 * uniform mu.  2D, LBEM_F32 storage (LBEM_ERR_ARG otherwise); the handle then
 * steps in pairs (lbem_set_temporal_blocking; with walls and layers each pair is
 * followed by a pass recomputing the bands next to the walls), with a dispersive
 * pole and walls one step per launch with the general kernel, bit-identical to
 * single steps either way; lbem_set_medium makes it isotropic again.  Batches
 * and the adjoint take isotropic handles only.  Synchronises the stream. */
lbem_status lbem_set_medium_aniso(lbem_t *h, const float *eps_r, double mu_xx, double mu_yy);

/* Initial fields (Eq. 8): sets g = g^(0)(E, B) at every site and t = 0, and
 * clears recorded traces.  E and B are [3][nsite] floats (host or device), or
 * NULL for zero.  In 2D only E_z, B_x and B_y are representable; the other
 * components are ignored.  Requires a medium (LBEM_ERR_STATE otherwise). */
lbem_status lbem_set_fields(lbem_t *h, const float *E, const float *B);

/* Point current sources (Eq. 3's -j/eps0 term): source k injects the current
 * density j_{comp[k]}(site[k], t) = amp[k*nt + t] for 0 <= t < nt (0 after).
 * site: [n] flat indices, comp: [n] in 0..2 (in 2D only comp 2, j_z, couples
 * to the TM fields; others are ignored), amp: [n*nt] floats.  All three are
 * HOST arrays, copied.  n = 0 removes all sources.  At most 65536 sources. */
lbem_status lbem_set_sources(lbem_t *h, int n, const long long *site, const int *comp, const float *amp, int nt);

/* Receivers: each step, before the collision, receiver r records field
 * comp[r] (0..2 = E_x..E_z, 3..5 = B_x..B_z) at site[r] into a handle-owned
 * trace buffer of `capacity` samples per receiver (steps beyond capacity are
 * not recorded).  site, comp: HOST arrays [n], copied.  n = 0 removes all
 * receivers.  Recording restarts at the next lbem_set_fields. */
lbem_status lbem_set_receivers(lbem_t *h, int n, const long long *site, const int *comp, int capacity);

/* ---------------------------------------------------------------- time stepping */

/* Advance nsteps steps: per site and step, pull-stream (Eq. 18), moments (Eqs.
 * 9-10), source (Eq. 3), equilibrium (Eq. 8), collision at tau = dt/2 (Eq. 17);
 * receivers sample the pre-collision fields.  One fused kernel launch per step,
 * or per two (three) steps where lbem_set_temporal_blocking enables it (two is
 * the default for 2D), enqueued on the stream (or replayed from
 * a cached CUDA graph when enabled by lbem_set_graphs).  Requires a medium.
 * nsteps >= 0. */
lbem_status lbem_step(lbem_t *h, int nsteps);

/* Walls and absorbing layers (2D and 3D, LBEM_F32 storage; the paper treats
 * periodic domains only and leaves other boundaries open).  kind[a] (a = x, y,
 * z; z must be LBEM_BC_PERIODIC in 2D) puts a wall half a site beyond the first
 * and the last site of axis a: a population that would cross it returns to the
 * site it left in the opposite direction (halfway bounce-back), each tensor
 * component g_bc times (b == a ? -1 : 1)(c == a ? -1 : 1) for LBEM_BC_PEC (the
 * geometric mirror) and minus that for LBEM_BC_PMC -- in 2D the single
 * component g_xy thus gets -1 (PEC) or +1 (PMC).  The state then evolves as the
 * periodic state on a domain twice as long holding the mirror image.  grad ln mu at the edge sites
 * uses the mirror image of mu.  layer > 0 (at most half the walled axis) adds
 * an absorbing layer inside every wall: after each collision the populations of
 * a site at distance i = 0 .. layer-1 from the wall-adjacent site are scaled by
 * 1 - gamma_max ((layer - i)/layer)^2 (both axes' factors at corners), which
 * damps E and B alike and keeps the medium's wave impedance; 0 <= gamma_max < 1.
 * Every stepping mode applies (single, two and three steps per launch, graphs):
 * in 2D, after each launch a small kernel recomputes that launch's steps on the
 * sites within max(layer, 1) + steps - 1 of a wall, so results stay
 * bit-identical across modes; in 3D the one-site-per-thread kernel applies the
 * walls and layers itself.  All-periodic kind[] removes the walls.
 * LBEM_ERR_ARG for other values or 16-bit storage; LBEM_ERR_STATE after lbem_forward_record (the
 * adjoint is periodic only).  Batches (lbem_batch_create) take periodic members
 * only.  Synchronises the stream. */
lbem_status lbem_set_boundaries(lbem_t *h, const int kind[3], int layer, double gamma_max);
lbem_status lbem_get_boundaries(const lbem_t *h, int kind[3], int *layer, double *gamma_max);

/* Frequency-dispersive permittivity (the convolution term of Eq. 3, which the
 * paper leaves to auxiliary differential equations): one Drude-Lorentz pole per
 * site, d_t J + gamma J + wr^2 P = wp^2 E with J = d_t P, i.e.
 * eps(omega) = eps_r (1 + wp^2 / (wr^2 - omega^2 - i gamma omega)) with eps_r of
 * lbem_set_medium as eps_infinity (lattice units: frequencies per step).  wp2,
 * wr2, gamma: [nsite] floats, host or device, copied; wr2 and gamma may be NULL
 * (zero); wp2 = NULL removes the pole.  The lattice's zeroth moment then
 * carries D/eps_r, E = D/eps_r - P is what lbem_fields, receivers and
 * lbem_diagnostics report, and P enters the equilibrium's second moment; J at
 * half steps and P at whole ones are stepped time-centred before each
 * collision (homogeneous lossless Drude medium: 4 sin^2(omega/2) =
 * 4 c^2 (sin^2(kx/2) + sin^2(ky/2)) + wp^2).  2D, LBEM_F32 storage
 * (LBEM_ERR_ARG otherwise), after lbem_set_medium (LBEM_ERR_STATE); validated in
 * FP64: LBEM_ERR_MEDIUM (nothing changed) unless every parameter is finite and
 * >= 0 and wp2 + wr2 <= 4 w0 (w0 the rest weight, 1 - 2 c_L^2 or 1 - c_x^2 - c_y^2: the stability
 * bound), which lbem_set_medium also checks against a new medium.  A dispersive
 * handle with walls or a mu array steps one step per launch with the general kernel (walls, layers and an
 * anisotropic medium included); without them it steps in pairs (lbem_set_temporal_blocking), bit-identical to
 * single steps.  The update J <- ((1 - gamma/2) J - wr2 P + wp2 E) / (1 + gamma/2) runs with three per-site
 * coefficients formed once here in FP64 (no division per step).  The handle holds a second P plane (every launch
 * writes P to the plane paired with its output
 * population buffer); lbem_set_fields starts the pole at rest (D = E); lbem_save_state
 * appends J and P (lbem_info's state_bytes counts them).  Batches and the
 * adjoint take non-dispersive handles only.  Synchronises the stream. */
lbem_status lbem_set_dispersion(lbem_t *h, const float *wp2, const float *wr2, const float *gamma);

/* Watchdog (off by default): with every > 0, lbem_step computes the FP64 field energy (as
 * lbem_diagnostics, synchronising) whenever t reaches a multiple of `every`, and stops with
 * LBEM_ERR_UNSTABLE (t left at the check) if the state is not finite or the energy grew by more than
 * max_growth (> 1) since the previous check.  every = 0 switches it off.  The scheme is neutral (no
 * growth without sources), so a jump means an over-driven source or a corrupted state. */
lbem_status lbem_set_watchdog(lbem_t *h, int every, double max_growth);

/* Temporal blocking (2D; 16-bit storage needs uniform mu and nx % 4 == 0; otherwise ignored).  With
 * steps_per_pass = 2 (the default) lbem_step advances pairs of steps with one kernel that stages a tile plus
 * a two-site halo in shared memory and performs both steps there, so the state crosses HBM once per two steps
 * (44 instead of 88 bytes per site and step pair for FP32); an odd last step is a single step.  For FP32
 * storage results are bit-identical to single steps; 16-bit storage is rounded once per launch (decode, two
 * FP32 steps, encode).  steps_per_pass = 3 (FP32 storage, uniform mu; otherwise as 2) advances triples of steps
 * through a three-site halo (44 bytes per site per three steps), a remaining pair with the two-step kernel;
 * again bit-identical to single steps.  1 makes every step a single-step launch (the kernel lbem_set_variant
 * selects).  With steps_per_pass = 3, tile_shape selects 0 = 6 rows, 384 threads, 3 CTAs per SM (also -1);
 * 1 = 4 rows, 288, 4; 2 = 8 rows, 448, 2.  With steps_per_pass = 2, tile_shape
 * selects the tile (128 sites wide) height, threads per CTA and CTAs per SM: 0 = 6 rows, 256 threads, 5
 * per SM (the default, also -1); 1 = 8 rows, 320, 3; 2 = 8 rows, 352, 3; 3 = 10 rows, 384, 3; 4 = 5 rows,
 * 224, 5; 5 = 4 rows, 192, 6; 6 = 14 rows, 512, 2; FP32 only: 7, 8 = no tiles: each warp streams a
 * 128-column strip down a segment of rows through registers (5 or 4 blocks of 128 threads per SM); 9 - 14 =
 * strip streaming: persistent CTAs take units of rows of a 128-column strip from a queue and stream them in
 * chunks through shared-memory stages (a producer warp loads chunks ahead by TMA), computing step t+1 one row
 * behind step t (chunk rows, stages, CTAs per SM, chunks per unit: 9 = 4, 4, 2, 16; 10 = 4, 3, 3, 12;
 * 11 = 6, 3, 2, 12; 12 = 3, 4, 3, 24; 13 = 4, 3, 3, 32; 14 = 3, 4, 3, 12).  With -1 (or never set), an FP32
 * grid of uniform mu with at least 12 000 000 sites takes shape 10, any other shape 0.  With
 * a heterogeneous mu (FP32; the two grad ln mu planes are staged beside c_L^2, 52 instead of 104 bytes per
 * site and step pair) only 0 = 6 rows, 256 threads, 4 per SM, 1 = 14 rows, 512, 2, and 2 = strip streaming
 * (4, 3, 2, 16; the default from 12 000 000 sites) exist; a larger shape set before the medium falls back to 0.  An anisotropic medium (lbem_set_medium_aniso) steps in pairs
 * with shape 0 (the tile kernel, 256 threads, 5 per SM) or 1 (the strip kernel, the default from 12 000 000
 * sites), walls and layers included; a dispersive pole without walls or a mu array with shape 0 at 4 per SM;
 * both bit-identical to their single steps.  With a pole and walls (or a pole with a mu array), and for
 * steps_per_pass = 3, every step of these media is a single step.
 * LBEM_ERR_ARG for values outside the current handle's set. */
lbem_status lbem_set_temporal_blocking(lbem_t *h, int steps_per_pass, int tile_shape);

/* Steps per launch in effect (2 or 3 only where that kernel is enabled and applies), the tile shape (the one
 * launched when two steps per launch are in effect, else as set or autotuned) and the number of tile shapes of
 * the selected steps per pass; any pointer may be NULL. */
lbem_status lbem_get_temporal_blocking(const lbem_t *h, int *steps_per_pass, int *tile_shape, int *nshapes);

/* Use (on != 0) or not CUDA-graph replay of runs of steps in lbem_step. */
lbem_status lbem_set_graphs(lbem_t *h, int on);

/* Steps taken since the last lbem_set_fields / lbem_load_state. */
lbem_status lbem_time(const lbem_t *h, long long *t);

/* ---------------------------------------------------------------- outputs */

/* Field extraction (Eqs. 9-10 and E_g = -1/2 eps_gab Lambda_ab): E, B of the
 * current (pre-collision) state, [3][nsite] floats each, host or device; either
 * may be NULL.  Components not representable in 2D are written as 0. */
lbem_status lbem_fields(lbem_t *h, float *E, float *B);

/* Energy density and Poynting vector of the current state (paper, Sec. "Heterogeneous media"):
 *   u[s]      = sum_a (B_a^2 + E_a^2 / c_eff^2)      ([nsite] floats; its sum is out[0] of lbem_diagnostics)
 *   P[a*n+s]  = eps_abc E_b B_c                       ([3][nsite] floats)
 * either may be NULL; host or device memory.  Uses the handle's staging area (allocated on first use). */
lbem_status lbem_energy_flux(lbem_t *h, float *u, float *P);

/* Receiver traces: out[r*nrec_steps + n] for n < nrec_steps = min(t, capacity),
 * host or device; *nrecorded (host, may be NULL) receives nrec_steps.  out may be
 * NULL to query the count only. */
lbem_status lbem_traces(lbem_t *h, float *out, int *nrecorded);

/* FP64 diagnostics of the current state (synchronising; result on the host):
 *   out[0] = sum_x sum_a (B_a^2 + E_a^2 / c_eff^2)       (field energy, Sec. "Heterogeneous media")
 *   out[1] = sum_x sum_i sum_ab g_iab^2 / w_i             (terms with w_i = 0 skipped)
 *   out[2] = sqrt(sum_x (div B)^2), periodic central differences
 * Deterministic: block partial sums in a handle-owned scratch array, reduced in
 * fixed order.  LBEM_ERR_UNSTABLE if any of the three is not finite. */
lbem_status lbem_diagnostics(lbem_t *h, double out[3]);

/* The three FP64 diagnostics of lbem_diagnostics, for callers that cannot
 * allocate device memory (for example a program that hands all device memory
 * to its own pool at start-up, or a loop whose memory budget is fixed after
 * initialisation); the paper has no counterpart.  It takes no handle and
 * allocates nothing: inputs and output are the caller's device memory, and
 * the only scratch (per-block partial sums, 192 KiB) is a static device array
 * of the library, held by every GPU that loads the library until exit.
 * Scope: the state of a periodic, isotropic, non-dispersive handle (no walls,
 * no lbem_set_medium_aniso tensor, no lbem_set_dispersion pole); for other
 * handles the sums are not those of lbem_diagnostics (use that call).
 *   state : FP32 distribution in the layout lbem_save_state writes for an
 *           LBEM_F32 handle of this geometry (device memory): npop planes
 *           (5 in 2D, 21 in 3D) of ny*nz rows of round_up(nx, 32) floats,
 *           4 * npop * round_up(nx, 32) * ny * nz bytes
 *   eps_r, mu_r : the medium as given to lbem_set_medium ([nsite] floats,
 *           device; mu_r may be NULL); c_ref2 as in lbem_desc (<= 0: default)
 *   out   : 3 doubles of device memory, written asynchronously on `stream`
 * LBEM_ERR_ARG, with nothing launched, for grids above 33554432 sites, host
 * pointers, or a buffer whose device allocation ends before the bytes above
 * (the allocation the driver knows: a buffer carved out of a larger pool
 * allocation is checked against the end of that pool allocation).
 * The first call on a device looks up the static array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the array: calls that overlap on the GPU race. */
lbem_status lbem_diagnostics_static(int dim, int nx, int ny, int nz, const void *state, const float *eps_r,
                                    const float *mu_r, double c_ref2, double *out, void *stream);

/* ---------------------------------------------------------------- checkpoint / resume */

/* Copy the distribution state (state_bytes from lbem_info) to dst / from src
 * (host or device).  lbem_load_state also sets t (for source and receiver time
 * indexing) to t_at_save. */
lbem_status lbem_save_state(lbem_t *h, void *dst);
lbem_status lbem_load_state(lbem_t *h, const void *src, long long t_at_save);

/* Verify the guard bands (256 patterned bytes) the library keeps on both sides of every handle-owned
 * device array (distribution, medium, events, traces, scratch); synchronises the stream.  LBEM_ERR_STATE
 * names the first array whose band was overwritten.  A check for out-of-bounds writes that needs no
 * device-side instrumentation. */
lbem_status lbem_check_guards(lbem_t *h);

/* Rows of one population plane of the current state, for spatial domain
 * decomposition: the state holds post-collision values laid out for pull
 * streaming (a site pulls population p from its neighbour across -c_p), so a
 * slab that keeps one ghost row on either side stays exact if, after each
 * single step, its ghost rows receive the populations the neighbouring slabs
 * send across the cut (2D: plane 2 of the last real row upwards, plane 4 of the
 * first real row downwards; 3D, slabs in z: planes 9-11 upwards and 18-20
 * downwards, ny rows each).  Copies nrows rows (2D: row = y; 3D: row = y + ny z)
 * starting at row0 of plane `plane` to (to_state = 0) or from (to_state = 1)
 * buf, [nrows][nx] floats, host or device.  LBEM_F32 storage; a decomposed
 * handle must step one step per launch (lbem_set_temporal_blocking(h, 1, -1)).  A
 * dispersive pole's J and P and an anisotropic tensor need no exchange (site-local
 * and uniform); walls may close the axes along the cuts, not the slab axis.
 * LBEM_ERR_ARG for planes or rows out of range.  Host buffers synchronise the
 * stream. */
lbem_status lbem_rows(lbem_t *h, int plane, int row0, int nrows, float *buf, int to_state);

/* Halo of a slab for spatial domain decomposition along y (2D, LBEM_F32 storage): a slab of ny rows is `halo`
 * ghost rows, its real rows, and `halo` ghost rows, stepped as its own periodic grid; after every `halo` steps each
 * slab sends its neighbours what their ghost rows need and writes what it receives into its own.  The state holds
 * post-collision values laid out for pull streaming (a row pulls g_2 from the row below, g_4 from the row above).
 *   halo = 1 (exchange after every single step): up goes g_2 of the last real row, down g_4 of the first
 *            (1 row of nx floats each way).
 *   halo = 2 (exchange after every two steps, so each slab steps two steps per launch): the inner ghost row's first
 *            collision feeds a real row, so up go g_0, g_1, g_2, g_3 of the last real row and g_2 of the row below
 *            it, down g_0, g_1, g_3, g_4 of the first real row and g_4 of the row above it (5 rows of nx floats
 *            each way, in that order).
 * lbem_halo_out writes what goes up into `up` and what goes down into `down`; lbem_halo_in writes the rows received
 * from the slab below into the lower ghost rows and those from above into the upper ones.  Buffers are device memory,
 * [rows][nx] floats; either may be NULL (that direction skipped).  One small kernel per direction on the handle's
 * stream.  LBEM_ERR_ARG for other storage or dimensions, halo outside {1, 2}, fewer than 3 * halo rows, or host
 * buffers.  A decomposed handle with halo = 1 must step one step per launch (lbem_set_temporal_blocking(h, 1, -1)).
 * Not in the paper (its runs were single-domain). */
lbem_status lbem_halo_out(lbem_t *h, int halo, float *up, float *down);
lbem_status lbem_halo_in(lbem_t *h, int halo, const float *from_below, const float *from_above);

/* ---------------------------------------------------------------- adjoint (not in the paper) */

/* Forward run that records what the adjoint needs: advances nsteps steps from
 * the current state (receivers record as in lbem_step) and keeps a copy of the
 * state every `checkpoint_every` steps in handle-owned device memory.  FP32
 * storage, uniform mu (LBEM_ERR_STATE otherwise). */
lbem_status lbem_forward_record(lbem_t *h, int nsteps, int checkpoint_every);

/* Reverse-time adjoint of the last lbem_forward_record: given the cotangent of
 * the receiver traces dL/dtrace ([nrec][nsteps] floats, host or device), writes
 * dL/d eps_r ([nsite] floats, host or device).  Recomputes each checkpoint
 * segment forward, then runs the hand-written adjoint stream-collide kernel
 * backwards through it; the gradient accumulates over time steps in FP64.
 * If grad_cL2 is not NULL it also receives dL/dc_L^2 ([nsite] doubles). */
lbem_status lbem_adjoint(lbem_t *h, const float *trace_cot, float *grad_eps, double *grad_cL2);

/* ---------------------------------------------------------------- tuning */

/* Time each launch shape of the stream-collide kernel on this handle for
 * trial_steps steps (the state is saved and restored) and keep the fastest.
 * *best (may be NULL) receives the chosen variant id.  Where two steps per
 * launch apply and are enabled (lbem_set_temporal_blocking), every tile shape
 * of that kernel is timed too; the fastest is kept, and two-step launches stay
 * on only if they beat the best single-step kernel. */
lbem_status lbem_autotune(lbem_t *h, int trial_steps, int *best);
lbem_status lbem_set_variant(lbem_t *h, int variant);
lbem_status lbem_get_variant(const lbem_t *h, int *variant, int *nvariants);

/* ---------------------------------------------------------------- batches of independent media */

/* A batch steps n independent 2D FP32 handles (members, of any sizes) with one
 * kernel launch per step, or per pair of steps, over a flattened work table of
 * all members; runs of steps are captured once into a CUDA graph and replayed.
 * Members keep their own medium, fields, sources, receivers and outputs (use
 * the calls above on them); all members must be at the same time t when
 * stepped.  The batch does not own the members.  Launch shapes (variants):
 * 0..8 advance one step per launch (rows of warps, one site per thread, a
 * persistent pipeline, lanes linear over each member's padded plane); 9 .. 13
 * advance two steps per launch through shared-memory tiles of 128 x 6 sites (5
 * or 4 blocks per SM), 128 x 8, 128 x 10 and 128 x 12 sites, over a packed copy
 * of the members' states with periodic halos that the batch keeps (filled at
 * the start of a call, written back into the members' buffers at its end; an
 * odd step count takes one single step first); 14, 15 advance two steps per
 * launch over the same packed copy by strip streaming (persistent CTAs take
 * units of 30 or 34 rows of a member's 128-column strip from a queue and stream
 * them in chunks of 4 or 3 rows through shared-memory stages).  Every variant
 * gives the same bits as each member stepped alone. */
lbem_status lbem_batch_create(int n, lbem_t *const *members, void *stream, lbem_batch_t **out);
lbem_status lbem_batch_step(lbem_batch_t *b, int nsteps);
/* Time every variant over trial_steps steps (members' states saved and restored) and keep the fastest; *best (may
 * be NULL) receives it.  The two-step variants pack and unpack the members once per call, so trials of a few hundred
 * steps rank them as the long runs they are meant for. */
lbem_status lbem_batch_autotune(lbem_batch_t *b, int trial_steps, int *best);
/* Choose the batched kernel's launch shape directly (0 <= variant < *nvariants of lbem_batch_get_variant). */
lbem_status lbem_batch_set_variant(lbem_batch_t *b, int variant);
lbem_status lbem_batch_get_variant(const lbem_batch_t *b, int *variant, int *nvariants);
void lbem_batch_destroy(lbem_batch_t *b);

#ifdef __cplusplus
}
#endif
#endif
