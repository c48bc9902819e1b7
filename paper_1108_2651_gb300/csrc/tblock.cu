// Two time steps per pass (temporal blocking), 2D, FP32 storage; uniform mu, and variants for a heterogeneous mu
// (MU: the grad ln mu planes staged beside c_L^2), an anisotropic tensor (AN) and a dispersive pole (POLE), the
// last two with the general kernel's site update (collide2d_an, pole_update), so that they too are bit-identical
// to single steps of general.cu.
//
// A persistent CTA takes tiles of 128 x TBY sites in turn.  For each it loads
// the post-collision state at t of the tile plus a halo of 2 sites (one per
// step of the pull stencil) and c_L^2 into shared memory, computes step t on
// the tile plus a ring of 1 site (Eqs. 17-18, the same site update as the
// single-step kernels), then step t+1 on the tile from those values, and writes
// only the final post-collision state.  The loads of the next tile (TMA boxes,
// or 16-byte asynchronous copies where the window wraps periodically) run
// while step t+1 of the current one is computed, and several CTAs share an SM.
//
// Each population plane is staged shifted by its pull offset in y, so that
// row r of every staged plane holds exactly what the update of tile row r
// pulls (the moving populations g2 from the row above and g4 from the row
// below), and a plane keeps only the rows that are read: TBY + 2 rows of each
// plane at t, TBY rows of each at t + 1.  A lane updates 4 consecutive sites
// of a row with 16-byte shared-memory accesses; one warp covers a tile row.
//
// HBM traffic per two site updates is 24 bytes read (5 populations and c_L^2)
// and 20 written, against 88 for two single steps.  The arithmetic of each
// site update is that of collide2d, so the results are bit-identical to two
// single steps.  Sources act at both steps on every site computed; receivers
// record at the owned sites only.
#include <cuda.h>
#include <string.h>

#include "lbem_internal.cuh"
#include "tma.cuh"

namespace lbk {

constexpr int TBX = 128;     // tile width: one warp of 4-site lanes
constexpr int TW = TBX + 8;  // staged columns x0-4 .. x0+TBX+3 (16-byte aligned); column j <-> x0-4+j

// Row shift of the staged planes: plane p row r of the t stage holds global row y0 - 1 + r + in_shift(p), and
// plane p row j of the t+1 stage holds global row y0 + j + in_shift(p).
__device__ __host__ constexpr int in_shift(int p) { return p == 2 ? -1 : p == 4 ? 1 : 0; }


// Shared-memory layout of a CTA (floats; regions start on 128-byte boundaries), then one mbarrier.  The
// medium stage holds c_L^2 and, with a heterogeneous permeability (MU), d_x ln mu and d_y ln mu after it, each
// R rows of TW (the two gradient planes are one TMA box, so R * TW floats must be a multiple of 128 bytes).
template <int TBY, bool MU = false, bool POLE = false>
struct TbGeom {
    static constexpr int R = TBY + 2;  // staged rows per plane at t (tile rows y0-1 .. y0+TBY), and of c_L^2
    static constexpr int NCL = MU ? 3 : 1;  // medium planes
    static constexpr int up32(int n) { return (n + 31) / 32 * 32; }
    // plane strides (each staged plane at t is a TMA destination: 128-byte aligned)
    static constexpr int IN_PL = up32(R * TW), P_PL = TBY * TW;
    static constexpr int IN_SZ = up32(5 * IN_PL), CL_SZ = up32(NCL * R * TW), P_SZ = up32(5 * P_PL);
    // with a dispersive pole: P at t over the window (R rows of TW), and J, wp2, wr2, gamma over the owned sites
    // (TBY rows of TBX, plane stride JS_PL), both staged with the window
    static constexpr int PS_SZ = POLE ? up32(R * TW) : 0, JS_PL = TBY * TBX, JS_SZ = POLE ? up32(4 * JS_PL) : 0;
    static constexpr int SZ = IN_SZ + CL_SZ + P_SZ + PS_SZ + JS_SZ;
    static constexpr size_t BYTES = sizeof(float) * SZ + sizeof(unsigned long long);
    static constexpr unsigned TMA_BYTES = sizeof(float) * ((5 + NCL) * R * TW + (POLE ? R * TW + 4 * JS_PL : 0));
    static_assert(!MU || (R * TW) % 32 == 0, "gradient planes 128-byte aligned");
    static_assert(!POLE || JS_PL % 32 == 0, "pole planes 128-byte aligned");
};

// Tensor maps of the pole's planes (P at t: box TW x (TBY+2) at (x0-4, y0-1); J, wp2, wr2, gamma: box TBX x TBY at
// (x0, y0)); an unused placeholder for kernels without a pole.
template <bool POLE>
struct PoleMaps {
    CUtensorMap P, J, wp, wr, gm;
};
template <>
struct PoleMaps<false> {
    int unused;
};

// Source plane k of the medium stage: c_L^2, then d_x ln mu and d_y ln mu.
__device__ __forceinline__ const float *medium_plane(const StepArgs &a, int k) {
    return k == 0 ? a.med.cL2 : a.med.dlnmu + (k - 1) * a.g.plane;
}

// Asynchronous copies of the pole's planes for one tile (as the window: 16 bytes per copy where every group of 4
// columns stays contiguous after the periodic wrap, else 4): P over the window's rows and columns into PS, J, wp2,
// wr2, gamma over the tile's own rows and columns into JS.
template <int TBY>
__device__ __forceinline__ void tb_issue_pole(const StepArgs &a, int x0, int y0, float *PS, float *JS, int nt) {
    constexpr int R = TbGeom<TBY>::R, JPL = TbGeom<TBY, false, true>::JS_PL, Q = TW / 4, QJ = TBX / 4;
    const Grid &G = a.g;
    const bool v16 = (x0 - 4 >= 0 && x0 + TBX + 4 <= G.nx) || (G.nx & 3) == 0;
    for (int k = threadIdx.x; k < R * Q; k += nt) {
        const int r = k / Q, q = k - r * Q;
        const float *src = a.med.Pr + (long long)wrapi(y0 - 1 + r, G.ny) * G.pitch;
        float *dst = PS + r * TW + 4 * q;
        if (v16)
            tb_cpa16(dst, src + wrapi(x0 - 4 + 4 * q, G.nx));
        else
            for (int j = 0; j < 4; j++) tb_cpa4(dst + j, src + wrapi(x0 - 4 + 4 * q + j, G.nx));
    }
    for (int k = threadIdx.x; k < 4 * TBY * QJ; k += nt) {
        const int pr = k / QJ, q = k - pr * QJ;
        const int pl = pr / TBY, r = pr - pl * TBY;
        const float *base = pl == 0 ? a.med.J : pl == 1 ? a.med.pc : pl == 2 ? a.med.pb : a.med.pa;
        const float *src = base + (long long)wrapi(y0 + r, G.ny) * G.pitch;
        float *dst = JS + pl * JPL + r * TBX + 4 * q;
        if (v16)
            tb_cpa16(dst, src + wrapi(x0 + 4 * q, G.nx));
        else
            for (int j = 0; j < 4; j++) tb_cpa4(dst + j, src + wrapi(x0 + 4 * q + j, G.nx));
    }
}

// Asynchronous copies of one tile's window with periodic wrap (16 bytes per copy when every group of 4
// columns stays contiguous after the wrap, else 4).
template <int TBY, bool MU = false>
__device__ __forceinline__ void tb_issue(const StepArgs &a, int x0, int y0, float *IN, float *CL, int nt) {
    constexpr int R = TbGeom<TBY>::R, PL = TbGeom<TBY>::IN_PL, Q = TW / 4, NP = 5 + TbGeom<TBY, MU>::NCL;
    const Grid &G = a.g;
    const float *in = static_cast<const float *>(a.in.data);
    const int tid = threadIdx.x;
    if (((x0 - 4 >= 0) && (x0 + TBX + 4 <= G.nx)) || (G.nx & 3) == 0) {
        for (int k = tid; k < NP * R * Q; k += nt) {
            const int pr = k / Q, q = k - pr * Q;  // pr = plane * R + row; planes 5.. are the medium stage
            const int pl = pr / R, r = pr - pl * R;
            const int gx = wrapi(x0 - 4 + 4 * q, G.nx);
            if (pl < 5) {
                const int gy = wrapi(y0 - 1 + r + in_shift(pl), G.ny);
                tb_cpa16(IN + pl * PL + r * TW + 4 * q, in + pl * G.plane + (long long)gy * G.pitch + gx);
            } else {
                const int gy = wrapi(y0 - 1 + r, G.ny);
                tb_cpa16(CL + (pl - 5) * R * TW + r * TW + 4 * q,
                         medium_plane(a, pl - 5) + (long long)gy * G.pitch + gx);
            }
        }
    } else {  // columns wrap inside a group: element copies
        for (int k = tid; k < NP * R * TW; k += nt) {
            const int pr = k / TW, c = k - pr * TW;
            const int pl = pr / R, r = pr - pl * R;
            const int gx = wrapi(x0 - 4 + c, G.nx);
            if (pl < 5) {
                const int gy = wrapi(y0 - 1 + r + in_shift(pl), G.ny);
                tb_cpa4(IN + pl * PL + r * TW + c, in + pl * G.plane + (long long)gy * G.pitch + gx);
            } else {
                const int gy = wrapi(y0 - 1 + r, G.ny);
                tb_cpa4(CL + (pl - 5) * R * TW + r * TW + c,
                        medium_plane(a, pl - 5) + (long long)gy * G.pitch + gx);
            }
        }
    }
}

// ---- tensor-memory-accelerator (TMA) window loads for tiles whose window needs no periodic wrap

__device__ int g_tb_timeouts = 0;  // set when a bounded wait of the two-step kernel gave up
// Limit of the bounded waits for a tile's TMA window, in ns of device time (lbem_set_wait_limit); 0 gives up at
// once, which exercises the give-up path with ordinary, in-bounds loads.  Read once per kernel.
__device__ unsigned long long g_wait_limit_ns = 2000000000ull;
// After giving up, a CTA still waits this long for its copies in flight to land before it exits (shared memory
// must not be written by a copy after its CTA is gone); independent of g_wait_limit_ns.
constexpr unsigned long long kDrainNs = 2000000000ull;

template <int TBY>
__device__ __forceinline__ bool tb_interior(int x0, int y0, const Grid &G) {
    return x0 - 4 >= 0 && x0 + TBX + 4 <= G.nx && y0 - 2 >= 0 && y0 + TBY + 2 <= G.ny;
}

// Start the loads of one tile's window: one thread issues six TMA copies (each population plane as a
// (TBY+2) x (TBX+8) box at its row shift, and c_L^2) for interior tiles; every thread issues its share of the
// asynchronous copies otherwise.
template <int TBY, bool MU = false, bool POLE = false>
__device__ __forceinline__ void tb_load(const StepArgs &a, int x0, int y0, float *IN, float *CL, unsigned mbar,
                                        bool tma, const CUtensorMap *tmIn, const CUtensorMap *tmCL, int nt,
                                        const CUtensorMap *tmDL = nullptr, float *PS = nullptr, float *JS = nullptr,
                                        const PoleMaps<POLE> *pm = nullptr) {
    if (tma) {
        if (threadIdx.x == 0) {
            // earlier generic-proxy accesses of the window (ordered by the preceding barrier) before the
            // asynchronous-proxy writes
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar),
                         "r"(TbGeom<TBY, MU, POLE>::TMA_BYTES)
                         : "memory");
#pragma unroll
            for (int p = 0; p < 5; p++)
                tma_load_3d(IN + p * TbGeom<TBY>::IN_PL, tmIn, x0 - 4, y0 - 1 + in_shift(p), p, mbar);
            tma_load_2d(CL, tmCL, x0 - 4, y0 - 1, mbar);
            if (MU) tma_load_3d(CL + TbGeom<TBY>::R * TW, tmDL, x0 - 4, y0 - 1, 0, mbar);
            if constexpr (POLE) {
                constexpr int JPL = TbGeom<TBY, false, true>::JS_PL;
                tma_load_2d(PS, &pm->P, x0 - 4, y0 - 1, mbar);
                tma_load_2d(JS, &pm->J, x0, y0, mbar);
                tma_load_2d(JS + JPL, &pm->wp, x0, y0, mbar);
                tma_load_2d(JS + 2 * JPL, &pm->wr, x0, y0, mbar);
                tma_load_2d(JS + 3 * JPL, &pm->gm, x0, y0, mbar);
            }
        }
    } else {
        tb_issue<TBY, MU>(a, x0, y0, IN, CL, nt);
        if constexpr (POLE) tb_issue_pole<TBY>(a, x0, y0, PS, JS, nt);
    }
}

// Whether tile rows y0-1 .. y0+TBY may hold a source or receiver (if not, the usual case, no per-site lookups).
template <int TBY>
__device__ __forceinline__ bool tb_events(const StepArgs &a, int y0) {
    const Grid &G = a.g;
    return a.evt.rowptr && !(y0 >= 1 && y0 + TBY + 1 <= G.ny &&
                             __ldg(a.evt.rowptr + y0 - 1) == __ldg(a.evt.rowptr + y0 + TBY + 1));
}

// Whether grid row gy (wrapped) holds a source or receiver: within an event tile, only such rows take the per-site
// event path (a warp-uniform test: one warp computes one row).
__device__ __forceinline__ bool row_events(const StepArgs &a, int gy) {
    const int y = wrapi(gy, a.g.ny);
    return __ldg(a.evt.rowptr + y) != __ldg(a.evt.rowptr + y + 1);
}

// Populations pulled by four consecutive sites at shared row `row`, column c (a multiple of 4) of a shifted
// stage S with plane stride PL: g0, g2, g4 from columns c.., g1 from c-1.., g3 from c+1.. (Eq. 17).
struct Pull4 {
    float4 g0, g1, g2, g3, g4;
    __device__ __forceinline__ Pull4(const float *S, int PL, int row, int c) {
        const float *r = S + row * TW + c;
        g0 = lds4(r);
        const float4 l1 = lds4(r + PL - 4), m1 = lds4(r + PL);
        g1 = make_float4(l1.w, m1.x, m1.y, m1.z);
        g2 = lds4(r + 2 * PL);
        const float4 m3 = lds4(r + 3 * PL), h3 = lds4(r + 3 * PL + 4);
        g3 = make_float4(m3.y, m3.z, m3.w, h3.x);
        g4 = lds4(r + 4 * PL);
    }
};

#define TB_COMP(v, k) (k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w)
#define TB_SET(v, k, val) (k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w) = (val)

// The dispersive pole at four sites: P at the current time, J half a step before, and its parameters.
struct Pole4 {
    float4 P, J, wp, wr, gm;
};

// Four values of a pitched plane at row gy, columns gx.. gx+3 (both wrapped periodically): one 16-byte load
// where the four are inside the grid, else four loads.
__device__ __forceinline__ float4 ld_plane4(const float *pl, const Grid &G, int gy, int gx) {
    const float *r = pl + (long long)wrapi(gy, G.ny) * G.pitch;
    if (gx >= 0 && gx + 3 < G.nx) return *reinterpret_cast<const float4 *>(r + gx);
    return make_float4(r[wrapi(gx, G.nx)], r[wrapi(gx + 1, G.nx)], r[wrapi(gx + 2, G.nx)], r[wrapi(gx + 3, G.nx)]);
}

// Four site updates (collide2d each) at global row gy, columns x0+4*lane.., time t.
// With a heterogeneous permeability (MU) the source carries B_x d_y ln mu - B_y d_x ln mu (dlx, dly: the
// gradient of ln mu at the four sites) at every site, as in the single-step kernels.
// With AN (an anisotropic medium, a.med.ar / a.med.amu) or POLE (a dispersive pole, state in *pp) the update is
// the general kernel's collide2d_an with P at t; on owned rows POLE also advances *pp by one step (pole_update).
template <bool EV, bool MU, class PULL, bool AN = false, bool POLE = false>
__device__ __forceinline__ void tb_update4m(const StepArgs &a, const PULL &g, float4 cl, float4 dlx, float4 dly,
                                            int x0, int gy, long long t, bool owned_row, float4 &o0, float4 &o1,
                                            float4 &o2, float4 &o3, float4 &o4, Pole4 *pp = nullptr) {
    const Grid &G = a.g;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const float q0 = TB_COMP(g.g0, k), q1 = TB_COMP(g.g1, k), q2 = TB_COMP(g.g2, k), q3 = TB_COMP(g.g3, k),
                    q4 = TB_COMP(g.g4, k), ck = TB_COMP(cl, k);
        Out5 o;
        const float shat0 = MU ? mu_source(q4 - q2, q1 - q3, TB_COMP(dlx, k), TB_COMP(dly, k)) : 0.f;
        if (AN || POLE) {
            // AN: a tensor (with or without a pole); POLE alone: an isotropic pole (r = 1, the products by r drop)
            const float r = AN ? a.med.ar : 1.f, ri = AN ? __fdiv_rn(1.f, r) : 1.f, fs = __fadd_rn(r, ri);
            const float pz = POLE ? TB_COMP(pp->P, k) : 0.f;
            float shat = 0.f;
            if (EV) {
                const int gx = x0 + 4 * lane + k;
                shat = site_events(a, wrapi(gx, G.nx), wrapi(gy, G.ny), t, owned_row && gx < G.nx && gy < G.ny, q0,
                                   q1, q2, q3, q4, ck, 0.f, pz, r, ri, AN ? a.med.amu : 1.f);
            }
            if (POLE && owned_row) {
                const float sig = __fadd_rn(__fadd_rn(__fadd_rn(q0, q1), __fadd_rn(q2, q3)), q4);
                float J = TB_COMP(pp->J, k), Pn = pz;
                pole_update(ck, sig, TB_COMP(pp->wp, k), TB_COMP(pp->wr, k), TB_COMP(pp->gm, k), J, Pn);
                TB_SET(pp->J, k, J);
                TB_SET(pp->P, k, Pn);
            }
            o = AN ? collide2d_an(q0, q1, q2, q3, q4, ck, shat, r, ri, fs, pz)
                   : collide2d_pole_iso(q0, q1, q2, q3, q4, ck, shat, pz);
        } else if (EV) {
            const int gx = x0 + 4 * lane + k;
            const float shat = site_events(a, wrapi(gx, G.nx), wrapi(gy, G.ny), t,
                                           owned_row && gx < G.nx && gy < G.ny, q0, q1, q2, q3, q4, ck, shat0);
            o = collide2d(q0, q1, q2, q3, q4, ck, shat);
        } else if (MU) {
            o = collide2d(q0, q1, q2, q3, q4, ck, shat0);
        } else {
            o = collide2d_free(q0, q1, q2, q3, q4, ck);
        }
        TB_SET(o0, k, o.o0);
        TB_SET(o1, k, o.o1);
        TB_SET(o2, k, o.o2);
        TB_SET(o3, k, o.o3);
        TB_SET(o4, k, o.o4);
    }
}

template <bool EV, class PULL>
__device__ __forceinline__ void tb_update4(const StepArgs &a, const PULL &g, float4 cl, int x0, int gy, long long t,
                                           bool owned_row, float4 &o0, float4 &o1, float4 &o2, float4 &o3,
                                           float4 &o4) {
    tb_update4m<EV, false>(a, g, cl, cl, cl, x0, gy, t, owned_row, o0, o1, o2, o3, o4);
}

// Step t on tile rows y0-1 .. y0+TBY (stage row py <-> global row y0-1+py), one warp per row, storing each
// plane's result only where step t+1 reads it (planes 0, 1, 3 at stage row py-1, plane 2 at py, plane 4 at
// py-2); then the ring sites x0-1 (plane 1 only) and x0+TBX (plane 3 only) of rows y0 .. y0+TBY-1.  Also
// reads into clb the c_L^2 of the warp's step-(t+1) row (and with MU into dbx, dby its gradient of ln mu), as
// the medium stage is reloaded before step t+1.
// With POLE (a dispersive pole) every warp computes one row (TBY + 2 warps) and step t+1 of row py runs on the
// same warp, so the pole's state of the warp's owned row stays in registers (Jh, Ph: J at t+1/2, P at t+1).
template <int TBY, int NT, bool EV, bool MU = false, bool AN = false, bool POLE = false>
__device__ __forceinline__ void tb_step_a(const StepArgs &a, const float *IN, const float *CL, float *P, int x0,
                                          int y0, long long t, float4 &clb, float4 &dbx, float4 &dby, Pole4 &ph,
                                          const float *PS = nullptr, const float *JS = nullptr) {
    using Gm = TbGeom<TBY>;
    constexpr int R = Gm::R, NW = NT / 32, PL = Gm::P_PL, DX = R * TW, DY = 2 * R * TW;
    static_assert(!POLE || NW == R, "with a pole: one warp per row of step t");
    const Grid &G = a.g;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int c = 4 + 4 * lane;
    const int bw = warp - (POLE ? 1 : 0);  // the warp's output row of step t+1
    if (bw >= 0 && bw < TBY) {
        clb = lds4(CL + (bw + 1) * TW + c);
        if (MU) {
            dbx = lds4(CL + DX + (bw + 1) * TW + c);
            dby = lds4(CL + DY + (bw + 1) * TW + c);
        }
    }
    for (int py = warp; py < R; py += NW) {
        const Pull4 g(IN, Gm::IN_PL, py, c);
        const float4 cl = lds4(CL + py * TW + c);
        const float4 dlx = MU ? lds4(CL + DX + py * TW + c) : cl, dly = MU ? lds4(CL + DY + py * TW + c) : cl;
        const bool own = py >= 1 && py <= TBY;
        Pole4 pp;
        if (POLE) {  // from the stages loaded with the window
            constexpr int JPL = TbGeom<TBY, false, true>::JS_PL;
            pp.P = lds4(PS + py * TW + c);
            pp.J = pp.wp = pp.wr = pp.gm = make_float4(0.f, 0.f, 0.f, 0.f);
            // J is updated in place by the tile owning the site.  Lanes past nx (rows past ny) of a ragged last
            // tile read J at wrapped sites of another tile, which may be updating them: their pole results only
            // ever reach the row padding or are dropped, while the collisions they feed use P at t, which no
            // launch writes in place.
            if (own) {
                const float *js = JS + (py - 1) * TBX + 4 * lane;
                pp.J = lds4(js);
                pp.wp = lds4(js + JPL);
                pp.wr = lds4(js + 2 * JPL);
                pp.gm = lds4(js + 3 * JPL);
            }
        }
        float4 o0, o1, o2, o3, o4;
        if (EV && row_events(a, y0 - 1 + py))
            tb_update4m<true, MU, Pull4, AN, POLE>(a, g, cl, dlx, dly, x0, y0 - 1 + py, t, own, o0, o1, o2, o3, o4,
                                                   &pp);
        else
            tb_update4m<false, MU, Pull4, AN, POLE>(a, g, cl, dlx, dly, x0, y0 - 1 + py, t, own, o0, o1, o2, o3, o4,
                                                    &pp);
        if (POLE && own) ph = pp;  // J(t+1/2), P(t+1) and the parameters stay with this warp for step t+1
        float *Pr = P + c;
        if (py >= 1 && py <= TBY) {
            sts4(Pr + 0 * PL + (py - 1) * TW, o0);
            sts4(Pr + 1 * PL + (py - 1) * TW, o1);
            sts4(Pr + 3 * PL + (py - 1) * TW, o3);
        }
        if (py < TBY) sts4(Pr + 2 * PL + py * TW, o2);
        if (py >= 2) sts4(Pr + 4 * PL + (py - 2) * TW, o4);
    }
    // ring sites go to the warps with one row fewer (from warp R % NW on)
    int k0 = tid - 32 * (R % NW);
    if (k0 < 0) k0 += NT;
    for (int k = k0; k < 2 * TBY; k += NT) {
        const int py = (k >> 1) + 1, cc = (k & 1) ? TBX + 4 : 3;
        const float *r = IN + py * TW + cc;
        const float q0 = r[0], q1 = r[Gm::IN_PL - 1], q2 = r[2 * Gm::IN_PL], q3 = r[3 * Gm::IN_PL + 1],
                    q4 = r[4 * Gm::IN_PL];
        const float ck = CL[py * TW + cc];
        float shat = MU ? mu_source(q4 - q2, q1 - q3, CL[DX + py * TW + cc], CL[DY + py * TW + cc]) : 0.f;
        Out5 o;
        if (AN || POLE) {
            const float r = AN ? a.med.ar : 1.f, ri = AN ? __fdiv_rn(1.f, r) : 1.f, fs = __fadd_rn(r, ri);
            const int gx = wrapi(x0 - 4 + cc, G.nx), gy = wrapi(y0 - 1 + py, G.ny);
            const float pz = POLE ? PS[py * TW + cc] : 0.f;
            if (EV)
                shat = site_events(a, gx, gy, t, false, q0, q1, q2, q3, q4, ck, 0.f, pz, r, ri, AN ? a.med.amu : 1.f);
            o = AN ? collide2d_an(q0, q1, q2, q3, q4, ck, shat, r, ri, fs, pz)
                   : collide2d_pole_iso(q0, q1, q2, q3, q4, ck, shat, pz);
        } else {
            if (EV)
                shat = site_events(a, wrapi(x0 - 4 + cc, G.nx), wrapi(y0 - 1 + py, G.ny), t, false, q0, q1, q2, q3,
                                   q4, ck, shat);
            o = collide2d(q0, q1, q2, q3, q4, ck, shat);
        }
        if (k & 1)
            P[3 * PL + (py - 1) * TW + cc] = o.o3;
        else
            P[1 * PL + (py - 1) * TW + cc] = o.o1;
    }
}

// Step t+1 on tile row y0 + warp from the t+1 stage, written as 16-byte streaming stores.
template <int TBY, bool EV, bool MU = false, bool AN = false, bool POLE = false>
__device__ __forceinline__ void tb_step_b(const StepArgs &a, const float *P, float4 clb, float4 dbx, float4 dby,
                                          int x0, int y0, long long t, const Pole4 &ph = Pole4()) {
    const Grid &G = a.g;
    const int lane = threadIdx.x & 31, oy = (threadIdx.x >> 5) - (POLE ? 1 : 0);
    const int gy = y0 + oy;
    if (oy < 0 || oy >= TBY || gy >= G.ny) return;
    const int c = 4 + 4 * lane;
    const Pull4 g(P, TbGeom<TBY>::P_PL, oy, c);
    Pole4 pp;
    if (POLE) pp = ph;
    float4 o0, o1, o2, o3, o4;
    if (EV && row_events(a, gy))
        tb_update4m<true, MU, Pull4, AN, POLE>(a, g, clb, dbx, dby, x0, gy, t + 1, true, o0, o1, o2, o3, o4, &pp);
    else
        tb_update4m<false, MU, Pull4, AN, POLE>(a, g, clb, dbx, dby, x0, gy, t + 1, true, o0, o1, o2, o3, o4, &pp);
    if (x0 + 4 * lane < G.pitch) {  // pitch is a multiple of 4: a lane's 4 columns are all in or all out
        const long long off = (long long)gy * G.pitch + x0 + 4 * lane;
        float4 *o = reinterpret_cast<float4 *>(static_cast<float *>(a.out.data) + off);
        const long long pl4 = G.plane / 4;
        __stcs(o, o0);
        __stcs(o + pl4, o1);
        __stcs(o + 2 * pl4, o2);
        __stcs(o + 3 * pl4, o3);
        __stcs(o + 4 * pl4, o4);
        if (POLE) {  // J in place (only this site reads it), P to the plane of the output's parity
            *reinterpret_cast<float4 *>(a.med.J + off) = pp.J;
            *reinterpret_cast<float4 *>(a.med.Pw + off) = pp.P;
        }
    }
}
#undef TB_SET

// One persistent CTA per SM slot; CTA b takes tiles b, b + gridDim.x, ... (row-major over the tile grid).
// The window of the next tile is loaded while step t+1 of the current one is computed.
template <int TBY, int NT, int MINB, bool MU = false, bool AN = false, bool POLE = false>
__global__ void __launch_bounds__(NT, MINB)
    step2d_tb2(StepArgs a, const __grid_constant__ CUtensorMap tmIn, const __grid_constant__ CUtensorMap tmCL,
               const __grid_constant__ CUtensorMap tmDL, const __grid_constant__ PoleMaps<POLE> pm, int use_tma,
               int ntx, int nty, int dq, int dr) {
    static_assert(NT / 32 >= TBY, "one warp per row of step t+1");
    using Gm = TbGeom<TBY, MU, POLE>;
    extern __shared__ __align__(1024) float sm[];
    float *IN = sm;              // [5][TBY+2][TW], shifted planes at t
    float *CL = sm + Gm::IN_SZ;  // [1 or 3][TBY+2][TW]: c_L^2 (and d_x ln mu, d_y ln mu)
    float *P = CL + Gm::CL_SZ;   // [5][TBY][TW], shifted planes at t+1
    float *PS = P + Gm::P_SZ;    // with a pole: [TBY+2][TW] P at t
    float *JS = PS + Gm::PS_SZ;  // with a pole: [4][TBY][TBX] J, wp2, wr2, gamma of the owned sites
    unsigned long long *mb = reinterpret_cast<unsigned long long *>(sm + Gm::SZ);
    const Grid &G = a.g;
    const int tid = threadIdx.x;
    if (smem_u32(sm) & 127) use_tma = 0;  // TMA destinations here are 128-byte aligned; else element copies
    int tx = blockIdx.x % ntx, ty = blockIdx.x / ntx;
    if (ty >= nty) return;
    const unsigned mbar = smem_u32(mb);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    unsigned parity = 0;  // next phase of the mbarrier to wait for
    const unsigned long long wait_limit = g_wait_limit_ns;
    tb_load<TBY, MU, POLE>(a, tx * TBX, ty * TBY, IN, CL, mbar, use_tma && tb_interior<TBY>(tx * TBX, ty * TBY, G),
                           &tmIn, &tmCL, NT, &tmDL, PS, JS, &pm);
    asm volatile("cp.async.commit_group;\n" ::);
    bool events = tb_events<TBY>(a, ty * TBY);
    const long long t = a.t;
    while (ty < nty) {
        int ntx_ = tx + dr, nty_ = ty + dq;  // next tile of this CTA
        if (ntx_ >= ntx) {
            ntx_ -= ntx;
            nty_++;
        }
        const bool has_next = nty_ < nty;
        const bool events_next = has_next && tb_events<TBY>(a, nty_ * TBY);  // latency hidden behind this tile
        const int x0 = tx * TBX, y0 = ty * TBY;
        asm volatile("cp.async.wait_group 0;\n" ::);
        bool ok = true;
        if (use_tma && tb_interior<TBY>(x0, y0, G)) {
            ok = mbar_wait(mbar, parity, wait_limit);
            parity ^= 1u;
        }
        // every thread's copies have landed, and step t+1 of the previous tile is done with P
        if (__syncthreads_or(!ok)) {  // a TMA load never completed: flag it, let it drain (bounded), stop
            if (tid == 0) atomicExch(&g_tb_timeouts, 1);
            mbar_wait(mbar, parity ^ 1u, kDrainNs);  // drain what is in flight
            return;
        }
        float4 clb = make_float4(0.f, 0.f, 0.f, 0.f), dbx = clb, dby = clb;
        Pole4 ph;
        if (events)
            tb_step_a<TBY, NT, true, MU, AN, POLE>(a, IN, CL, P, x0, y0, t, clb, dbx, dby, ph, PS, JS);
        else
            tb_step_a<TBY, NT, false, MU, AN, POLE>(a, IN, CL, P, x0, y0, t, clb, dbx, dby, ph, PS, JS);
        __syncthreads();
        if (has_next)  // the t stage, the medium stage (and the pole's stages) are free: load the next tile
            tb_load<TBY, MU, POLE>(a, ntx_ * TBX, nty_ * TBY, IN, CL, mbar,
                                   use_tma && tb_interior<TBY>(ntx_ * TBX, nty_ * TBY, G), &tmIn, &tmCL, NT, &tmDL,
                                   PS, JS, &pm);
        asm volatile("cp.async.commit_group;\n" ::);
        if (events)
            tb_step_b<TBY, true, MU, AN, POLE>(a, P, clb, dbx, dby, x0, y0, t, ph);
        else
            tb_step_b<TBY, false, MU, AN, POLE>(a, P, clb, dbx, dby, x0, y0, t, ph);
        tx = ntx_;
        ty = nty_;
        events = events_next;
    }
    asm volatile("cp.async.wait_group 0;\n" ::);
}

// =====================================================================================================
// Two steps per launch over a batch of independent media (FP32, uniform mu, periodic).  The batch keeps its members'
// states in a packed layout of its own: member m occupies packed rows r0[m] .. r0[m] + ny + 3 of planes W floats
// wide, packed row r0[m] + 2 + y <-> member row y in [-2, ny + 1] and packed column x + 4 <-> member column x.  The
// two rows and columns just outside the member hold its periodic images (a halo), so every tile's window (rows
// y0 - 2 .. y0 + TBY + 1, columns x0 - 4 .. x0 + TBX + 3) is one TMA box without wrap, as for an interior tile of a
// single grid.  A launch reads one packed buffer and writes the other; a tile writes each output site and its images
// in the halo (sites within two of an edge), so the next launch finds the halo current.  Sources and receivers use
// each member's own tables and coordinates, and the site updates are those of step2d_tb2, so every member's result
// is bit-identical to its single steps.  The state is packed at the start of a call and unpacked into each member's
// own buffer at its end (batch_pack_kernel).

// Pack (unpack == 0) or unpack a batch's states, one block per packed row (its member found by bisection of r0):
// pack writes rows -2 .. ny+1 and columns -2 .. nx+1 of the five planes and of c_L^2 from the member's buffer (the
// periodic images outside it); unpack writes rows 0 .. ny-1, columns 0 .. nx-1 back.  The member's buffer is that
// of args[2 m + par]'s input.
__global__ void batch_pack_kernel(const StepArgs *__restrict__ args, int par, const int *__restrict__ r0, int n,
                                  BatchPacked pk, int which, int unpack) {
    const int b = blockIdx.x;
    int lo = 0, hi = n;  // r0[lo] <= b < r0[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(r0 + mid) <= b) lo = mid;
        else hi = mid;
    }
    const StepArgs &a = args[2 * lo + par];
    const int nx = a.g.nx, ny = a.g.ny, pitch = a.g.pitch;
    const long long plane = a.g.plane;
    const int y = b - __ldg(r0 + lo) - 2;
    float *pb = (which ? pk.buf[1] : pk.buf[0]) + (long long)b * pk.W + 4;
    float *mem = static_cast<float *>(a.in.data);
    if (unpack) {
        if (y < 0 || y >= ny) return;
        for (int x = threadIdx.x; x < nx; x += blockDim.x)
            for (int p = 0; p < 5; p++) mem[p * plane + (long long)y * pitch + x] = pb[p * pk.plane + x];
        return;
    }
    const long long yr = (long long)wrapi(y, ny) * pitch;
    float *pc = pk.cl + (long long)b * pk.W + 4;
    for (int x = (int)threadIdx.x - 2; x <= nx + 1; x += blockDim.x) {
        const long long src = yr + wrapi(x, nx);
        for (int p = 0; p < 5; p++) pb[p * pk.plane + x] = mem[p * plane + src];
        pc[x] = a.med.cL2[src];
    }
}

// Step t+1 on tile row y0 + warp, written to the packed output with the row's and the lane's halo images.
template <int TBY, bool EV>
__device__ __forceinline__ void tb_step_b_packed(const StepArgs &a, const float *P, float4 clb, int x0, int y0,
                                                 long long t, float *out, long long pplane, int W, int prow0, int nx,
                                                 int ny) {
    const int lane = threadIdx.x & 31, oy = threadIdx.x >> 5;
    const int gy = y0 + oy;
    if (oy >= TBY || gy >= ny) return;
    const int c = 4 + 4 * lane;
    const Pull4 g(P, TbGeom<TBY>::P_PL, oy, c);
    float4 o[5];
    Pole4 pp;
    if (EV && row_events(a, gy))
        tb_update4m<true, false, Pull4>(a, g, clb, clb, clb, x0, gy, t + 1, true, o[0], o[1], o[2], o[3], o[4], &pp);
    else
        tb_update4m<false, false, Pull4>(a, g, clb, clb, clb, x0, gy, t + 1, true, o[0], o[1], o[2], o[3], o[4], &pp);
    const int xs = x0 + 4 * lane;  // the lane's first site
    if (xs >= nx) return;
    auto row_at = [&](int yy) { return out + (long long)(prow0 + 2 + yy) * W + 4; };
    auto store_row = [&](int yy) {
        float *r = row_at(yy) + xs;
        if (xs + 3 < nx) {
#pragma unroll
            for (int p = 0; p < 5; p++) __stcs(reinterpret_cast<float4 *>(r + p * pplane), o[p]);
        } else {
#pragma unroll
            for (int j = 0; j < 3; j++)
                if (xs + j < nx)
#pragma unroll
                    for (int p = 0; p < 5; p++) r[p * pplane + j] = TB_COMP(o[p], j);
        }
    };
    store_row(gy);
    for (int yy = gy + ny; yy <= ny + 1; yy += ny) store_row(yy);  // images in the upper halo rows
    for (int yy = gy - ny; yy >= -2; yy -= ny) store_row(yy);      // and in the lower ones
    if (xs < 2 || xs + 3 >= nx - 2) {  // sites within two of the left or right edge: their column images
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int x = xs + j;
            if (x >= nx) break;
            for (int xi = x + nx; xi <= nx + 1; xi += nx)
                for (int yy = gy - ((gy + 2) / ny) * ny; yy <= ny + 1; yy += ny)
#pragma unroll
                    for (int p = 0; p < 5; p++) row_at(yy)[p * pplane + xi] = TB_COMP(o[p], j);
            for (int xi = x - nx; xi >= -2; xi -= nx)
                for (int yy = gy - ((gy + 2) / ny) * ny; yy <= ny + 1; yy += ny)
#pragma unroll
                    for (int p = 0; p < 5; p++) row_at(yy)[p * pplane + xi] = TB_COMP(o[p], j);
        }
    }
}

template <int TBY, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    step2d_batch_tb2(const StepArgs *__restrict__ args, const BatchTile *__restrict__ tiles, long long ntiles,
                     const long long *__restrict__ t0p, int toff, int par, BatchPacked pk,
                     const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                     const __grid_constant__ CUtensorMap tmCL) {
    static_assert(NT / 32 >= TBY, "one warp per row of step t+1");
    using Gm = TbGeom<TBY>;
    extern __shared__ __align__(1024) float sm[];
    float *IN = sm;
    float *CL = sm + Gm::IN_SZ;
    float *P = CL + Gm::CL_SZ;
    unsigned long long *mb = reinterpret_cast<unsigned long long *>(sm + Gm::SZ);
    const int tid = threadIdx.x;
    long long k = blockIdx.x;
    if (k >= ntiles) return;
    if (smem_u32(sm) & 127) return;  // the launch checks alignment on the host side too (TMA destinations)
    const CUtensorMap *tmIn = par ? &tmB : &tmA;
    float *out = par ? pk.buf[0] : pk.buf[1];  // (a select: an index into the parameter would copy it to the stack)
    const unsigned mbar = smem_u32(mb);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    const unsigned long long wait_limit = g_wait_limit_ns;
    unsigned parity = 0;
    const long long t = *t0p + toff;
    // the window of a tile: five shifted planes and c_L^2 as TMA boxes (member column x0 - 4 <-> packed x0,
    // member row y0 - 1 <-> packed row py)
    auto load = [&](int x0, int py) {
        if (tid == 0) {
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(Gm::TMA_BYTES)
                         : "memory");
#pragma unroll
            for (int p = 0; p < 5; p++) tma_load_3d(IN + p * Gm::IN_PL, tmIn, x0, py + in_shift(p), p, mbar);
            tma_load_2d(CL, &tmCL, x0, py, mbar);
        }
    };
    BatchTile cur = tiles[k];
    load(cur.x0, cur.py);
    while (true) {
        const long long kn = k + gridDim.x;
        const bool has_next = kn < ntiles;
        BatchTile nxt;
        if (has_next) nxt = tiles[kn];  // one 32-byte descriptor, in flight while this tile is computed
        const StepArgs &a = args[2 * cur.m];
        const int x0 = cur.x0, y0 = cur.y0;
        const bool events = cur.ev;
        const bool ok = mbar_wait(mbar, parity, wait_limit);
        parity ^= 1u;
        // the window has landed, and step t+1 of the previous tile is done with P
        if (__syncthreads_or(!ok)) {  // a TMA load never completed: flag it, let it drain (bounded), stop
            if (tid == 0) atomicExch(&g_tb_timeouts, 1);
            mbar_wait(mbar, parity ^ 1u, kDrainNs);  // drain what is in flight
            return;
        }
        float4 clb = make_float4(0.f, 0.f, 0.f, 0.f), dbx = clb, dby = clb;
        Pole4 ph;
        if (events)
            tb_step_a<TBY, NT, true>(a, IN, CL, P, x0, y0, t, clb, dbx, dby, ph);
        else
            tb_step_a<TBY, NT, false>(a, IN, CL, P, x0, y0, t, clb, dbx, dby, ph);
        __syncthreads();
        if (has_next) load(nxt.x0, nxt.py);  // the t stage and c_L^2 are free
        const int prow0 = cur.py - y0 - 1;  // the member's first packed row
        if (events)
            tb_step_b_packed<TBY, true>(a, P, clb, x0, y0, t, out, pk.plane, pk.W, prow0, cur.nx, cur.ny);
        else
            tb_step_b_packed<TBY, false>(a, P, clb, x0, y0, t, out, pk.plane, pk.W, prow0, cur.nx, cur.ny);
        if (!has_next) break;
        k = kn;
        cur = nxt;
    }
}

// Tensor maps of the packed buffers ([5][rows][W] floats, box: one plane of TBY+2 rows of TW) and of the packed
// c_L^2; false if unavailable.
template <int TBY>
static bool make_batch_maps(const BatchPacked &pk, long long rows, CUtensorMap *mA, CUtensorMap *mB,
                            CUtensorMap *mCL) {
    EncodeTiled fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims3[3] = {(cuuint64_t)pk.W, (cuuint64_t)rows, 5};
    const cuuint64_t str3[2] = {(cuuint64_t)pk.W * 4, (cuuint64_t)pk.plane * 4};
    const cuuint32_t box3[3] = {(cuuint32_t)TW, (cuuint32_t)(TBY + 2), 1};
    const cuuint32_t one[3] = {1, 1, 1};
    for (int k = 0; k < 2; k++)
        if (fn(k ? mB : mA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, pk.buf[k], dims3, str3, box3, one,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    const cuuint64_t dims2[2] = {(cuuint64_t)pk.W, (cuuint64_t)rows};
    const cuuint64_t str2[1] = {(cuuint64_t)pk.W * 4};
    const cuuint32_t box2[2] = {(cuuint32_t)TW, (cuuint32_t)(TBY + 2)};
    return fn(mCL, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(pk.cl), dims2, str2, box2, one,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int TBY, int NT, int MINB>
static cudaError_t launch_batch_tb(const StepArgs *args, const BatchTile *tiles, long long ntiles,
                                   const long long *t0p, int toff, int par, const BatchPacked &pk, long long rows,
                                   cudaStream_t s) {
    using Gm = TbGeom<TBY>;
    static int per_sm = 0, nsm = 0;
    if (!per_sm) {
        cudaError_t e = cudaFuncSetAttribute(step2d_batch_tb2<TBY, NT, MINB>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Gm::BYTES);
        if (e != cudaSuccess) return e;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step2d_batch_tb2<TBY, NT, MINB>, NT, Gm::BYTES);
        if (per_sm < 1) per_sm = 1;
    }
    CUtensorMap mA, mB, mCL;
    if (!make_batch_maps<TBY>(pk, rows, &mA, &mB, &mCL)) return cudaErrorNotSupported;
    const long long slots = (long long)per_sm * nsm;
    const unsigned blocks = (unsigned)(ntiles < slots ? ntiles : slots);
    if (blocks == 0) return cudaSuccess;
    step2d_batch_tb2<TBY, NT, MINB><<<blocks, NT, Gm::BYTES, s>>>(args, tiles, ntiles, t0p, toff, par, pk, mA, mB, mCL);
    return cudaGetLastError();
}

int batch_tb2_rows(int shape) { return shape == 2 ? 8 : shape == 3 ? 10 : shape == 4 ? 12 : 6; }

cudaError_t launch_batch_tb2(const StepArgs *args, const BatchTile *tiles, long long ntiles, const long long *t0p,
                             int toff, int par, const BatchPacked &pk, long long rows, int shape, cudaStream_t s) {
    switch (shape) {
        case 1: return launch_batch_tb<6, 256, 4>(args, tiles, ntiles, t0p, toff, par, pk, rows, s);
        case 2: return launch_batch_tb<8, 320, 3>(args, tiles, ntiles, t0p, toff, par, pk, rows, s);
        case 3: return launch_batch_tb<10, 384, 3>(args, tiles, ntiles, t0p, toff, par, pk, rows, s);
        case 4: return launch_batch_tb<12, 448, 2>(args, tiles, ntiles, t0p, toff, par, pk, rows, s);
        default: return launch_batch_tb<6, 256, 5>(args, tiles, ntiles, t0p, toff, par, pk, rows, s);
    }
}

cudaError_t launch_batch_pack(const StepArgs *args, int par, const int *r0, int n, long long rows,
                              const BatchPacked &pk, int which, bool unpack, cudaStream_t s) {
    if (rows <= 0) return cudaSuccess;
    batch_pack_kernel<<<(unsigned)rows, 256, 0, s>>>(args, par, r0, n, pk, which, unpack ? 1 : 0);
    return cudaGetLastError();
}

// =====================================================================================================
// Three steps per launch, FP32 storage.  Stage S0 (state at t, staged from HBM) -> step A -> S1 (t+1) -> step B
// -> S2 (t+2) -> step C -> HBM (t+3).  Output rows y0 .. y0+TBY-1; step B computes rows y0-1 .. y0+TBY and
// columns x0-1 .. x0+TBX (one ring column), step A rows y0-2 .. y0+TBY+1 and columns x0-2 .. x0+TBX+1 (two).
// Every stage is staged shifted by the pull offsets, so a stage stores plane p of its row r at row
// r - 1 - in_shift(p) of the next stage (when that row exists), exactly as in the two-step kernel; all columns
// are indexed as in the two-step kernel (shared column j <-> x0-4+j).  HBM traffic: 44 bytes per site per three
// steps.
template <int TBY>
struct TbGeom3 {
    static constexpr int R0 = TBY + 4, R1 = TBY + 2, R2 = TBY;  // rows per plane of S0, S1, S2
    static constexpr int up32(int n) { return (n + 31) / 32 * 32; }
    static constexpr int S0_PL = up32(R0 * TW), S1_PL = R1 * TW, S2_PL = R2 * TW;
    static constexpr int S0_SZ = up32(5 * S0_PL), CL_SZ = up32(R0 * TW), S1_SZ = up32(5 * S1_PL);
    static constexpr int S2_SZ = up32(5 * S2_PL);
    static constexpr int SZ = S0_SZ + CL_SZ + S1_SZ + S2_SZ;
    static constexpr size_t BYTES = sizeof(float) * SZ + sizeof(unsigned long long);
    static constexpr unsigned TMA_BYTES = sizeof(float) * 6 * R0 * TW;
};

template <int TBY>
__device__ __forceinline__ bool tb3_interior(int x0, int y0, const Grid &G) {
    return x0 - 4 >= 0 && x0 + TBX + 4 <= G.nx && y0 - 3 >= 0 && y0 + TBY + 3 <= G.ny;
}

// Window of a tile: S0 plane p rows 0 .. TBY+3 <-> global rows y0-2+r+in_shift(p); c_L^2 rows y0-2 .. y0+TBY+1.
template <int TBY>
__device__ __forceinline__ void tb3_load(const StepArgs &a, int x0, int y0, float *S0, float *CL, unsigned mbar,
                                         bool tma, const CUtensorMap *tmIn, const CUtensorMap *tmCL, int nt) {
    using Gm = TbGeom3<TBY>;
    constexpr int R = Gm::R0, Q = TW / 4;
    if (tma) {
        if (threadIdx.x == 0) {
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(Gm::TMA_BYTES)
                         : "memory");
#pragma unroll
            for (int p = 0; p < 5; p++) tma_load_3d(S0 + p * Gm::S0_PL, tmIn, x0 - 4, y0 - 2 + in_shift(p), p, mbar);
            tma_load_2d(CL, tmCL, x0 - 4, y0 - 2, mbar);
        }
        return;
    }
    const Grid &G = a.g;
    const float *in = static_cast<const float *>(a.in.data);
    const int tid = threadIdx.x;
    if (((x0 - 4 >= 0) && (x0 + TBX + 4 <= G.nx)) || (G.nx & 3) == 0) {
        for (int k = tid; k < 6 * R * Q; k += nt) {
            const int pr = k / Q, q = k - pr * Q;
            const int pl = pr / R, r = pr - pl * R;
            const int gx = wrapi(x0 - 4 + 4 * q, G.nx);
            if (pl < 5) {
                const int gy = wrapi(y0 - 2 + r + in_shift(pl), G.ny);
                tb_cpa16(S0 + pl * Gm::S0_PL + r * TW + 4 * q, in + pl * G.plane + (long long)gy * G.pitch + gx);
            } else {
                const int gy = wrapi(y0 - 2 + r, G.ny);
                tb_cpa16(CL + r * TW + 4 * q, a.med.cL2 + (long long)gy * G.pitch + gx);
            }
        }
    } else {
        for (int k = tid; k < 6 * R * TW; k += nt) {
            const int pr = k / TW, c = k - pr * TW;
            const int pl = pr / R, r = pr - pl * R;
            const int gx = wrapi(x0 - 4 + c, G.nx);
            if (pl < 5) {
                const int gy = wrapi(y0 - 2 + r + in_shift(pl), G.ny);
                tb_cpa4(S0 + pl * Gm::S0_PL + r * TW + c, in + pl * G.plane + (long long)gy * G.pitch + gx);
            } else {
                const int gy = wrapi(y0 - 2 + r, G.ny);
                tb_cpa4(CL + r * TW + c, a.med.cL2 + (long long)gy * G.pitch + gx);
            }
        }
    }
}

// Store the five outputs of stage row r at column(s) c of the next stage D (rows RD, plane stride DPL):
// plane p goes to row r - 1 - in_shift(p) when 0 <= that < RD.
template <int RD, int DPL>
__device__ __forceinline__ void tb3_store4(float *D, int r, int c, float4 o0, float4 o1, float4 o2, float4 o3,
                                           float4 o4) {
    float *d = D + c;
    if (r >= 1 && r <= RD) {
        sts4(d + 0 * DPL + (r - 1) * TW, o0);
        sts4(d + 1 * DPL + (r - 1) * TW, o1);
        sts4(d + 3 * DPL + (r - 1) * TW, o3);
    }
    if (r < RD) sts4(d + 2 * DPL + r * TW, o2);
    if (r >= 2 && r <= RD + 1) sts4(d + 4 * DPL + (r - 2) * TW, o4);
}
template <int RD, int DPL>
__device__ __forceinline__ void tb3_store1(float *D, int r, int c, const Out5 &o) {
    if (r >= 1 && r <= RD) {
        D[0 * DPL + (r - 1) * TW + c] = o.o0;
        D[1 * DPL + (r - 1) * TW + c] = o.o1;
        D[3 * DPL + (r - 1) * TW + c] = o.o3;
    }
    if (r < RD) D[2 * DPL + r * TW + c] = o.o2;
    if (r >= 2 && r <= RD + 1) D[4 * DPL + (r - 2) * TW + c] = o.o4;
}

// One site of a ring column cc of stage S (plane stride SPL) at stage row r, c_L^2 ck, global (gx, gy), time t.
template <bool EV>
__device__ __forceinline__ Out5 tb3_site(const StepArgs &a, const float *S, int SPL, int r, int cc, float ck, int gx,
                                         int gy, long long t, bool owned) {
    const float *q = S + r * TW + cc;
    const float q0 = q[0], q1 = q[SPL - 1], q2 = q[2 * SPL], q3 = q[3 * SPL + 1], q4 = q[4 * SPL];
    if (EV) {
        const Grid &G = a.g;
        const float shat = site_events(a, wrapi(gx, G.nx), wrapi(gy, G.ny), t, owned, q0, q1, q2, q3, q4, ck);
        return collide2d(q0, q1, q2, q3, q4, ck, shat);
    }
    return collide2d_free(q0, q1, q2, q3, q4, ck);
}

// Steps A and B of a tile (the staged window in S0/CL must be complete).  Reads into clb / clc the c_L^2 of the
// warp's step-B and step-C rows and into clr the ring sites' c_L^2 of step B, as c_L^2 is reloaded after A.
template <int TBY, int NT, bool EV>
__device__ __forceinline__ void tb3_step_a(const StepArgs &a, const float *S0, const float *CL, float *S1, int x0,
                                           int y0, long long t, float4 &clb, float4 &clc, float &clr) {
    using Gm = TbGeom3<TBY>;
    constexpr int NW = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int c = 4 + 4 * lane;
    // c_L^2 row of global row g is g - (y0 - 2)
    if (warp < Gm::R1) clb = lds4(CL + (warp + 1) * TW + c);
    if (warp < Gm::R2) clc = lds4(CL + (warp + 2) * TW + c);
    {
        const int k = tid - 32 * Gm::R0;  // step-B ring sites (rows 0 .. TBY+1, columns 3 and TBX+4) on spare warps
        if (k >= 0 && k < 2 * Gm::R1) clr = CL[((k >> 1) + 1) * TW + ((k & 1) ? TBX + 4 : 3)];
    }
    for (int r = warp; r < Gm::R0; r += NW) {
        const Pull4 g(S0, Gm::S0_PL, r, c);
        const float4 cl = lds4(CL + r * TW + c);
        float4 o0, o1, o2, o3, o4;
        tb_update4<EV>(a, g, cl, x0, y0 - 2 + r, t, r >= 2 && r < TBY + 2, o0, o1, o2, o3, o4);
        tb3_store4<Gm::R1, Gm::S1_PL>(S1, r, c, o0, o1, o2, o3, o4);
    }
    // ring columns x0-2, x0-1, x0+TBX, x0+TBX+1 (shared columns 2, 3, TBX+4, TBX+5), on the warps after the rows
    for (int k = tid - 32 * Gm::R0; k >= 0 && k < 4 * Gm::R0; k += NT) {
        const int r = k >> 2, cc = (k & 3) < 2 ? 2 + (k & 3) : TBX + 2 + (k & 3);
        const Out5 o = tb3_site<EV>(a, S0, Gm::S0_PL, r, cc, CL[r * TW + cc], x0 - 4 + cc, y0 - 2 + r, t, false);
        tb3_store1<Gm::R1, Gm::S1_PL>(S1, r, cc, o);
    }
}

template <int TBY, int NT, bool EV>
__device__ __forceinline__ void tb3_step_b(const StepArgs &a, const float *S1, float *S2, int x0, int y0, long long t,
                                           float4 clb, float clr) {
    using Gm = TbGeom3<TBY>;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int c = 4 + 4 * lane;
    if (warp < Gm::R1) {
        const int r = warp;
        const Pull4 g(S1, Gm::S1_PL, r, c);
        float4 o0, o1, o2, o3, o4;
        tb_update4<EV>(a, g, clb, x0, y0 - 1 + r, t + 1, r >= 1 && r <= TBY, o0, o1, o2, o3, o4);
        tb3_store4<Gm::R2, Gm::S2_PL>(S2, r, c, o0, o1, o2, o3, o4);
    }
    const int k = tid - 32 * Gm::R0;
    if (k >= 0 && k < 2 * Gm::R1) {  // ring columns x0-1 (plane 1 needed) and x0+TBX (plane 3)
        const int r = k >> 1, cc = (k & 1) ? TBX + 4 : 3;
        const Out5 o = tb3_site<EV>(a, S1, Gm::S1_PL, r, cc, clr, x0 - 4 + cc, y0 - 1 + r, t + 1, false);
        if (r >= 1 && r <= TBY) {
            if (k & 1)
                S2[3 * Gm::S2_PL + (r - 1) * TW + cc] = o.o3;
            else
                S2[1 * Gm::S2_PL + (r - 1) * TW + cc] = o.o1;
        }
    }
}

template <int TBY, bool EV>
__device__ __forceinline__ void tb3_step_c(const StepArgs &a, const float *S2, int x0, int y0, long long t,
                                           float4 clc) {
    const Grid &G = a.g;
    const int lane = threadIdx.x & 31, oy = threadIdx.x >> 5;
    const int gy = y0 + oy;
    if (oy >= TBY || gy >= G.ny) return;
    const int c = 4 + 4 * lane;
    const Pull4 g(S2, TbGeom3<TBY>::S2_PL, oy, c);
    float4 o0, o1, o2, o3, o4;
    tb_update4<EV>(a, g, clc, x0, gy, t + 2, true, o0, o1, o2, o3, o4);
    if (x0 + 4 * lane < G.pitch) {
        float4 *o = reinterpret_cast<float4 *>(static_cast<float *>(a.out.data) + (long long)gy * G.pitch + x0 +
                                               4 * lane);
        const long long pl4 = G.plane / 4;
        __stcs(o, o0);
        __stcs(o + pl4, o1);
        __stcs(o + 2 * pl4, o2);
        __stcs(o + 3 * pl4, o3);
        __stcs(o + 4 * pl4, o4);
    }
}

template <int TBY>
__device__ __forceinline__ bool tb3_events(const StepArgs &a, int y0) {
    const Grid &G = a.g;
    return a.evt.rowptr && !(y0 >= 2 && y0 + TBY + 2 <= G.ny &&
                             __ldg(a.evt.rowptr + y0 - 2) == __ldg(a.evt.rowptr + y0 + TBY + 2));
}

// Persistent like step2d_tb2; the window of the next tile loads during steps B and C of the current one.
template <int TBY, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    step2d_tb3(StepArgs a, const __grid_constant__ CUtensorMap tmIn, const __grid_constant__ CUtensorMap tmCL,
               int use_tma, int ntx, int nty, int dq, int dr) {
    using Gm = TbGeom3<TBY>;
    static_assert(NT / 32 >= Gm::R0 + 1, "one warp per step-A row, spare threads for the ring columns");
    static_assert(NT - 32 * Gm::R0 >= 4 * Gm::R0, "one thread per step-A ring site");
    extern __shared__ __align__(1024) float sm[];
    float *S0 = sm;
    float *CL = sm + Gm::S0_SZ;
    float *S1 = CL + Gm::CL_SZ;
    float *S2 = S1 + Gm::S1_SZ;
    const unsigned mbar = smem_u32(S2 + Gm::S2_SZ);
    const Grid &G = a.g;
    const int tid = threadIdx.x;
    if (smem_u32(sm) & 127) use_tma = 0;
    int tx = blockIdx.x % ntx, ty = blockIdx.x / ntx;
    if (ty >= nty) return;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    unsigned parity = 0;
    const unsigned long long wait_limit = g_wait_limit_ns;
    tb3_load<TBY>(a, tx * TBX, ty * TBY, S0, CL, mbar, use_tma && tb3_interior<TBY>(tx * TBX, ty * TBY, G), &tmIn,
                  &tmCL, NT);
    asm volatile("cp.async.commit_group;\n" ::);
    bool events = tb3_events<TBY>(a, ty * TBY);
    const long long t = a.t;
    while (ty < nty) {
        int ntx_ = tx + dr, nty_ = ty + dq;
        if (ntx_ >= ntx) {
            ntx_ -= ntx;
            nty_++;
        }
        const bool has_next = nty_ < nty;
        const bool events_next = has_next && tb3_events<TBY>(a, nty_ * TBY);
        const int x0 = tx * TBX, y0 = ty * TBY;
        asm volatile("cp.async.wait_group 0;\n" ::);
        bool ok = true;
        if (use_tma && tb3_interior<TBY>(x0, y0, G)) {
            ok = mbar_wait(mbar, parity, wait_limit);
            parity ^= 1u;
        }
        // every thread's copies have landed, and step C of the previous tile is done with S2
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicExch(&g_tb_timeouts, 1);
            mbar_wait(mbar, parity ^ 1u, kDrainNs);  // drain what is in flight
            return;
        }
        float4 clb = make_float4(0.f, 0.f, 0.f, 0.f), clc = clb;
        float clr = 0.f;
        if (events)
            tb3_step_a<TBY, NT, true>(a, S0, CL, S1, x0, y0, t, clb, clc, clr);
        else
            tb3_step_a<TBY, NT, false>(a, S0, CL, S1, x0, y0, t, clb, clc, clr);
        __syncthreads();
        if (has_next)  // S0 and c_L^2 are free: start the loads of the next tile
            tb3_load<TBY>(a, ntx_ * TBX, nty_ * TBY, S0, CL, mbar,
                          use_tma && tb3_interior<TBY>(ntx_ * TBX, nty_ * TBY, G), &tmIn, &tmCL, NT);
        asm volatile("cp.async.commit_group;\n" ::);
        if (events)
            tb3_step_b<TBY, NT, true>(a, S1, S2, x0, y0, t, clb, clr);
        else
            tb3_step_b<TBY, NT, false>(a, S1, S2, x0, y0, t, clb, clr);
        __syncthreads();
        if (events)
            tb3_step_c<TBY, true>(a, S2, x0, y0, t, clc);
        else
            tb3_step_c<TBY, false>(a, S2, x0, y0, t, clc);
        tx = ntx_;
        ty = nty_;
        events = events_next;
    }
    asm volatile("cp.async.wait_group 0;\n" ::);
}

// Tensor maps of the populations ([5][ny][pitch] floats, box: one plane of TBY+2 rows) and c_L^2
// ([ny][pitch], box: TBY+2 rows); false if unavailable.
template <int TBY>
static bool make_maps(const StepArgs &a, CUtensorMap *mIn, CUtensorMap *mCL) {
    constexpr int R = TbGeom<TBY>::R;
    EncodeTiled fn = encode_fn();
    if (!fn || a.g.nx < TW || a.g.ny < TBY + 4) return false;
    const cuuint64_t dims3[3] = {(cuuint64_t)a.g.nx, (cuuint64_t)a.g.ny, 5};
    const cuuint64_t str3[2] = {(cuuint64_t)a.g.pitch * 4, (cuuint64_t)a.g.plane * 4};
    const cuuint32_t box3[3] = {(cuuint32_t)TW, (cuuint32_t)R, 1};
    const cuuint32_t one[3] = {1, 1, 1};
    if (fn(mIn, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(a.in.data), dims3, str3, box3, one,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    const cuuint64_t dims2[2] = {(cuuint64_t)a.g.nx, (cuuint64_t)a.g.ny};
    const cuuint64_t str2[1] = {(cuuint64_t)a.g.pitch * 4};
    const cuuint32_t box2[2] = {(cuuint32_t)TW, (cuuint32_t)R};
    return fn(mCL, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(a.med.cL2), dims2, str2, box2, one,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor map of the gradient of ln mu ([2][ny][pitch] floats: d_x, d_y), box: both planes of TBY+2 rows.
template <int TBY>
static bool make_dl_map(const StepArgs &a, CUtensorMap *mDL) {
    EncodeTiled fn = encode_fn();
    if (!fn || !a.med.dlnmu) return false;
    const cuuint64_t dims3[3] = {(cuuint64_t)a.g.nx, (cuuint64_t)a.g.ny, 2};
    const cuuint64_t str3[2] = {(cuuint64_t)a.g.pitch * 4, (cuuint64_t)a.g.plane * 4};
    const cuuint32_t box3[3] = {(cuuint32_t)TW, (cuuint32_t)TbGeom<TBY>::R, 2};
    const cuuint32_t one[3] = {1, 1, 1};
    return fn(mDL, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(a.med.dlnmu), dims3, str3, box3, one,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor maps of the pole's planes for the tile kernel: P at t (pitched [ny][pitch], box TW x (TBY+2)) and J, wp2,
// wr2, gamma (box TBX x TBY); false if unavailable.
template <int TBY>
static bool make_pole_maps(const StepArgs &a, PoleMaps<true> *pm) {
    EncodeTiled fn = encode_fn();
    if (!fn || !a.med.Pr) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)a.g.nx, (cuuint64_t)a.g.ny};
    const cuuint64_t str[1] = {(cuuint64_t)a.g.pitch * 4};
    const cuuint32_t boxP[2] = {(cuuint32_t)TW, (cuuint32_t)(TBY + 2)}, boxJ[2] = {(cuuint32_t)TBX, (cuuint32_t)TBY};
    const cuuint32_t one[2] = {1, 1};
    auto enc = [&](CUtensorMap *m, const float *base, const cuuint32_t *box) {
        return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, str, box, one,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    return enc(&pm->P, a.med.Pr, boxP) && enc(&pm->J, a.med.J, boxJ) && enc(&pm->wp, a.med.pc, boxJ) &&
           enc(&pm->wr, a.med.pb, boxJ) && enc(&pm->gm, a.med.pa, boxJ);
}

template <int TBY, int NT, int MINB, bool MU = false, bool AN = false, bool POLE = false>
static cudaError_t launch_tb(const StepArgs &a, cudaStream_t s) {
    using Gm = TbGeom<TBY, MU, POLE>;
    static int per_sm = 0, nsm = 0;
    if (!per_sm) {
        cudaError_t e = cudaFuncSetAttribute(step2d_tb2<TBY, NT, MINB, MU, AN, POLE>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Gm::BYTES);
        if (e != cudaSuccess) return e;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step2d_tb2<TBY, NT, MINB, MU, AN, POLE>, NT,
                                                      Gm::BYTES);
        if (per_sm < 1) per_sm = 1;
    }
    CUtensorMap mIn, mCL, mDL;
    PoleMaps<POLE> pm;
    memset(&mIn, 0, sizeof mIn);
    memset(&mCL, 0, sizeof mCL);
    memset(&mDL, 0, sizeof mDL);
    memset(&pm, 0, sizeof pm);
    bool tma = make_maps<TBY>(a, &mIn, &mCL) && (!MU || make_dl_map<TBY>(a, &mDL));
    if constexpr (POLE) tma = tma && make_pole_maps<TBY>(a, &pm);
    const int use_tma = tma ? 1 : 0;
    const int ntx = (a.g.nx + TBX - 1) / TBX, nty = (a.g.ny + TBY - 1) / TBY;
    const int ntiles = ntx * nty;
    const int blocks = ntiles < per_sm * nsm ? ntiles : per_sm * nsm;
    step2d_tb2<TBY, NT, MINB, MU, AN, POLE>
        <<<blocks, NT, Gm::BYTES, s>>>(a, mIn, mCL, mDL, pm, use_tma, ntx, nty, blocks / ntx, blocks % ntx);
    return cudaGetLastError();
}

// =====================================================================================================
// 16-bit storage (LBEM_F16, LBEM_BF16, LBEM_I16B).  Same tiles and steps; the t stage holds the stored 16-bit
// values (half the shared memory), each value is decoded once as step t pulls it, the t+1 stage is FP32, and
// step t+1 encodes what it writes.  So a launch rounds the state to the storage format once per two steps
// (the single-step kernels round at every step); the arithmetic is FP32 as everywhere.  Needs nx % 4 == 0,
// so that every group of 4 columns (one block-int16 exponent) stays contiguous across the periodic wrap.

constexpr int THW = TBX + 16;  // staged 16-bit columns x0-8 .. x0+TBX+7 (16-bit TMA boxes start at x = 8k)
constexpr int TEX = 64;        // staged exponent groups per row: group x0/4-16+k at column k (byte boxes: x = 16k)

template <int ST, int TBY>
struct TbGeomH {
    static constexpr int R = TBY + 2;
    static constexpr int up(int n, int m) { return (n + m - 1) / m * m; }
    static constexpr int INH_PL = up(R * THW * 2, 128);                    // bytes per staged 16-bit plane
    static constexpr int EX_PL = ST == LBEM_I16B ? up(R * TEX, 128) : 0;  // bytes per staged exponent plane
    static constexpr int P_PL = TBY * TW;                                 // floats per t+1 plane
    static constexpr int OFF_EX = 5 * INH_PL, OFF_CL = OFF_EX + 5 * EX_PL, OFF_P = OFF_CL + up(R * TW * 4, 128);
    static constexpr int OFF_MB = OFF_P + up(5 * P_PL * 4, 128);
    static constexpr size_t BYTES = OFF_MB + sizeof(unsigned long long);
    static constexpr unsigned TMA_BYTES = 5 * R * THW * 2 + R * TW * 4 + (ST == LBEM_I16B ? 5 * R * TEX : 0);
};

// One stored 16-bit value to FP32 (as Codec<ST>::load4 does): f is inv_scale (F16) or the block's 2^(e-15)
// (I16B, 0 for a zero block).
template <int ST>
__device__ __forceinline__ float dec16(unsigned h, float f) {
    if (ST == LBEM_F16) return __fmul_rn(__half2float(__ushort_as_half((unsigned short)h)), f);
    if (ST == LBEM_BF16) return __uint_as_float(h << 16);
    return __fmul_rn(i16_to_f((short)h), f);
}
__device__ __forceinline__ float ex_factor(int e) { return i16b_factor(e); }

// The two stored values packed in w (low half first), decoded as dec16 does.
template <int ST>
__device__ __forceinline__ float2 dec16x2(unsigned w, float f) {
    if constexpr (ST == LBEM_I16B) {
        return i16x2_to_f2(w, f);
    } else if constexpr (ST == LBEM_F16) {
        const float2 v = __half22float2(*reinterpret_cast<const __half2 *>(&w));
        return make_float2(__fmul_rn(v.x, f), __fmul_rn(v.y, f));
    } else {
        return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
    }
}

__device__ __forceinline__ void tb_cpa8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(dst)), "l"(src));
}

// Pulled populations of four sites at stage row `row`, lane L (16-bit stage column j = 8 + 4L <-> x0+4L).
template <int ST, int TBY>
struct Pull4h {
    float4 g0, g1, g2, g3, g4;
    __device__ __forceinline__ Pull4h(const char *INh, const signed char *EX, int row, int L, float inv_scale) {
        using Gm = TbGeomH<ST, TBY>;
        const int j = 8 + 4 * L;
        const char *r = INh + (row * THW + j) * 2;
        const uint2 r0 = *reinterpret_cast<const uint2 *>(r);
        const uint2 a1 = *reinterpret_cast<const uint2 *>(r + Gm::INH_PL - 8);
        const uint2 b1 = *reinterpret_cast<const uint2 *>(r + Gm::INH_PL);
        const uint2 r2 = *reinterpret_cast<const uint2 *>(r + 2 * Gm::INH_PL);
        const uint2 r3 = *reinterpret_cast<const uint2 *>(r + 3 * Gm::INH_PL);
        const uint2 c3 = *reinterpret_cast<const uint2 *>(r + 3 * Gm::INH_PL + 8);
        const uint2 r4 = *reinterpret_cast<const uint2 *>(r + 4 * Gm::INH_PL);
        float f0 = inv_scale, f1a = inv_scale, f1b = inv_scale, f2 = inv_scale, f3a = inv_scale, f3b = inv_scale,
              f4 = inv_scale;
        if (ST == LBEM_I16B) {  // exponent column of stage column j: 14 + j/4
            const signed char *e = EX + row * TEX + 16 + L;
            f0 = ex_factor(e[0]);
            f1a = ex_factor(e[Gm::EX_PL - 1]);
            f1b = ex_factor(e[Gm::EX_PL]);
            f2 = ex_factor(e[2 * Gm::EX_PL]);
            f3a = ex_factor(e[3 * Gm::EX_PL]);
            f3b = ex_factor(e[3 * Gm::EX_PL + 1]);
            f4 = ex_factor(e[4 * Gm::EX_PL]);
        }
        const float2 p0a = dec16x2<ST>(r0.x, f0), p0b = dec16x2<ST>(r0.y, f0);
        const float2 p1a = dec16x2<ST>(a1.y, f1a), p1b = dec16x2<ST>(b1.x, f1b), p1c = dec16x2<ST>(b1.y, f1b);
        const float2 p2a = dec16x2<ST>(r2.x, f2), p2b = dec16x2<ST>(r2.y, f2);
        const float2 p3a = dec16x2<ST>(r3.x, f3a), p3b = dec16x2<ST>(r3.y, f3a), p3c = dec16x2<ST>(c3.x, f3b);
        const float2 p4a = dec16x2<ST>(r4.x, f4), p4b = dec16x2<ST>(r4.y, f4);
        g0 = make_float4(p0a.x, p0a.y, p0b.x, p0b.y);
        g1 = make_float4(p1a.y, p1b.x, p1b.y, p1c.x);
        g2 = make_float4(p2a.x, p2a.y, p2b.x, p2b.y);
        g3 = make_float4(p3a.y, p3b.x, p3b.y, p3c.x);
        g4 = make_float4(p4a.x, p4a.y, p4b.x, p4b.y);
    }
};

// One decoded value of the 16-bit stage (plane p, row, stage column j).
template <int ST, int TBY>
__device__ __forceinline__ float stage16(const char *INh, const signed char *EX, int p, int row, int j, float inv_scale) {
    using Gm = TbGeomH<ST, TBY>;
    const unsigned h = *reinterpret_cast<const unsigned short *>(INh + p * Gm::INH_PL + (row * THW + j) * 2);
    const float f = ST == LBEM_I16B ? ex_factor(EX[p * Gm::EX_PL + row * TEX + 14 + j / 4]) : inv_scale;
    return dec16<ST>(h, f);
}

template <int TBY>
__device__ __forceinline__ bool tb_interior16(int x0, int y0, const Grid &G) {
    return x0 - 8 >= 0 && x0 + TBX + 8 <= G.nx && y0 - 2 >= 0 && y0 + TBY + 2 <= G.ny;
}

// Loads of one tile's window: TMA boxes for interior tiles (one thread), asynchronous copies of 4-column
// groups with periodic wrap otherwise (nx % 4 == 0), exponent bytes by plain loads.
template <int ST, int TBY>
__device__ __forceinline__ void tb_load16(const StepArgs &a, int x0, int y0, char *sm, unsigned mbar, bool tma,
                                          const CUtensorMap *tmIn, const CUtensorMap *tmCL, const CUtensorMap *tmEx,
                                          int nt) {
    using Gm = TbGeomH<ST, TBY>;
    constexpr int R = Gm::R;
    char *INh = sm;
    signed char *EX = reinterpret_cast<signed char *>(sm + Gm::OFF_EX);
    float *CL = reinterpret_cast<float *>(sm + Gm::OFF_CL);
    if (tma) {
        if (threadIdx.x == 0) {
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(Gm::TMA_BYTES)
                         : "memory");
#pragma unroll
            for (int p = 0; p < 5; p++) tma_load_3d(INh + p * Gm::INH_PL, tmIn, x0 - 8, y0 - 1 + in_shift(p), p, mbar);
            tma_load_2d(CL, tmCL, x0 - 4, y0 - 1, mbar);
            if (ST == LBEM_I16B) {
#pragma unroll
                for (int p = 0; p < 5; p++)
                    tma_load_3d(EX + p * Gm::EX_PL, tmEx, x0 / 4 - 16, y0 - 1 + in_shift(p), p, mbar);
            }
        }
        return;
    }
    const Grid &G = a.g;
    const unsigned short *in = static_cast<const unsigned short *>(a.in.data);
    constexpr int QH = THW / 4, QC = TW / 4;
    for (int k = threadIdx.x; k < 5 * R * QH; k += nt) {
        const int pr = k / QH, q = k - pr * QH;
        const int pl = pr / R, r = pr - pl * R;
        const int gy = wrapi(y0 - 1 + r + in_shift(pl), G.ny), gx = wrapi(x0 - 8 + 4 * q, G.nx);
        tb_cpa8(INh + pl * Gm::INH_PL + (r * THW + 4 * q) * 2, in + pl * G.plane + (long long)gy * G.pitch + gx);
        if (ST == LBEM_I16B)
            EX[pl * Gm::EX_PL + r * TEX + 14 + q] = __ldg(a.in.ex + pl * a.in.explane + (long long)gy * a.in.expitch + gx / 4);
    }
    for (int k = threadIdx.x; k < R * QC; k += nt) {
        const int r = k / QC, q = k - r * QC;
        const int gy = wrapi(y0 - 1 + r, G.ny), gx = wrapi(x0 - 4 + 4 * q, G.nx);
        tb_cpa16(CL + r * TW + 4 * q, a.med.cL2 + (long long)gy * G.pitch + gx);
    }
}

// Step t from the 16-bit stage into the FP32 t+1 stage (as tb_step_a).
template <int ST, int TBY, int NT, bool EV>
__device__ __forceinline__ void tb_step_a16(const StepArgs &a, const char *INh, const signed char *EX, const float *CL,
                                            float *P, int x0, int y0, long long t, float4 &clb) {
    using Gm = TbGeomH<ST, TBY>;
    constexpr int R = Gm::R, NW = NT / 32, PL = Gm::P_PL;
    const Grid &G = a.g;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int c = 4 + 4 * lane;
    const float is = a.in.inv_scale;
    if (warp < TBY) clb = lds4(CL + (warp + 1) * TW + c);
    for (int py = warp; py < R; py += NW) {
        const Pull4h<ST, TBY> g(INh, EX, py, lane, is);
        const float4 cl = lds4(CL + py * TW + c);
        float4 o0, o1, o2, o3, o4;
        tb_update4<EV>(a, g, cl, x0, y0 - 1 + py, t, py >= 1 && py <= TBY, o0, o1, o2, o3, o4);
        float *Pr = P + c;
        if (py >= 1 && py <= TBY) {
            sts4(Pr + 0 * PL + (py - 1) * TW, o0);
            sts4(Pr + 1 * PL + (py - 1) * TW, o1);
            sts4(Pr + 3 * PL + (py - 1) * TW, o3);
        }
        if (py < TBY) sts4(Pr + 2 * PL + py * TW, o2);
        if (py >= 2) sts4(Pr + 4 * PL + (py - 2) * TW, o4);
    }
    int k0 = tid - 32 * (R % NW);
    if (k0 < 0) k0 += NT;
    for (int k = k0; k < 2 * TBY; k += NT) {
        const int py = (k >> 1) + 1, j = (k & 1) ? TBX + 8 : 7;  // 16-bit stage column of x0-1 / x0+TBX
        const int cc = j - 4;                                    // FP32 column of the same site
        const float q0 = stage16<ST, TBY>(INh, EX, 0, py, j, is), q1 = stage16<ST, TBY>(INh, EX, 1, py, j - 1, is),
                    q2 = stage16<ST, TBY>(INh, EX, 2, py, j, is), q3 = stage16<ST, TBY>(INh, EX, 3, py, j + 1, is),
                    q4 = stage16<ST, TBY>(INh, EX, 4, py, j, is);
        const float ck = CL[py * TW + cc];
        float shat = 0.f;
        if (EV)
            shat = site_events(a, wrapi(x0 - 4 + cc, G.nx), wrapi(y0 - 1 + py, G.ny), t, false, q0, q1, q2, q3, q4,
                               ck);
        const Out5 o = collide2d(q0, q1, q2, q3, q4, ck, shat);
        if (k & 1)
            P[3 * PL + (py - 1) * TW + cc] = o.o3;
        else
            P[1 * PL + (py - 1) * TW + cc] = o.o1;
    }
}

// Step t+1 on tile row y0 + warp, encoded to the storage format as it is written.
template <int ST, int TBY, bool EV>
__device__ __forceinline__ void tb_step_b16(const StepArgs &a, const float *P, float4 clb, int x0, int y0, long long t) {
    const Grid &G = a.g;
    const int lane = threadIdx.x & 31, oy = threadIdx.x >> 5;
    const int gy = y0 + oy;
    if (oy >= TBY || gy >= G.ny) return;
    const int c = 4 + 4 * lane;
    const Pull4 g(P, TbGeomH<ST, TBY>::P_PL, oy, c);
    float4 o[5];
    tb_update4<EV>(a, g, clb, x0, gy, t + 1, true, o[0], o[1], o[2], o[3], o[4]);
    if (x0 + 4 * lane < G.pitch) {
        unsigned short *out = static_cast<unsigned short *>(a.out.data) + (long long)gy * G.pitch + x0 + 4 * lane;
#pragma unroll
        for (int p = 0; p < 5; p++) {
            uint2 r;
            if constexpr (ST == LBEM_I16B) {
                const int e = Codec<LBEM_I16B>::enc4e(o[p], r);
                a.out.ex[p * a.out.explane + (long long)gy * a.out.expitch + x0 / 4 + lane] = (int8_t)e;
            } else {
                r = Codec<ST>::enc4(a.out, o[p]);
            }
            __stcs(reinterpret_cast<uint2 *>(out + p * G.plane), r);
        }
    }
}

template <int ST, int TBY, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    step2d_tb2h(StepArgs a, const __grid_constant__ CUtensorMap tmIn, const __grid_constant__ CUtensorMap tmCL,
                const __grid_constant__ CUtensorMap tmEx, int use_tma, int ntx, int nty, int dq, int dr) {
    static_assert(NT / 32 >= TBY, "one warp per row of step t+1");
    using Gm = TbGeomH<ST, TBY>;
    extern __shared__ __align__(1024) char smb[];
    const char *INh = smb;
    const signed char *EX = reinterpret_cast<const signed char *>(smb + Gm::OFF_EX);
    const float *CL = reinterpret_cast<const float *>(smb + Gm::OFF_CL);
    float *P = reinterpret_cast<float *>(smb + Gm::OFF_P);
    const unsigned mbar = smem_u32(smb + Gm::OFF_MB);
    const Grid &G = a.g;
    const int tid = threadIdx.x;
    if (smem_u32(smb) & 127) use_tma = 0;
    int tx = blockIdx.x % ntx, ty = blockIdx.x / ntx;
    if (ty >= nty) return;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    unsigned parity = 0;
    const unsigned long long wait_limit = g_wait_limit_ns;
    tb_load16<ST, TBY>(a, tx * TBX, ty * TBY, smb, mbar, use_tma && tb_interior16<TBY>(tx * TBX, ty * TBY, G), &tmIn,
                       &tmCL, &tmEx, NT);
    asm volatile("cp.async.commit_group;\n" ::);
    bool events = tb_events<TBY>(a, ty * TBY);
    const long long t = a.t;
    while (ty < nty) {
        int ntx_ = tx + dr, nty_ = ty + dq;
        if (ntx_ >= ntx) {
            ntx_ -= ntx;
            nty_++;
        }
        const bool has_next = nty_ < nty;
        const bool events_next = has_next && tb_events<TBY>(a, nty_ * TBY);
        const int x0 = tx * TBX, y0 = ty * TBY;
        asm volatile("cp.async.wait_group 0;\n" ::);
        bool ok = true;
        if (use_tma && tb_interior16<TBY>(x0, y0, G)) {
            ok = mbar_wait(mbar, parity, wait_limit);
            parity ^= 1u;
        }
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicExch(&g_tb_timeouts, 1);
            mbar_wait(mbar, parity ^ 1u, kDrainNs);  // drain what is in flight
            return;
        }
        float4 clb = make_float4(0.f, 0.f, 0.f, 0.f);
        if (events)
            tb_step_a16<ST, TBY, NT, true>(a, INh, EX, CL, P, x0, y0, t, clb);
        else
            tb_step_a16<ST, TBY, NT, false>(a, INh, EX, CL, P, x0, y0, t, clb);
        __syncthreads();
        if (has_next)
            tb_load16<ST, TBY>(a, ntx_ * TBX, nty_ * TBY, smb, mbar,
                               use_tma && tb_interior16<TBY>(ntx_ * TBX, nty_ * TBY, G), &tmIn, &tmCL, &tmEx, NT);
        asm volatile("cp.async.commit_group;\n" ::);
        if (events)
            tb_step_b16<ST, TBY, true>(a, P, clb, x0, y0, t);
        else
            tb_step_b16<ST, TBY, false>(a, P, clb, x0, y0, t);
        tx = ntx_;
        ty = nty_;
        events = events_next;
    }
    asm volatile("cp.async.wait_group 0;\n" ::);
}

template <int TBY, int NT, int MINB>
static cudaError_t launch_tb3(const StepArgs &a, cudaStream_t s) {
    using Gm = TbGeom3<TBY>;
    static int per_sm = 0, nsm = 0;
    if (!per_sm) {
        cudaError_t e = cudaFuncSetAttribute(step2d_tb3<TBY, NT, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)Gm::BYTES);
        if (e != cudaSuccess) return e;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step2d_tb3<TBY, NT, MINB>, NT, Gm::BYTES);
        if (per_sm < 1) per_sm = 1;
    }
    CUtensorMap mIn, mCL;
    memset(&mIn, 0, sizeof mIn);
    memset(&mCL, 0, sizeof mCL);
    // boxes of TBY+4 rows: the two-step map builder with the row count of a (TBY+2)-row tile
    const int use_tma = (a.g.ny >= TBY + 6 && make_maps<TBY + 2>(a, &mIn, &mCL)) ? 1 : 0;
    const int ntx = (a.g.nx + TBX - 1) / TBX, nty = (a.g.ny + TBY - 1) / TBY;
    const int ntiles = ntx * nty;
    const int blocks = ntiles < per_sm * nsm ? ntiles : per_sm * nsm;
    step2d_tb3<TBY, NT, MINB><<<blocks, NT, Gm::BYTES, s>>>(a, mIn, mCL, use_tma, ntx, nty, blocks / ntx,
                                                            blocks % ntx);
    return cudaGetLastError();
}

int tb3_nshapes() { return 3; }

cudaError_t launch_step_2d_tb3(const StepArgs &a, int shape, cudaStream_t s) {
    switch (shape) {
        case 1: return launch_tb3<4, 288, 4>(a, s);
        case 2: return launch_tb3<8, 448, 2>(a, s);
        default: return launch_tb3<6, 384, 3>(a, s);
    }
}

// Tensor maps of the 16-bit populations (box: one plane of TBY+2 rows of THW values), c_L^2 and, for block-int16,
// the exponent planes (box: TEX bytes of TBY+2 rows); false if unavailable or the strides do not allow it.
template <int ST, int TBY>
static bool make_maps16(const StepArgs &a, CUtensorMap *mIn, CUtensorMap *mCL, CUtensorMap *mEx) {
    constexpr int R = TbGeomH<ST, TBY>::R;
    EncodeTiled fn = encode_fn();
    if (!fn || a.g.nx < THW || a.g.ny < TBY + 4) return false;
    const cuuint32_t one[3] = {1, 1, 1};
    const cuuint64_t dims3[3] = {(cuuint64_t)a.g.nx, (cuuint64_t)a.g.ny, 5};
    const cuuint64_t str3[2] = {(cuuint64_t)a.g.pitch * 2, (cuuint64_t)a.g.plane * 2};
    const cuuint32_t box3[3] = {(cuuint32_t)THW, (cuuint32_t)R, 1};
    if (fn(mIn, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, const_cast<void *>(a.in.data), dims3, str3, box3, one,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    const cuuint64_t dims2[2] = {(cuuint64_t)a.g.nx, (cuuint64_t)a.g.ny};
    const cuuint64_t str2[1] = {(cuuint64_t)a.g.pitch * 4};
    const cuuint32_t box2[2] = {(cuuint32_t)TW, (cuuint32_t)R};
    if (fn(mCL, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(a.med.cL2), dims2, str2, box2, one,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    if (ST != LBEM_I16B) return true;
    if (a.in.expitch % 16 || a.in.explane % 16) return false;
    const cuuint64_t dimsE[3] = {(cuuint64_t)a.in.expitch, (cuuint64_t)a.g.ny, 5};
    const cuuint64_t strE[2] = {(cuuint64_t)a.in.expitch, (cuuint64_t)a.in.explane};
    const cuuint32_t boxE[3] = {(cuuint32_t)TEX, (cuuint32_t)R, 1};
    return fn(mEx, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, a.in.ex, dimsE, strE, boxE, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

template <int ST, int TBY, int NT, int MINB>
static cudaError_t launch_tb16(const StepArgs &a, cudaStream_t s) {
    using Gm = TbGeomH<ST, TBY>;
    static int per_sm = 0, nsm = 0;
    if (!per_sm) {
        cudaError_t e = cudaFuncSetAttribute(step2d_tb2h<ST, TBY, NT, MINB>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Gm::BYTES);
        if (e != cudaSuccess) return e;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step2d_tb2h<ST, TBY, NT, MINB>, NT, Gm::BYTES);
        if (per_sm < 1) per_sm = 1;
    }
    CUtensorMap mIn, mCL, mEx;
    memset(&mIn, 0, sizeof mIn);
    memset(&mCL, 0, sizeof mCL);
    memset(&mEx, 0, sizeof mEx);
    const int use_tma = make_maps16<ST, TBY>(a, &mIn, &mCL, &mEx) ? 1 : 0;
    const int ntx = (a.g.nx + TBX - 1) / TBX, nty = (a.g.ny + TBY - 1) / TBY;
    const int ntiles = ntx * nty;
    const int blocks = ntiles < per_sm * nsm ? ntiles : per_sm * nsm;
    step2d_tb2h<ST, TBY, NT, MINB><<<blocks, NT, Gm::BYTES, s>>>(a, mIn, mCL, mEx, use_tma, ntx, nty, blocks / ntx,
                                                                 blocks % ntx);
    return cudaGetLastError();
}

template <int ST>
static cudaError_t launch_16(const StepArgs &a, int shape, cudaStream_t s) {
    switch (shape) {
        case 1: return launch_tb16<ST, 6, 256, 4>(a, s);
        case 2: return launch_tb16<ST, 8, 320, 4>(a, s);
        case 3: return launch_tb16<ST, 8, 320, 3>(a, s);
        case 4: return launch_tb16<ST, 4, 192, 6>(a, s);
        case 5: return launch_tb16<ST, 10, 384, 3>(a, s);
        case 6: return launch_tb16<ST, 14, 512, 2>(a, s);
        default: return launch_tb16<ST, 6, 256, 5>(a, s);
    }
}

// Tile shapes (rows, threads, CTAs per SM).  Measured on 4096^2 (heterogeneous medium, FP32): 6 rows at five
// CTAs per SM is the fastest; the others remain selectable for other sizes and for the bit-identity tests.
// With a heterogeneous permeability (FP32 only): 6 rows at four CTAs per SM (51 KB), 14 rows at two, or the strip
// kernel (sstream.cu).
// With an anisotropic medium (FP32, no mu array) only tile shape 0.
int tb2_nshapes(int storage, bool has_mu) {
    if (has_mu) return storage == LBEM_F32 ? 3 : 0;
    return storage == LBEM_F32 ? 7 + rs2_nshapes() + ss2_nshapes() : 7;
}

cudaError_t launch_step_2d_tb2(const StepArgs &a, int storage, int shape, cudaStream_t s) {
    switch (storage) {
        case LBEM_F16: return launch_16<LBEM_F16>(a, shape, s);
        case LBEM_BF16: return launch_16<LBEM_BF16>(a, shape, s);
        case LBEM_I16B: return launch_16<LBEM_I16B>(a, shape, s);
        default: break;
    }
    if (a.med.wp2)  // a dispersive pole: with a tensor (AN and POLE), or isotropic (POLE alone)
        return (a.med.ar != 1.f || a.med.amu != 1.f) ? launch_tb<6, 256, 3, false, true, true>(a, s)
                                                       : launch_tb<6, 256, 3, false, false, true>(a, s);
    if (a.med.ar != 1.f || a.med.amu != 1.f)  // anisotropic: the tile kernel (shape 0) or the strip kernel (1)
        return shape == 1 ? launch_step_2d_ss2_an(a, s) : launch_tb<6, 256, 5, false, true>(a, s);
    if (a.med.dlnmu)  // heterogeneous mu: two tile shapes, then the strip kernel
        return shape == 2   ? launch_step_2d_ss2_mu(a, s)
               : shape == 1 ? launch_tb<14, 512, 2, true>(a, s)
                            : launch_tb<6, 256, 4, true>(a, s);
    if (shape >= 7 + rs2_nshapes()) return launch_step_2d_ss2(a, shape - 7 - rs2_nshapes(), s);  // sstream.cu
    if (shape >= 7) return launch_step_2d_rs2(a, shape - 7, s);  // register streaming (rstream.cu)
    switch (shape) {
        case 1: return launch_tb<8, 320, 3>(a, s);
        case 2: return launch_tb<8, 352, 3>(a, s);   // ring sites on the 11th warp
        case 3: return launch_tb<10, 384, 3>(a, s);
        case 4: return launch_tb<5, 224, 5>(a, s);
        case 5: return launch_tb<4, 192, 6>(a, s);
        case 6: return launch_tb<14, 512, 2>(a, s);
        default: return launch_tb<6, 256, 5>(a, s);  // 42 KB of shared memory
    }
}

cudaError_t tb_set_wait_limit(unsigned long long ns) {
    const cudaError_t e = cudaMemcpyToSymbol(g_wait_limit_ns, &ns, sizeof ns);
    return e != cudaSuccess ? e : ss_set_wait_limit(ns);
}

bool tb2_take_timeouts() {
    const bool ss = ss2_take_timeouts();
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_tb_timeouts, sizeof v) != cudaSuccess) return false;
    if (v) {
        const int z = 0;
        cudaMemcpyToSymbol(g_tb_timeouts, &z, sizeof z);
    }
    return v != 0 || ss;
}

}  // namespace lbk
