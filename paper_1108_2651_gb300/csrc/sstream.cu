// Two time steps per launch by streaming a strip of rows through a ring of shared-memory stages (2D, FP32 storage):
// uniform mu; variants for a heterogeneous mu (the two grad ln mu planes staged as planes 6-7) and for an
// anisotropic tensor (the per-axis collision); and the batch of independent media over their packed copy.
//
// A CTA owns a strip of 128 columns (x0 .. x0+127) and a run of rows ys .. ye-1 and walks down the run in chunks of
// TBY rows.  A chunk of the state at t (the five population planes, each staged shifted by its pull offset in y so
// that staged row w of every plane holds what the update of chunk row w pulls, and c_L^2) arrives in one of S
// stages, ahead of the one being computed.  Phase g computes step t on the rows of chunk g (Eqs.
// 17-18) and step t+1 on the rows one behind the previous chunk, whose pulls are then all computed: the step-t
// results at a row are the next step's g0, g1, g3 there, g2 one row below and g4 one row above.  Step t therefore
// stores each result plane at the row that will pull it, in a ring of 2 TBY + 2 rows (with c_L^2 beside them for
// step t+1), and one barrier of the warps that compute, per phase, is the only synchronisation between the two
// steps: the rows step t writes in a phase and the rows step t+1 reads in it are disjoint.
//
// Warps 0 .. 2 TBY - 1 consume: TBY rows of step t, and TBY rows of step t+1 with the chunk's ring sites (the
// column left and right of the strip, which give step t+1 plane 1 at x0-1 and plane 3 at x0+128).  The last warp
// produces: it runs up to S chunks ahead of them (full and empty mbarriers per stage) and takes units of work from a
// queue.  Chunks inside the grid are six TMA boxes.  In the first and last strip the boxes reach past the grid's
// columns (the copy fills zeros there) and six more boxes of 4 columns bring the periodic images into a side buffer,
// from which those few pulls read.  Chunks whose rows wrap periodically, and ragged grids, are staged by the producer
// warp's asynchronous copies, which arrive on the stage's mbarrier as they land.
//
// A chunk's sources and receivers are staged beside its descriptor by the producer (row boundaries read a unit
// ahead, records copied asynchronously on the stage's mbarrier); a row holding some matches them against its lanes'
// sites in one pass, writes the receivers from the pulled populations and adds the sources' terms after the plain
// collision, which is the collision with S^ operation for operation.
//
// HBM traffic per two site updates: 24 bytes read and 20 written; the two rows outside a run and the four columns
// either side of a strip are read again, mostly from L2.  Nothing is computed twice except those rows and the ring
// sites.  The site updates are collide2d / collide2d_free, so the results are bit-identical to two single steps.
#include <cuda.h>
#include <string.h>

#include "lbem_internal.cuh"
#include "tma.cuh"

namespace lbk {

namespace {
constexpr int SBX = 128;     // strip width: one warp of 4-site lanes
constexpr int SW = SBX + 8;  // staged columns x0-4 .. x0+131 (16-byte aligned boxes); column j <-> x0-4+j

// Row shift of the staged planes: plane p row w of chunk k's stage holds global row s_k + w + ss_shift(p).
__device__ __host__ constexpr int ss_shift(int p) { return p == 2 ? -1 : p == 4 ? 1 : 0; }
}  // namespace

__device__ int g_ss_timeouts = 0;  // set when a bounded wait of the strip kernel gave up
// Limit of the strip kernel's bounded waits for a chunk, in ns of device time (0 gives up at once).
__device__ unsigned long long g_ss_wait_limit_ns = 2000000000ull;
constexpr unsigned long long kSsDrainNs = 2000000000ull;  // after giving up: wait for copies in flight

// Shared memory of a CTA (floats): S stages of a chunk (six planes of TBY rows of SW, each plane 128-byte aligned,
// a TMA destination), S side buffers of the periodic images of an edge strip (six planes of TBY rows of 4), the
// step-(t+1) ring (six planes of M rows of SW: populations 0..4, then c_L^2), the chunk descriptors, then two
// mbarriers per stage (full: staged; empty: read by every consumer warp).
// The sources and receivers of a chunk's rows s-1 .. s+TBY-1 (window rows 0 .. TBY), staged in shared memory so that
// the site updates match against a short list instead of walking the event tables: the records of the tables' row
// range, copied asynchronously by the producer (tracked by the stage's mbarrier), and per window row the first
// record of that row (b[i]; b[TBY + 1] = n).  At most SS_EMAX records; a chunk with more, or whose window wraps
// periodically, is not staged.
constexpr int SS_EMAX = 12, SS_RMAX = 10;
struct SsEvList {
    int n, b[SS_RMAX + 1];
    Event rec[SS_EMAX];
};
// A chunk's descriptor slot: two int4 (d0: the unit's x0, ys, ye and k | flags; d1: the batch member's m, packed row,
// size) and the chunk's event list.
struct SsDesc {
    int4 d0, d1;
    SsEvList ev;
};

template <int TBY, int S, bool BATCH = false, bool MU = false>
struct SsGeom {
    static constexpr int up32(int n) { return (n + 31) / 32 * 32; }
    static constexpr int NPL = MU ? 8 : 6;  // staged planes: populations 0..4, c_L^2 (and d_x ln mu, d_y ln mu)
    static constexpr int M = 2 * TBY + 2;
    static constexpr int PL_IN = up32(TBY * SW), STAGE = NPL * PL_IN;
    static constexpr int EPL = up32(4 * TBY), ESTAGE = NPL * EPL;
    static constexpr int PL_P = M * SW;
    static constexpr int IN_SZ = S * STAGE, E_SZ = BATCH ? 0 : S * ESTAGE, P_SZ = up32(NPL * PL_P);  // (no images:
    // the batch's packed members carry theirs)
    static constexpr int DS = S + 2;  // chunk descriptor slots (SsDesc) after the ring, then the mbarriers
    // (the batch kernel keeps a copy of each chunk's member arguments beside the descriptors)
    static constexpr int SZ = IN_SZ + E_SZ + P_SZ + DS * (int)(sizeof(SsDesc) / 4) +
                              (BATCH ? DS * (int)(sizeof(StepArgs) / 4) : 0);
    static constexpr size_t BYTES = sizeof(float) * SZ + 2 * S * sizeof(unsigned long long);
    static constexpr unsigned TMA_BYTES = sizeof(float) * NPL * TBY * SW, E_BYTES = sizeof(float) * NPL * TBY * 4;
};

// Which columns of the strip wrap: 0 none (x0-4 .. x0+131 inside the grid), 1 the first strip (x0 = 0, the images
// of columns nx-4 .. nx-1 left of it), 2 the last strip of a grid of whole strips (the images of columns 0 .. 3
// right of it), 3 anything else (a single strip, or a last strip reaching past nx), staged by element copies.
__device__ __forceinline__ int ss_xmode(const Grid &G, int x0) {
    if (x0 - 4 >= 0 && x0 + SBX + 4 <= G.nx) return 0;
    if ((G.nx & 3) == 0 && x0 == 0 && SBX + 4 <= G.nx) return 1;
    if ((G.nx & 3) == 0 && x0 >= SBX && x0 + SBX == G.nx) return 2;
    return 3;
}

// How chunk rows s .. s+TBY-1 are staged: 0 six TMA boxes, 1 six boxes and the six boxes of the images (xmode 1
// or 2), 2 every thread's asynchronous copies (rows that wrap, xmode 3, or no tensor maps).
template <int TBY>
__device__ __forceinline__ int ss_chunk_mode(const Grid &G, int xm, int s, bool tma) {
    if (!tma || xm == 3 || s < 1 || s + TBY + 1 > G.ny) return 2;
    return xm == 0 ? 0 : 1;
}

// Stage the chunk of step-t rows s .. s+TBY-1 into `st` (and `es`), by the producer warp, arriving on the stage's
// full mbarrier (count 1): the five population planes at their row shifts, c_L^2 and, with MU, d_x ln mu and d_y ln mu.
// Modes 0 and 1: lane 0 arrives with the transaction bytes, then lanes issue one box each (lane p plane p, lane
// NPL + p its images).  Mode 2: every lane issues its share of asynchronous copies (16 bytes where every group of 4
// columns stays contiguous after the periodic wrap, else 4), each lane's copies tracked by the mbarrier (its pending
// count rises until they land), then lane 0 arrives.
template <int TBY, int S, bool MU = false>
__device__ __forceinline__ void ss_issue(const StepArgs &a, int x0, int xm, int s, int mode, float *st, float *es,
                                         unsigned mbar, const CUtensorMap *tmIn, const CUtensorMap *tmCL,
                                         const CUtensorMap *tmIn4, const CUtensorMap *tmCL4,
                                         const CUtensorMap *tmDL = nullptr, const CUtensorMap *tmDL4 = nullptr) {
    using Gm = SsGeom<TBY, S, false, MU>;
    constexpr int NPL = Gm::NPL;
    const Grid &G = a.g;
    const int lane = threadIdx.x & 31;
    if (mode != 2) {
        if (lane == 0) {
            const unsigned bytes = Gm::TMA_BYTES + (mode == 1 ? Gm::E_BYTES : 0u);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes)
                         : "memory");
        }
        __syncwarp();
        const bool image = lane >= NPL;
        const int p = image ? lane - NPL : lane;
        if (lane < (mode == 1 ? 2 * NPL : NPL)) {
            // the consumers' reads of this stage (ordered by the empty mbarrier) before the async-proxy writes
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            const int x = image ? (xm == 1 ? G.nx - 4 : 0) : x0 - 4;
            float *dst = image ? es + p * Gm::EPL : st + p * Gm::PL_IN;
            if (p < 5)
                tma_load_3d(dst, image ? tmIn4 : tmIn, x, s + ss_shift(p), p, mbar);
            else if (p == 5)
                tma_load_2d(dst, image ? tmCL4 : tmCL, x, s, mbar);
            else
                tma_load_3d(dst, image ? tmDL4 : tmDL, x, s, p - 6, mbar);
        }
        return;
    }
    const float *in = static_cast<const float *>(a.in.data);
    auto row_of = [&](int p, int w) -> const float * {  // plane p's source row for staged row w
        if (p < 5) return in + p * G.plane + (long long)wrapi(s + w + ss_shift(p), G.ny) * G.pitch;
        const float *base = p == 5 ? a.med.cL2 : a.med.dlnmu + (p - 6) * G.plane;
        return base + (long long)wrapi(s + w, G.ny) * G.pitch;
    };
    if (xm == 0 || (G.nx & 3) == 0) {
        constexpr int Q = SW / 4;
        for (int k = lane; k < NPL * TBY * Q; k += 32) {
            const int pr = k / Q, q = k - pr * Q;  // pr = plane * TBY + row
            const int p = pr / TBY, w = pr - p * TBY;
            tb_cpa16(st + p * Gm::PL_IN + w * SW + 4 * q, row_of(p, w) + wrapi(x0 - 4 + 4 * q, G.nx));
        }
    } else {
        for (int k = lane; k < NPL * TBY * SW; k += 32) {
            const int pr = k / SW, c = k - pr * SW;
            const int p = pr / TBY, w = pr - p * TBY;
            tb_cpa4(st + p * Gm::PL_IN + w * SW + c, row_of(p, w) + wrapi(x0 - 4 + c, G.nx));
        }
    }
    asm volatile("cp.async.mbarrier.arrive.shared::cta.b64 [%0];\n" ::"r"(mbar) : "memory");
    __syncwarp();
    if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(mbar) : "memory");
}

// site_events (source current at column x of window row i and time t, receiver writes where owned) from a staged
// list: the same arithmetic in the same order.  Uniform mu only.
// With an anisotropic medium (site_events' sbx, sby, jmu: B_x, B_y scaled by r and 1/r, j_z by mubar; 1 leaves every
// value unchanged).
// With a heterogeneous permeability the sum starts from the B x grad ln mu term shat0 and a source's current is scaled
// by mu at the site (wrapped row y).
__device__ __forceinline__ float ss_list_events(const StepArgs &a, const SsEvList *L, int i, int x, long long t,
                                                bool owned, float g0, float g1, float g2, float g3, float g4,
                                                float cl, float sbx = 1.f, float sby = 1.f, float jmu = 1.f,
                                                float shat0 = 0.f, int y = 0) {
    float shat = shat0;
    for (int j = L->b[i]; j < L->b[i + 1]; j++) {
        const Event ev = L->rec[j];
        if (ev.x != x) continue;
        if (ev.kind == 0) {
            if (ev.comp == 2 && t < a.evt.nt) {
                float jz = __ldg(a.evt.amp + (long long)ev.index * a.evt.nt + t);
                if (a.med.mu) jz = __fmul_rn(jz, __ldg(a.med.mu + (long long)y * a.g.pitch + x));
                shat = __fsub_rn(shat, __fmul_rn(jz, jmu));
            }
        } else if (owned && t < a.evt.cap) {
            const float s = ((g0 + g1) + (g2 + g3)) + g4;
            float v = field2d(ev.comp, cl, s, g4 - g2, g1 - g3);
            if (ev.comp == 3) v = __fmul_rn(v, sbx);
            if (ev.comp == 4) v = __fmul_rn(v, sby);
            a.evt.traces[(long long)ev.index * a.evt.cap + t] = v;
        }
    }
    return shat;
}

// The staged events of window row i for a lane's four sites (columns gx0 .. gx0+3, wrapped into 0 .. nx-1), in one
// pass over the row's records: S^ of each site (shat0 minus mu j_z of the site's sources, in record order, as
// ss_list_events forms it) and the receiver writes of the pre-collision fields of the owned sites (`owned`: the
// row is the caller's; a site is owned when also gx < nx, so an owned column appears at most once).
__device__ __forceinline__ float4 ss_list_events4(const StepArgs &a, const SsEvList *L, int i, int gx0, int nx,
                                                  long long t, bool owned, const float4 (&q)[5], float4 cl,
                                                  float sbx, float sby, float jmu, float4 sh, int y, bool &src) {
    const int w0 = wrapi(gx0, nx);
    for (int j = L->b[i]; j < L->b[i + 1]; j++) {
        const Event ev = L->rec[j];
        int dx = ev.x - w0;  // site k sits at column ev.x when k = dx + a multiple of nx (several only if nx < 4)
        if (dx < 0) dx += nx;
        const bool m0 = dx == 0, m1 = dx == 1 || (dx == 0 && nx == 1),
                   m2 = dx == 2 || (dx < 2 && (2 - dx) % nx == 0), m3 = dx == 3 || (dx < 3 && (3 - dx) % nx == 0);
        if (!(m0 || m1 || m2 || m3)) continue;
        if (ev.kind == 0) {
            if (ev.comp == 2 && t < a.evt.nt) {
                float jz = __ldg(a.evt.amp + (long long)ev.index * a.evt.nt + t);
                if (a.med.mu) jz = __fmul_rn(jz, __ldg(a.med.mu + (long long)y * a.g.pitch + ev.x));
                const float d = __fmul_rn(jz, jmu);
                src = true;
                if (m0) sh.x = __fsub_rn(sh.x, d);
                if (m1) sh.y = __fsub_rn(sh.y, d);
                if (m2) sh.z = __fsub_rn(sh.z, d);
                if (m3) sh.w = __fsub_rn(sh.w, d);
            }
        } else if (owned && t < a.evt.cap) {
            const int lo = a.wx0, hi = min(a.wx1, nx);  // owned columns (the write window's, inside the grid)
            const bool r0 = m0 && gx0 >= lo && gx0 < hi, r1 = m1 && gx0 + 1 >= lo && gx0 + 1 < hi,
                       r2 = m2 && gx0 + 2 >= lo && gx0 + 2 < hi, r3 = m3 && gx0 + 3 >= lo && gx0 + 3 < hi;
            if (r0 || r1 || r2 || r3) {
                const int k = r0 ? 0 : r1 ? 1 : r2 ? 2 : 3;
                const float g0 = get(q[0], k), g1 = get(q[1], k), g2 = get(q[2], k), g3 = get(q[3], k),
                            g4 = get(q[4], k);
                const float s = ((g0 + g1) + (g2 + g3)) + g4;
                float v = field2d(ev.comp, get(cl, k), s, g4 - g2, g1 - g3);
                if (ev.comp == 3) v = __fmul_rn(v, sbx);
                if (ev.comp == 4) v = __fmul_rn(v, sby);
                a.evt.traces[(long long)ev.index * a.evt.cap + t] = v;
            }
        }
    }
    return sh;
}

// Whether window row i of a staged list holds an event.
__device__ __forceinline__ bool ss_list_has_row(const SsEvList *L, int i) { return L->b[i + 1] > L->b[i]; }

// The row pointers of rows ys-2+q (q = lane + 32 j, j < 3) of a unit, -1 outside 0 .. ny.
__device__ __forceinline__ void ss_load_rowptr(const int *rowptr, int ny, int ys, int (&rp)[3]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < 3; j++) {
        const int r = ys - 2 + lane + 32 * j;
        rp[j] = rowptr && r >= 0 && r <= ny ? __ldg(rowptr + r) : -1;
    }
}

// For chunk k of a unit whose row pointers are rp (rows ys-2 ..): whether its rows s-1 .. s+TBY may hold an event
// (bit 25 of the descriptor), and whether they are staged into L (bit 26): the window's row boundaries written, the
// records copied asynchronously, each lane's copies tracked by the stage's mbarrier.  Every lane of the producer warp
// calls it; it ends with __syncwarp, before the producer's arrival on the stage.
template <int TBY>
__device__ __forceinline__ int ss_stage_chunk(const int (&rp)[3], const Event *ev, bool has_events, int ny, int s,
                                              int k, SsEvList *L, unsigned mbar) {
    const int lane = threadIdx.x & 31;
    if (!has_events) return 0;
    const int q = k * TBY + (lane <= TBY + 1 ? lane : 0);  // window row boundary `lane` <-> row s-1+lane
    const int v0 = __shfl_sync(0xffffffffu, rp[0], q & 31), v1 = __shfl_sync(0xffffffffu, rp[1], q & 31),
              v2 = __shfl_sync(0xffffffffu, rp[2], q & 31);
    const int v = (q >> 5) == 0 ? v0 : (q >> 5) == 1 ? v1 : v2;
    const int b0 = __shfl_sync(0xffffffffu, v, 0), bend = __shfl_sync(0xffffffffu, v, TBY + 1);
    const bool inside = s - 1 >= 0 && s + TBY <= ny && k * TBY + TBY + 1 < 96;
    if (!inside) return 1 << 25;  // not staged: the site updates walk the tables
    const int n = bend - b0;
    if (n == 0) return 0;
    if (n > SS_EMAX) return 1 << 25;
    if (lane <= TBY + 1) L->b[lane] = v - b0;
    if (lane == 0) L->n = n;
    if (lane < n) {
        tb_cpa16(reinterpret_cast<float *>(&L->rec[lane]), reinterpret_cast<const float *>(ev + b0 + lane));
        asm volatile("cp.async.mbarrier.arrive.shared::cta.b64 [%0];\n" ::"r"(mbar) : "memory");
    }
    __syncwarp();
    return 3 << 25;
}

// Four site updates at global row gy, columns x0+4*lane.., from the pulled populations q[0..4] and c_L^2.  Without
// EV the sources and receivers, if any, come from a staged list `el` (window row li): the row takes the plain path,
// collide2d_free, and a lane with a source adds the collision's S^ terms afterwards (collide2d is collide2d_free
// followed by those additions, so the bits are collide2d's).  With EV they come from a staged list `el`, or with
// none (a chunk not staged) are looked up per site in the global tables, and every site takes collide2d.
//
// With AN (a uniform in-plane permeability tensor, a.med.ar / a.med.amu) the site update is the general kernel's
// collide2d_an with its per-axis speeds (r, 1/r) and no pole, and the events scale as in site_events; its event
// rows take the EV path (folded into the plain path they slowed its plain rows).
//
// With MU (a heterogeneous permeability: d_x ln mu, d_y ln mu of the four sites in dlx, dly) each site's S^ carries
// B_x d_y ln mu - B_y d_x ln mu (mu_source), as in the single-step kernels.
template <bool EV, bool AN = false, bool MU = false>
__device__ __forceinline__ void ss_update4(const StepArgs &a, const float4 (&q)[5], float4 cl, int x0, int gy,
                                           long long t, bool owned, float4 (&o)[5], const SsEvList *el = nullptr,
                                           int li = 0, float4 dlx = float4(), float4 dly = float4()) {
    const Grid &G = a.g;
    const int lane = threadIdx.x & 31;
    const float ar = AN ? a.med.ar : 1.f, ri = AN ? __fdiv_rn(1.f, ar) : 1.f, fs = __fadd_rn(ar, ri);
    owned = owned && gy >= a.wy0 && gy < a.wy1;  // receivers only inside the write window
    if (!EV) {
        // S^ of the four sites: the permeability term (MU), minus mu j_z of the sources of a staged list `el`, whose
        // receivers are written here from the pre-collision populations
        float4 sh = make_float4(0.f, 0.f, 0.f, 0.f);
        if (MU) {
#pragma unroll
            for (int k = 0; k < 4; k++)
                set(sh, k, mu_source(get(q[4], k) - get(q[2], k), get(q[1], k) - get(q[3], k), get(dlx, k),
                                     get(dly, k)));
        }
        bool src = false;
        if (!AN && el)
            sh = ss_list_events4(a, el, li, x0 + 4 * lane, G.nx, t, owned && gy < G.ny, q, cl, ar, ri,
                                 AN ? a.med.amu : 1.f, sh, wrapi(gy, G.ny), src);
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const float q0 = get(q[0], k), q1 = get(q[1], k), q2 = get(q[2], k), q3 = get(q[3], k),
                        q4 = get(q[4], k), ck = get(cl, k);
            const Out5 r = AN   ? collide2d_an(q0, q1, q2, q3, q4, ck, 0.f, ar, ri, fs, 0.f)
                           : MU ? collide2d(q0, q1, q2, q3, q4, ck, get(sh, k))
                                : collide2d_free(q0, q1, q2, q3, q4, ck);
            set(o[0], k, r.o0);
            set(o[1], k, r.o1);
            set(o[2], k, r.o2);
            set(o[3], k, r.o3);
            set(o[4], k, r.o4);
        }
        if (!MU && src) {  // the source terms added as the collision with S^ adds them (+0 S^ adds -0: no change)
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const float ck = get(cl, k), h = get(sh, k);
                const float w0 = __fsub_rn(1.f, 2.f * ck);
                const float Tm = __fmul_rn(-0.5f * ck, h), T0 = __fmul_rn(-w0, h);
                set(o[0], k, __fadd_rn(get(o[0], k), T0));
                set(o[1], k, __fadd_rn(get(o[1], k), Tm));
                set(o[2], k, __fadd_rn(get(o[2], k), Tm));
                set(o[3], k, __fadd_rn(get(o[3], k), Tm));
                set(o[4], k, __fadd_rn(get(o[4], k), Tm));
            }
        }
        return;
    }
    if (AN && el) {  // EV with a staged list (the anisotropic medium's event rows): one pass, then collide2d_an with S^
        float4 sh = make_float4(0.f, 0.f, 0.f, 0.f);
        bool src = false;
        sh = ss_list_events4(a, el, li, x0 + 4 * lane, G.nx, t, owned && gy < G.ny, q, cl, ar, ri,
                             AN ? a.med.amu : 1.f, sh, wrapi(gy, G.ny), src);
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const Out5 r = collide2d_an(get(q[0], k), get(q[1], k), get(q[2], k), get(q[3], k), get(q[4], k),
                                        get(cl, k), get(sh, k), ar, ri, fs, 0.f);
            set(o[0], k, r.o0);
            set(o[1], k, r.o1);
            set(o[2], k, r.o2);
            set(o[3], k, r.o3);
            set(o[4], k, r.o4);
        }
        return;
    }
    // EV: a chunk whose events were not staged, each site's events looked up in the global tables
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const float q0 = get(q[0], k), q1 = get(q[1], k), q2 = get(q[2], k), q3 = get(q[3], k), q4 = get(q[4], k),
                    ck = get(cl, k);
        const float shat0 = MU ? mu_source(q4 - q2, q1 - q3, get(dlx, k), get(dly, k)) : 0.f;
        const int gx = x0 + 4 * lane + k;
        const bool own = owned && gx < G.nx && gy < G.ny && gx >= a.wx0 && gx < a.wx1;
        const float jmu = AN ? a.med.amu : 1.f;
        const float shat = AN ? site_events(a, wrapi(gx, G.nx), wrapi(gy, G.ny), t, own, q0, q1, q2, q3, q4, ck, 0.f,
                                            0.f, ar, ri, jmu)
                              : site_events(a, wrapi(gx, G.nx), wrapi(gy, G.ny), t, own, q0, q1, q2, q3, q4, ck, shat0);
        const Out5 r = AN ? collide2d_an(q0, q1, q2, q3, q4, ck, shat, ar, ri, fs, 0.f)
                          : collide2d(q0, q1, q2, q3, q4, ck, shat);
        set(o[0], k, r.o0);
        set(o[1], k, r.o1);
        set(o[2], k, r.o2);
        set(o[3], k, r.o3);
        set(o[4], k, r.o4);
    }
}

// The populations pulled by a lane's four sites at row `row` of a stage S with plane stride PL: g0, g2, g4 from
// columns c.., g1 from c-1.., g3 from c+1.. (Eq. 17), and c_L^2 from plane 5.
__device__ __forceinline__ void ss_pull(const float *S, int PL, int row, int c, float4 (&q)[5], float4 &cl,
                                        float4 *dlx = nullptr, float4 *dly = nullptr) {
    const float *r = S + row * SW + c;
    if (dlx) {  // planes 6 and 7: d_x ln mu, d_y ln mu
        *dlx = lds4(r + 6 * PL);
        *dly = lds4(r + 7 * PL);
    }
    q[0] = lds4(r);
    const float4 l1 = lds4(r + PL - 4), m1 = lds4(r + PL);
    q[1] = make_float4(l1.w, m1.x, m1.y, m1.z);
    q[2] = lds4(r + 2 * PL);
    const float4 m3 = lds4(r + 3 * PL), h3 = lds4(r + 3 * PL + 4);
    q[3] = make_float4(m3.y, m3.z, m3.w, h3.x);
    q[4] = lds4(r + 4 * PL);
    cl = lds4(r + 5 * PL);
}

__device__ __forceinline__ bool ss_row_events(const StepArgs &a, int gy) {
    const int y = wrapi(gy, a.g.ny);
    return __ldg(a.evt.rowptr + y) != __ldg(a.evt.rowptr + y + 1);
}

// Step t on row w of the chunk in stage `st` (global row r = s + w), the lane's four sites; results go to the ring at
// the rows that pull them (ring row u = r - ys + 2 for planes 0, 1, 3 and c_L^2, u + 1 for plane 2, u - 1 for plane
// 4).  With the images in `es` (emode 1: left of the strip, 2: right of it) lane 0's g1 or lane 31's g3 come from
// there.
template <int TBY, int S, bool EV, bool AN = false, bool MU = false>
__device__ __forceinline__ void ss_step_a(const StepArgs &a, const float *st, const float *es, int emode, float *P,
                                          int x0, int ys, int ye, int r, int w, int u, long long t,
                                          const SsEvList *el) {
    using Gm = SsGeom<TBY, S>;
    constexpr int M = Gm::M, PP = Gm::PL_P;
    const int lane = threadIdx.x & 31, c = 4 + 4 * lane;
    float4 q[5], cl, o[5], dlx = make_float4(0.f, 0.f, 0.f, 0.f), dly = dlx;
    ss_pull(st, Gm::PL_IN, w, c, q, cl, MU ? &dlx : nullptr, MU ? &dly : nullptr);
    if (emode == 1 && lane == 0) q[1].x = es[Gm::EPL + w * 4 + 3];        // column x0-1 = nx-1
    if (emode == 2 && lane == 31) q[3].w = es[3 * Gm::EPL + w * 4 + 0];   // column x0+128 = 0
    ss_update4<EV, AN, MU>(a, q, cl, x0, r, t, r >= ys && r < ye, o, el, w + 1, dlx, dly);
    const int s0 = u % M, s2 = s0 == M - 1 ? 0 : s0 + 1, s4 = s0 == 0 ? M - 1 : s0 - 1;
    float *p0 = P + s0 * SW + c;
    sts4(p0, o[0]);
    sts4(p0 + PP, o[1]);
    sts4(p0 + 3 * PP, o[3]);
    sts4(p0 + 5 * PP, cl);
    if (MU) {  // the medium of the row, for step t+1
        sts4(p0 + 6 * PP, dlx);
        sts4(p0 + 7 * PP, dly);
    }
    sts4(P + 2 * PP + s2 * SW + c, o[2]);
    sts4(P + 4 * PP + s4 * SW + c, o[4]);
}

// The ring sites of the chunk in stage `st`, by the ring warp: lane 2w takes column x0-1 of chunk row w (plane 1
// only), lane 2w+1 column x0+128 (plane 3 only), at ring row p TBY + w + 1 (p: the CTA's phase); with the images in
// `es` the columns outside the grid come from there.
template <int TBY, int S, bool AN = false, bool MU = false>
__device__ __forceinline__ void ss_ring(const StepArgs &a, const float *st, const float *es, int emode, float *P,
                                        int x0, int s, int p, bool events, long long t, const SsEvList *el) {
    using Gm = SsGeom<TBY, S>;
    const int lane = threadIdx.x & 31;
    if (lane >= 2 * TBY) return;
    const int w = lane >> 1, right = lane & 1, cc = right ? SBX + 4 : 3, r = s + w;
    auto v = [&](int pl, int col) -> float {
        if (emode == 1 && col < 4) return es[pl * Gm::EPL + w * 4 + col];
        if (emode == 2 && col >= SBX + 4) return es[pl * Gm::EPL + w * 4 + col - (SBX + 4)];
        return st[pl * Gm::PL_IN + w * SW + col];
    };
    const float q0 = v(0, cc), q1 = v(1, cc - 1), q2 = v(2, cc), q3 = v(3, cc + 1), q4 = v(4, cc), ck = v(5, cc);
    const float ar = AN ? a.med.ar : 1.f, ri = AN ? __fdiv_rn(1.f, ar) : 1.f, fs = __fadd_rn(ar, ri);
    const float jmu = AN ? a.med.amu : 1.f;
    const float shat0 = MU ? mu_source(q4 - q2, q1 - q3, v(6, cc), v(7, cc)) : 0.f;
    float shat = shat0;
    if (el)
        shat = ss_list_events(a, el, w + 1, wrapi(x0 - 4 + cc, a.g.nx), t, false, q0, q1, q2, q3, q4, ck, ar, ri, jmu,
                              shat0, wrapi(r, a.g.ny));
    else if (events && ss_row_events(a, r))
        shat = AN ? site_events(a, wrapi(x0 - 4 + cc, a.g.nx), wrapi(r, a.g.ny), t, false, q0, q1, q2, q3, q4, ck, 0.f,
                                0.f, ar, ri, jmu)
                  : site_events(a, wrapi(x0 - 4 + cc, a.g.nx), wrapi(r, a.g.ny), t, false, q0, q1, q2, q3, q4, ck,
                                shat0);
    const Out5 ro = AN ? collide2d_an(q0, q1, q2, q3, q4, ck, shat, ar, ri, fs, 0.f)
                       : collide2d(q0, q1, q2, q3, q4, ck, shat);
    const int s0 = (p * TBY + w + 1) % Gm::M;
    if (right)
        P[3 * Gm::PL_P + s0 * SW + cc] = ro.o3;
    else
        P[Gm::PL_P + s0 * SW + cc] = ro.o1;
}

// Step t+1 on global row rb (ring row ub), written as 16-byte streaming stores.
template <int TBY, int S, bool EV, bool AN = false, bool MU = false>
__device__ __forceinline__ void ss_step_b(const StepArgs &a, const float *P, int x0, int rb, int ub, long long t,
                                          const SsEvList *el, int w) {
    using Gm = SsGeom<TBY, S>;
    const Grid &G = a.g;
    const int lane = threadIdx.x & 31, c = 4 + 4 * lane;
    float4 q[5], cl, o[5], dlx = make_float4(0.f, 0.f, 0.f, 0.f), dly = dlx;
    ss_pull(P, Gm::PL_P, ub % Gm::M, c, q, cl, MU ? &dlx : nullptr, MU ? &dly : nullptr);
    ss_update4<EV, AN, MU>(a, q, cl, x0, rb, t + 1, true, o, el, w, dlx, dly);
    const int xs = x0 + 4 * lane;
    if (xs < G.pitch) {  // pitch is a multiple of 4: a lane's 4 columns are all in or all out
        float *op = static_cast<float *>(a.out.data) + (long long)rb * G.pitch + xs;
        // the write window (walls: the bands next to them are the edge pass's); columns past nx are padding
        unsigned m = 15u;
        if (a.wx0 > 0 || a.wy0 > 0 || a.wx1 < G.pitch || a.wy1 < G.ny) {  // (a window: walls)
            const bool rowin = rb >= a.wy0 && rb < a.wy1;
            m = 0u;
#pragma unroll
            for (int j = 0; j < 4; j++)
                m |= (xs + j >= G.nx || (rowin && xs + j >= a.wx0 && xs + j < a.wx1)) ? 1u << j : 0u;
        }
        if (m == 15u) {
            float4 *op4 = reinterpret_cast<float4 *>(op);
            const long long pl4 = G.plane / 4;
            __stcs(op4, o[0]);
            __stcs(op4 + pl4, o[1]);
            __stcs(op4 + 2 * pl4, o[2]);
            __stcs(op4 + 3 * pl4, o[3]);
            __stcs(op4 + 4 * pl4, o[4]);
        } else if (m) {
#pragma unroll
            for (int j = 0; j < 4; j++)
                if ((m >> j) & 1u)
#pragma unroll
                    for (int p = 0; p < 5; p++) op[p * G.plane + j] = get(o[p], j);
        }
    }
}

// A chunk's descriptor (in shared memory, DS = S + 2 of them in a ring): the unit's strip x0 and rows ys .. ye-1, and
// w = the chunk's index k in the unit | staging mode << 16 | column mode << 20 | 1 << 24 (0: the stream has ended)
// | 1 << 25 when rows s-1 .. s+TBY of the chunk may hold a source or receiver.
__device__ __forceinline__ bool ss_valid(int4 d) { return (d.w >> 24) & 1; }
__device__ __forceinline__ bool ss_events(int4 d) { return (d.w >> 25) & 1; }

// Block barrier 1 of the n consumer threads, returning whether any of them passed true.
__device__ __forceinline__ bool ss_consumers_or(bool v, int n) {
    int r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.s32 q, %1, 0;\n bar.red.or.pred p, 1, %2, q;\n selp.s32 %0, 1, 0, p;\n}\n"
        : "=r"(r)
        : "r"((int)v), "r"(n)
        : "memory");
    return r != 0;
}

// The queue of units: the first nbig are strip u % nstrip, rows (u / nstrip) H .. + H - 1; the rest, from row
// Yb = (nbig / nstrip) H on, strip j % nstrip, runs of Hs rows (j = u - nbig), so that the last units taken are short.
struct SsUnits {
    int nstrip, H, Hs, nbig, nunits;
};
__device__ __forceinline__ void ss_unit(const SsUnits &U, int ny, int u, int &x0, int &ys, int &ye) {
    if (u < U.nbig) {
        x0 = (u % U.nstrip) * SBX;
        ys = (u / U.nstrip) * U.H;
        ye = min(ys + U.H, ny);
    } else {
        const int j = u - U.nbig;
        x0 = (j % U.nstrip) * SBX;
        ys = (U.nbig / U.nstrip) * U.H + (j / U.nstrip) * U.Hs;
        ye = min(ys + U.Hs, ny);
    }
}

// Persistent CTAs over the queue of units, taken in order from the handle's counter, so that CTAs slowed down by
// sources, receivers or the memory they read take fewer units.  The chunks of a CTA's successive units form one
// stream.
//
// The producer warp (the last) runs ahead of the others: for stream chunk c it waits until stage c % S is free (its
// empty mbarrier: the warps that read the stage are done with chunk c - S), writes the chunk's descriptor and stages
// it (full mbarrier); after the last chunk it writes an end descriptor.  It takes the next unit from the queue when it
// starts a unit, and loads that unit's row pointers (one chunk per lane) then, so that their event flags are ready.
//
// The other warps run phase p on stream chunk p: warps 0 .. TBY-1 step t on its rows, warps TBY .. 2 TBY - 1 step t+1
// one behind chunk p - 1 (whatever units the two chunks belong to), the ring warp its ring sites; ring rows are
// numbered by the phase (rows of step t+1 that would pull across a unit boundary lie outside their unit and are
// skipped).  The step-t and ring warps release the stage once they have read it; a barrier of these 2 TBY + 1 warps
// closes the phase.
template <int TBY, int S, int MINB, bool AN = false, bool MU = false>
__global__ void __launch_bounds__((2 * TBY + 2) * 32, MINB)
    step2d_ss2(StepArgs a, const __grid_constant__ CUtensorMap tmIn, const __grid_constant__ CUtensorMap tmCL,
               const __grid_constant__ CUtensorMap tmIn4, const __grid_constant__ CUtensorMap tmCL4,
               const __grid_constant__ CUtensorMap tmDL, const __grid_constant__ CUtensorMap tmDL4, int use_tma,
               SsUnits U) {
    using Gm = SsGeom<TBY, S, false, MU>;
    constexpr int NC = 2 * TBY + 1, DS = Gm::DS;  // consumer warps (the ring warp is warp 2 TBY)
    extern __shared__ __align__(1024) float sm[];
    float *E = sm + Gm::IN_SZ;
    float *P = E + Gm::E_SZ;
    SsDesc *desc = reinterpret_cast<SsDesc *>(P + Gm::P_SZ);
    unsigned long long *mb = reinterpret_cast<unsigned long long *>(desc + DS);  // full[S], then empty[S]
    const Grid &G = a.g;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool tma = use_tma && !(smem_u32(sm) & 127);  // TMA destinations here are 128-byte aligned
    const unsigned full0 = smem_u32(mb), empty0 = full0 + 8 * S;
    if (tid < S) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(full0 + 8 * tid) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(empty0 + 8 * tid), "r"(TBY + 1) : "memory");
    }
    if (tid == 0) asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    __syncthreads();
    const unsigned long long wait_limit = g_ss_wait_limit_ns;
    if (warp == NC) {
        // ---- producer (every lane keeps the same unit state)
        if (lane < (MU ? 6 : 4)) {  // the tensor maps, into the copy engine's descriptor cache
            const CUtensorMap *m = lane == 0   ? &tmIn
                                   : lane == 1 ? &tmCL
                                   : lane == 2 ? &tmIn4
                                   : lane == 3 ? &tmCL4
                                   : lane == 4 ? &tmDL
                                               : &tmDL4;
            asm volatile("prefetch.tensormap [%0];\n" ::"l"(m) : "memory");
        }
        int cK = 0, ck = 0, cx0 = 0, cys = 0, cye = 0, cxm = 0;
        int nu = 0, rpc[3], rpn[3];  // the next unit; row pointers of the current and the next unit (rows ys-2 ..)
        auto fetch_next = [&]() {
            int u = 0;
            if (lane == 0) u = atomicAdd(a.sched, 1);
            nu = __shfl_sync(0xffffffffu, u, 0);
            if (nu < U.nunits && a.evt.rowptr) {  // loaded now, used when the unit starts
                int x0, ys, ye;
                ss_unit(U, G.ny, nu, x0, ys, ye);
                ss_load_rowptr(a.evt.rowptr, G.ny, ys, rpn);
            }
        };
        fetch_next();
        int c = 0;
        bool ok = true;
        for (;; c++) {
            if (c >= S && !mbar_wait(empty0 + 8 * (c % S), (unsigned)(c / S - 1) & 1u, wait_limit)) {
                ok = false;
                break;
            }
            if (ck == cK && nu < U.nunits) {  // start the next unit
                ss_unit(U, G.ny, nu, cx0, cys, cye);
                cK = (cye - cys + 2 + TBY - 1) / TBY;  // step-t chunks: rows ys-1 .. ys-2+K*TBY (through ye)
                cxm = ss_xmode(G, cx0);
                ck = 0;
#pragma unroll
                for (int j = 0; j < 3; j++) rpc[j] = rpn[j];
                fetch_next();
            }
            int4 d = make_int4(0, 0, 0, 0);
            if (ck < cK) {
                const int s = cys - 1 + ck * TBY, mode = ss_chunk_mode<TBY>(G, cxm, s, tma);
                d = make_int4(cx0, cys, cye, ck | mode << 16 | cxm << 20 | 1 << 24);
                d.w |= ss_stage_chunk<TBY>(rpc, a.evt.ev, a.evt.rowptr != nullptr, G.ny, s, ck, &desc[c % DS].ev,
                                           full0 + 8 * (c % S));
                ck++;
            }
            if (lane == 0) desc[c % DS].d0 = d;
            if (!ss_valid(d)) {  // end of the stream: the consumers find the end descriptor
                __syncwarp();
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(full0 + 8 * (c % S)) : "memory");
                break;
            }
            ss_issue<TBY, S, MU>(a, d.x, cxm, d.y - 1 + (d.w & 0xffff) * TBY, (d.w >> 16) & 15,
                                 sm + (c % S) * Gm::STAGE, E + (c % S) * Gm::ESTAGE, full0 + 8 * (c % S), &tmIn, &tmCL,
                                 &tmIn4, &tmCL4, &tmDL, &tmDL4);
        }
        if (!ok) {  // the consumers stopped: flag it, let this warp's copies in flight land (bounded)
            if (lane == 0) atomicExch(&g_ss_timeouts, 1);
            for (int k = c > S ? c - S : 0; k < c; k++)
                mbar_wait(full0 + 8 * (k % S), (unsigned)(k / S) & 1u, kSsDrainNs);
        }
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        __threadfence();  // the queue accesses before the CTA counts itself out
    } else {
        // ---- step t, step t+1 and the ring sites
        const long long t = a.t;
        for (int p = 0;; p++) {
            const bool ok = mbar_wait(full0 + 8 * (p % S), (unsigned)(p / S) & 1u, wait_limit);
            const int4 da = desc[p % DS].d0, db = desc[(p + DS - 1) % DS].d0;
            const bool va = ok && ss_valid(da), vb = p >= 1 && ss_valid(db);
            const SsEvList *ela = (da.w >> 26) & 1 ? &desc[p % DS].ev : nullptr;
            const SsEvList *elb = (db.w >> 26) & 1 ? &desc[(p + DS - 1) % DS].ev : nullptr;
            const float *st = sm + (p % S) * Gm::STAGE, *es = E + (p % S) * Gm::ESTAGE;
            const int emode = ((da.w >> 16) & 15) == 1 ? (da.w >> 20) & 15 : 0, s = da.y - 1 + (da.w & 0xffff) * TBY;
            if (warp < TBY) {
                if (va) {
                    const int r = s + warp;
                    const bool ev = ss_events(da) && (ela ? ss_list_has_row(ela, warp + 1) : ss_row_events(a, r));
                    if (ev && (!ela || AN))  // (a chunk whose events were not staged walks the global tables)
                        ss_step_a<TBY, S, true, AN, MU>(a, st, es, emode, P, da.x, da.y, da.z, r, warp,
                                                        p * TBY + warp + 1, t, ela);
                    else
                        ss_step_a<TBY, S, false, AN, MU>(a, st, es, emode, P, da.x, da.y, da.z, r, warp,
                                                         p * TBY + warp + 1, t, ev ? ela : nullptr);
                }
            } else if (warp < 2 * TBY) {
                const int w = warp - TBY;
                if (vb) {
                    const int rb = db.y - 2 + (db.w & 0xffff) * TBY + w;
                    if (rb >= db.y && rb < db.z) {
                        const bool ev = ss_events(db) && (elb ? ss_list_has_row(elb, w) : ss_row_events(a, rb));
                        if (ev && (!elb || AN))
                            ss_step_b<TBY, S, true, AN, MU>(a, P, db.x, rb, (p - 1) * TBY + w, t, elb, w);
                        else
                            ss_step_b<TBY, S, false, AN, MU>(a, P, db.x, rb, (p - 1) * TBY + w, t, ev ? elb : nullptr,
                                                             w);
                    }
                }
            } else if (va) {
                ss_ring<TBY, S, AN, MU>(a, st, es, emode, P, da.x, s, p, ss_events(da), t, ela);
            }
            if (va && (warp < TBY || warp == 2 * TBY)) {  // this warp has read the stage: release it to the producer
                __syncwarp();
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(empty0 + 8 * (p % S)) : "memory");
            }
            // the phase's ring writes before the next phase's reads
            if (ss_consumers_or(!ok, NC * 32)) {  // a chunk never arrived: flag it and stop (the producer drains)
                if (tid == 0) atomicExch(&g_ss_timeouts, 1);
                break;
            }
            if (!ss_valid(da)) break;  // the end descriptor: step t+1 of the last chunk was this phase's
        }
    }
    // count this CTA out; the last one resets the queue for the next launch
    __syncthreads();
    if (tid == 0 && atomicAdd(a.sched + 1, 1) == (int)gridDim.x - 1) {
        a.sched[0] = 0;
        a.sched[1] = 0;
    }
}

// Tensor maps of the populations ([5][ny][pitch] floats, box: one plane of TBY rows of `w` columns) and c_L^2;
// false if unavailable (every chunk is then staged by asynchronous copies).
static bool ss_make_maps(const StepArgs &a, int tby, int w, CUtensorMap *mIn, CUtensorMap *mCL) {
    EncodeTiled fn = encode_fn();
    if (!fn || a.g.nx < SW || a.g.ny < tby + 2) return false;
    const cuuint64_t dims3[3] = {(cuuint64_t)a.g.nx, (cuuint64_t)a.g.ny, 5};
    const cuuint64_t str3[2] = {(cuuint64_t)a.g.pitch * 4, (cuuint64_t)a.g.plane * 4};
    const cuuint32_t box3[3] = {(cuuint32_t)w, (cuuint32_t)tby, 1};
    const cuuint32_t one[3] = {1, 1, 1};
    if (fn(mIn, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(a.in.data), dims3, str3, box3, one,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    const cuuint64_t dims2[2] = {(cuuint64_t)a.g.nx, (cuuint64_t)a.g.ny};
    const cuuint64_t str2[1] = {(cuuint64_t)a.g.pitch * 4};
    const cuuint32_t box2[2] = {(cuuint32_t)w, (cuuint32_t)tby};
    return fn(mCL, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(a.med.cL2), dims2, str2, box2, one,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor map of the gradient of ln mu ([2][ny][pitch] floats: d_x, d_y; box: one plane of TBY rows of `w` columns).
static bool ss_make_dl_map(const StepArgs &a, int tby, int w, CUtensorMap *m) {
    EncodeTiled fn = encode_fn();
    if (!fn || !a.med.dlnmu || a.g.nx < SW || a.g.ny < tby + 2) return false;
    const cuuint64_t dims3[3] = {(cuuint64_t)a.g.nx, (cuuint64_t)a.g.ny, 2};
    const cuuint64_t str3[2] = {(cuuint64_t)a.g.pitch * 4, (cuuint64_t)a.g.plane * 4};
    const cuuint32_t box3[3] = {(cuuint32_t)w, (cuuint32_t)tby, 1};
    const cuuint32_t one[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(a.med.dlnmu), dims3, str3, box3, one,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Persistent CTAs (as many as are resident, at most one per unit) over units of MCH TBY - 2 rows (MCH chunks each),
// and units of 2 TBY - 2 rows (two chunks) for the last rows: about two short units per CTA.
template <int TBY, int S, int MINB, int MCH, bool AN = false, bool MU = false>
static cudaError_t launch_ss(const StepArgs &a, cudaStream_t s) {
    using Gm = SsGeom<TBY, S, false, MU>;
    constexpr int NT = (2 * TBY + 2) * 32;
    static_assert(MCH <= 32, "a unit's event flags are one 32-bit mask");
    if (!a.sched) return cudaErrorInvalidValue;
    static int per_sm = 0, nsm = 0;
    if (!per_sm) {
        cudaError_t e = cudaFuncSetAttribute(step2d_ss2<TBY, S, MINB, AN, MU>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Gm::BYTES);
        if (e != cudaSuccess) return e;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step2d_ss2<TBY, S, MINB, AN, MU>, NT, Gm::BYTES);
        if (per_sm < 1) per_sm = 1;
    }
    CUtensorMap mIn, mCL, mIn4, mCL4, mDL, mDL4;
    memset(&mIn, 0, sizeof mIn);
    memset(&mCL, 0, sizeof mCL);
    memset(&mIn4, 0, sizeof mIn4);
    memset(&mCL4, 0, sizeof mCL4);
    memset(&mDL, 0, sizeof mDL);
    memset(&mDL4, 0, sizeof mDL4);
    const int use_tma = ss_make_maps(a, TBY, SW, &mIn, &mCL) && ss_make_maps(a, TBY, 4, &mIn4, &mCL4) &&
                                (!MU || (ss_make_dl_map(a, TBY, SW, &mDL) && ss_make_dl_map(a, TBY, 4, &mDL4)))
                            ? 1
                            : 0;
    SsUnits U;
    U.nstrip = (a.g.nx + SBX - 1) / SBX;
    U.H = MCH * TBY - 2;
    U.Hs = 2 * TBY - 2;
    const long long slots = (long long)per_sm * nsm;
    const long long small_rows = (2 * slots + U.nstrip - 1) / U.nstrip * U.Hs;  // about two short units per CTA
    const long long big_runs = small_rows >= a.g.ny ? 0 : (a.g.ny - small_rows) / U.H;
    U.nbig = (int)(big_runs * U.nstrip);
    const long long rest = a.g.ny - big_runs * U.H;
    const long long nunits = U.nbig + (long long)U.nstrip * ((rest + U.Hs - 1) / U.Hs);
    if (nunits > (1 << 30)) return cudaErrorInvalidValue;
    U.nunits = (int)nunits;
    const int blocks = (int)(nunits < slots ? nunits : slots);
    step2d_ss2<TBY, S, MINB, AN, MU><<<blocks, NT, Gm::BYTES, s>>>(a, mIn, mCL, mIn4, mCL4, mDL, mDL4, use_tma, U);
    return cudaGetLastError();
}

// Shapes (rows per chunk, stages, CTAs per SM, chunks per tall unit); shared memory 86, 73, 106, 68, 73 and 68 KB.
// Measured on 4096^2 (heterogeneous medium): 257-261k Mlups for shapes 0, 1 and 5, against 247k for the tile kernel,
// before later changes; shape 1 (the default) with 12 chunks per unit 271.8k, with 16 268.8k, 24 266.9k, 8 271.6k.
int ss2_nshapes() { return 6; }

cudaError_t launch_step_2d_ss2(const StepArgs &a, int shape, cudaStream_t s) {
    switch (shape) {
        case 1: return launch_ss<4, 3, 3, 12>(a, s);
        case 2: return launch_ss<6, 3, 2, 12>(a, s);
        case 3: return launch_ss<3, 4, 3, 24>(a, s);
        case 4: return launch_ss<4, 3, 3, 32>(a, s);
        case 5: return launch_ss<3, 4, 3, 12>(a, s);
        default: return launch_ss<4, 4, 2, 16>(a, s);
    }
}

// =====================================================================================================
// The batch over its packed states (the layout of step2d_batch_tb2: member m from packed row r0[m], packed row
// r0[m] + 2 + y <-> member row y in [-2, ny + 1], packed column x + 4 <-> member column x, two rows and columns of
// periodic images around each member).  The strip kernel's phases run over units of one member each; every chunk is
// six TMA boxes of the packed input (the images make a window never wrap), and step t+1 writes each output site and,
// within two of an edge, its images, so the next launch finds the halo current.  The site updates are those of
// step2d_ss2, so every member's result is bit-identical to its single steps.

// Step t+1 on member row rb (ring row ub), written to the packed output with the row's and the lane's images.
template <int TBY, int S, bool EV>
__device__ __forceinline__ void ss_step_b_packed(const StepArgs &a, const float *P, int x0, int rb, int ub, long long t,
                                                 float *out, long long pplane, int W, int prow0, int nx, int ny,
                                                 const SsEvList *el, int w) {
    using Gm = SsGeom<TBY, S>;
    const int lane = threadIdx.x & 31, c = 4 + 4 * lane;
    float4 q[5], cl, o[5];
    ss_pull(P, Gm::PL_P, ub % Gm::M, c, q, cl);
    ss_update4<EV>(a, q, cl, x0, rb, t + 1, true, o, el, w);
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
                    for (int p = 0; p < 5; p++) r[p * pplane + j] = get(o[p], j);
        }
    };
    store_row(rb);
    for (int yy = rb + ny; yy <= ny + 1; yy += ny) store_row(yy);  // images in the upper halo rows
    for (int yy = rb - ny; yy >= -2; yy -= ny) store_row(yy);      // and in the lower ones
    if (xs < 2 || xs + 3 >= nx - 2) {  // sites within two of the left or right edge: their column images
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int x = xs + j;
            const float v0 = get(o[0], j), v1 = get(o[1], j), v2 = get(o[2], j), v3 = get(o[3], j), v4 = get(o[4], j);
            auto put = [&](int yy, int xi) {
                float *r = row_at(yy) + xi;
                r[0] = v0;
                r[pplane] = v1;
                r[2 * pplane] = v2;
                r[3 * pplane] = v3;
                r[4 * pplane] = v4;
            };
            if (x < nx) {
                for (int xi = x + nx; xi <= nx + 1; xi += nx)
                    for (int yy = rb - ((rb + 2) / ny) * ny; yy <= ny + 1; yy += ny) put(yy, xi);
                for (int xi = x - nx; xi >= -2; xi -= nx)
                    for (int yy = rb - ((rb + 2) / ny) * ny; yy <= ny + 1; yy += ny) put(yy, xi);
            }
        }
    }
}

// Persistent CTAs over the queue of units (taken in order from the counters `sched`), a producer warp running ahead
// of the step-t, step-t+1 and ring warps, as step2d_ss2.  A chunk's descriptor is two int4: the unit's x0, ys, ye and
// k | 1 << 24 | event flag << 25, then its member m, packed row prow0 and size; the producer reads the next unit's
// table entry (one word per lane) when it starts a unit.
template <int TBY, int S, int MINB>
__global__ void __launch_bounds__((2 * TBY + 2) * 32, MINB)
    step2d_batch_ss2(const StepArgs *__restrict__ args, const BatchUnit *__restrict__ units, int nunits, int *sched,
                     const long long *__restrict__ t0p, int toff, int par, BatchPacked pk,
                     const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                     const __grid_constant__ CUtensorMap tmCL) {
    using Gm = SsGeom<TBY, S, true>;
    constexpr int NC = 2 * TBY + 1, DS = Gm::DS;
    constexpr int NA = (int)(sizeof(StepArgs) / 16);  // 16-byte pieces of a member's arguments
    static_assert(sizeof(StepArgs) % 16 == 0 && NA <= 32, "arguments copied by one warp in 16-byte pieces");
    extern __shared__ __align__(1024) float sm[];
    float *P = sm + Gm::IN_SZ + Gm::E_SZ;
    SsDesc *desc = reinterpret_cast<SsDesc *>(P + Gm::P_SZ);
    // per descriptor slot its member's arguments: the site updates' event path reads them from shared memory (global
    // loads of them missed L1, which shared memory fills, and stalled each event row)
    StepArgs *sargs = reinterpret_cast<StepArgs *>(desc + DS);
    unsigned long long *mb = reinterpret_cast<unsigned long long *>(sargs + DS);  // full[S], then empty[S]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const unsigned full0 = smem_u32(mb), empty0 = full0 + 8 * S;
    if (tid < S) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(full0 + 8 * tid) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(empty0 + 8 * tid), "r"(TBY + 1) : "memory");
    }
    if (tid == 0) asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    __syncthreads();
    const unsigned long long wait_limit = g_ss_wait_limit_ns;
    const bool aligned = !(smem_u32(sm) & 127);  // TMA destinations here are 128-byte aligned (checked on the host too)
    if (warp == NC) {
        // ---- producer
        const CUtensorMap *tmIn = par ? &tmB : &tmA;
        if (lane < 2) asm volatile("prefetch.tensormap [%0];\n" ::"l"(lane == 0 ? tmIn : &tmCL) : "memory");
        int cK = 0, ck = 0, nu = 0, nd = 0;
        int cm = 0, cx0 = 0, cys = 0, cye = 0, cpr = 0, cnx = 0, cny = 0;
        const int *crp = nullptr;
        const Event *cev = nullptr;
        int rpc[3], rpn[3];  // row pointers of the current and the next unit's rows ys-2 ..
        bool rpn_ready = false;
        auto field = [&](int f) { return __shfl_sync(0xffffffffu, nd, f); };
        auto ptr = [&](int f) {  // a pointer field of the next unit's table entry (two words)
            return (const void *)(((unsigned long long)(unsigned)field(f + 1) << 32) | (unsigned)field(f));
        };
        auto fetch_next = [&]() {  // the next unit and its table entry (one word per lane), in flight from here
            int u = 0;
            if (lane == 0) u = atomicAdd(sched, 1);
            nu = __shfl_sync(0xffffffffu, u, 0);
            nd = nu < nunits && lane < 12 ? __ldg(reinterpret_cast<const int *>(units + nu) + lane) : 0;
            rpn_ready = false;
        };
        auto load_next_rowptr = [&]() {  // once the entry has landed: the next unit's row pointers
            ss_load_rowptr(static_cast<const int *>(ptr(8)), field(6), field(2), rpn);
            rpn_ready = true;
        };
        fetch_next();
        int c = 0;
        bool ok = aligned;
        for (; ok; c++) {
            if (c >= S && !mbar_wait(empty0 + 8 * (c % S), (unsigned)(c / S - 1) & 1u, wait_limit)) {
                ok = false;
                break;
            }
            if (ck == cK && nu < nunits) {  // start the next unit
                if (!rpn_ready) load_next_rowptr();
                cm = field(0);
                cx0 = field(1);
                cys = field(2);
                cye = field(3);
                cpr = field(4);
                cnx = field(5);
                cny = field(6);
                crp = static_cast<const int *>(ptr(8));
                cev = static_cast<const Event *>(ptr(10));
#pragma unroll
                for (int j = 0; j < 3; j++) rpc[j] = rpn[j];
                cK = (cye - cys + 2 + TBY - 1) / TBY;
                ck = 0;
                fetch_next();
            } else if (!rpn_ready && nu < nunits) {
                load_next_rowptr();
            }
            int4 d0 = make_int4(0, 0, 0, 0), d1 = make_int4(0, 0, 0, 0);
            if (ck < cK) {
                const int s = cys - 1 + ck * TBY;
                d0 = make_int4(cx0, cys, cye, ck | 1 << 24);
                if (lane < NA) {  // the member's arguments beside the descriptor (tracked by the stage's mbarrier)
                    tb_cpa16(reinterpret_cast<float *>(sargs + c % DS) + 4 * lane,
                             reinterpret_cast<const float *>(args + 2 * cm) + 4 * lane);
                    asm volatile("cp.async.mbarrier.arrive.shared::cta.b64 [%0];\n" ::"r"(full0 + 8 * (c % S))
                                 : "memory");
                }
                __syncwarp();  // the copies' arrivals before lane 0's
                d0.w |= ss_stage_chunk<TBY>(rpc, cev, crp != nullptr, cny, s, ck, &desc[c % DS].ev,
                                            full0 + 8 * (c % S));
                d1 = make_int4(cm, cpr, cnx, cny);
                ck++;
            }
            if (lane == 0) {
                desc[c % DS].d0 = d0;
                desc[c % DS].d1 = d1;
            }
            if (!ss_valid(d0)) {  // end of the stream
                __syncwarp();
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(full0 + 8 * (c % S)) : "memory");
                break;
            }
            // six boxes, one per lane: member column x0 - 4 <-> packed column x0, member row y <-> prow0 + 2 + y
            const unsigned mbar = full0 + 8 * (c % S);
            float *st = sm + (c % S) * Gm::STAGE;
            const int s = cys - 1 + (ck - 1) * TBY, py = cpr + 2 + s;
            if (lane == 0)
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(Gm::TMA_BYTES)
                             : "memory");
            __syncwarp();
            if (lane < 6) {
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                if (lane < 5)
                    tma_load_3d(st + lane * Gm::PL_IN, tmIn, cx0, py + ss_shift(lane), lane, mbar);
                else
                    tma_load_2d(st + 5 * Gm::PL_IN, &tmCL, cx0, py, mbar);
            }
        }
        if (!ok) {  // the consumers stopped (or shared memory is misaligned): flag it, let the copies land (bounded)
            if (lane == 0) atomicExch(&g_ss_timeouts, 1);
            for (int k = c > S ? c - S : 0; k < c; k++)
                mbar_wait(full0 + 8 * (k % S), (unsigned)(k / S) & 1u, kSsDrainNs);
            if (!aligned && lane == 0)  // the consumers wait for an end descriptor in stage 0
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(full0) : "memory");
        }
        __threadfence();  // the queue accesses before the CTA counts itself out
    } else {
        // ---- step t, step t+1 and the ring sites
        const long long t = *t0p + toff;
        float *out = par ? pk.buf[0] : pk.buf[1];  // (a select: an index into the parameter would copy it to the stack)
        for (int p = 0;; p++) {
            const bool ok = mbar_wait(full0 + 8 * (p % S), (unsigned)(p / S) & 1u, wait_limit);
            const int4 da = desc[p % DS].d0;
            const int4 db = desc[(p + DS - 1) % DS].d0, dbm = desc[(p + DS - 1) % DS].d1;
            const bool va = ok && ss_valid(da), vb = p >= 1 && ss_valid(db);
            const SsEvList *ela = (da.w >> 26) & 1 ? &desc[p % DS].ev : nullptr;
            const SsEvList *elb = (db.w >> 26) & 1 ? &desc[(p + DS - 1) % DS].ev : nullptr;
            const float *st = sm + (p % S) * Gm::STAGE;
            const int s = da.y - 1 + (da.w & 0xffff) * TBY;
            if (warp < TBY) {
                if (va) {
                    const StepArgs &am = sargs[p % DS];
                    const int r = s + warp;
                    const bool ev = ss_events(da) && (ela ? ss_list_has_row(ela, warp + 1) : ss_row_events(am, r));
                    if (ev && !ela)
                        ss_step_a<TBY, S, true>(am, st, st, 0, P, da.x, da.y, da.z, r, warp, p * TBY + warp + 1, t,
                                                nullptr);
                    else
                        ss_step_a<TBY, S, false>(am, st, st, 0, P, da.x, da.y, da.z, r, warp, p * TBY + warp + 1, t,
                                                 ev ? ela : nullptr);
                }
            } else if (warp < 2 * TBY) {
                const int w = warp - TBY;
                if (vb) {
                    const int rb = db.y - 2 + (db.w & 0xffff) * TBY + w;
                    if (rb >= db.y && rb < db.z) {
                        const StepArgs &bm = sargs[(p + DS - 1) % DS];
                        const bool ev = ss_events(db) && (elb ? ss_list_has_row(elb, w) : ss_row_events(bm, rb));
                        if (ev && !elb)
                            ss_step_b_packed<TBY, S, true>(bm, P, db.x, rb, (p - 1) * TBY + w, t, out, pk.plane, pk.W,
                                                           dbm.y, dbm.z, dbm.w, nullptr, w);
                        else
                            ss_step_b_packed<TBY, S, false>(bm, P, db.x, rb, (p - 1) * TBY + w, t, out, pk.plane, pk.W,
                                                            dbm.y, dbm.z, dbm.w, ev ? elb : nullptr, w);
                    }
                }
            } else if (va) {
                ss_ring<TBY, S>(sargs[p % DS], st, st, 0, P, da.x, s, p, ss_events(da), t, ela);
            }
            if (va && (warp < TBY || warp == 2 * TBY)) {  // this warp has read the stage: release it to the producer
                __syncwarp();
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(empty0 + 8 * (p % S)) : "memory");
            }
            if (ss_consumers_or(!ok, NC * 32)) {  // a chunk never arrived: flag it and stop (the producer drains)
                if (tid == 0) atomicExch(&g_ss_timeouts, 1);
                break;
            }
            if (!ss_valid(da)) break;
        }
    }
    __syncthreads();
    if (tid == 0 && atomicAdd(sched + 1, 1) == (int)gridDim.x - 1) {
        sched[0] = 0;
        sched[1] = 0;
    }
}

// Tensor maps of the packed buffers ([5][rows][W] floats, box: one plane of TBY rows of SW) and of the packed c_L^2.
static bool ss_batch_maps(const BatchPacked &pk, long long rows, int tby, CUtensorMap *mA, CUtensorMap *mB,
                          CUtensorMap *mCL) {
    EncodeTiled fn = encode_fn();
    if (!fn || pk.W < SW) return false;
    const cuuint64_t dims3[3] = {(cuuint64_t)pk.W, (cuuint64_t)rows, 5};
    const cuuint64_t str3[2] = {(cuuint64_t)pk.W * 4, (cuuint64_t)pk.plane * 4};
    const cuuint32_t box3[3] = {(cuuint32_t)SW, (cuuint32_t)tby, 1};
    const cuuint32_t one[3] = {1, 1, 1};
    for (int b = 0; b < 2; b++)
        if (fn(b ? mB : mA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, pk.buf[b], dims3, str3, box3, one,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    const cuuint64_t dims2[2] = {(cuuint64_t)pk.W, (cuuint64_t)rows};
    const cuuint64_t str2[1] = {(cuuint64_t)pk.W * 4};
    const cuuint32_t box2[2] = {(cuuint32_t)SW, (cuuint32_t)tby};
    return fn(mCL, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, pk.cl, dims2, str2, box2, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int TBY, int S, int MINB>
static cudaError_t launch_bss(const StepArgs *args, const BatchUnit *units, int nunits, int *sched,
                              const long long *t0p, int toff, int par, const BatchPacked &pk, long long rows,
                              cudaStream_t s) {
    using Gm = SsGeom<TBY, S, true>;
    constexpr int NT = (2 * TBY + 2) * 32;
    static int per_sm = 0, nsm = 0;
    if (!per_sm) {
        cudaError_t e = cudaFuncSetAttribute(step2d_batch_ss2<TBY, S, MINB>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Gm::BYTES);
        if (e != cudaSuccess) return e;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step2d_batch_ss2<TBY, S, MINB>, NT, Gm::BYTES);
        if (per_sm < 1) per_sm = 1;
    }
    CUtensorMap mA, mB, mCL;
    memset(&mA, 0, sizeof mA);
    memset(&mB, 0, sizeof mB);
    memset(&mCL, 0, sizeof mCL);
    if (!ss_batch_maps(pk, rows, TBY, &mA, &mB, &mCL)) return cudaErrorNotSupported;
    const long long slots = (long long)per_sm * nsm;
    const int blocks = (int)(nunits < slots ? nunits : slots);
    if (blocks < 1) return cudaSuccess;
    step2d_batch_ss2<TBY, S, MINB>
        <<<blocks, NT, Gm::BYTES, s>>>(args, units, nunits, sched, t0p, toff, par, pk, mA, mB, mCL);
    return cudaGetLastError();
}

// Shapes of the batch's strip kernel (chunk rows, stages, CTAs per SM, chunks per unit).  Shape 0's units are 30 rows
// (8 chunks): with 256 media of 64-512 rows, taller units lengthened the tail (on 256 media: 16 chunks 184.5k Mlups,
// 8 chunks 192.3k, 32 chunks 140k).
int batch_ss2_nshapes() { return 2; }
int batch_ss2_rows(int shape) { return shape == 1 ? 3 : 4; }
int batch_ss2_chunks(int shape) { return shape == 1 ? 12 : 8; }

cudaError_t launch_batch_ss2(const StepArgs *args, const BatchUnit *units, int nunits, int *sched, const long long *t0p,
                             int toff, int par, const BatchPacked &pk, long long rows, int shape, cudaStream_t s) {
    if (shape == 1) return launch_bss<3, 4, 3>(args, units, nunits, sched, t0p, toff, par, pk, rows, s);
    return launch_bss<4, 3, 3>(args, units, nunits, sched, t0p, toff, par, pk, rows, s);
}

// An anisotropic medium (uniform tensor, no pole): the strip kernel with the general kernel's site update, chunk
// rows, stages, CTAs per SM and chunks per unit of shape 1.
cudaError_t launch_step_2d_ss2_an(const StepArgs &a, cudaStream_t s) { return launch_ss<4, 3, 3, 12, true>(a, s); }

// A heterogeneous permeability: the strip kernel with the d_x ln mu, d_y ln mu planes staged beside c_L^2 (and kept
// with it for step t+1), 4-row chunks, 3 stages, 2 CTAs per SM (96 KB), 16 chunks per unit (12: 1.4 % slower).
cudaError_t launch_step_2d_ss2_mu(const StepArgs &a, cudaStream_t s) {
    return launch_ss<4, 3, 2, 16, false, true>(a, s);
}

cudaError_t ss_set_wait_limit(unsigned long long ns) {
    return cudaMemcpyToSymbol(g_ss_wait_limit_ns, &ns, sizeof ns);
}

bool ss2_take_timeouts() {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_ss_timeouts, sizeof v) != cudaSuccess) return false;
    if (v) {
        const int z = 0;
        cudaMemcpyToSymbol(g_ss_timeouts, &z, sizeof z);
    }
    return v != 0;
}

}  // namespace lbk
