// Two time steps per launch by streaming rows through registers (2D, FP32 storage, uniform mu).
//
// A warp owns a strip of 128 columns (x0 .. x0+127, 4 per lane) and a segment of rows y0 .. y0+H-1.  It walks
// down the rows keeping in registers what the next updates pull: for row a it computes step t (Eqs. 17-18,
// the site update of the single-step kernels) and then step t+1 for row a-1, whose pulls are then all
// available: the populations of step t at rows a-2 (g2), a-1 (g0, g1, g3 and their x-neighbours) and a (g4).
// The x-neighbours come from the adjacent lanes by warp shuffles; the columns just outside the strip
// (x0-1, x0+128) are one extra site of step t computed by lanes 0 and 31 (the ring), whose own inputs lanes 0
// and 31 load beside their quads.  Every lane's columns are taken modulo nx (periodic), so a strip that runs
// past the last column computes the wrapped sites again: that provides the ring of the last columns and makes
// ragged and tiny grids need no special case; only sites x < nx are recorded by receivers, and stores go to
// x < pitch (duplicates land in the row padding).
//
// HBM traffic per two site updates: 24 bytes read and 20 written (rows at the segment edges are read twice,
// mostly from L2), against 88 for two single steps.  Loads are staged through a small per-warp shared-memory
// ring (cp.async, three rows deep; each lane reads back only what it copied) and there are no block-level
// barriers.  The site updates are collide2d / collide2d_free, so the results are bit-identical to two single
// steps.
#include "lbem_internal.cuh"

namespace lbk {

// Per-warp staging of the inputs of step t at one row a (cp.async; each lane copies and later reads back only
// its own slots, so no synchronisation between lanes is needed):
//   q[0..5][lane] = planes 0, 1, 3, c_L^2 at row a, plane 2 at row a-1, plane 4 at row a+1 (4 sites per lane)
//   e[0][0..5]    = lane 0's ring inputs:  IN0[a][xl], IN1[a][xl], IN1[a][xll], IN2[a-1][xl], IN4[a+1][xl], CL[a][xl]
//   e[1][0..5]    = lane 31's ring inputs: IN0[a][xr], IN2[a-1][xr], IN3[a][xr], IN3[a][xrr], IN4[a+1][xr], CL[a][xr]
// with xl = x0-1, xll = x0-2, xr = x0+128, xrr = x0+129.
struct RsStage {
    float4 q[6][32];
    float e[2][8];
};
constexpr int RS_NS = 3;  // stages per warp: rows a, a+1, a+2 in flight

struct RsLane {
    int x;        // first column of the lane (unwrapped)
    bool direct;  // the 4 columns are x .. x+3 < nx (one 16-byte copy)
    int xa, xb;   // lane 0: x0-1, x0-2; lane 31: x0+128, x0+129 (wrapped)
};

__device__ __forceinline__ void rs_cp16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src));
}
__device__ __forceinline__ void rs_cp4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src));
}

__device__ __forceinline__ void rs_quad(float4 *dst, const float *base, const RsLane &L, int nx) {
    if (L.direct) {
        rs_cp16(dst, base + L.x);
    } else {
        float *d = reinterpret_cast<float *>(dst);
#pragma unroll
        for (int k = 0; k < 4; k++) rs_cp4(d + k, base + wrapi(L.x + k, nx));
    }
}

// Issue the copies of row `row`'s inputs into stage S (one commit group per call).
__device__ __forceinline__ void rs_issue(const StepArgs &a, const RsLane &L, int lane, int row, RsStage &S) {
    const Grid &G = a.g;
    const float *in = static_cast<const float *>(a.in.data);
    const long long ra = (long long)wrapi(row, G.ny) * G.pitch;
    const long long rm = (long long)wrapi(row - 1, G.ny) * G.pitch;
    const long long rp = (long long)wrapi(row + 1, G.ny) * G.pitch;
    const float *P0 = in, *P1 = in + G.plane, *P2 = in + 2 * G.plane, *P3 = in + 3 * G.plane, *P4 = in + 4 * G.plane;
    rs_quad(&S.q[0][lane], P0 + ra, L, G.nx);
    rs_quad(&S.q[1][lane], P1 + ra, L, G.nx);
    rs_quad(&S.q[2][lane], P3 + ra, L, G.nx);
    rs_quad(&S.q[3][lane], a.med.cL2 + ra, L, G.nx);
    rs_quad(&S.q[4][lane], P2 + rm, L, G.nx);
    rs_quad(&S.q[5][lane], P4 + rp, L, G.nx);
    if (lane == 0) {
        rs_cp4(&S.e[0][0], P0 + ra + L.xa);
        rs_cp4(&S.e[0][1], P1 + ra + L.xa);
        rs_cp4(&S.e[0][2], P1 + ra + L.xb);
        rs_cp4(&S.e[0][3], P2 + rm + L.xa);
        rs_cp4(&S.e[0][4], P4 + rp + L.xa);
        rs_cp4(&S.e[0][5], a.med.cL2 + ra + L.xa);
    } else if (lane == 31) {
        rs_cp4(&S.e[1][0], P0 + ra + L.xa);
        rs_cp4(&S.e[1][1], P2 + rm + L.xa);
        rs_cp4(&S.e[1][2], P3 + ra + L.xa);
        rs_cp4(&S.e[1][3], P3 + ra + L.xb);
        rs_cp4(&S.e[1][4], P4 + rp + L.xa);
        rs_cp4(&S.e[1][5], a.med.cL2 + ra + L.xa);
    }
}

#define RS_COMP(v, k) (k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w)
#define RS_SET(v, k, val) (k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w) = (val)

// Four site updates of one lane at row `row` (unwrapped), time t.
template <bool EV>
__device__ __forceinline__ void rs_update4(const StepArgs &a, const RsLane &L, float4 g0, float4 g1, float4 g2,
                                           float4 g3, float4 g4, float4 cl, int row, long long t, bool owned_row,
                                           float4 &o0, float4 &o1, float4 &o2, float4 &o3, float4 &o4) {
    const Grid &G = a.g;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const float q0 = RS_COMP(g0, k), q1 = RS_COMP(g1, k), q2 = RS_COMP(g2, k), q3 = RS_COMP(g3, k),
                    q4 = RS_COMP(g4, k), ck = RS_COMP(cl, k);
        Out5 o;
        if (EV) {
            const float shat = site_events(a, wrapi(L.x + k, G.nx), wrapi(row, G.ny), t,
                                           owned_row && L.x + k < G.nx, q0, q1, q2, q3, q4, ck);
            o = collide2d(q0, q1, q2, q3, q4, ck, shat);
        } else {
            o = collide2d_free(q0, q1, q2, q3, q4, ck);
        }
        RS_SET(o0, k, o.o0);
        RS_SET(o1, k, o.o1);
        RS_SET(o2, k, o.o2);
        RS_SET(o3, k, o.o3);
        RS_SET(o4, k, o.o4);
    }
}

__device__ __forceinline__ bool rs_row_events(const StepArgs &a, int row) {
    if (!a.evt.rowptr) return false;
    const int r = wrapi(row, a.g.ny);
    return __ldg(a.evt.rowptr + r) != __ldg(a.evt.rowptr + r + 1);
}

template <int MINB>
__global__ void __launch_bounds__(128, MINB) step2d_rs2(StepArgs a, int nstrips, int nseg, int H) {
    __shared__ RsStage stage[4][RS_NS];  // per warp
    const Grid &G = a.g;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int w = blockIdx.x * 4 + wib;
    if (w >= nstrips * nseg) return;  // warp-uniform
    RsStage *st = stage[wib];
    const int sx = w % nstrips, sy = w / nstrips;
    const int x0 = sx * 128, y0 = sy * H;
    const int y1 = min(y0 + H, G.ny);  // output rows y0 .. y1-1
    RsLane L;
    L.x = x0 + 4 * lane;
    L.direct = L.x + 3 < G.nx;
    L.xa = lane == 0 ? wrapi(x0 - 1, G.nx) : wrapi(x0 + 128, G.nx);
    L.xb = lane == 0 ? wrapi(x0 - 2, G.nx) : wrapi(x0 + 129, G.nx);
    const long long t = a.t;
    float *out = static_cast<float *>(a.out.data);
    const bool store_ok = L.x < G.pitch;  // pitch is a multiple of 4: a lane's 4 columns are all in or all out
    const int ei = lane == 0 ? 0 : 1;

    // window of step-t results: plane 2 at rows r-2 and r-1, planes 0, 1, 3 and c_L^2 at row r-1, and the ring
    // value at row r-1 (lane 0: plane 1 at x0-1; lane 31: plane 3 at x0+128)
    float4 w2m = make_float4(0.f, 0.f, 0.f, 0.f), w2 = w2m, w0 = w2m, w1 = w2m, w3 = w2m, wcl = w2m;
    float wr = 0.f;
#pragma unroll
    for (int k = 0; k < RS_NS - 1; k++) {
        if (y0 - 1 + k <= y1) rs_issue(a, L, lane, y0 - 1 + k, st[k]);
        asm volatile("cp.async.commit_group;\n" ::);
    }
    int si = 0;  // stage of the current row
    for (int row = y0 - 1; row <= y1; row++) {  // step t at `row`, step t+1 at row-1
        // the copies of row+RS_NS-1 go into the stage freed by the previous row
        const int sn = si == 0 ? RS_NS - 1 : si - 1;
        if (row + RS_NS - 1 <= y1) rs_issue(a, L, lane, row + RS_NS - 1, st[sn]);
        asm volatile("cp.async.commit_group;\n" ::);
        asm volatile("cp.async.wait_group %0;\n" ::"n"(RS_NS - 1));  // this lane's copies of `row` have landed
        const RsStage &S = st[si];
        const float4 p0 = S.q[0][lane], p1 = S.q[1][lane], p3 = S.q[2][lane], cl = S.q[3][lane];
        const float4 p2 = S.q[4][lane], p4 = S.q[5][lane];
        // ---- step t, row `row`
        float up = __shfl_up_sync(FULL, p1.w, 1);
        float dn = __shfl_down_sync(FULL, p3.x, 1);
        if (lane == 0) up = S.e[0][1];
        if (lane == 31) dn = S.e[1][2];
        const float4 g1 = make_float4(up, p1.x, p1.y, p1.z);
        const float4 g3 = make_float4(p3.y, p3.z, p3.w, dn);
        const bool ev_a = rs_row_events(a, row);
        const bool own_a = row >= y0 && row < y1;
        float4 o0, o1, o2, o3, o4;
        if (ev_a)
            rs_update4<true>(a, L, p0, g1, p2, g3, p4, cl, row, t, own_a, o0, o1, o2, o3, o4);
        else
            rs_update4<false>(a, L, p0, g1, p2, g3, p4, cl, row, t, own_a, o0, o1, o2, o3, o4);
        // ring site of step t: lane 0 at x0-1 (keeps plane 1), lane 31 at x0+128 (keeps plane 3)
        float ring = 0.f;
        if (lane == 0 || lane == 31) {
            const float *e = S.e[ei];
            const float r1 = lane == 0 ? e[2] : p1.w;
            const float r2 = lane == 0 ? e[3] : e[1];
            const float r3 = lane == 0 ? p3.x : e[3];
            Out5 o;
            if (ev_a) {
                const float shat = site_events(a, L.xa, wrapi(row, G.ny), t, false, e[0], r1, r2, r3, e[4], e[5]);
                o = collide2d(e[0], r1, r2, r3, e[4], e[5], shat);
            } else {
                o = collide2d_free(e[0], r1, r2, r3, e[4], e[5]);
            }
            ring = lane == 0 ? o.o1 : o.o3;
        }
        // ---- step t+1, row `row` - 1 (an output row from y0 on)
        if (row - 1 >= y0) {
            const int b = row - 1;
            float bu = __shfl_up_sync(FULL, w1.w, 1);
            float bd = __shfl_down_sync(FULL, w3.x, 1);
            if (lane == 0) bu = wr;
            if (lane == 31) bd = wr;
            const float4 h1 = make_float4(bu, w1.x, w1.y, w1.z);
            const float4 h3 = make_float4(w3.y, w3.z, w3.w, bd);
            float4 q0, q1, q2, q3, q4;
            if (rs_row_events(a, b))
                rs_update4<true>(a, L, w0, h1, w2m, h3, o4, wcl, b, t + 1, true, q0, q1, q2, q3, q4);
            else
                rs_update4<false>(a, L, w0, h1, w2m, h3, o4, wcl, b, t + 1, true, q0, q1, q2, q3, q4);
            if (store_ok) {
                float4 *o = reinterpret_cast<float4 *>(out + (long long)b * G.pitch + L.x);
                const long long pl4 = G.plane / 4;
                __stcs(o, q0);
                __stcs(o + pl4, q1);
                __stcs(o + 2 * pl4, q2);
                __stcs(o + 3 * pl4, q3);
                __stcs(o + 4 * pl4, q4);
            }
        }
        // ---- shift the window
        w2m = w2;
        w2 = o2;
        w0 = o0;
        w1 = o1;
        w3 = o3;
        wr = ring;
        wcl = cl;
        si = si == RS_NS - 1 ? 0 : si + 1;
    }
    asm volatile("cp.async.wait_group 0;\n" ::);
}
#undef RS_COMP
#undef RS_SET

template <int MINB>
static cudaError_t launch_rs(const StepArgs &a, cudaStream_t s) {
    static int per_sm = 0, nsm = 0;
    if (!per_sm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step2d_rs2<MINB>, 128, 0);
        if (per_sm < 1) per_sm = 1;
    }
    const int nstrips = (a.g.nx + 127) / 128;
    // one wave: about as many (strip, segment) warps as fit on the GPU at once, segments of at least 8 rows
    const long long resident = (long long)per_sm * nsm * 4;
    int nseg = (int)(resident / nstrips);
    if (nseg < 1) nseg = 1;
    int H = (a.g.ny + nseg - 1) / nseg;
    if (H < 8) H = 8;
    nseg = (a.g.ny + H - 1) / H;
    const long long warps = (long long)nstrips * nseg;
    step2d_rs2<MINB><<<(unsigned)((warps + 3) / 4), 128, 0, s>>>(a, nstrips, nseg, H);
    return cudaGetLastError();
}

// 90 registers at five blocks of four warps per SM (4096^2: 245k Mlups, level with the tile kernel); four blocks
// leave 106 registers.  Six blocks would spill.
int rs2_nshapes() { return 2; }

cudaError_t launch_step_2d_rs2(const StepArgs &a, int shape, cudaStream_t s) {
    if (shape == 1) return launch_rs<4>(a, s);
    return launch_rs<5>(a, s);
}

}  // namespace lbk
