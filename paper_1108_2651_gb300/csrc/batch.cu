// Batched stepping of many independent 2D FP32 media of uneven sizes: one
// kernel launch per step covers every member through a flattened table of
// warps (each warp = 128 sites of one row of one member, R rows per warp for
// the variant R), and runs of steps are captured once into a CUDA graph.
//
// Per call, a small table of member descriptors (buffers, medium, events,
// grid) is uploaded, and the start time t0 is written to device memory; the
// captured launches read t0 and carry only their step offset and the
// ping-pong parity, so one graph serves every call with the same number of
// steps and the same members.
#include <algorithm>
#include <vector>

#include "lbem_internal.cuh"

namespace lbk {

struct Member {
    Grid g;
    PopBuf a, b;  // a = buffer holding the state at the call's start
    Medium med;
    Events evt;
};

// Same site update as step2d<F32, mu = false, R> (kernels2d.cu), with the grid,
// buffers and events taken from the member this warp belongs to.
__device__ __forceinline__ void pull_f32(const PopBuf &in, const Grid &G, int row, int c, int lane, float4 g[5]) {
    using C = Codec<LBEM_F32>;
    const int x0 = 4 * c;
    const bool active = c < G.nchunk;
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
    if (c == G.nchunk - 1) set(g[3], G.nx - 1 - x0, C::load1(in, 3, row, 0));
}

template <int R, int MINB = 1>
__global__ void __launch_bounds__(BLOCK, MINB) step2d_batch(const Member *__restrict__ M, const long long *__restrict__ wstart,
                                                      const int *__restrict__ wmember, long long nwarps,
                                                      const long long *__restrict__ t0p, int offset) {
    using C = Codec<LBEM_F32>;
    const int lane = threadIdx.x & 31;
    const long long wg = ((long long)blockIdx.x * BLOCK + threadIdx.x) >> 5;
    if (wg >= nwarps) return;
    const int lo = __ldg(wmember + wg);  // member of this warp
    const Member &m = M[lo];
    const Grid &G = m.g;
    const long long lw = wg - wstart[lo];
    const int wpr = G.nchunk_pad >> 5;
    const int rg = (int)(lw / wpr);
    const int c = (int)(lw - (long long)rg * wpr) * 32 + lane;
    const int row0 = rg * R;
    if (row0 >= G.ny) return;
    const bool active = c < G.nchunk;
    const PopBuf &in = (offset & 1) ? m.b : m.a;
    const PopBuf &out = (offset & 1) ? m.a : m.b;
    const long long t = *t0p + offset;
    float4 g[R][5], cl[R];
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int row = min(row0 + r, G.ny - 1);
        pull_f32(in, G, row, c, lane, g[r]);
        cl[r] = active ? __ldg(reinterpret_cast<const float4 *>(m.med.cL2 + (long long)row * G.pitch) + c)
                       : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int row = row0 + r;
        if (row >= G.ny) break;
        float4 shat = make_float4(0.f, 0.f, 0.f, 0.f);
        if (m.evt.rowptr) {
            const int e0 = __ldg(m.evt.rowptr + row), e1 = __ldg(m.evt.rowptr + row + 1);
            for (int e = e0; e < e1; e++) {
                const Event ev = m.evt.ev[e];
                if ((ev.x >> 2) != c || !active) continue;
                const int j = ev.x & 3;
                if (ev.kind == 0) {
                    if (ev.comp == 2 && t < m.evt.nt)
                        set(shat, j, get(shat, j) - __ldg(m.evt.amp + (long long)ev.index * m.evt.nt + t));
                } else if (t < m.evt.cap) {
                    const float s = ((get(g[r][0], j) + get(g[r][1], j)) + (get(g[r][2], j) + get(g[r][3], j))) +
                                    get(g[r][4], j);
                    const float bx = get(g[r][4], j) - get(g[r][2], j), by = get(g[r][1], j) - get(g[r][3], j);
                    float v = 0.f;
                    if (ev.comp == 2) v = -get(cl[r], j) * s;
                    else if (ev.comp == 3) v = bx;
                    else if (ev.comp == 4) v = by;
                    m.evt.traces[(long long)ev.index * m.evt.cap + t] = v;
                }
            }
        }
        float4 o[5];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const float g0 = get(g[r][0], j), g1 = get(g[r][1], j), g2 = get(g[r][2], j), g3 = get(g[r][3], j),
                        g4 = get(g[r][4], j), q = get(cl[r], j), sh = get(shat, j);
            const Out5 u = collide2d(g0, g1, g2, g3, g4, q, sh);
            set(o[0], j, u.o0);
            set(o[1], j, u.o1);
            set(o[2], j, u.o2);
            set(o[3], j, u.o3);
            set(o[4], j, u.o4);
        }
        if (active)
            for (int i = 0; i < 5; i++) C::store4(out, i, row, c, o[i]);
    }
}

// Flattened mapping: one site per thread, sites of a member numbered x + nx*y
// and cut into blocks of BLOCK consecutive sites (a block never spans two
// members), so no lane idles except in a member's last block.
__global__ void __launch_bounds__(BLOCK) step2d_batch_site(const Member *__restrict__ M, const int *__restrict__ bmember,
                                                           const long long *__restrict__ bstart,
                                                           const long long *__restrict__ t0p, int offset) {
    const int mi = __ldg(bmember + blockIdx.x);
    const Member &m = M[mi];
    const Grid &G = m.g;
    const long long s = (long long)(blockIdx.x - bstart[mi]) * BLOCK + threadIdx.x;
    if (s >= (long long)G.nx * G.ny) return;
    const int row = (int)(s / G.nx), x = (int)(s - (long long)row * G.nx);
    const int xm = x == 0 ? G.nx - 1 : x - 1, xp = x == G.nx - 1 ? 0 : x + 1;
    const int ym = row == 0 ? G.ny - 1 : row - 1, yp = row == G.ny - 1 ? 0 : row + 1;
    const PopBuf &in = (offset & 1) ? m.b : m.a;
    const PopBuf &out = (offset & 1) ? m.a : m.b;
    const float *ip = static_cast<const float *>(in.data);
    const long long P = G.plane, W = G.pitch;
    const float g0 = __ldg(ip + (long long)row * W + x);
    const float g1 = __ldg(ip + P + (long long)row * W + xm);
    const float g2 = __ldg(ip + 2 * P + (long long)ym * W + x);
    const float g3 = __ldg(ip + 3 * P + (long long)row * W + xp);
    const float g4 = __ldg(ip + 4 * P + (long long)yp * W + x);
    const float q = __ldg(m.med.cL2 + (long long)row * W + x);
    const long long t = *t0p + offset;
    float sh = 0.f;
    if (m.evt.rowptr) {
        const int e0 = __ldg(m.evt.rowptr + row), e1 = __ldg(m.evt.rowptr + row + 1);
        for (int e = e0; e < e1; e++) {
            const Event ev = m.evt.ev[e];
            if (ev.x != x) continue;
            if (ev.kind == 0) {
                if (ev.comp == 2 && t < m.evt.nt) sh -= __ldg(m.evt.amp + (long long)ev.index * m.evt.nt + t);
            } else if (t < m.evt.cap) {
                const float sg = ((g0 + g1) + (g2 + g3)) + g4;
                float v = 0.f;
                if (ev.comp == 2) v = -q * sg;
                else if (ev.comp == 3) v = g4 - g2;
                else if (ev.comp == 4) v = g1 - g3;
                m.evt.traces[(long long)ev.index * m.evt.cap + t] = v;
            }
        }
    }
    const Out5 u = collide2d(g0, g1, g2, g3, g4, q, sh);
    float *op = static_cast<float *>(out.data) + (long long)row * W + x;
    __stcs(op, u.o0);
    __stcs(op + P, u.o1);
    __stcs(op + 2 * P, u.o2);
    __stcs(op + 3 * P, u.o3);
    __stcs(op + 4 * P, u.o4);
}

// Linear mapping over the padded plane: lane L of a member covers 4 sites at
// row = L / (pitch/4), chunk c = L % (pitch/4); warps may span row ends, so only
// the pitch padding idles lanes.  A lane at a row start or end takes its +-x
// neighbour from the periodic wrap, a lane at a warp edge by a scalar load, any
// other lane by shuffle from its neighbour (which is then in the same row).
template <int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) step2d_batch_lin(const Member *__restrict__ M,
                                                                const long long *__restrict__ wstart,
                                                                const int *__restrict__ wmember, long long nwarps,
                                                                const long long *__restrict__ t0p, int offset) {
    using C = Codec<LBEM_F32>;
    const int lane = threadIdx.x & 31;
    const long long wg = ((long long)blockIdx.x * BLOCK + threadIdx.x) >> 5;
    if (wg >= nwarps) return;
    const int mi = __ldg(wmember + wg);
    const Member &m = M[mi];
    const Grid &G = m.g;
    const int cpr = G.pitch >> 2;  // chunks per padded row
    const long long L = (wg - wstart[mi]) * 32 + lane;
    const int row = (int)(L / cpr);
    const int c = (int)(L - (long long)row * cpr);
    const bool inrow = row < G.ny;
    const bool active = inrow && c < G.nchunk;
    const int rr = inrow ? row : G.ny - 1;
    const PopBuf &in = (offset & 1) ? m.b : m.a;
    const PopBuf &out = (offset & 1) ? m.a : m.b;
    const long long t = *t0p + offset;
    const int x0 = 4 * c;
    const int ym = rr == 0 ? G.ny - 1 : rr - 1, yp = rr == G.ny - 1 ? 0 : rr + 1;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 g[5];
    g[0] = active ? C::load4(in, 0, rr, c) : z4;
    float4 a1 = active ? C::load4(in, 1, rr, c) : z4;
    g[2] = active ? C::load4(in, 2, ym, c) : z4;
    float4 a3 = active ? C::load4(in, 3, rr, c) : z4;
    g[4] = active ? C::load4(in, 4, yp, c) : z4;
    const float4 cl = active ? __ldg(reinterpret_cast<const float4 *>(m.med.cL2 + (long long)rr * G.pitch) + c) : z4;
    float prev = __shfl_up_sync(FULL, a1.w, 1);
    float next = __shfl_down_sync(FULL, a3.x, 1);
    if (active && (lane == 0 || c == 0)) prev = C::load1(in, 1, rr, c == 0 ? G.nx - 1 : x0 - 1);
    if (active && lane == 31 && x0 + 4 < G.nx) next = C::load1(in, 3, rr, x0 + 4);
    if (!active) return;
    g[1] = make_float4(prev, a1.x, a1.y, a1.z);
    g[3] = make_float4(a3.y, a3.z, a3.w, next);
    if (c == G.nchunk - 1) set(g[3], G.nx - 1 - x0, C::load1(in, 3, rr, 0));
    float4 shat = z4;
    if (m.evt.rowptr) {
        const int e0 = __ldg(m.evt.rowptr + rr), e1 = __ldg(m.evt.rowptr + rr + 1);
        for (int e = e0; e < e1; e++) {
            const Event ev = m.evt.ev[e];
            if ((ev.x >> 2) != c) continue;
            const int j = ev.x & 3;
            if (ev.kind == 0) {
                if (ev.comp == 2 && t < m.evt.nt)
                    set(shat, j, get(shat, j) - __ldg(m.evt.amp + (long long)ev.index * m.evt.nt + t));
            } else if (t < m.evt.cap) {
                const float s = ((get(g[0], j) + get(g[1], j)) + (get(g[2], j) + get(g[3], j))) + get(g[4], j);
                const float bx = get(g[4], j) - get(g[2], j), by = get(g[1], j) - get(g[3], j);
                float v = 0.f;
                if (ev.comp == 2) v = -get(cl, j) * s;
                else if (ev.comp == 3) v = bx;
                else if (ev.comp == 4) v = by;
                m.evt.traces[(long long)ev.index * m.evt.cap + t] = v;
            }
        }
    }
    float4 o[5];
    // rows without a source have S^ = +0 everywhere: collide2d_free gives the same bits
    if (m.evt.rowptr && __ldg(m.evt.rowptr + rr) != __ldg(m.evt.rowptr + rr + 1)) {
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const Out5 u = collide2d(get(g[0], j), get(g[1], j), get(g[2], j), get(g[3], j), get(g[4], j),
                                     get(cl, j), get(shat, j));
            set(o[0], j, u.o0);
            set(o[1], j, u.o1);
            set(o[2], j, u.o2);
            set(o[3], j, u.o3);
            set(o[4], j, u.o4);
        }
    } else {
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const Out5 u = collide2d_free(get(g[0], j), get(g[1], j), get(g[2], j), get(g[3], j), get(g[4], j),
                                          get(cl, j));
            set(o[0], j, u.o0);
            set(o[1], j, u.o1);
            set(o[2], j, u.o2);
            set(o[3], j, u.o3);
            set(o[4], j, u.o4);
        }
    }
    for (int i = 0; i < 5; i++) C::store4(out, i, rr, c, o[i]);
}

// Persistent row mapping: warp w walks the contiguous units [w*k, (w+1)*k) of the
// flattened table (nearly always one member), keeps that member's descriptor in
// registers, and issues the loads of its next unit before it computes the current one.
struct RawB {
    float4 v0, a1, v2, a3, v4, cl;
    float s1, s3, sw;
};

__device__ __forceinline__ void batch_raw(const Member &m, const PopBuf &in, int row, int c, int lane, RawB &r) {
    using C = Codec<LBEM_F32>;
    const Grid &G = m.g;
    const bool active = c < G.nchunk;
    const int x0 = 4 * c;
    const int ym = row == 0 ? G.ny - 1 : row - 1, yp = row == G.ny - 1 ? 0 : row + 1;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    r.v0 = active ? C::load4(in, 0, row, c) : z4;
    r.a1 = active ? C::load4(in, 1, row, c) : z4;
    r.v2 = active ? C::load4(in, 2, ym, c) : z4;
    r.a3 = active ? C::load4(in, 3, row, c) : z4;
    r.v4 = active ? C::load4(in, 4, yp, c) : z4;
    r.cl = active ? __ldg(reinterpret_cast<const float4 *>(m.med.cL2 + (long long)row * G.pitch) + c) : z4;
    r.s1 = (lane == 0 && active) ? C::load1(in, 1, row, c == 0 ? G.nx - 1 : x0 - 1) : 0.f;
    r.s3 = (lane == 31 && x0 + 4 < G.nx) ? C::load1(in, 3, row, x0 + 4) : 0.f;
    r.sw = (c == G.nchunk - 1) ? C::load1(in, 3, row, 0) : 0.f;
}

__global__ void __launch_bounds__(BLOCK) step2d_batch_pipe(const Member *__restrict__ M, const long long *__restrict__ wstart,
                                                           const int *__restrict__ wmember, long long nunits,
                                                           long long per_warp, const long long *__restrict__ t0p,
                                                           int offset) {
    using C = Codec<LBEM_F32>;
    const int lane = threadIdx.x & 31;
    const long long w = ((long long)blockIdx.x * BLOCK + threadIdx.x) >> 5;
    long long u = w * per_warp;
    const long long uend = min(nunits, u + per_warp);
    if (u >= uend) return;  // warp-uniform
    const long long t = *t0p + offset;
    int mi = __ldg(wmember + u);
    const Member *mp = M + mi;
    long long ubase = __ldg(wstart + mi);
    auto rc = [&](const Member &mm, long long uu, long long base, int &row, int &c) {
        const int wpr = mm.g.nchunk_pad >> 5;
        const long long lu = uu - base;
        row = (int)(lu / wpr);
        c = (int)(lu - (long long)row * wpr) * 32 + lane;
    };
    int row, c;
    rc(*mp, u, ubase, row, c);
    RawB cur;
    batch_raw(*mp, (offset & 1) ? mp->b : mp->a, row, c, lane, cur);
    while (true) {
        const long long un = u + 1;
        const bool more = un < uend;
        int nmi = mi, nrow = 0, nc = 0;
        const Member *nmp = mp;
        long long nbase = ubase;
        RawB nxt;
        if (more) {
            nmi = __ldg(wmember + un);
            if (nmi != mi) {  // warp-uniform: the next unit starts a new member
                nmp = M + nmi;
                nbase = __ldg(wstart + nmi);
            }
            rc(*nmp, un, nbase, nrow, nc);
            batch_raw(*nmp, (offset & 1) ? nmp->b : nmp->a, nrow, nc, lane, nxt);
        }
        const Member &m = *mp;
        const Grid &G = m.g;
        const bool active = c < G.nchunk;
        const int x0 = 4 * c;
        float prev = __shfl_up_sync(FULL, cur.a1.w, 1);
        float next = __shfl_down_sync(FULL, cur.a3.x, 1);
        if (lane == 0) prev = cur.s1;
        if (lane == 31 && x0 + 4 < G.nx) next = cur.s3;
        float4 g[5];
        g[0] = cur.v0;
        g[1] = make_float4(prev, cur.a1.x, cur.a1.y, cur.a1.z);
        g[2] = cur.v2;
        g[3] = make_float4(cur.a3.y, cur.a3.z, cur.a3.w, next);
        g[4] = cur.v4;
        if (c == G.nchunk - 1) set(g[3], G.nx - 1 - x0, cur.sw);
        float4 shat = make_float4(0.f, 0.f, 0.f, 0.f);
        if (m.evt.rowptr) {
            const int e0 = __ldg(m.evt.rowptr + row), e1 = __ldg(m.evt.rowptr + row + 1);
            for (int e = e0; e < e1; e++) {
                const Event ev = m.evt.ev[e];
                if ((ev.x >> 2) != c || !active) continue;
                const int j = ev.x & 3;
                if (ev.kind == 0) {
                    if (ev.comp == 2 && t < m.evt.nt)
                        set(shat, j, get(shat, j) - __ldg(m.evt.amp + (long long)ev.index * m.evt.nt + t));
                } else if (t < m.evt.cap) {
                    const float s = ((get(g[0], j) + get(g[1], j)) + (get(g[2], j) + get(g[3], j))) + get(g[4], j);
                    const float bx = get(g[4], j) - get(g[2], j), by = get(g[1], j) - get(g[3], j);
                    float v = 0.f;
                    if (ev.comp == 2) v = -get(cur.cl, j) * s;
                    else if (ev.comp == 3) v = bx;
                    else if (ev.comp == 4) v = by;
                    m.evt.traces[(long long)ev.index * m.evt.cap + t] = v;
                }
            }
        }
        float4 o[5];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const float g0 = get(g[0], j), g1 = get(g[1], j), g2 = get(g[2], j), g3 = get(g[3], j), g4 = get(g[4], j),
                        q = get(cur.cl, j), sh = get(shat, j);
            const Out5 u = collide2d(g0, g1, g2, g3, g4, q, sh);
            set(o[0], j, u.o0);
            set(o[1], j, u.o1);
            set(o[2], j, u.o2);
            set(o[3], j, u.o3);
            set(o[4], j, u.o4);
        }
        if (active) {
            const PopBuf &out = (offset & 1) ? m.a : m.b;
            for (int i = 0; i < 5; i++) C::store4(out, i, row, c, o[i]);
        }
        if (!more) break;
        u = un;
        mp = nmp;
        mi = nmi;
        ubase = nbase;
        row = nrow;
        c = nc;
        cur = nxt;
    }
}

}  // namespace lbk

struct lbem_batch {
    int n = 0;
    std::vector<lbem_t *> members;
    cudaStream_t stream = nullptr;
    lbk::Member *d_members = nullptr;
    long long *d_wstart = nullptr;  // [n + 1] first warp (row variants) or block (site variant) of each member
    int *d_map = nullptr;           // warp -> member (row variants) or block -> member (site variant)
    size_t map_cap = 0;
    long long *d_t0 = nullptr;
    long long total_warps = 0, total_blocks = 0;
    // two steps per launch: per member its step arguments for both buffer parities, a tile -> member table and
    // each member's first tile (tile rows tb_rows)
    lbk::StepArgs *d_args = nullptr;
    lbk::BatchTile *d_tiles = nullptr;
    size_t tiles_cap = 0;
    long long ntiles = 0;
    int tb_rows = 0;
    // the strip kernel's units (sstream.cu) and its work queue (two counters, zero between launches)
    lbk::BatchUnit *d_units = nullptr;
    size_t units_cap = 0;
    int nunits = 0;
    int *d_sched = nullptr;
    // the two-step kernels' packed states with halos: two population buffers and c_L^2, [rows][W] per plane, member m
    // from packed row r0[m] (d_r0, n + 1 entries)
    float *d_pack = nullptr;  // 11 planes: buffer 0 (5), buffer 1 (5), c_L^2 (1)
    size_t pack_bytes = 0;
    int *d_r0 = nullptr;
    int pack_W = 0;
    long long pack_rows = 0;
    lbk::BatchPacked packed() const {
        lbk::BatchPacked k;
        const long long pl = pack_rows * pack_W;
        k.buf[0] = d_pack;
        k.buf[1] = d_pack + 5 * pl;
        k.cl = d_pack + 10 * pl;
        k.r0 = d_r0;
        k.W = pack_W;
        k.plane = pl;
        return k;
    }
    int variant = 0;
    cudaGraphExec_t graph = nullptr;
    int graph_steps = 0, graph_variant = -1;
};

using namespace lbk;

// variants 0..2: row mapping with R = 1, 2, 4 rows per warp; variant 3: flattened one-site-per-thread mapping;
// variant 4: persistent row mapping (R = 1 table) with contiguous unit ranges and prefetch;
// variants 5, 6: R = 1 with registers capped for 5 / 6 resident blocks per SM;
// variants 7, 8: linear mapping over the padded plane (uncapped / capped for 5 blocks per SM)
// Variants: R = 1, 2, 4 rows per warp; 0 one site per thread; -1 persistent register pipeline; -5, -6 R = 1
// capped for 5 / 6 blocks per SM; -7, -8 linear over each member's padded plane (uncapped / 5 blocks per SM);
// 100 + k: two steps per launch through shared-memory tiles, tile shape k (launch_batch_tb2); 200 + k: two steps per
// launch by strip streaming, shape k (launch_batch_ss2).
static const int kRowsB[] = {1, 2, 4, 0, -1, -5, -6, -7, -8, 100, 101, 102, 103, 104, 200, 201};
static const int kBatchVariants = (int)(sizeof(kRowsB) / sizeof(kRowsB[0]));
static const int kLinVariant = 7;  // the single-step kernel that takes the odd step of a two-step variant
static bool two_step(int variant) { return kRowsB[variant] >= 100; }
static bool strip_variant(int variant) { return kRowsB[variant] >= 200; }

static void drop_batch_graph(lbem_batch_t *b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_steps = 0;
    b->graph_variant = -1;
}

// Every member's step arguments for both buffer parities (args[2 k]: state in buffer a, written to b; args[2 k + 1]:
// the reverse) and the packed layout of the two-step kernels: member k from packed row r0[k], its rows and two halo
// rows on either side, rows W floats wide so that every window (member columns x0 - 4 .. x0 + 131 of a 128-column
// tile or strip) lies inside a row.  Uploads the arguments and r0, (re)allocates the packed buffers; r0 to the caller.
static lbem_status upload_packed_layout(lbem_batch_t *b, std::vector<int> &r0) {
    std::vector<StepArgs> args(2 * (size_t)b->n);
    r0.assign(b->n + 1, 0);
    int maxw = 0;
    for (int k = 0; k < b->n; k++) {
        lbem_t *h = b->members[k];
        args[2 * k] = step_args(h, h->cur);
        args[2 * k + 1] = step_args(h, h->cur ^ 1);
        if ((long long)r0[k] + h->grid.ny + 4 > 0x7fffffffLL)
            return fail(LBEM_ERR_ARG, "lbem_batch: members too tall for the packed layout");
        r0[k + 1] = r0[k] + h->grid.ny + 4;
        maxw = std::max(maxw, (h->grid.nx + 127) / 128 * 128);
    }
    const int W = round_up(maxw + 8, 32);
    const long long prows = r0[b->n];
    const size_t need = sizeof(float) * 11 * (size_t)prows * W;
    if (b->pack_bytes < need) {
        drop_batch_graph(b);  // a captured graph may refer to the old buffers
        cudaFree(b->d_pack);
        b->d_pack = nullptr;
        b->pack_bytes = 0;
        if (cudaMalloc((void **)&b->d_pack, need) != cudaSuccess) {
            cudaGetLastError();
            return fail(LBEM_ERR_NOMEM, "lbem_batch: no room for the packed states");
        }
        b->pack_bytes = need;
        LBEM_CUDA(cudaMemsetAsync(b->d_pack, 0, need, b->stream));
    }
    b->pack_W = W;
    b->pack_rows = prows;
    LBEM_CUDA(cudaMemcpyAsync(b->d_r0, r0.data(), sizeof(int) * (b->n + 1), cudaMemcpyHostToDevice, b->stream));
    LBEM_CUDA(cudaMemcpyAsync(b->d_args, args.data(), sizeof(StepArgs) * args.size(), cudaMemcpyHostToDevice,
                              b->stream));
    LBEM_CUDA(cudaStreamSynchronize(b->stream));  // host vectors go out of scope
    return LBEM_OK;
}

// Rows of member h that hold a source or receiver.
static std::vector<char> event_rows(const lbem_t *h) {
    const int nx = h->grid.nx, ny = h->grid.ny;
    std::vector<char> evrow(ny, 0);
    for (long long site : h->src_site) evrow[(site / nx) % ny] = 1;
    for (long long site : h->rec_site) evrow[(site / nx) % ny] = 1;
    return evrow;
}

// Tile tables of the two-step tile kernel (tiles of 128 x rows sites) over the packed layout.
static lbem_status upload_tile_tables(lbem_batch_t *b, int rows) {
    std::vector<int> r0;
    lbem_status st = upload_packed_layout(b, r0);
    if (st != LBEM_OK) return st;
    std::vector<long long> ts(b->n + 1, 0);
    for (int k = 0; k < b->n; k++) {
        const lbem_t *h = b->members[k];
        ts[k + 1] = ts[k] + (long long)((h->grid.nx + 127) / 128) * ((h->grid.ny + rows - 1) / rows);
    }
    const long long total = ts[b->n];
    // tile descriptors: member, origin, packed row of the window's first c_L^2 row, size, and whether the window's
    // rows (periodic) hold a source or receiver
    std::vector<BatchTile> tl((size_t)total);
    for (int k = 0; k < b->n; k++) {
        lbem_t *h = b->members[k];
        const int nx = h->grid.nx, ny = h->grid.ny, ntx = (nx + 127) / 128;
        const std::vector<char> evrow = event_rows(h);
        for (long long u = ts[k]; u < ts[k + 1]; u++) {
            const int local = (int)(u - ts[k]), ty = local / ntx, tx = local - ty * ntx;
            BatchTile d;
            d.m = k;
            d.x0 = tx * 128;
            d.y0 = ty * rows;
            d.py = r0[k] + 2 + d.y0 - 1;
            d.nx = nx;
            d.ny = ny;
            d.ev = 0;
            for (int r = -1; r <= rows && !d.ev; r++) d.ev = evrow[(((d.y0 + r) % ny) + ny) % ny];
            d.pad = 0;
            tl[(size_t)(u)] = d;
        }
    }
    if (b->tiles_cap < tl.size()) {
        cudaFree(b->d_tiles);
        b->d_tiles = nullptr;
        b->tiles_cap = 0;
        if (cudaMalloc((void **)&b->d_tiles, sizeof(BatchTile) * tl.size()) != cudaSuccess) {
            cudaGetLastError();
            return fail(LBEM_ERR_NOMEM, "lbem_batch: no room for the tile table");
        }
        b->tiles_cap = tl.size();
    }
    LBEM_CUDA(cudaMemcpyAsync(b->d_tiles, tl.data(), sizeof(BatchTile) * tl.size(), cudaMemcpyHostToDevice,
                              b->stream));
    LBEM_CUDA(cudaStreamSynchronize(b->stream));  // host vectors go out of scope
    b->ntiles = total;
    b->tb_rows = rows;
    return LBEM_OK;
}

// Unit table of the strip kernel over the packed layout: per member and 128-column strip, runs of
// chunks * rows - 2 rows (the strip kernel's step t covers rows ys-1 .. ye in whole chunks), with the member's event
// tables; tall units first so that the ragged ones come last in the queue.
static lbem_status upload_unit_tables(lbem_batch_t *b, int shape) {
    std::vector<int> r0;
    lbem_status st = upload_packed_layout(b, r0);
    if (st != LBEM_OK) return st;
    const int tby = batch_ss2_rows(shape), H = batch_ss2_chunks(shape) * tby - 2;
    std::vector<BatchUnit> ul;
    for (int k = 0; k < b->n; k++) {
        const lbem_t *h = b->members[k];
        const int nx = h->grid.nx, ny = h->grid.ny;
        for (int ys = 0; ys < ny; ys += H)
            for (int x0 = 0; x0 < nx; x0 += 128) {
                BatchUnit u;
                u.m = k;
                u.x0 = x0;
                u.ys = ys;
                u.ye = std::min(ys + H, ny);
                u.prow0 = r0[k];
                u.nx = nx;
                u.ny = ny;
                u.pad = 0;
                u.rowptr = h->nev ? h->d_rowptr : nullptr;
                u.ev = h->d_ev;
                ul.push_back(u);
            }
    }
    std::stable_sort(ul.begin(), ul.end(),
                     [](const BatchUnit &a, const BatchUnit &c) { return a.ye - a.ys > c.ye - c.ys; });
    if (ul.size() > (size_t)(1 << 30)) return fail(LBEM_ERR_ARG, "lbem_batch: too many units");
    if (b->units_cap < ul.size()) {
        cudaFree(b->d_units);
        b->d_units = nullptr;
        b->units_cap = 0;
        if (cudaMalloc((void **)&b->d_units, sizeof(BatchUnit) * ul.size()) != cudaSuccess) {
            cudaGetLastError();
            return fail(LBEM_ERR_NOMEM, "lbem_batch: no room for the unit table");
        }
        b->units_cap = ul.size();
    }
    LBEM_CUDA(cudaMemcpyAsync(b->d_units, ul.data(), sizeof(BatchUnit) * ul.size(), cudaMemcpyHostToDevice,
                              b->stream));
    LBEM_CUDA(cudaStreamSynchronize(b->stream));  // host vector goes out of scope
    b->nunits = (int)ul.size();
    return LBEM_OK;
}

static lbem_status upload_tables(lbem_batch_t *b, int variant) {
    if (two_step(variant)) {  // the pair kernel's tiles, and the linear single-step kernel's table for an odd step
        lbem_status st = strip_variant(variant) ? upload_unit_tables(b, kRowsB[variant] - 200)
                                                : upload_tile_tables(b, batch_tb2_rows(kRowsB[variant] - 100));
        if (st != LBEM_OK) return st;
        variant = kLinVariant;
    }
    const int R = kRowsB[variant] < 0 ? 1 : kRowsB[variant];  // persistent and capped variants use the R = 1 table
    std::vector<Member> hm(b->n);
    std::vector<long long> ws(b->n + 1, 0);
    for (int k = 0; k < b->n; k++) {
        lbem_t *h = b->members[k];
        StepArgs a = step_args(h, h->cur);
        hm[k].g = a.g;
        hm[k].a = a.in;
        hm[k].b = a.out;
        hm[k].med = a.med;
        hm[k].evt = a.evt;
        const bool lin = kRowsB[variant] == -7 || kRowsB[variant] == -8;
        const long long units = lin ? ((long long)h->grid.ny * (h->grid.pitch / 4) + 31) / 32
                                : R ? (long long)((h->grid.ny + R - 1) / R) * (h->grid.nchunk_pad / 32)
                                    : ((long long)h->grid.nx * h->grid.ny + BLOCK - 1) / BLOCK;
        ws[k + 1] = ws[k] + units;
    }
    const long long total = ws[b->n];
    if (R) {
        b->total_warps = total;
        b->total_blocks = (total * 32 + BLOCK - 1) / BLOCK;
    } else {
        b->total_warps = total * (BLOCK / 32);
        b->total_blocks = total;
    }
    std::vector<int> map((size_t)total);
    for (int k = 0; k < b->n; k++)
        for (long long u = ws[k]; u < ws[k + 1]; u++) map[(size_t)u] = k;
    if (b->map_cap < map.size()) {
        cudaFree(b->d_map);
        b->d_map = nullptr;
        b->map_cap = 0;
        if (cudaMalloc((void **)&b->d_map, sizeof(int) * map.size()) != cudaSuccess) {
            cudaGetLastError();
            return fail(LBEM_ERR_NOMEM, "lbem_batch: no room for the work table");
        }
        b->map_cap = map.size();
    }
    LBEM_CUDA(cudaMemcpyAsync(b->d_members, hm.data(), sizeof(Member) * b->n, cudaMemcpyHostToDevice, b->stream));
    LBEM_CUDA(cudaMemcpyAsync(b->d_wstart, ws.data(), sizeof(long long) * (b->n + 1), cudaMemcpyHostToDevice, b->stream));
    LBEM_CUDA(cudaMemcpyAsync(b->d_map, map.data(), sizeof(int) * map.size(), cudaMemcpyHostToDevice, b->stream));
    LBEM_CUDA(cudaStreamSynchronize(b->stream));  // host vectors go out of scope
    return LBEM_OK;
}

static cudaError_t launch_batch(lbem_batch_t *b, int variant, int offset) {
    const unsigned blocks = (unsigned)b->total_blocks;
    const long long nw = b->total_warps;
    switch (kRowsB[variant]) {
        case 1: step2d_batch<1><<<blocks, BLOCK, 0, b->stream>>>(b->d_members, b->d_wstart, b->d_map, nw, b->d_t0, offset); break;
        case 2: step2d_batch<2><<<blocks, BLOCK, 0, b->stream>>>(b->d_members, b->d_wstart, b->d_map, nw, b->d_t0, offset); break;
        case 4: step2d_batch<4><<<blocks, BLOCK, 0, b->stream>>>(b->d_members, b->d_wstart, b->d_map, nw, b->d_t0, offset); break;
        case 0: step2d_batch_site<<<blocks, BLOCK, 0, b->stream>>>(b->d_members, b->d_map, b->d_wstart, b->d_t0, offset); break;
        case -5: step2d_batch<1, 5><<<blocks, BLOCK, 0, b->stream>>>(b->d_members, b->d_wstart, b->d_map, nw, b->d_t0, offset); break;
        case -6: step2d_batch<1, 6><<<blocks, BLOCK, 0, b->stream>>>(b->d_members, b->d_wstart, b->d_map, nw, b->d_t0, offset); break;
        case -7: step2d_batch_lin<1><<<blocks, BLOCK, 0, b->stream>>>(b->d_members, b->d_wstart, b->d_map, nw, b->d_t0, offset); break;
        case -8: step2d_batch_lin<5><<<blocks, BLOCK, 0, b->stream>>>(b->d_members, b->d_wstart, b->d_map, nw, b->d_t0, offset); break;
        default: {
            static int per_sm = 0, nsm = 0;
            if (!per_sm) {
                int dev = 0;
                cudaGetDevice(&dev);
                cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step2d_batch_pipe, BLOCK, 0);
                if (per_sm < 1) per_sm = 1;
            }
            const long long warps = (long long)per_sm * nsm * (BLOCK / 32);
            const long long per_warp = (nw + warps - 1) / warps;
            const long long used = (nw + per_warp - 1) / per_warp;
            const unsigned pb = (unsigned)((used * 32 + BLOCK - 1) / BLOCK);
            step2d_batch_pipe<<<pb, BLOCK, 0, b->stream>>>(b->d_members, b->d_wstart, b->d_map, nw, per_warp, b->d_t0, offset);
            break;
        }
    }
    return cudaGetLastError();
}

// Enqueue nsteps steps of `variant` from the members' current state (t0 in device memory): one launch per step, or
// for a two-step variant one launch per pair of steps, after a single step first when nsteps is odd.  Returns the
// number of launches (each one flips the members' buffers) in *nlaunch.
static cudaError_t enqueue_batch(lbem_batch_t *b, int variant, int nsteps, int *nlaunch) {
    if (!two_step(variant)) {
        for (int k = 0; k < nsteps; k++) {
            cudaError_t e = launch_batch(b, variant, k);
            if (e != cudaSuccess) return e;
        }
        *nlaunch = nsteps;
        return cudaSuccess;
    }
    // an odd step first, on the members' own buffers (the state then sits in their other buffer: parity 1)
    int n = 0, toff = 0, par = 0;
    if (nsteps & 1) {
        cudaError_t e = launch_batch(b, kLinVariant, 0);
        if (e != cudaSuccess) return e;
        n = toff = par = 1;
    }
    if (nsteps >= 2) {  // pack, pairs of steps between the packed buffers, unpack into the members' state buffers
        const BatchPacked pk = b->packed();
        cudaError_t e = launch_batch_pack(b->d_args, par, b->d_r0, b->n, b->pack_rows, pk, 0, false, b->stream);
        int j = 0;
        for (; e == cudaSuccess && toff + 2 <= nsteps; toff += 2, j++, n++)
            e = strip_variant(variant)
                    ? launch_batch_ss2(b->d_args, b->d_units, b->nunits, b->d_sched, b->d_t0, toff, j & 1, pk,
                                       b->pack_rows, kRowsB[variant] - 200, b->stream)
                    : launch_batch_tb2(b->d_args, b->d_tiles, b->ntiles, b->d_t0, toff, j & 1, pk, b->pack_rows,
                                       kRowsB[variant] - 100, b->stream);
        if (e == cudaSuccess)
            e = launch_batch_pack(b->d_args, par, b->d_r0, b->n, b->pack_rows, pk, j & 1, true, b->stream);
        if (e != cudaSuccess) return e;
    }
    *nlaunch = n;
    return cudaSuccess;
}


static lbem_status check_members(lbem_batch_t *b) {
    const long long t = b->members[0]->t;
    for (lbem_t *h : b->members) {
        if (!h->has_medium) return fail(LBEM_ERR_STATE, "lbem_batch_step: every member needs a medium");
        if (h->has_mu || h->walls() || h->general())
            return fail(LBEM_ERR_STATE,
                        "lbem_batch_step: members need uniform mu, periodic boundaries and no dispersive pole");
        if (h->t != t) return fail(LBEM_ERR_STATE, "lbem_batch_step: members are at different times");
        if (h->stream != b->stream) {
            // members may have work queued on their own streams: order it before the batch
            LBEM_CUDA(cudaStreamSynchronize(h->stream));
        }
    }
    return LBEM_OK;
}

extern "C" {

lbem_status lbem_batch_create(int n, lbem_t *const *members, void *stream, lbem_batch_t **out) {
    if (!out || !members || n < 1) return fail(LBEM_ERR_ARG, "lbem_batch_create: need n >= 1 members");
    *out = nullptr;
    for (int k = 0; k < n; k++) {
        const lbem_t *h = members[k];
        if (!h) return fail(LBEM_ERR_ARG, "lbem_batch_create: null member");
        if (h->dim != 2 || h->storage != LBEM_F32 || h->has_mu || h->walls() || h->general())
            return fail(LBEM_ERR_ARG,
                        "lbem_batch_create: members must be 2D, LBEM_F32 storage, uniform mu, periodic boundaries");
        for (int j = 0; j < k; j++)
            if (members[j] == h) return fail(LBEM_ERR_ARG, "lbem_batch_create: a member appears twice");
    }
    lbem_batch_t *b = new lbem_batch_t();
    b->n = n;
    b->members.assign(members, members + n);
    b->stream = (cudaStream_t)stream;
    cudaError_t e = cudaMalloc((void **)&b->d_members, sizeof(Member) * n);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_wstart, sizeof(long long) * (n + 1));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_args, sizeof(StepArgs) * 2 * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_r0, sizeof(int) * (n + 1));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_t0, sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_sched, sizeof(int) * 2);
    if (e == cudaSuccess) e = cudaMemset(b->d_sched, 0, sizeof(int) * 2);
    if (e != cudaSuccess) {
        cudaGetLastError();
        lbem_batch_destroy(b);
        return fail(LBEM_ERR_NOMEM, "lbem_batch_create: device allocation failed");
    }
    *out = b;
    return LBEM_OK;
}

lbem_status lbem_batch_step(lbem_batch_t *b, int nsteps) {
    if (!b) return fail(LBEM_ERR_ARG, "null batch");
    if (nsteps < 0) return fail(LBEM_ERR_ARG, "lbem_batch_step: nsteps < 0");
    if (nsteps == 0) return LBEM_OK;
    lbem_status st = check_members(b);
    if (st != LBEM_OK) return st;
    st = upload_tables(b, b->variant);
    if (st != LBEM_OK) return st;
    const long long t0 = b->members[0]->t;
    LBEM_CUDA(cudaMemcpyAsync(b->d_t0, &t0, sizeof(long long), cudaMemcpyHostToDevice, b->stream));
    LBEM_CUDA(cudaStreamSynchronize(b->stream));
    if (b->stream != nullptr) {
        if (!(b->graph && b->graph_steps == nsteps && b->graph_variant == b->variant)) {
            drop_batch_graph(b);
            LBEM_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
            int nl = 0;
            cudaError_t e = enqueue_batch(b, b->variant, nsteps, &nl);
            if (e != cudaSuccess) {
                cudaGraph_t g = nullptr;
                cudaStreamEndCapture(b->stream, &g);
                if (g) cudaGraphDestroy(g);
                return cuda_fail(e, "lbem_batch_step (capture)");
            }
            cudaGraph_t g = nullptr;
            LBEM_CUDA(cudaStreamEndCapture(b->stream, &g));
            e = cudaGraphInstantiate(&b->graph, g, 0);
            cudaGraphDestroy(g);
            LBEM_CUDA(e);
            b->graph_steps = nsteps;
            b->graph_variant = b->variant;
        }
        LBEM_CUDA(cudaGraphLaunch(b->graph, b->stream));
    } else {
        int nl = 0;
        LBEM_CUDA(enqueue_batch(b, b->variant, nsteps, &nl));
    }
    // each single-step launch flips the members' buffers; the two-step variants unpack the pairs' result into the
    // buffer they packed from, so only their odd first step flips
    const int flips = two_step(b->variant) ? (nsteps & 1) : nsteps;
    for (lbem_t *h : b->members) {
        h->cur ^= (flips & 1);
        h->t += nsteps;
    }
    // members' own streams must see the batch's work before their next call
    if (b->stream != b->members[0]->stream) LBEM_CUDA(cudaStreamSynchronize(b->stream));
    return LBEM_OK;
}

lbem_status lbem_batch_autotune(lbem_batch_t *b, int trial_steps, int *best) {
    if (!b) return fail(LBEM_ERR_ARG, "null batch");
    if (trial_steps < 1) return fail(LBEM_ERR_ARG, "lbem_batch_autotune: trial_steps >= 1");
    lbem_status st = check_members(b);
    if (st != LBEM_OK) return st;
    // the trials step every member in place; the states are saved and restored
    std::vector<void *> saves(b->n, nullptr);
    for (int k = 0; k < b->n; k++) {
        size_t bytes = 0;
        lbem_info(b->members[k], nullptr, &bytes);
        if (cudaMalloc(&saves[k], bytes) != cudaSuccess) {
            cudaGetLastError();
            for (void *p : saves) cudaFree(p);
            return fail(LBEM_ERR_NOMEM, "lbem_batch_autotune: no room to save member states");
        }
        if ((st = lbem_save_state(b->members[k], saves[k])) != LBEM_OK) break;
    }
    const long long t0 = b->members[0]->t;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_ms = 1e30f;
    int best_v = b->variant;
    for (int v = 0; v < kBatchVariants && st == LBEM_OK; v++) {
        if ((st = upload_tables(b, v)) != LBEM_OK) break;
        LBEM_CUDA(cudaMemcpyAsync(b->d_t0, &t0, sizeof(long long), cudaMemcpyHostToDevice, b->stream));
        for (int rep = 0; rep < 2; rep++) {
            cudaEventRecord(e0, b->stream);
            int nl = 0;
            LBEM_CUDA(enqueue_batch(b, v, trial_steps, &nl));
            cudaEventRecord(e1, b->stream);
        }
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
            best_ms = ms;
            best_v = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (int k = 0; k < b->n && st == LBEM_OK; k++) st = lbem_load_state(b->members[k], saves[k], t0);
    cudaStreamSynchronize(b->stream);
    for (lbem_t *h : b->members) cudaStreamSynchronize(h->stream);
    for (void *p : saves) cudaFree(p);
    if (st != LBEM_OK) return st;
    b->variant = best_v;
    drop_batch_graph(b);
    if (best) *best = best_v;
    return LBEM_OK;
}

lbem_status lbem_batch_set_variant(lbem_batch_t *b, int variant) {
    if (!b) return fail(LBEM_ERR_ARG, "null batch");
    if (variant < 0 || variant >= kBatchVariants) return fail(LBEM_ERR_ARG, "lbem_batch_set_variant: out of range");
    b->variant = variant;
    drop_batch_graph(b);
    return LBEM_OK;
}

lbem_status lbem_batch_get_variant(const lbem_batch_t *b, int *variant, int *nvariants) {
    if (!b) return fail(LBEM_ERR_ARG, "null batch");
    if (variant) *variant = b->variant;
    if (nvariants) *nvariants = kBatchVariants;
    return LBEM_OK;
}

void lbem_batch_destroy(lbem_batch_t *b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    drop_batch_graph(b);
    cudaFree(b->d_members);
    cudaFree(b->d_wstart);
    cudaFree(b->d_map);
    cudaFree(b->d_t0);
    cudaFree(b->d_args);
    cudaFree(b->d_tiles);
    cudaFree(b->d_units);
    cudaFree(b->d_sched);
    cudaFree(b->d_r0);
    cudaFree(b->d_pack);
    delete b;
}

}  // extern "C"
