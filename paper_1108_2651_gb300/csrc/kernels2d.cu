// 2D (D2Q5) kernels of the lattice-Boltzmann Maxwell scheme of Hanasoge,
// Succi & Orszag (arXiv:1108.2651): fused pull-stream + moments + source +
// BGK collision (Eqs. 3, 8, 17, 18), initial state (Eq. 8), field extraction
// (Eqs. 9-10) and FP64 diagnostics.
//
// The single independent tensor component g_i = g_{i,xy} is stored per
// direction i (D2Q5 order c_0 = 0, c_1 = +x, c_2 = +y, c_3 = -x, c_4 = -y).
// With tau = dt/2 (Delta t / tau = 2) and the weights of moving particles
// equal to c_L^2/2, the collision of Eq. 17 with the equilibrium of Eq. 8
// reduces per site to (sigma = sum_i g_i, Lambda = c_L^2 sigma = -E_z,
// B_y = g_1 - g_3, B_x = g_4 - g_2):
//   g'_1 = Lambda - g_3 + T_m    g'_3 = Lambda - g_1 + T_m
//   g'_2 = Lambda - g_4 + T_m    g'_4 = Lambda - g_2 + T_m
//   g'_0 = 2 w0 sigma - g_0 + T_0,   w0 = 1 - 2 c_L^2,
// since 2 g^(0)_1 = Lambda + B_y etc.  The source of Eq. 3 is S_z = c_L^2 S^
// with S^ = B_x d_y ln mu - B_y d_x ln mu - mu j_z, and the tensor source
// T_i = -(w_i / c_L^2) S_z gives T_m = -c_L^2 S^/2, T_0 = -w0 S^.
//
// Thread mapping: one warp covers 128 consecutive sites of one row, 4 per
// lane, loaded as one 4-element vector per population.  The +x / -x pulls are
// shifted by one site: the neighbouring lane's element arrives by a warp
// shuffle; the first and last lane of a warp fetch one element each.
#include "lbem_internal.cuh"

namespace lbk {

// pull2d (the pulls of 4 sites of a row by one lane), collide2d and field2d are in lbem_internal.cuh.

template <int ST, bool MU, int R>
__global__ void __launch_bounds__(BLOCK) step2d(StepArgs a) {
    using C = Codec<ST>;
    const Grid &G = a.g;
    const int lane = threadIdx.x & 31;
    const long long wg = ((long long)blockIdx.x * BLOCK + threadIdx.x) >> 5;
    const int wpr = G.nchunk_pad >> 5;
    const int rg = (int)(wg / wpr);
    const int c = (int)(wg - (long long)rg * wpr) * 32 + lane;
    const int row0 = rg * R;
    if (row0 >= G.ny) return;  // warp-uniform
    const bool active = c < G.nchunk;

    float4 g[R][5];
    float4 cl[R];
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int row = min(row0 + r, G.ny - 1);
        pull2d<ST>(a.in, G, row, c, lane, g[r]);
        cl[r] = active ? __ldg(reinterpret_cast<const float4 *>(a.med.cL2 + (long long)row * G.pitch) + c)
                       : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int row = row0 + r;
        if (row >= G.ny) break;  // warp-uniform
        float4 shat = make_float4(0.f, 0.f, 0.f, 0.f);
        if (MU && active) {
            const float4 dx = __ldg(reinterpret_cast<const float4 *>(a.med.dlnmu + (long long)row * G.pitch) + c);
            const float4 dy =
                __ldg(reinterpret_cast<const float4 *>(a.med.dlnmu + G.plane + (long long)row * G.pitch) + c);
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const float bx = get(g[r][4], j) - get(g[r][2], j), by = get(g[r][1], j) - get(g[r][3], j);
                set(shat, j, mu_source(bx, by, get(dx, j), get(dy, j)));
            }
        }
        if (a.evt.rowptr) {
            const int e0 = __ldg(a.evt.rowptr + row), e1 = __ldg(a.evt.rowptr + row + 1);
            for (int e = e0; e < e1; e++) {
                const Event ev = a.evt.ev[e];
                if ((ev.x >> 2) != c || !active) continue;
                const int j = ev.x & 3;
                if (ev.kind == 0) {
                    if (ev.comp == 2 && a.t < a.evt.nt) {
                        float jz = __ldg(a.evt.amp + (long long)ev.index * a.evt.nt + a.t);
                        if (MU) jz = __fmul_rn(jz, __ldg(a.med.mu + (long long)row * G.pitch + ev.x));
                        set(shat, j, __fsub_rn(get(shat, j), jz));
                    }
                } else if (a.t < a.evt.cap) {
                    const float gj[5] = {get(g[r][0], j), get(g[r][1], j), get(g[r][2], j), get(g[r][3], j),
                                         get(g[r][4], j)};
                    const float s = ((gj[0] + gj[1]) + (gj[2] + gj[3])) + gj[4];
                    a.evt.traces[(long long)ev.index * a.evt.cap + a.t] =
                        field2d(ev.comp, get(cl[r], j), s, gj[4] - gj[2], gj[1] - gj[3]);
                }
            }
        }
        float4 o0, o1, o2, o3, o4;
        // rows without a source (and mu uniform) have S^ = +0 everywhere: collide2d_free gives the same bits
        const bool src = MU || (a.evt.rowptr && __ldg(a.evt.rowptr + row) != __ldg(a.evt.rowptr + row + 1));
        if (src) {
#pragma unroll
            for (int j = 0; j < 4; j++) {
                Out5 o = collide2d(get(g[r][0], j), get(g[r][1], j), get(g[r][2], j), get(g[r][3], j),
                                   get(g[r][4], j), get(cl[r], j), get(shat, j));
                set(o0, j, o.o0);
                set(o1, j, o.o1);
                set(o2, j, o.o2);
                set(o3, j, o.o3);
                set(o4, j, o.o4);
            }
        } else {
#pragma unroll
            for (int j = 0; j < 4; j++) {
                Out5 o = collide2d_free(get(g[r][0], j), get(g[r][1], j), get(g[r][2], j), get(g[r][3], j),
                                        get(g[r][4], j), get(cl[r], j));
                set(o0, j, o.o0);
                set(o1, j, o.o1);
                set(o2, j, o.o2);
                set(o3, j, o.o3);
                set(o4, j, o.o4);
            }
        }
        if (active) {
            C::store4(a.out, 0, row, c, o0);
            C::store4(a.out, 1, row, c, o1);
            C::store4(a.out, 2, row, c, o2);
            C::store4(a.out, 3, row, c, o3);
            C::store4(a.out, 4, row, c, o4);
        }
    }
}

// ------------------------------------------------------------------ persistent, software-pipelined variant
// Each warp walks units of 128 sites (one row segment) with a grid-sized
// stride and issues the loads of its next unit before it shuffles, collides
// and stores the current one, so the memory system always has a unit's loads
// in flight per warp even while it computes.
struct Raw2 {
    float4 v0, a1, v2, a3, v4, cl;
    float s1, s3, sw;
};

template <int ST>
__device__ __forceinline__ void load_raw(const StepArgs &a, int row, int c, int lane, Raw2 &r) {
    using C = Codec<ST>;
    const Grid &G = a.g;
    const bool active = c < G.nchunk;
    const int x0 = 4 * c;
    const int ym = row == 0 ? G.ny - 1 : row - 1, yp = row == G.ny - 1 ? 0 : row + 1;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    r.v0 = active ? C::load4(a.in, 0, row, c) : z4;
    r.a1 = active ? C::load4(a.in, 1, row, c) : z4;
    r.v2 = active ? C::load4(a.in, 2, ym, c) : z4;
    r.a3 = active ? C::load4(a.in, 3, row, c) : z4;
    r.v4 = active ? C::load4(a.in, 4, yp, c) : z4;
    r.cl = active ? __ldg(reinterpret_cast<const float4 *>(a.med.cL2 + (long long)row * G.pitch) + c) : z4;
    r.s1 = (lane == 0 && active) ? C::load1(a.in, 1, row, c == 0 ? G.nx - 1 : x0 - 1) : 0.f;
    r.s3 = (lane == 31 && x0 + 4 < G.nx) ? C::load1(a.in, 3, row, x0 + 4) : 0.f;
    r.sw = (c == G.nchunk - 1) ? C::load1(a.in, 3, row, 0) : 0.f;
}

template <int ST, bool MU>
__global__ void __launch_bounds__(BLOCK) step2d_pipe(StepArgs a) {
    using C = Codec<ST>;
    const Grid &G = a.g;
    const int lane = threadIdx.x & 31;
    const int wpr = G.nchunk_pad >> 5;
    const long long nunits = (long long)G.ny * wpr;
    const long long nwarps = (long long)gridDim.x * (BLOCK / 32);
    long long u = ((long long)blockIdx.x * BLOCK + threadIdx.x) >> 5;
    if (u >= nunits) return;  // warp-uniform
    Raw2 cur;
    int row = (int)(u / wpr), c = (int)(u - (long long)row * wpr) * 32 + lane;
    load_raw<ST>(a, row, c, lane, cur);
    while (true) {
        const long long un = u + nwarps;
        const bool more = un < nunits;  // warp-uniform
        int nrow = 0, nc = 0;
        Raw2 nxt;
        if (more) {
            nrow = (int)(un / wpr);
            nc = (int)(un - (long long)nrow * wpr) * 32 + lane;
            load_raw<ST>(a, nrow, nc, lane, nxt);
        }
        // finish the pull of the current unit
        const int x0 = 4 * c;
        const bool active = c < G.nchunk;
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
        if (MU && active) {
            const float4 dx = __ldg(reinterpret_cast<const float4 *>(a.med.dlnmu + (long long)row * G.pitch) + c);
            const float4 dy =
                __ldg(reinterpret_cast<const float4 *>(a.med.dlnmu + G.plane + (long long)row * G.pitch) + c);
            for (int j = 0; j < 4; j++) {
                const float bx = get(g[4], j) - get(g[2], j), by = get(g[1], j) - get(g[3], j);
                set(shat, j, mu_source(bx, by, get(dx, j), get(dy, j)));
            }
        }
        if (a.evt.rowptr) {
            const int e0 = __ldg(a.evt.rowptr + row), e1 = __ldg(a.evt.rowptr + row + 1);
            for (int e = e0; e < e1; e++) {
                const Event ev = a.evt.ev[e];
                if ((ev.x >> 2) != c || !active) continue;
                const int j = ev.x & 3;
                if (ev.kind == 0) {
                    if (ev.comp == 2 && a.t < a.evt.nt) {
                        float jz = __ldg(a.evt.amp + (long long)ev.index * a.evt.nt + a.t);
                        if (MU) jz = __fmul_rn(jz, __ldg(a.med.mu + (long long)row * G.pitch + ev.x));
                        set(shat, j, __fsub_rn(get(shat, j), jz));
                    }
                } else if (a.t < a.evt.cap) {
                    const float s = ((get(g[0], j) + get(g[1], j)) + (get(g[2], j) + get(g[3], j))) + get(g[4], j);
                    a.evt.traces[(long long)ev.index * a.evt.cap + a.t] =
                        field2d(ev.comp, get(cur.cl, j), s, get(g[4], j) - get(g[2], j), get(g[1], j) - get(g[3], j));
                }
            }
        }
        float4 o0, o1, o2, o3, o4;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            Out5 o = collide2d(get(g[0], j), get(g[1], j), get(g[2], j), get(g[3], j), get(g[4], j),
                               get(cur.cl, j), get(shat, j));
            set(o0, j, o.o0);
            set(o1, j, o.o1);
            set(o2, j, o.o2);
            set(o3, j, o.o3);
            set(o4, j, o.o4);
        }
        if (active) {
            C::store4(a.out, 0, row, c, o0);
            C::store4(a.out, 1, row, c, o1);
            C::store4(a.out, 2, row, c, o2);
            C::store4(a.out, 3, row, c, o3);
            C::store4(a.out, 4, row, c, o4);
        }
        if (!more) break;
        u = un;
        row = nrow;
        c = nc;
        cur = nxt;
    }
}

template <int ST, bool MU>
static cudaError_t launch_pipe(const StepArgs &a, cudaStream_t s) {
    static int per_sm = 0, nsm = 0;  // resident blocks per SM of this instantiation, SM count
    if (!per_sm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step2d_pipe<ST, MU>, BLOCK, 0);
        if (per_sm < 1) per_sm = 1;
    }
    const long long units = (long long)a.g.ny * (a.g.nchunk_pad / 32);
    long long blocks = (units * 32 + BLOCK - 1) / BLOCK;
    blocks = blocks < (long long)per_sm * nsm ? blocks : (long long)per_sm * nsm;
    step2d_pipe<ST, MU><<<(unsigned)blocks, BLOCK, 0, s>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ persistent variant with cp.async staging
// Each lane copies its own unit data (the five population vectors, c_L^2, the
// halo words of the +-x pulls and, for LBEM_I16B, the exponent words)
// asynchronously into a private slot of a KS-stage shared-memory ring, KS-1
// units ahead of the unit it computes.  Only the lane that issued a copy reads
// it, so a cp.async.wait_group is the only wait (no barrier, no spin).
constexpr int KS = 3;          // pipeline stages
constexpr int SLOT = 112;      // bytes per lane and stage

__device__ __forceinline__ void cpa4(void *dst, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src));
}
__device__ __forceinline__ void cpa8(void *dst, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src));
}
__device__ __forceinline__ void cpa16(void *dst, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src));
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cpa_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// slot layout: [0,80) five population vectors (16 B each; 8 B used for 16-bit storage),
// [80,96) c_L^2 float4, [96,100) word holding x0-1 of plane 1, [100,104) word holding x0+4 of plane 3,
// [104,108) word holding x = 0 of plane 3; LBEM_I16B exponent words in [80,100) reuse is avoided by
// placing them after: own exponents at [108,112) would not fit five, so I16B keeps its exponent bytes
// in a second slot array (see ExSlot).
struct ExSlot {
    unsigned own[5];      // words holding the chunk exponent of each plane
    unsigned s1, s3, sw;  // exponent words of the three halo elements
};

template <int ST>
__device__ __forceinline__ const char *plane_row(const PopBuf &b, int p, int row) {
    return static_cast<const char *>(b.data) + (p * b.plane + (long long)row * b.pitch) * Codec<ST>::bytes;
}

template <int ST>
__device__ __forceinline__ void issue_unit(const StepArgs &a, int row, int c, int lane, char *slot, ExSlot *ex) {
    const Grid &G = a.g;
    if (c >= G.nchunk) return;
    const int x0 = 4 * c;
    const int ym = row == 0 ? G.ny - 1 : row - 1, yp = row == G.ny - 1 ? 0 : row + 1;
    const int rows[5] = {row, row, ym, row, yp};
    constexpr int VB = 4 * Codec<ST>::bytes;  // bytes of one 4-site vector
#pragma unroll
    for (int p = 0; p < 5; p++) {
        const char *src = plane_row<ST>(a.in, p, rows[p]) + (long long)c * VB;
        if (VB == 16) cpa16(slot + 16 * p, src);
        else cpa8(slot + 16 * p, src);
    }
    cpa16(slot + 80, a.med.cL2 + (long long)row * G.pitch + x0);
    constexpr int EB = Codec<ST>::bytes;
    auto word = [&](int p, int x) {  // the aligned 4-byte word holding element x of plane p, row `row`
        const int e = (EB == 4) ? x : (x & ~1);
        return plane_row<ST>(a.in, p, row) + (long long)e * EB;
    };
    const int x1 = c == 0 ? G.nx - 1 : x0 - 1;
    if (lane == 0) cpa4(slot + 96, word(1, x1));
    if (lane == 31 && x0 + 4 < G.nx) cpa4(slot + 100, word(3, x0 + 4));
    if (c == G.nchunk - 1) cpa4(slot + 104, word(3, 0));
    if (ST == LBEM_I16B) {
        auto exw = [&](int p, int r, int ch) {
            return reinterpret_cast<const char *>(a.in.ex + p * a.in.explane + (long long)r * a.in.expitch + (ch & ~3));
        };
#pragma unroll
        for (int p = 0; p < 5; p++) cpa4(&ex->own[p], exw(p, rows[p], c));
        if (lane == 0) cpa4(&ex->s1, exw(1, row, x1 >> 2));
        if (lane == 31 && x0 + 4 < G.nx) cpa4(&ex->s3, exw(3, row, (x0 + 4) >> 2));
        if (c == G.nchunk - 1) cpa4(&ex->sw, exw(3, row, 0));
    }
}

// decode a 4-site vector / one element staged in shared memory
template <int ST>
__device__ __forceinline__ float4 dec4(const PopBuf &b, const char *v, unsigned exword, int c) {
    if (ST == LBEM_F32) return *reinterpret_cast<const float4 *>(v);
    const uint2 r = *reinterpret_cast<const uint2 *>(v);
    if (ST == LBEM_F16) {
        const float4 f = h4_to_f4(r);
        return make_float4(f.x * b.inv_scale, f.y * b.inv_scale, f.z * b.inv_scale, f.w * b.inv_scale);
    }
    if (ST == LBEM_BF16)
        return make_float4(__uint_as_float(r.x << 16), __uint_as_float(r.x & 0xffff0000u), __uint_as_float(r.y << 16),
                           __uint_as_float(r.y & 0xffff0000u));
    const int e = (int)(signed char)((exword >> (8 * (c & 3))) & 0xffu);
    const float f = i16b_factor(e);
    const float2 lo = i16x2_to_f2(r.x, f), hi = i16x2_to_f2(r.y, f);
    return make_float4(lo.x, lo.y, hi.x, hi.y);
}

template <int ST>
__device__ __forceinline__ float dec1(const PopBuf &b, unsigned w, int x, unsigned exword) {
    if (ST == LBEM_F32) return __uint_as_float(w);
    const unsigned short hbits = (unsigned short)((x & 1) ? (w >> 16) : (w & 0xffffu));
    if (ST == LBEM_F16) return __half2float(__ushort_as_half(hbits)) * b.inv_scale;
    if (ST == LBEM_BF16) return __uint_as_float(((unsigned)hbits) << 16);
    const int e = (int)(signed char)((exword >> (8 * ((x >> 2) & 3))) & 0xffu);
    return i16_to_f((short)hbits) * i16b_factor(e);
}

template <int ST, bool MU>
__global__ void __launch_bounds__(BLOCK) step2d_async(StepArgs a) {
    using C = Codec<ST>;
    extern __shared__ __align__(16) char smem[];
    const Grid &G = a.g;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int wpr = G.nchunk_pad >> 5;
    const long long nunits = (long long)G.ny * wpr;
    const long long nwarps = (long long)gridDim.x * (BLOCK / 32);
    const long long u0 = ((long long)blockIdx.x * BLOCK + threadIdx.x) >> 5;
    if (u0 >= nunits) return;  // warp-uniform
    char *slots = smem + ((size_t)wib * KS * 32 + lane) * SLOT;  // stage k at slots + k * 32 * SLOT
    ExSlot *exs = reinterpret_cast<ExSlot *>(smem + (size_t)(BLOCK / 32) * KS * 32 * SLOT) + (wib * KS * 32 + lane);
    auto unit_rc = [&](long long u, int &row, int &c) {
        row = (int)(u / wpr);
        c = (int)(u - (long long)row * wpr) * 32 + lane;
    };
    // prologue: KS-1 units in flight
#pragma unroll
    for (int k = 0; k < KS - 1; k++) {
        const long long u = u0 + k * nwarps;
        if (u < nunits) {
            int row, c;
            unit_rc(u, row, c);
            issue_unit<ST>(a, row, c, lane, slots + (size_t)k * 32 * SLOT, exs + k * 32);
        }
        cpa_commit();
    }
    for (long long k = 0;; k++) {
        const long long u = u0 + k * nwarps;
        if (u >= nunits) break;  // warp-uniform
        {
            const long long un = u + (KS - 1) * nwarps;
            const int sn = (int)((k + KS - 1) % KS);
            if (un < nunits) {
                int row, c;
                unit_rc(un, row, c);
                issue_unit<ST>(a, row, c, lane, slots + (size_t)sn * 32 * SLOT, exs + sn * 32);
            }
            cpa_commit();
        }
        cpa_wait<KS - 1>();  // this lane's copies of unit k are complete
        const int sk = (int)(k % KS);
        const char *sl = slots + (size_t)sk * 32 * SLOT;
        const ExSlot &ex = exs[sk * 32];
        int row, c;
        unit_rc(u, row, c);
        const bool active = c < G.nchunk;
        const int x0 = 4 * c;
        float4 g[5];
        float4 a1 = make_float4(0.f, 0.f, 0.f, 0.f), a3 = a1, cl = a1;
        if (active) {
            g[0] = dec4<ST>(a.in, sl + 0, ST == LBEM_I16B ? ex.own[0] : 0u, c);
            a1 = dec4<ST>(a.in, sl + 16, ST == LBEM_I16B ? ex.own[1] : 0u, c);
            g[2] = dec4<ST>(a.in, sl + 32, ST == LBEM_I16B ? ex.own[2] : 0u, c);
            a3 = dec4<ST>(a.in, sl + 48, ST == LBEM_I16B ? ex.own[3] : 0u, c);
            g[4] = dec4<ST>(a.in, sl + 64, ST == LBEM_I16B ? ex.own[4] : 0u, c);
            cl = *reinterpret_cast<const float4 *>(sl + 80);
        } else {
            g[0] = g[2] = g[4] = a1;
        }
        float prev = __shfl_up_sync(FULL, a1.w, 1);
        float next = __shfl_down_sync(FULL, a3.x, 1);
        if (lane == 0 && active)
            prev = dec1<ST>(a.in, *reinterpret_cast<const unsigned *>(sl + 96), c == 0 ? G.nx - 1 : x0 - 1, ex.s1);
        if (lane == 31 && x0 + 4 < G.nx) next = dec1<ST>(a.in, *reinterpret_cast<const unsigned *>(sl + 100), x0 + 4, ex.s3);
        g[1] = make_float4(prev, a1.x, a1.y, a1.z);
        g[3] = make_float4(a3.y, a3.z, a3.w, next);
        if (c == G.nchunk - 1) set(g[3], G.nx - 1 - x0, dec1<ST>(a.in, *reinterpret_cast<const unsigned *>(sl + 104), 0, ex.sw));
        float4 shat = make_float4(0.f, 0.f, 0.f, 0.f);
        if (MU && active) {
            const float4 dx = __ldg(reinterpret_cast<const float4 *>(a.med.dlnmu + (long long)row * G.pitch) + c);
            const float4 dy =
                __ldg(reinterpret_cast<const float4 *>(a.med.dlnmu + G.plane + (long long)row * G.pitch) + c);
            for (int j = 0; j < 4; j++) {
                const float bx = get(g[4], j) - get(g[2], j), by = get(g[1], j) - get(g[3], j);
                set(shat, j, mu_source(bx, by, get(dx, j), get(dy, j)));
            }
        }
        if (a.evt.rowptr) {
            const int e0 = __ldg(a.evt.rowptr + row), e1 = __ldg(a.evt.rowptr + row + 1);
            for (int e = e0; e < e1; e++) {
                const Event ev = a.evt.ev[e];
                if ((ev.x >> 2) != c || !active) continue;
                const int j = ev.x & 3;
                if (ev.kind == 0) {
                    if (ev.comp == 2 && a.t < a.evt.nt) {
                        float jz = __ldg(a.evt.amp + (long long)ev.index * a.evt.nt + a.t);
                        if (MU) jz = __fmul_rn(jz, __ldg(a.med.mu + (long long)row * G.pitch + ev.x));
                        set(shat, j, __fsub_rn(get(shat, j), jz));
                    }
                } else if (a.t < a.evt.cap) {
                    const float s = ((get(g[0], j) + get(g[1], j)) + (get(g[2], j) + get(g[3], j))) + get(g[4], j);
                    a.evt.traces[(long long)ev.index * a.evt.cap + a.t] =
                        field2d(ev.comp, get(cl, j), s, get(g[4], j) - get(g[2], j), get(g[1], j) - get(g[3], j));
                }
            }
        }
        float4 o0, o1, o2, o3, o4;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            Out5 o = collide2d(get(g[0], j), get(g[1], j), get(g[2], j), get(g[3], j), get(g[4], j), get(cl, j),
                               get(shat, j));
            set(o0, j, o.o0);
            set(o1, j, o.o1);
            set(o2, j, o.o2);
            set(o3, j, o.o3);
            set(o4, j, o.o4);
        }
        if (active) {
            C::store4(a.out, 0, row, c, o0);
            C::store4(a.out, 1, row, c, o1);
            C::store4(a.out, 2, row, c, o2);
            C::store4(a.out, 3, row, c, o3);
            C::store4(a.out, 4, row, c, o4);
        }
    }
    cpa_wait<0>();  // nothing may stay in flight into a slot when the block exits
}

template <int ST, bool MU>
static cudaError_t launch_async(const StepArgs &a, cudaStream_t s) {
    static int per_sm = 0, nsm = 0;
    const size_t smem = (size_t)(BLOCK / 32) * KS * 32 * (SLOT + sizeof(ExSlot));
    if (!per_sm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaError_t e = cudaFuncSetAttribute(step2d_async<ST, MU>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step2d_async<ST, MU>, BLOCK, smem);
        if (per_sm < 1) per_sm = 1;
    }
    const long long units = (long long)a.g.ny * (a.g.nchunk_pad / 32);
    long long blocks = (units * 32 + BLOCK - 1) / BLOCK;
    blocks = blocks < (long long)per_sm * nsm ? blocks : (long long)per_sm * nsm;
    step2d_async<ST, MU><<<(unsigned)blocks, BLOCK, smem, s>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ 16-bit storage, 8 sites per lane
// One 16-byte load per population and lane (eight 16-bit values), so a warp
// request is 512 bytes as in the FP32 kernel; a warp covers 256 sites.
struct F8 {
    float v[8];
};

template <int ST>
__device__ __forceinline__ F8 load8(const PopBuf &b, int p, int row, int c8) {
    F8 f;
    const uint4 r = __ldg(reinterpret_cast<const uint4 *>(static_cast<const char *>(b.data) +
                                                         (p * b.plane + (long long)row * b.pitch) * 2) + c8);
    const unsigned w[4] = {r.x, r.y, r.z, r.w};
    if (ST == LBEM_F16) {
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const float2 t = __half22float2(*reinterpret_cast<const __half2 *>(&w[k]));
            f.v[2 * k] = t.x * b.inv_scale;
            f.v[2 * k + 1] = t.y * b.inv_scale;
        }
    } else if (ST == LBEM_BF16) {
#pragma unroll
        for (int k = 0; k < 4; k++) {
            f.v[2 * k] = __uint_as_float(w[k] << 16);
            f.v[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
        }
    } else {
        const unsigned short e2 = __ldg(reinterpret_cast<const unsigned short *>(b.ex + p * b.explane +
                                                                                 (long long)row * b.expitch) + c8);
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int e = (int)(signed char)((e2 >> (8 * (k >> 1))) & 0xffu);
            const float2 d = i16x2_to_f2(w[k], i16b_factor(e));
            f.v[2 * k] = d.x;
            f.v[2 * k + 1] = d.y;
        }
    }
    return f;
}

template <int ST>
__device__ __forceinline__ void store8(const PopBuf &b, int p, int row, int c8, const F8 &f) {
    using C = Codec<ST>;
    // each 4-site half is encoded exactly as the 4-site codec encodes it; one 16-byte store per lane
    const float4 lo = make_float4(f.v[0], f.v[1], f.v[2], f.v[3]), hi = make_float4(f.v[4], f.v[5], f.v[6], f.v[7]);
    uint2 r0, r1;
    unsigned short e2 = 0;
    if (ST == LBEM_I16B) {
        const int e0 = Codec<LBEM_I16B>::enc4e(lo, r0), e1 = Codec<LBEM_I16B>::enc4e(hi, r1);
        e2 = (unsigned short)((unsigned)(e0 & 0xff) | ((unsigned)(e1 & 0xff) << 8));
    } else if (ST == LBEM_F16) {
        r0 = Codec<LBEM_F16>::enc4(b, lo);
        r1 = Codec<LBEM_F16>::enc4(b, hi);
    } else {
        r0 = Codec<LBEM_BF16>::enc4(b, lo);
        r1 = Codec<LBEM_BF16>::enc4(b, hi);
    }
    uint4 *q = reinterpret_cast<uint4 *>(static_cast<char *>(b.data) + (p * b.plane + (long long)row * b.pitch) * 2);
    __stcs(q + c8, make_uint4(r0.x, r0.y, r1.x, r1.y));
    if (ST == LBEM_I16B)
        reinterpret_cast<unsigned short *>(b.ex + p * b.explane + (long long)row * b.expitch)[c8] = e2;
    (void)sizeof(C);
}

template <int ST, bool MU, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) step2d_w8(StepArgs a) {
    using C = Codec<ST>;
    const Grid &G = a.g;
    const int lane = threadIdx.x & 31;
    const int n8 = (G.nx + 7) / 8, n8p = (n8 + 31) / 32 * 32;
    const long long wg = ((long long)blockIdx.x * BLOCK + threadIdx.x) >> 5;
    const int wpr = n8p >> 5;
    const int row = (int)(wg / wpr);
    const int c8 = (int)(wg - (long long)row * wpr) * 32 + lane;
    if (row >= G.ny) return;
    const bool active = c8 < n8 && 8 * c8 < G.nx;
    const int x0 = 8 * c8;
    const int ym = row == 0 ? G.ny - 1 : row - 1, yp = row == G.ny - 1 ? 0 : row + 1;
    F8 g0{}, a1{}, g2{}, a3{}, g4{};
    if (active) {
        g0 = load8<ST>(a.in, 0, row, c8);
        a1 = load8<ST>(a.in, 1, row, c8);
        g2 = load8<ST>(a.in, 2, ym, c8);
        a3 = load8<ST>(a.in, 3, row, c8);
        g4 = load8<ST>(a.in, 4, yp, c8);
    }
    float prev = __shfl_up_sync(FULL, a1.v[7], 1);
    float next = __shfl_down_sync(FULL, a3.v[0], 1);
    if (lane == 0 && active) prev = C::load1(a.in, 1, row, c8 == 0 ? G.nx - 1 : x0 - 1);
    if (lane == 31 && x0 + 8 < G.nx) next = C::load1(a.in, 3, row, x0 + 8);
    if (!active) return;
    F8 g1, g3;
    g1.v[0] = prev;
#pragma unroll
    for (int k = 1; k < 8; k++) g1.v[k] = a1.v[k - 1];
#pragma unroll
    for (int k = 0; k < 7; k++) g3.v[k] = a3.v[k + 1];
    g3.v[7] = next;
    if (x0 + 8 >= G.nx) {  // periodic wrap at x = nx-1 inside this lane's 8 sites
        const float w = C::load1(a.in, 3, row, 0);
#pragma unroll
        for (int k = 0; k < 8; k++)
            if (x0 + k == G.nx - 1) g3.v[k] = w;
    }
    const float4 cA = __ldg(reinterpret_cast<const float4 *>(a.med.cL2 + (long long)row * G.pitch) + 2 * c8);
    const float4 cB = __ldg(reinterpret_cast<const float4 *>(a.med.cL2 + (long long)row * G.pitch) + 2 * c8 + 1);
    const float cl[8] = {cA.x, cA.y, cA.z, cA.w, cB.x, cB.y, cB.z, cB.w};
    float shat[8];
#pragma unroll
    for (int k = 0; k < 8; k++) shat[k] = 0.f;
    if (MU) {
        const float *dxr = a.med.dlnmu + (long long)row * G.pitch, *dyr = a.med.dlnmu + G.plane + (long long)row * G.pitch;
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const float bx = g4.v[k] - g2.v[k], by = g1.v[k] - g3.v[k];
            shat[k] = mu_source(bx, by, __ldg(dxr + x0 + k), __ldg(dyr + x0 + k));
        }
    }
    if (a.evt.rowptr) {
        const int e0 = __ldg(a.evt.rowptr + row), e1 = __ldg(a.evt.rowptr + row + 1);
        for (int e = e0; e < e1; e++) {
            const Event ev = a.evt.ev[e];
            if ((ev.x >> 3) != c8) continue;
            const int j = ev.x & 7;
#pragma unroll
            for (int k = 0; k < 8; k++) {
                if (k != j) continue;
                if (ev.kind == 0) {
                    if (ev.comp == 2 && a.t < a.evt.nt) {
                        float jz = __ldg(a.evt.amp + (long long)ev.index * a.evt.nt + a.t);
                        if (MU) jz = __fmul_rn(jz, __ldg(a.med.mu + (long long)row * G.pitch + ev.x));
                        shat[k] = __fsub_rn(shat[k], jz);
                    }
                } else if (a.t < a.evt.cap) {
                    const float sg = ((g0.v[k] + g1.v[k]) + (g2.v[k] + g3.v[k])) + g4.v[k];
                    a.evt.traces[(long long)ev.index * a.evt.cap + a.t] =
                        field2d(ev.comp, cl[k], sg, g4.v[k] - g2.v[k], g1.v[k] - g3.v[k]);
                }
            }
        }
    }
    F8 o0, o1, o2, o3, o4;
    // rows without a source (and mu uniform) have S^ = +0 everywhere: collide2d_free gives the same bits
    const bool src = MU || (a.evt.rowptr && __ldg(a.evt.rowptr + row) != __ldg(a.evt.rowptr + row + 1));
    if (src) {
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const Out5 o = collide2d(g0.v[k], g1.v[k], g2.v[k], g3.v[k], g4.v[k], cl[k], shat[k]);
            o0.v[k] = o.o0;
            o1.v[k] = o.o1;
            o2.v[k] = o.o2;
            o3.v[k] = o.o3;
            o4.v[k] = o.o4;
        }
    } else {
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const Out5 o = collide2d_free(g0.v[k], g1.v[k], g2.v[k], g3.v[k], g4.v[k], cl[k]);
            o0.v[k] = o.o0;
            o1.v[k] = o.o1;
            o2.v[k] = o.o2;
            o3.v[k] = o.o3;
            o4.v[k] = o.o4;
        }
    }
    store8<ST>(a.out, 0, row, c8, o0);
    store8<ST>(a.out, 1, row, c8, o1);
    store8<ST>(a.out, 2, row, c8, o2);
    store8<ST>(a.out, 3, row, c8, o3);
    store8<ST>(a.out, 4, row, c8, o4);
}

template <int ST, bool MU>
static cudaError_t launch_w8(const StepArgs &a, cudaStream_t s, int minb) {
    const int n8 = (a.g.nx + 7) / 8, n8p = (n8 + 31) / 32 * 32;
    const long long warps = (long long)a.g.ny * (n8p / 32);
    const unsigned blocks = (unsigned)((warps * 32 + BLOCK - 1) / BLOCK);
    // minb: registers capped so that minb blocks of 256 threads are resident per SM
    if (minb == 5) step2d_w8<ST, MU, 5><<<blocks, BLOCK, 0, s>>>(a);
    else if (minb == 4) step2d_w8<ST, MU, 4><<<blocks, BLOCK, 0, s>>>(a);
    else step2d_w8<ST, MU, 1><<<blocks, BLOCK, 0, s>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ launchers
static const int kRows2d[] = {1, 2, 4};
// rows per warp 1, 2, 4; 3 = persistent pipelined; 4 = cp.async staged; 5 = 8 sites per lane (16-bit storage);
// 6, 7 = variant 5 with registers capped for 4 / 5 resident blocks per SM
int nvariants_2d() { return 8; }

template <int ST, bool MU>
static cudaError_t launch_st(const StepArgs &a, int variant, cudaStream_t s) {
    if (variant == 3) return launch_pipe<ST, MU>(a, s);
    if (variant == 4) return launch_async<ST, MU>(a, s);
    if (variant >= 5 && variant <= 7) {
        if (ST == LBEM_F32) variant = 0;  // FP32 already issues 16-byte loads with 4 sites per lane
        else return launch_w8<ST, MU>(a, s, variant == 5 ? 1 : variant - 2);
    }
    const int R = kRows2d[variant];
    const long long warps = (long long)((a.g.ny + R - 1) / R) * (a.g.nchunk_pad / 32);
    const long long blocks = (warps * 32 + BLOCK - 1) / BLOCK;
    switch (R) {
        case 1: step2d<ST, MU, 1><<<(unsigned)blocks, BLOCK, 0, s>>>(a); break;
        case 2: step2d<ST, MU, 2><<<(unsigned)blocks, BLOCK, 0, s>>>(a); break;
        default: step2d<ST, MU, 4><<<(unsigned)blocks, BLOCK, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_step_2d(const StepArgs &a, int storage, bool has_mu, int variant, cudaStream_t s) {
    if (variant < 0 || variant >= nvariants_2d()) variant = 0;
#define LBEM_CASE(ST)                                                                               \
    case ST: return has_mu ? launch_st<ST, true>(a, variant, s) : launch_st<ST, false>(a, variant, s);
    switch (storage) {
        LBEM_CASE(LBEM_F32)
        LBEM_CASE(LBEM_F16)
        LBEM_CASE(LBEM_BF16)
        LBEM_CASE(LBEM_I16B)
        default: return cudaErrorInvalidValue;
    }
#undef LBEM_CASE
}

// ------------------------------------------------------------------ walls in the state's readout
// The stored state is post-collision: site x pulls g_i(x) = buf_i(x - c_i).  Across a wall (walls.cu) the pull is
// the site's own opposite population times the wall sign: g_i(x) = s buf_opp(i)(x).
__device__ __forceinline__ int opp2d(int i) { return i == 0 ? 0 : (i <= 2 ? i + 2 : i - 2); }
__device__ __forceinline__ float wall_sign(int kind) { return kind == 1 ? -1.f : 1.f; }

// ------------------------------------------------------------------ initial state: buf_i(x) = g^(0)_i(x + c_i)
// (with walls, where x + c_i lies beyond a wall, buf_i(x) is what site x pulls back: s g^(0)_opp(i)(x))
// (anisotropic medium, ratio r = c_x / c_y: moving particles of axis x get (r/2)(Lambda + c_x B_y), of axis y
// (1/(2r))(Lambda - c_y B_x), the rest one (w0/c^2) Lambda with w0 = 1 - c^2 (r + 1/r))
template <int ST>
__global__ void __launch_bounds__(BLOCK) init2d(Grid G, PopBuf out, const float *cL2, const float *E, const float *B,
                                                long long nsite, Walls w, float r) {
    using C = Codec<ST>;
    const long long tid = (long long)blockIdx.x * BLOCK + threadIdx.x;
    const int row = (int)(tid / G.nchunk_pad);
    const int c = (int)(tid - (long long)row * G.nchunk_pad);
    if (row >= G.ny || c >= G.nchunk) return;
    const int cx[5] = {0, 1, 0, -1, 0}, cy[5] = {0, 0, 1, 0, -1};
    for (int i = 0; i < 5; i++) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int j = 0; j < 4; j++) {
            const int x = 4 * c + j;
            if (x >= G.nx) break;
            int xs = x + cx[i], ys = row + cy[i], ie = i;
            float sg = 1.f;
            if (w.kind[0] && (xs < 0 || xs >= G.nx)) {
                xs = x;
                ie = opp2d(i);
                sg = wall_sign(w.kind[0]);
            } else if (w.kind[1] && (ys < 0 || ys >= G.ny)) {
                ys = row;
                ie = opp2d(i);
                sg = wall_sign(w.kind[1]);
            }
            xs = (xs + G.nx) % G.nx;
            ys = (ys + G.ny) % G.ny;
            const long long sd = (long long)ys * G.nx + xs;
            const float cl = cL2[(long long)ys * G.pitch + xs];
            const float Lam = E ? -E[2 * nsite + sd] : 0.f;
            const float bx = B ? B[sd] : 0.f, by = B ? B[nsite + sd] : 0.f;
            // Eq. 8: g^(0)_i = (w_i / c_L^2) [Lambda + c_ix B_y - c_iy B_x]
            float wc;
            if (r == 1.f) wc = (ie == 0) ? (1.f - 2.f * cl) / cl : 0.5f;
            else wc = (ie == 0) ? (1.f - (r + 1.f / r) * cl) / cl : (cx[ie] ? 0.5f * r : 0.5f / r);
            set(v, j, sg * (wc * (Lam + cx[ie] * by - cy[ie] * bx)));
        }
        C::store4(out, i, row, c, v);
    }
}

static Walls handle_walls(const lbem_t *h) {
    Walls w;
    w.kind[0] = h->bc[0];
    w.kind[1] = h->bc[1];
    return w;
}

cudaError_t launch_init_2d(const lbem_t *h, const float *E, const float *B, cudaStream_t s) {
    const Grid &G = h->grid;
    const long long n = (long long)G.ny * G.nchunk_pad;
    const unsigned blocks = (unsigned)((n + BLOCK - 1) / BLOCK);
    const PopBuf &o = h->buf[h->cur];
    const Walls w = handle_walls(h);
    const float r = h->aniso_r;
    switch (h->storage) {
        case LBEM_F32: init2d<LBEM_F32><<<blocks, BLOCK, 0, s>>>(G, o, h->cL2, E, B, h->nsite, w, r); break;
        case LBEM_F16: init2d<LBEM_F16><<<blocks, BLOCK, 0, s>>>(G, o, h->cL2, E, B, h->nsite, w, r); break;
        case LBEM_BF16: init2d<LBEM_BF16><<<blocks, BLOCK, 0, s>>>(G, o, h->cL2, E, B, h->nsite, w, r); break;
        default: init2d<LBEM_I16B><<<blocks, BLOCK, 0, s>>>(G, o, h->cL2, E, B, h->nsite, w, r); break;
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------ field extraction (dense [3][nsite] outputs)
template <int ST>
__global__ void __launch_bounds__(BLOCK) fields2d(Grid G, PopBuf in, const float *cL2, float *E, float *B,
                                                  long long nsite, Walls w, const float *Pz, float r) {
    using C = Codec<ST>;
    const int lane = threadIdx.x & 31;
    const long long wg = ((long long)blockIdx.x * BLOCK + threadIdx.x) >> 5;
    const int wpr = G.nchunk_pad >> 5;
    const int row = (int)(wg / wpr);
    const int c = (int)(wg - (long long)row * wpr) * 32 + lane;
    if (row >= G.ny) return;
    float4 g[5];
    pull2d<ST>(in, G, row, c, lane, g);
    if (c >= G.nchunk) return;
    const float4 cl = __ldg(reinterpret_cast<const float4 *>(cL2 + (long long)row * G.pitch) + c);
    for (int j = 0; j < 4; j++) {
        const int x = 4 * c + j;
        if (x >= G.nx) break;
        // pulls across a wall
        if (w.kind[0] && x == 0) set(g[1], j, wall_sign(w.kind[0]) * C::load1(in, 3, row, x));
        if (w.kind[0] && x == G.nx - 1) set(g[3], j, wall_sign(w.kind[0]) * C::load1(in, 1, row, x));
        if (w.kind[1] && row == 0) set(g[2], j, wall_sign(w.kind[1]) * C::load1(in, 4, row, x));
        if (w.kind[1] && row == G.ny - 1) set(g[4], j, wall_sign(w.kind[1]) * C::load1(in, 2, row, x));
        const long long sd = (long long)row * G.nx + x;
        const float s = ((get(g[0], j) + get(g[1], j)) + (get(g[2], j) + get(g[3], j))) + get(g[4], j);
        if (E) {
            E[sd] = 0.f;
            E[nsite + sd] = 0.f;
            const float ez = -get(cl, j) * s;
            E[2 * nsite + sd] = Pz ? __fsub_rn(ez, Pz[(long long)row * G.pitch + x]) : ez;  // E = D/eps_inf - P
        }
        if (B) {  // anisotropic medium: B_x = r (g_4 - g_2), B_y = (g_1 - g_3) / r
            const float bx = get(g[4], j) - get(g[2], j), by = get(g[1], j) - get(g[3], j);
            B[sd] = r == 1.f ? bx : __fmul_rn(r, bx);
            B[nsite + sd] = r == 1.f ? by : __fmul_rn(__fdiv_rn(1.f, r), by);
            B[2 * nsite + sd] = 0.f;
        }
    }
}

cudaError_t launch_fields_2d(const lbem_t *h, float *E, float *B, cudaStream_t s) {
    const Grid &G = h->grid;
    const long long warps = (long long)G.ny * (G.nchunk_pad / 32);
    const unsigned blocks = (unsigned)((warps * 32 + BLOCK - 1) / BLOCK);
    const PopBuf &in = h->buf[h->cur];
    const Walls w = handle_walls(h);
    const float *Pz = h->disp ? h->pole_P(h->cur) : nullptr;
    const float r = h->aniso_r;
    switch (h->storage) {
        case LBEM_F32: fields2d<LBEM_F32><<<blocks, BLOCK, 0, s>>>(G, in, h->cL2, E, B, h->nsite, w, Pz, r); break;
        case LBEM_F16: fields2d<LBEM_F16><<<blocks, BLOCK, 0, s>>>(G, in, h->cL2, E, B, h->nsite, w, Pz, r); break;
        case LBEM_BF16: fields2d<LBEM_BF16><<<blocks, BLOCK, 0, s>>>(G, in, h->cL2, E, B, h->nsite, w, Pz, r); break;
        default: fields2d<LBEM_I16B><<<blocks, BLOCK, 0, s>>>(G, in, h->cL2, E, B, h->nsite, w, Pz, r); break;
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------ FP64 diagnostics
template <int ST>
__device__ __forceinline__ double pop2d(const PopBuf &in, const Grid &G, const Walls &w, int i, int x, int y) {
    // pre-collision g_i at (x, y): buf_i(x - c_i), or s buf_opp(i)(x, y) across a wall
    const int cx[5] = {0, 1, 0, -1, 0}, cy[5] = {0, 0, 1, 0, -1};
    const int xu = x - cx[i], yu = y - cy[i];
    if (w.kind[0] && (xu < 0 || xu >= G.nx))
        return (double)wall_sign(w.kind[0]) * (double)Codec<ST>::load1(in, opp2d(i), y, x);
    if (w.kind[1] && (yu < 0 || yu >= G.ny))
        return (double)wall_sign(w.kind[1]) * (double)Codec<ST>::load1(in, opp2d(i), y, x);
    const int xs = (xu + G.nx) % G.nx, ys = (yu + G.ny) % G.ny;
    return (double)Codec<ST>::load1(in, i, ys, xs);
}

template <int ST>
__device__ __forceinline__ void bfield2d(const PopBuf &in, const Grid &G, const Walls &w, int x, int y, double &bx,
                                         double &by) {
    bx = pop2d<ST>(in, G, w, 4, x, y) - pop2d<ST>(in, G, w, 2, x, y);
    by = pop2d<ST>(in, G, w, 1, x, y) - pop2d<ST>(in, G, w, 3, x, y);
}

__device__ __forceinline__ double block_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < BLOCK / 32; k++) r += sh[k];
    return r;  // valid in thread 0
}

template <int ST>
__global__ void __launch_bounds__(BLOCK) diag2d(Grid G, PopBuf in, const float *cL2, double *partials, Walls w,
                                                const float *Pz, float r) {
    __shared__ double sh[BLOCK / 32];
    double en = 0.0, inv = 0.0, dv = 0.0;
    const long long nsite = (long long)G.nx * G.ny;
    for (long long s = (long long)blockIdx.x * BLOCK + threadIdx.x; s < nsite; s += (long long)gridDim.x * BLOCK) {
        const int y = (int)(s / G.nx), x = (int)(s - (long long)y * G.nx);
        double g[5], sum = 0.0;
        for (int i = 0; i < 5; i++) {
            g[i] = pop2d<ST>(in, G, w, i, x, y);
            sum += g[i];
        }
        const double cl = (double)cL2[(long long)y * G.pitch + x];
        const double rd = r, Ez = -cl * sum - (Pz ? (double)Pz[(long long)y * G.pitch + x] : 0.0), bx = rd * (g[4] - g[2]),
                     by = (g[1] - g[3]) / rd;
        en += bx * bx + by * by + Ez * Ez / cl;  // c_eff^2 = c_L^2 in 2D
        // weights: c_x^2 / 2 = r c_L^2 / 2 for x-movers, c_L^2 / (2 r) for y-movers (r = 1: isotropic)
        const double w0 = 1.0 - (rd + 1.0 / rd) * cl, wx = 0.5 * rd * cl, wy = 0.5 * cl / rd;
        double q = (g[1] * g[1] + g[3] * g[3]) / wx + (g[2] * g[2] + g[4] * g[4]) / wy;
        if (w0 != 0.0) q += g[0] * g[0] / w0;
        inv += 2.0 * q;  // g_xy and g_yx = -g_xy both count
        double bxp, byp, bxm, bym, t1, t2;
        // (periodic central differences, also next to walls)
        bfield2d<ST>(in, G, w, (x + 1) % G.nx, y, bxp, t1);
        bfield2d<ST>(in, G, w, (x - 1 + G.nx) % G.nx, y, bxm, t2);
        bfield2d<ST>(in, G, w, x, (y + 1) % G.ny, t1, byp);
        bfield2d<ST>(in, G, w, x, (y - 1 + G.ny) % G.ny, t2, bym);
        const double div = 0.5 * (bxp - bxm) + 0.5 * (byp - bym);
        dv += div * div;
    }
    const double a = block_sum(en, sh), b = block_sum(inv, sh), c = block_sum(dv, sh);
    if (threadIdx.x == 0) {
        partials[3 * blockIdx.x + 0] = a;
        partials[3 * blockIdx.x + 1] = b;
        partials[3 * blockIdx.x + 2] = c;
    }
}

// The same three sums for a periodic grid (no walls), rows strided over the blocks and columns over the threads:
// the energy and sum g^2/w terms of a site formed in FP32 (its pulled FP32 populations, one division each) and
// added in FP64; the divergence from the eight FP32 populations its four neighbours' B need, differenced in FP64
// (each B component is exact there).  GB300's FP64 rate made the all-FP64 site terms of diag2d the cost of a call.
template <int ST>
__global__ void __launch_bounds__(BLOCK) diag2d_periodic(Grid G, PopBuf in, const float *cL2, double *partials,
                                                         const float *Pz, float r) {
    __shared__ double sh[BLOCK / 32];
    double en = 0.0, inv = 0.0, dv = 0.0;
    const float ri = 1.f / r;
    const double fs64 = (double)r + 1.0 / (double)r;  // for w0 of an anisotropic medium (it can be small there)
    for (int y = blockIdx.x; y < G.ny; y += gridDim.x) {
        const int ym = y == 0 ? G.ny - 1 : y - 1, yp = y + 1 == G.ny ? 0 : y + 1;
        for (int x = threadIdx.x; x < G.nx; x += BLOCK) {
            const int xm = x == 0 ? G.nx - 1 : x - 1, xp = x + 1 == G.nx ? 0 : x + 1;
            const float g0 = Codec<ST>::load1(in, 0, y, x), g1 = Codec<ST>::load1(in, 1, y, xm),
                        g2 = Codec<ST>::load1(in, 2, ym, x), g3 = Codec<ST>::load1(in, 3, y, xp),
                        g4 = Codec<ST>::load1(in, 4, yp, x);
            const long long o = (long long)y * G.pitch + x;
            const float cl = cL2[o];
            const float Ez = -cl * (((g0 + g1) + (g2 + g3)) + g4) - (Pz ? Pz[o] : 0.f);
            const float bx = r * (g4 - g2), by = (g1 - g3) * ri;
            en += (double)(bx * bx + by * by + Ez * Ez / cl);
            const float wx = 0.5f * r * cl, wy = 0.5f * cl * ri;
            const float q = (g1 * g1 + g3 * g3) / wx + (g2 * g2 + g4 * g4) / wy;
            double q0 = 0.0;  // g0^2 / w0; isotropic w0 = 1 - 2 c_L^2 is exact in FP32 wherever it is below 1/2
            if (r == 1.f) {
                const float w0 = 1.f - 2.f * cl;
                if (w0 != 0.f) q0 = (double)(g0 * g0 / w0);
            } else {
                const double w0 = 1.0 - fs64 * (double)cl;
                if (w0 != 0.0) q0 = (double)g0 * (double)g0 / w0;
            }
            inv += 2.0 * ((double)q + q0);  // g_xy and g_yx = -g_xy both count
            // B at the four neighbours: B_x = g4 - g2 at (x +- 1, y), B_y = g1 - g3 at (x, y +- 1)
            const double bxp = (double)Codec<ST>::load1(in, 4, yp, xp) - (double)Codec<ST>::load1(in, 2, ym, xp);
            const double bxm = (double)Codec<ST>::load1(in, 4, yp, xm) - (double)Codec<ST>::load1(in, 2, ym, xm);
            const double byp = (double)Codec<ST>::load1(in, 1, yp, xm) - (double)Codec<ST>::load1(in, 3, yp, xp);
            const double bym = (double)Codec<ST>::load1(in, 1, ym, xm) - (double)Codec<ST>::load1(in, 3, ym, xp);
            const double div = 0.5 * (bxp - bxm) + 0.5 * (byp - bym);
            dv += div * div;
        }
    }
    const double a = block_sum(en, sh), b = block_sum(inv, sh), c = block_sum(dv, sh);
    if (threadIdx.x == 0) {
        partials[3 * blockIdx.x + 0] = a;
        partials[3 * blockIdx.x + 1] = b;
        partials[3 * blockIdx.x + 2] = c;
    }
}

cudaError_t launch_diag_2d(const lbem_t *h, double *partials, int nblocks, cudaStream_t s) {
    const PopBuf &in = h->buf[h->cur];
    const Walls w = handle_walls(h);
    const float *Pz = h->disp ? h->pole_P(h->cur) : nullptr;
    const float r = h->aniso_r;
    if (!w.kind[0] && !w.kind[1]) {
        switch (h->storage) {
            case LBEM_F32: diag2d_periodic<LBEM_F32><<<nblocks, BLOCK, 0, s>>>(h->grid, in, h->cL2, partials, Pz, r); break;
            case LBEM_F16: diag2d_periodic<LBEM_F16><<<nblocks, BLOCK, 0, s>>>(h->grid, in, h->cL2, partials, Pz, r); break;
            case LBEM_BF16: diag2d_periodic<LBEM_BF16><<<nblocks, BLOCK, 0, s>>>(h->grid, in, h->cL2, partials, Pz, r); break;
            default: diag2d_periodic<LBEM_I16B><<<nblocks, BLOCK, 0, s>>>(h->grid, in, h->cL2, partials, Pz, r); break;
        }
        return cudaGetLastError();
    }
    switch (h->storage) {
        case LBEM_F32: diag2d<LBEM_F32><<<nblocks, BLOCK, 0, s>>>(h->grid, in, h->cL2, partials, w, Pz, r); break;
        case LBEM_F16: diag2d<LBEM_F16><<<nblocks, BLOCK, 0, s>>>(h->grid, in, h->cL2, partials, w, Pz, r); break;
        case LBEM_BF16: diag2d<LBEM_BF16><<<nblocks, BLOCK, 0, s>>>(h->grid, in, h->cL2, partials, w, Pz, r); break;
        default: diag2d<LBEM_I16B><<<nblocks, BLOCK, 0, s>>>(h->grid, in, h->cL2, partials, w, Pz, r); break;
    }
    return cudaGetLastError();
}

}  // namespace lbk
