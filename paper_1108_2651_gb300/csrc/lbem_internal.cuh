// Internal declarations of the lbem CUDA library (not part of the C ABI).
//
// Data layout in device memory (structure of arrays):
//   * The distribution is stored as one plane per independent component:
//     2D: 5 planes g_i = g_{i,xy} (i = 0..4, the D2Q5 order of the paper's
//     Sec. "Lattice BGK formulation"); 3D: 21 planes h_{i,gamma} =
//     (g_{i,yz}, g_{i,zx}, g_{i,xy}), plane index i*3 + gamma, i = 0..6 with
//     c_1..c_3 = +x,+y,+z and c_4..c_6 = -x,-y,-z.
//   * A plane is nrows = ny*nz rows of `pitch` elements, pitch = nx rounded up
//     to a multiple of 32 (128-byte aligned FP32 rows).  Threads: a row is cut
//     into nchunk = ceil(nx/4) chunks of 4 sites, one per lane, padded to
//     nchunk_pad = 32*ceil(nchunk/32) lanes, so one warp covers 128
//     consecutive sites of one row; lanes past the row end load nothing.
//   * Ping-pong: buffer `cur` holds the post-collision values g'_i(x, t-1)
//     stored at the WRITING site x; the pre-collision state at time t is
//     g_i(x, t) = buf[i](x - c_i) (pull streaming, Eq. 18).
//   * Medium: c_L^2 per site in a pitched plane (FP32); mu and grad ln mu
//     planes only when a non-uniform mu was given.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/lbem.h"

namespace lbk {

constexpr unsigned FULL = 0xffffffffu;
constexpr int BLOCK = 256;  // threads per block of the stencil kernels

// ------------------------------------------------------------------ storage
struct PopBuf {
    void *data = nullptr;    // npop planes of elements (float / half / bf16 / int16)
    int8_t *ex = nullptr;    // LBEM_I16B: npop planes of per-chunk exponents
    long long plane = 0;     // elements per plane
    long long explane = 0;   // exponent bytes per plane
    int pitch = 0;           // elements per row
    int expitch = 0;         // exponents per row (= pitch / 4)
    float scale = 1.f;       // LBEM_F16: stored = scale * value
    float inv_scale = 1.f;
};

template <int ST>
struct Codec;

template <>
struct Codec<LBEM_F32> {
    static constexpr int bytes = 4;
    __device__ static __forceinline__ float4 load4(const PopBuf &b, int p, int row, int c) {
        const float4 *q = reinterpret_cast<const float4 *>(static_cast<const float *>(b.data) + p * b.plane +
                                                           (long long)row * b.pitch);
        return __ldg(q + c);
    }
    __device__ static __forceinline__ float load1(const PopBuf &b, int p, int row, int x) {
        return __ldg(static_cast<const float *>(b.data) + p * b.plane + (long long)row * b.pitch + x);
    }
    __device__ static __forceinline__ void store4(const PopBuf &b, int p, int row, int c, float4 v) {
        float4 *q = reinterpret_cast<float4 *>(static_cast<float *>(b.data) + p * b.plane + (long long)row * b.pitch);
        __stcs(q + c, v);
    }
};

__device__ __forceinline__ float4 h4_to_f4(uint2 r) {
    __half2 a = *reinterpret_cast<__half2 *>(&r.x), c = *reinterpret_cast<__half2 *>(&r.y);
    float2 fa = __half22float2(a), fc = __half22float2(c);
    return make_float4(fa.x, fa.y, fc.x, fc.y);
}

template <>
struct Codec<LBEM_F16> {
    static constexpr int bytes = 2;
    __device__ static __forceinline__ float4 load4(const PopBuf &b, int p, int row, int c) {
        const uint2 *q = reinterpret_cast<const uint2 *>(static_cast<const __half *>(b.data) + p * b.plane +
                                                         (long long)row * b.pitch);
        float4 v = h4_to_f4(__ldg(q + c));
        return make_float4(v.x * b.inv_scale, v.y * b.inv_scale, v.z * b.inv_scale, v.w * b.inv_scale);
    }
    __device__ static __forceinline__ float load1(const PopBuf &b, int p, int row, int x) {
        const __half *q = static_cast<const __half *>(b.data) + p * b.plane + (long long)row * b.pitch + x;
        return __half2float(__ldg(q)) * b.inv_scale;
    }
    __device__ static __forceinline__ uint2 enc4(const PopBuf &b, float4 v) {
        __half2 a = __floats2half2_rn(v.x * b.scale, v.y * b.scale);
        __half2 d = __floats2half2_rn(v.z * b.scale, v.w * b.scale);
        uint2 r;
        r.x = *reinterpret_cast<unsigned *>(&a);
        r.y = *reinterpret_cast<unsigned *>(&d);
        return r;
    }
    __device__ static __forceinline__ void store4(const PopBuf &b, int p, int row, int c, float4 v) {
        uint2 *q = reinterpret_cast<uint2 *>(static_cast<__half *>(b.data) + p * b.plane + (long long)row * b.pitch);
        __stcs(q + c, enc4(b, v));
    }
};

template <>
struct Codec<LBEM_BF16> {
    static constexpr int bytes = 2;
    __device__ static __forceinline__ float4 load4(const PopBuf &b, int p, int row, int c) {
        const uint2 *q = reinterpret_cast<const uint2 *>(static_cast<const __nv_bfloat16 *>(b.data) + p * b.plane +
                                                         (long long)row * b.pitch);
        uint2 r = __ldg(q + c);
        // bf16 -> f32 is a 16-bit left shift of the bit pattern
        return make_float4(__uint_as_float(r.x << 16), __uint_as_float(r.x & 0xffff0000u),
                           __uint_as_float(r.y << 16), __uint_as_float(r.y & 0xffff0000u));
    }
    __device__ static __forceinline__ float load1(const PopBuf &b, int p, int row, int x) {
        const unsigned short *q = reinterpret_cast<const unsigned short *>(
            static_cast<const __nv_bfloat16 *>(b.data) + p * b.plane + (long long)row * b.pitch + x);
        return __uint_as_float(((unsigned)__ldg(q)) << 16);
    }
    __device__ static __forceinline__ uint2 enc4(const PopBuf &b, float4 v) {
        (void)b;
        __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y);
        __nv_bfloat162 d = __floats2bfloat162_rn(v.z, v.w);
        uint2 r;
        r.x = *reinterpret_cast<unsigned *>(&a);
        r.y = *reinterpret_cast<unsigned *>(&d);
        return r;
    }
    __device__ static __forceinline__ void store4(const PopBuf &b, int p, int row, int c, float4 v) {
        uint2 *q = reinterpret_cast<uint2 *>(static_cast<__nv_bfloat16 *>(b.data) + p * b.plane +
                                             (long long)row * b.pitch);
        __stcs(q + c, enc4(b, v));
    }
};

// Block floating point: 4 consecutive sites of one plane row share exponent e
// (int8); value = q * 2^(e - 15), q an int16 with |q| <= 32767.  Encoding picks
// e = floor(log2(max|v|)) + 1, so max|v| < 2^e and q = rint(v * 2^(15 - e)):
// the quantisation step is 2^-15 of the power of two above the block maximum.
// Blocks whose maximum is below 2^-100 are stored as zero (e = -128).
constexpr int I16B_ZERO = -128;

__device__ __forceinline__ float pow2f(int k) {  // 2^k for -126 <= k <= 127
    return __int_as_float((k + 127) << 23);
}

// Exact int16 <-> float conversions on the FP32 adder instead of the reduced-rate
// conversion unit: for |q| < 2^22 the float 1.5*2^23 + q has q in its low mantissa
// bits, and adding 1.5*2^23 to a float of magnitude < 2^22 rounds it to the nearest
// integer (ties to even), exactly as __float2int_rn does.
constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23
constexpr int kMagicBits = 0x4B400000;
__device__ __forceinline__ float i16_to_f(int q) { return __int_as_float(kMagicBits + q) - kMagic; }
__device__ __forceinline__ int f_to_int_rn(float v) { return __float_as_int(v + kMagic) - kMagicBits; }

// The factor 2^(e-15) of a block-int16 block with exponent e, 0 for a zero block (e = -128): the encoder writes
// e in [-99, 100] or 127, so e + 112 is a positive biased exponent, and max(e + 112, 0) maps e = -128 to +0.
__device__ __forceinline__ float i16b_factor(int e) { return __int_as_float(max(e + 112, 0) << 23); }

// Block-int16 decoding of the two values packed in w (low half first), f = 2^(e-15) (0 for a zero block):
// h ^ 0x8000 = q + 2^15 placed under the exponent of 1.5 * 2^23 gives the float 1.5 * 2^23 + 2^15 + q exactly,
// and one rounding of (that float) * f - (1.5 * 2^23 + 2^15) * f is q * f, the same value as float(q) * f.
constexpr float kMagic16 = 12615680.0f;  // 1.5 * 2^23 + 2^15
__device__ __forceinline__ float2 i16x2_to_f2(unsigned w, float f) {
    const unsigned u = w ^ 0x80008000u;
    const float nf = -kMagic16 * f;  // exact: f is a power of two or zero
    return make_float2(__fmaf_rn(__uint_as_float(__byte_perm(u, 0x4B40u, 0x5410)), f, nf),
                       __fmaf_rn(__uint_as_float(__byte_perm(u, 0x4B40u, 0x5432)), f, nf));
}

template <>
struct Codec<LBEM_I16B> {
    static constexpr int bytes = 2;
    __device__ static __forceinline__ float4 load4(const PopBuf &b, int p, int row, int c) {
        const uint2 *q = reinterpret_cast<const uint2 *>(static_cast<const int16_t *>(b.data) + p * b.plane +
                                                         (long long)row * b.pitch);
        uint2 r = __ldg(q + c);
        const float f = i16b_factor(__ldg(b.ex + p * b.explane + (long long)row * b.expitch + c));
        const float2 lo = i16x2_to_f2(r.x, f), hi = i16x2_to_f2(r.y, f);
        return make_float4(lo.x, lo.y, hi.x, hi.y);
    }
    __device__ static __forceinline__ float load1(const PopBuf &b, int p, int row, int x) {
        short v = __ldg(static_cast<const short *>(b.data) + p * b.plane + (long long)row * b.pitch + x);
        int e = __ldg(b.ex + p * b.explane + (long long)row * b.expitch + (x >> 2));
        return (e == I16B_ZERO) ? 0.f : i16_to_f(v) * pow2f(e - 15);
    }
    // encoded 4-site block: mantissas in r, exponent returned
    __device__ static __forceinline__ int enc4e(float4 v, uint2 &r) {
        const float m = fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w)));
        // the ordinary block, computed for every block (no divergent branches); the two special cases below
        // replace its result.  For 2^-100 <= m < 2^100 the exponent e lies in [-99, 100], so the clamp is idle.
        const int e = ((__float_as_int(m) >> 23) & 0xff) - 127 + 1;
        const float s = pow2f(15 - min(max(e, -99), 100));
        // |v * s| <= 2^15 here; clamping to the integers +-32767 before the rounding equals clamping after it.
        // The adder-based rounding leaves q in the low 16 bits of the sum's bit pattern (two's complement).
        const unsigned b0 = __float_as_uint(fminf(fmaxf(__fmul_rn(v.x, s), -32767.f), 32767.f) + kMagic);
        const unsigned b1 = __float_as_uint(fminf(fmaxf(__fmul_rn(v.y, s), -32767.f), 32767.f) + kMagic);
        const unsigned b2 = __float_as_uint(fminf(fmaxf(__fmul_rn(v.z, s), -32767.f), 32767.f) + kMagic);
        const unsigned b3 = __float_as_uint(fminf(fmaxf(__fmul_rn(v.w, s), -32767.f), 32767.f) + kMagic);
        const bool huge = !(m < 0x1p+100f);  // huge or NaN: saturate, so the state stays visibly wrong
        const bool tiny = m < 0x1p-100f;     // negligible block -> exact zero
        r.x = huge ? 0x7fff7fffu : tiny ? 0u : __byte_perm(b0, b1, 0x5410);
        r.y = huge ? 0x7fff7fffu : tiny ? 0u : __byte_perm(b2, b3, 0x5410);
        return huge ? 127 : tiny ? I16B_ZERO : e;
    }
    __device__ static __forceinline__ void store4(const PopBuf &b, int p, int row, int c, float4 v) {
        uint2 r;
        const int e = enc4e(v, r);
        uint2 *q = reinterpret_cast<uint2 *>(static_cast<int16_t *>(b.data) + p * b.plane + (long long)row * b.pitch);
        __stcs(q + c, r);
        b.ex[p * b.explane + (long long)row * b.expitch + c] = (int8_t)e;
    }
};

__device__ __forceinline__ float get(const float4 &v, int j) {
    return j == 0 ? v.x : (j == 1 ? v.y : (j == 2 ? v.z : v.w));
}
__device__ __forceinline__ void set(float4 &v, int j, float a) {
    if (j == 0) v.x = a;
    else if (j == 1) v.y = a;
    else if (j == 2) v.z = a;
    else v.w = a;
}

// ------------------------------------------------------------------ 2D site update
// Collision of one D2Q5 site at tau = dt/2 (Eqs. 8 and 17 in closed form, derived in kernels2d.cu), used by
// every 2D kernel so that all launch shapes compute bit-identical results.  shat = S^ (zero without sources).
struct Out5 {
    float o0, o1, o2, o3, o4;
};
// Written with explicitly rounded operations (never contracted into FMAs), so that every kernel that calls it
// performs the same sequence of roundings whatever the compiler schedules around it.
__device__ __forceinline__ Out5 collide2d(float g0, float g1, float g2, float g3, float g4, float cl, float shat) {
    const float s = __fadd_rn(__fadd_rn(__fadd_rn(g0, g1), __fadd_rn(g2, g3)), g4);
    const float L = __fmul_rn(cl, s);
    const float w0 = __fsub_rn(1.f, 2.f * cl);          // 2 cl is exact
    const float Tm = __fmul_rn(-0.5f * cl, shat);        // -cl/2 is exact
    const float T0 = __fmul_rn(-w0, shat);
    Out5 o;
    o.o1 = __fadd_rn(__fsub_rn(L, g3), Tm);
    o.o3 = __fadd_rn(__fsub_rn(L, g1), Tm);
    o.o2 = __fadd_rn(__fsub_rn(L, g4), Tm);
    o.o4 = __fadd_rn(__fsub_rn(L, g2), Tm);
    o.o0 = __fadd_rn(__fsub_rn(__fmul_rn(2.f * w0, s), g0), T0);  // 2 w0 is exact
    return o;
}

// The site update of the general kernel (general.cu), in its exact operation order: per-axis speeds
// c_x^2 = r c^2, c_y^2 = c^2 / r (ri = 1/r, fs = r + 1/r; r = 1 isotropic) and the pole's P at t (+0 without a
// pole, its terms kept so that zeros keep their signs).
__device__ __forceinline__ Out5 collide2d_an(float g0, float g1, float g2, float g3, float g4, float cl, float shat,
                                             float r, float ri, float fs, float P = 0.f) {
    const float sig = __fadd_rn(__fadd_rn(__fadd_rn(g0, g1), __fadd_rn(g2, g3)), g4);
    const float Lam = __fadd_rn(__fmul_rn(cl, sig), P);
    const float Lx = __fmul_rn(r, Lam), Ly = __fmul_rn(ri, Lam);
    const float w0 = __fsub_rn(1.f, __fmul_rn(fs, cl));
    const float Tm = __fmul_rn(-0.5f * cl, shat), T0 = __fmul_rn(-w0, shat);
    const float Tx = __fmul_rn(r, Tm), Ty = __fmul_rn(ri, Tm);
    Out5 o;
    o.o0 = __fadd_rn(__fsub_rn(__fsub_rn(__fmul_rn(2.f * w0, sig), g0), __fmul_rn(2.f * fs, P)), T0);
    o.o1 = __fadd_rn(__fsub_rn(Lx, g3), Tx);
    o.o2 = __fadd_rn(__fsub_rn(Ly, g4), Ty);
    o.o3 = __fadd_rn(__fsub_rn(Lx, g1), Tx);
    o.o4 = __fadd_rn(__fsub_rn(Ly, g2), Ty);
    return o;
}

// One step of the dispersive pole at a site (the displacement form of the auxiliary equation, reading R17):
// E = -c_L^2 sigma - P, J <- ((1 - gam/2) J - wr^2 P + wp^2 E) / (1 + gam/2), P <- P + J, with the division
// folded into per-site coefficients computed once at upload: pa = (1 - gam/2)/(1 + gam/2), pb = wr^2/(1 + gam/2),
// pc = wp^2/(1 + gam/2) (pole_coefficients in general.cu).  Shared by the single-step general kernel and the two-step
// tile kernel so both round identically.
__device__ __forceinline__ void pole_update(float cl, float sig, float pc, float pb, float pa, float &J, float &P) {
    const float E = __fsub_rn(__fmul_rn(-cl, sig), P);
    J = __fadd_rn(__fsub_rn(__fmul_rn(pa, J), __fmul_rn(pb, P)), __fmul_rn(pc, E));
    P = __fadd_rn(P, J);
}

// collide2d_an of an isotropic medium with a pole (r = 1/r = 1, fs = 2): the products it drops are by 1, and 2 fs = 4
// is a power of two, so the results are those of collide2d_an bit for bit.
__device__ __forceinline__ Out5 collide2d_pole_iso(float g0, float g1, float g2, float g3, float g4, float cl,
                                                   float shat, float P) {
    const float sig = __fadd_rn(__fadd_rn(__fadd_rn(g0, g1), __fadd_rn(g2, g3)), g4);
    const float Lam = __fadd_rn(__fmul_rn(cl, sig), P);
    const float w0 = __fsub_rn(1.f, 2.f * cl);
    const float Tm = __fmul_rn(-0.5f * cl, shat), T0 = __fmul_rn(-w0, shat);
    Out5 o;
    o.o0 = __fadd_rn(__fsub_rn(__fsub_rn(__fmul_rn(2.f * w0, sig), g0), 4.f * P), T0);
    o.o1 = __fadd_rn(__fsub_rn(Lam, g3), Tm);
    o.o2 = __fadd_rn(__fsub_rn(Lam, g4), Tm);
    o.o3 = __fadd_rn(__fsub_rn(Lam, g1), Tm);
    o.o4 = __fadd_rn(__fsub_rn(Lam, g2), Tm);
    return o;
}

// collide2d at a site without a source (S^ = +0): there T_m and T_0 are -0 (c_L^2 > 0, w0 >= 0), and adding
// -0 leaves every value unchanged, so dropping them gives the same bits as collide2d(..., 0.f).
__device__ __forceinline__ Out5 collide2d_free(float g0, float g1, float g2, float g3, float g4, float cl) {
    const float s = __fadd_rn(__fadd_rn(__fadd_rn(g0, g1), __fadd_rn(g2, g3)), g4);
    const float L = __fmul_rn(cl, s);
    const float w0 = __fsub_rn(1.f, 2.f * cl);
    Out5 o;
    o.o1 = __fsub_rn(L, g3);
    o.o3 = __fsub_rn(L, g1);
    o.o2 = __fsub_rn(L, g4);
    o.o4 = __fsub_rn(L, g2);
    o.o0 = __fsub_rn(__fmul_rn(2.f * w0, s), g0);
    return o;
}

__device__ __forceinline__ float field2d(int comp, float cl, float s, float bx, float by) {
    switch (comp) {
        case 2: return -cl * s;  // E_z = -Lambda_xy
        case 3: return bx;
        case 4: return by;
        default: return 0.f;  // E_x, E_y, B_z are not representable in 2D
    }
}

// ------------------------------------------------------------------ site events
// Sources and receivers, sorted by row, with a CSR row pointer.  Event:
//   x     : column
//   kind  : 0 = point source (index = source k), 1 = receiver (index = receiver r)
//   comp  : source current component 0..2 / receiver field 0..5
struct Event {
    int x, kind, index, comp;
};

struct Events {
    const int *rowptr = nullptr;  // [nrows + 1] or null if no events
    const Event *ev = nullptr;
    const float *amp = nullptr;   // [nsrc][nt]
    int nt = 0;
    float *traces = nullptr;      // [nrec][cap]
    int cap = 0;
};

// ------------------------------------------------------------------ launch parameters
struct Grid {
    int nx, ny, nz, nrows;   // nrows = ny*nz
    int nchunk, nchunk_pad;  // chunks of 4 sites per row (active / padded to 32)
    int pitch;               // elements per plane row
    long long plane;         // elements per plane
};

struct Medium {
    const float *cL2 = nullptr;    // [plane]
    const float *mu = nullptr;     // [plane] or null
    const float *dlnmu = nullptr;  // [D][plane] or null
    // anisotropic medium (general.cu): r = c_x / c_y = sqrt(mu_xx / mu_yy), mubar = sqrt(mu_xx mu_yy); 1, 1: isotropic
    float ar = 1.f, amu = 1.f;
    // one dispersive pole per site (null without; pitched planes): its parameters (wp2 non-null marks a pole), the
    // per-site coefficients of its update (pole_update: pc, pb, pa), J (updated in place) and P, read from Pr
    // (time t) and written to Pw (the plane of the output state's parity)
    const float *wp2 = nullptr, *wr2 = nullptr, *gam = nullptr, *Pr = nullptr;
    const float *pc = nullptr, *pb = nullptr, *pa = nullptr;
    float *J = nullptr, *Pw = nullptr;
};

// Walls and absorbing layers (walls.cu): per axis x, y 0 = periodic, 1 = PEC wall, 2 = PMC wall; layer
// damping factors per column / row (null: no layer on that axis).
struct Walls {
    int kind[3] = {0, 0, 0};
    const float *fx = nullptr, *fy = nullptr, *fz = nullptr;
};
// What the general single-step kernel (general.cu) adds to a step: one Drude-Lorentz pole per site (parameters
// and state as planes with the grid's pitch, J at t - 1/2 (in place), P at t read from P and written to Pn; wp2
// null: no pole) and a uniform in-plane permeability tensor
// (axis speeds c_x^2 = r cbar^2, c_y^2 = cbar^2 / r with cbar^2 the stored c_L^2; mubar = sqrt(mu_xx mu_yy)).
struct General {
    const float *wp2 = nullptr, *wr2 = nullptr, *gam = nullptr;
    const float *pc = nullptr, *pb = nullptr, *pa = nullptr;  // pole_update's per-site coefficients
    float *J = nullptr;        // updated in place
    const float *P = nullptr;  // P at t
    float *Pn = nullptr;       // P at t + 1 (the other plane: neighbouring tiles of a multi-step launch read P at t)
    float r = 1.f, mubar = 1.f;
};
// Output rectangle of one edge tile: columns x0 .. x0+w-1, rows y0 .. y0+h-1.
struct EdgeTile {
    int x0, y0, w, h;
};

struct StepArgs {
    Grid g;
    PopBuf in, out;
    Medium med;
    Events evt;
    long long t;  // time of the pre-collision state being collided
    // work queue of the strip-streaming kernel (sstream.cu), two counters of the handle: [0] the next unit to take,
    // [1] the CTAs that finished; both zero between launches (the last CTA out resets them)
    int *sched = nullptr;
    // the strip-streaming kernel writes sites and receiver samples only with wx0 <= x < wx1 and wy0 <= y < wy1: with
    // walls its launches leave the bands next to them to the edge pass running beside it (everything otherwise)
    int wx0 = 0, wx1 = 1 << 30, wy0 = 0, wy1 = 1 << 30;
};

// Periodic index, cheap when v is already in range (the common case).
__device__ __forceinline__ int wrapi(int v, int n) {
    if ((unsigned)v < (unsigned)n) return v;
    v %= n;
    return v < 0 ? v + n : v;
}

// S^ of Eq. 3 from a heterogeneous permeability, B_x d_y ln mu - B_y d_x ln mu, explicitly rounded so that every
// kernel forms it with the same roundings.
__device__ __forceinline__ float mu_source(float bx, float by, float dlx, float dly) {
    return __fsub_rn(__fmul_rn(bx, dly), __fmul_rn(by, dlx));
}

// Source current at global site (x, y) and time t, and the receiver write of the pre-collision fields (only
// when `owned`), for the multi-step kernels.  Returns S^: shat0 (the permeability term, 0 for uniform mu)
// minus mu j_z of the sources at the site.
// Pre-collision populations of the 4 sites (row, 4c..4c+3): g_i(x) = buf_i(x - c_i).
// Must be called by all 32 lanes of a warp (shuffles); lanes with c >= nchunk
// load nothing and their results are discarded by the caller.
template <int ST>
__device__ __forceinline__ void pull2d(const PopBuf &in, const Grid &G, int row, int c, int lane, float4 g[5]) {
    using C = Codec<ST>;
    const int x0 = 4 * c;
    const bool active = c < G.nchunk;  // lanes past the row end load nothing
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
    if (c == G.nchunk - 1) set(g[3], G.nx - 1 - x0, C::load1(in, 3, row, 0));  // periodic wrap at x = nx-1
}

// shat0: the source already formed at the site; pz, sbx, sby, jmu: what the general kernel adds (E_z = -c^2 sigma
// - pz, B_x and B_y scaled by sbx, sby, j_z by jmu; 0, 1, 1, 1 leave every value unchanged).
__device__ __forceinline__ float site_events(const StepArgs &a, int x, int y, long long t, bool owned, float g0,
                                             float g1, float g2, float g3, float g4, float cl, float shat0 = 0.f,
                                             float pz = 0.f, float sbx = 1.f, float sby = 1.f, float jmu = 1.f) {
    float shat = shat0;
    if (!a.evt.rowptr) return shat;
    const int e0 = __ldg(a.evt.rowptr + y), e1 = __ldg(a.evt.rowptr + y + 1);
    for (int e = e0; e < e1; e++) {
        const Event ev = a.evt.ev[e];
        if (ev.x != x) continue;
        if (ev.kind == 0) {
            if (ev.comp == 2 && t < a.evt.nt) {
                float jz = __ldg(a.evt.amp + (long long)ev.index * a.evt.nt + t);
                if (a.med.mu) jz = __fmul_rn(jz, __ldg(a.med.mu + (long long)y * a.g.pitch + x));
                jz = __fmul_rn(jz, jmu);
                shat = __fsub_rn(shat, jz);
            }
        } else if (owned && t < a.evt.cap) {
            const float s = ((g0 + g1) + (g2 + g3)) + g4;
            float v = field2d(ev.comp, cl, s, g4 - g2, g1 - g3);
            if (ev.comp == 2) v = __fsub_rn(v, pz);  // with a dispersive pole E = D/eps_inf - P (else pz = +0)
            if (ev.comp == 3) v = __fmul_rn(v, sbx);
            if (ev.comp == 4) v = __fmul_rn(v, sby);
            a.evt.traces[(long long)ev.index * a.evt.cap + t] = v;
        }
    }
    return shat;
}

// ------------------------------------------------------------------ handle
struct AdjointState;  // defined in adjoint.cu

}  // namespace lbk

struct lbem {
    int dim = 2, storage = LBEM_F32, npop = 5;
    double c_ref2 = 0.5;
    cudaStream_t stream = nullptr;
    lbk::Grid grid{};
    long long nsite = 0;
    lbk::PopBuf buf[2];
    int cur = 0;
    void *pool = nullptr;  // population buffers
    size_t pool_bytes = 0;
    float *cL2 = nullptr, *mu = nullptr, *dlnmu = nullptr;
    bool has_medium = false, has_mu = false;
    long long t = 0;
    // events
    int *d_rowptr = nullptr;
    lbk::Event *d_ev = nullptr;
    float *d_amp = nullptr;
    float *d_traces = nullptr;
    int nsrc = 0, nrec = 0, nt = 0, cap = 0, nev = 0;
    std::vector<long long> src_site;
    std::vector<int> src_comp;
    std::vector<float> src_amp;
    std::vector<long long> rec_site;
    std::vector<int> rec_comp;
    // scratch
    double *d_partials = nullptr;
    int n_partials = 0;
    double *d_diag = nullptr;     // [3]
    unsigned *d_counter = nullptr; // [0] validation / max-abs scratch, [2..3] the strip kernel's work queue
    float *d_stage = nullptr;      // staging for host <-> device copies of grid fields
    size_t stage_bytes = 0;
    // graphs
    bool use_graphs = false;
    cudaGraphExec_t graph = nullptr;
    long long graph_t0 = -1;
    int graph_steps = 0, graph_cur = -1, graph_variant = -1, graph_cur_end = 0;
    // tuning
    int variant = 0;
    int tblock = 2;  // steps per pass (lbem_set_temporal_blocking)
    int tb_shape = 0;  // tile shape of the two-step kernel
    bool tb_shape_set = false;  // set by lbem_set_temporal_blocking (a shape >= 0) or lbem_autotune; else by grid size
    // watchdog (lbem_set_watchdog)
    int wd_every = 0;
    double wd_growth = 0.0, wd_last = -1.0;
    // walls and absorbing layers (lbem_set_boundaries); edge tiles per steps-per-launch k = 1..3
    int bc[3] = {0, 0, 0};
    int layer = 0;
    double gamma_max = 0.0;
    float *d_fx = nullptr, *d_fy = nullptr, *d_fz = nullptr;
    lbk::EdgeTile *d_tiles[4] = {nullptr, nullptr, nullptr, nullptr};
    int ntiles[4] = {0, 0, 0, 0};
    // 2D walls: the stream the edge pass runs on beside a strip-streaming launch, and the events that fork it from
    // and join it to the handle's stream
    cudaStream_t edge_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // frequency-dispersive permittivity (lbem_set_dispersion): pole parameters and state, planes (pitch layout)
    // P has two planes, paired with the population buffers: P at the time of buf[c] is pole_P(c), so a launch
    // reads P from the plane of its input's parity and writes the other one (every launch flips cur).
    float *d_wp2 = nullptr, *d_wr2 = nullptr, *d_gam = nullptr, *d_J = nullptr, *d_P = nullptr, *d_P2 = nullptr;
    float *d_pc = nullptr, *d_pb = nullptr, *d_pa = nullptr;  // pole_update's coefficients (pole_coefficients)
    float *pole_P(int c) const { return c ? d_P2 : d_P; }
    bool disp = false;
    // anisotropic medium (lbem_set_medium_aniso): r = sqrt(mu_xx / mu_yy), mubar = sqrt(mu_xx mu_yy)
    bool aniso = false;
    float aniso_r = 1.f, aniso_mu = 1.f;
    // media the general kernel steps (general.cu); without mu planes (and a pole without walls) also two steps
    // per launch
    bool general() const { return disp || aniso; }
    float aniso_fsum() const { return aniso ? aniso_r + 1.f / aniso_r : 2.f; }  // (c_x^2 + c_y^2) / cbar^2
    size_t tile_smem[4] = {0, 0, 0, 0}, tile_smem_mu[4] = {0, 0, 0, 0};  // uniform / heterogeneous mu
    bool walls() const { return bc[0] || bc[1] || bc[2]; }
    // adjoint
    lbk::AdjointState *adj = nullptr;
    // guard bands around every array above (see lbem_check_guards)
    struct Guarded {
        void *user;
        size_t bytes;
        const char *name;
    };
    std::vector<Guarded> guarded;
};

namespace lbk {

// errors (lbem_api.cu)
lbem_status fail(lbem_status s, const std::string &msg);
lbem_status cuda_fail(cudaError_t e, const char *what);
#define LBEM_CUDA(call)                                          \
    do {                                                         \
        cudaError_t _e = (call);                                 \
        if (_e != cudaSuccess) return ::lbk::cuda_fail(_e, #call); \
    } while (0)

inline int round_up(int a, int b) { return (a + b - 1) / b * b; }

StepArgs step_args(const lbem_t *h, int cur_in);

// 2D (kernels2d.cu)
int nvariants_2d();
cudaError_t launch_step_2d(const StepArgs &a, int storage, bool has_mu, int variant, cudaStream_t s);
// two steps per launch (tblock.cu): FP32 (uniform or heterogeneous mu), 16-bit storage (uniform mu, nx % 4 == 0)
int tb2_nshapes(int storage, bool has_mu);
// two steps per launch by register streaming (rstream.cu): FP32 storage, uniform mu
int rs2_nshapes();
cudaError_t launch_step_2d_rs2(const StepArgs &a, int shape, cudaStream_t s);
int ss2_nshapes();  // strip streaming (sstream.cu): two steps per launch, FP32, uniform mu
cudaError_t launch_step_2d_ss2(const StepArgs &a, int shape, cudaStream_t s);
cudaError_t launch_step_2d_ss2_an(const StepArgs &a, cudaStream_t s);  // anisotropic medium, no pole
cudaError_t launch_step_2d_ss2_mu(const StepArgs &a, cudaStream_t s);  // heterogeneous permeability
bool ss2_take_timeouts();  // reads and clears the strip kernel's wait-timeout flag
cudaError_t ss_set_wait_limit(unsigned long long ns);
bool tb2_take_timeouts();  // reads and clears the two-step kernel's wait-timeout flag
cudaError_t tb_set_wait_limit(unsigned long long ns);  // limit of its bounded waits (current device)
// three steps per launch (tblock.cu): FP32 storage, uniform mu
int tb3_nshapes();
cudaError_t launch_step_2d_tb3(const StepArgs &a, int shape, cudaStream_t s);
cudaError_t launch_step_2d_tb2(const StepArgs &a, int storage, int shape, cudaStream_t s);
// two steps per launch over a batch (tblock.cu): tiles of every member from a flattened table over the batch's packed
// states with halos (BatchPacked); args[2 m + par] are member m's step arguments for buffer parity par of its own
// buffers (the kernels use args[2 m] for the grid and events); tile rows of each shape: batch_tb2_rows
struct BatchPacked {
    float *buf[2];    // packed population buffers: [5][rows][W]
    float *cl;        // packed c_L^2: [rows][W]
    const int *r0;    // per member its first packed row; r0[n] = rows
    int W;            // packed row width (floats, a multiple of 32)
    long long plane;  // rows * W
};
// One tile of the batch's two-step kernel: member m, origin (x0, y0), the packed row py of member row y0 - 1 (the
// window's first c_L^2 row), the member's size, and whether rows y0 - 1 .. y0 + TBY (periodic) hold a source or a
// receiver.  Built on the host, one 32-byte load per tile.
struct __align__(16) BatchTile {
    int m, x0, y0, py;
    int nx, ny, ev, pad;
};
int batch_tb2_rows(int shape);
cudaError_t launch_batch_tb2(const StepArgs *args, const BatchTile *tiles, long long ntiles, const long long *t0p,
                             int toff, int par, const BatchPacked &pk, long long rows, int shape, cudaStream_t s);
cudaError_t launch_batch_pack(const StepArgs *args, int par, const int *r0, int n, long long rows,
                              const BatchPacked &pk, int which, bool unpack, cudaStream_t s);
// One unit of the batch's strip-streaming kernel (sstream.cu): member m, its 128-column strip from column x0 and rows
// ys .. ye-1, its packed row prow0 (member row -2) and size, and the member's event tables (row pointer and records;
// null without events).  Built on the host, tall units first.
struct __align__(16) BatchUnit {
    int m, x0, ys, ye;
    int prow0, nx, ny, pad;
    const int *rowptr;
    const Event *ev;
};
int batch_ss2_nshapes();
int batch_ss2_rows(int shape);    // chunk rows (TBY) of a shape
int batch_ss2_chunks(int shape);  // chunks of a full unit
cudaError_t launch_batch_ss2(const StepArgs *args, const BatchUnit *units, int nunits, int *sched, const long long *t0p,
                             int toff, int par, const BatchPacked &pk, long long rows, int shape, cudaStream_t s);
cudaError_t launch_init_2d(const lbem_t *h, const float *E, const float *B, cudaStream_t s);
cudaError_t launch_fields_2d(const lbem_t *h, float *E, float *B, cudaStream_t s);
cudaError_t launch_diag_2d(const lbem_t *h, double *partials, int nblocks, cudaStream_t s);
// 3D (kernels3d.cu)
int nvariants_3d();
cudaError_t launch_step_3d(const StepArgs &a, bool has_mu, int variant, cudaStream_t s, const Walls *w = nullptr);
cudaError_t launch_init_3d(const lbem_t *h, const float *E, const float *B, cudaStream_t s);
cudaError_t launch_fields_3d(const lbem_t *h, float *E, float *B, cudaStream_t s);
cudaError_t launch_diag_3d(const lbem_t *h, double *partials, int nblocks, cudaStream_t s);
// shared small kernels (medium.cu)
// fsum = sum of the axis speeds over c_L^2 (D, or r + 1/r anisotropic), mubar = sqrt(mu_xx mu_yy) (else 1)
cudaError_t launch_medium(lbem_t *h, const float *eps, const float *mu, double fsum, double mubar, unsigned *bad,
                          cudaStream_t s);
cudaError_t launch_maxabs(const float *a, long long n, unsigned *out, cudaStream_t s);
cudaError_t launch_reduce_partials(const double *partials, int n, double *out, cudaStream_t s);
int diag_blocks(long long nsite);
cudaError_t launch_medium_write(lbem_t *h, const float *eps, const float *mu, double mubar, cudaStream_t s);
cudaError_t launch_energy_flux(const lbem_t *h, const float *E, const float *B, float *u, float *P, cudaStream_t s);
// guarded device allocations (lbem_api.cu): `bytes` usable bytes between two patterned guard bands
cudaError_t gmalloc(lbem_t *h, void **p, size_t bytes, const char *name);
void gfree(lbem_t *h, void *p);
// adjoint.cu
void adjoint_free(lbem_t *h);
// walls.cu: the k steps of a launch recomputed on the bands next to walls and in layers
std::vector<EdgeTile> edge_tiles(const Grid &G, const int kind[2], int layer, int k);
size_t edge_smem_bytes(int k, const std::vector<EdgeTile> &tiles, bool mu);
cudaError_t launch_edge_2d(const StepArgs &a, const Walls &w, const EdgeTile *d_tiles, int ntiles, size_t smem, int k,
                           bool aniso, cudaStream_t s);
cudaError_t launch_medium_grad_walls(const lbem_t *h, cudaStream_t s);
// general.cu: single steps with a dispersive pole and / or an anisotropic medium (walls and layers applied in the
// kernel)
cudaError_t launch_step_2d_gen(const StepArgs &a, const Walls &w, const General &q, cudaStream_t s);
cudaError_t launch_disp_check(const lbem_t *h, const float *eps, const float *mu, double fsum, double mubar,
                              const float *wp2, const float *wr2, const float *gam, bool pitched, unsigned *bad,
                              cudaStream_t s);
cudaError_t launch_to_plane(const lbem_t *h, const float *src, float *dst, cudaStream_t s);
// the pole's per-site update coefficients (pole_update) from its parameter planes
cudaError_t launch_pole_coefficients(const lbem_t *h, cudaStream_t s);

}  // namespace lbk
