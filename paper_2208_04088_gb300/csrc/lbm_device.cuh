// lbm_device.cuh -- device-side building blocks of the solid-LBM kernels:
// storage conversion, raw-moment collision, pull streaming and the boundary
// rules of Sec. 4.  Included by the single-solver kernels (lbm_kernels.cu) and
// the batched kernels (lbm_batch.cu), so both run the same arithmetic.
#pragma once

#include <cstdint>
#include <cstring>
#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "lbm_internal.h"

namespace lbm {

// ---------------------------------------------------------------------------
// Storage of one population value (FP32, or 16-bit scaled deviations).
template <class T>
struct Store;

template <>
struct Store<float> {
    static __device__ __forceinline__ float ld(const float *p, float) { return __ldg(p); }
    static __device__ __forceinline__ void st(float *p, float v, float) { *p = v; }
};

template <>
struct Store<__half> {
    static __device__ __forceinline__ float ld(const __half *p, float inv_scale) {
        return __half2float(__ldg(p)) * inv_scale;
    }
    static __device__ __forceinline__ void st(__half *p, float v, float scale) {
        *p = __float2half_rn(v * scale);
    }
};

template <>
struct Store<__nv_bfloat16> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16 *p, float inv_scale) {
        return __bfloat162float(__ldg(p)) * inv_scale;
    }
    static __device__ __forceinline__ void st(__nv_bfloat16 *p, float v, float scale) {
        *p = __float2bfloat16_rn(v * scale);
    }
};

// The scales of step t with FP16 storage: L.inv_scale for the values the step
// reads (stored by step t - 1) and L.scale for the values it stores (the
// scale of step t - 1, halved if one of its values passed kScaleOver).  Other
// storage forms keep their fixed scale.  Every kernel of a step computes the
// same pair from the solver's scale record.
//
// t mod 3 for t >= 0 from the two 32-bit halves (2^32 = 1 mod 3), without a
// 64-bit division.
__host__ __device__ __forceinline__ int mod3(int64_t t) {
    const uint32_t lo = (uint32_t)t, hi = (uint32_t)((uint64_t)t >> 32);
    return (int)((lo % 3u + hi % 3u) % 3u);
}

// 1/s of a power of two s = 2^e, -127 <= e <= 126, exactly: the biased
// exponent 127 + e becomes 127 - e (the scales lie in [2^-126, 2^60]).
__device__ __forceinline__ float pow2_reciprocal(float s) {
    return __int_as_float(0x7f000000 - __float_as_int(s));
}

template <class T> __device__ __forceinline__ void step_scales(Lattice &L, int64_t t) {
    if constexpr (std::is_same<T, __half>::value) {
        if (L.sc) {
            const int p = mod3(t + 2);
            const float prev = L.sc->s[p];
            L.inv_scale = pow2_reciprocal(prev);
            L.scale = L.sc->over[p] ? fmaxf(__fmul_rn(prev, 0.5f), kScaleMin) : prev;
            L.over = L.sc->over + mod3(t);
        }
    }
}

// Step t's scale into the record, and the flag of step t + 1 cleared (it
// holds step t - 2's, which no kernel of step t reads).  One thread per step.
template <class T> __device__ __forceinline__ void publish_scale(const Lattice &L, int64_t t) {
    if constexpr (std::is_same<T, __half>::value) {
        if (L.sc) {
            L.sc->s[mod3(t)] = L.scale;
            L.sc->over[mod3(t + 1)] = 0u;
        }
    }
}

// Flags the step (L as step_scales left it) when a value it stores, scaled,
// passes kScaleOver.
template <class T> __device__ __forceinline__ void note_range(const Lattice &L, float v) {
    if constexpr (std::is_same<T, __half>::value) {
        if (L.over && fabsf(__fmul_rn(v, L.scale)) > kScaleOver &&
            !*reinterpret_cast<volatile uint32_t *>(L.over))
            atomicExch(L.over, 1u);
    }
}

// D2Q9 velocity components and opposite directions as constant expressions.
__host__ __device__ constexpr int c_cx(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : (i == 3 || i == 6 || i == 7) ? -1 : 0;
}
__host__ __device__ constexpr int c_cy(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : (i == 4 || i == 7 || i == 8) ? -1 : 0;
}
__host__ __device__ constexpr int opp(int i) {
    return i == 0 ? 0 : (i <= 4 ? (i + 1) % 4 + 1 : (i - 3) % 4 + 5);
}
static_assert(opp(1) == 3 && opp(2) == 4 && opp(3) == 1 && opp(4) == 2 && opp(5) == 7 &&
                  opp(6) == 8 && opp(7) == 5 && opp(8) == 6,
              "opposite directions");

// ---------------------------------------------------------------------------
// Explicitly rounded arithmetic.  The relaxation, the displacement update and
// the boundary rules are written with it (products, sums and fused
// multiply-adds in a fixed order), so every kernel that evaluates them -- the
// one-step kernels, the batched kernels and the temporally blocked kernel --
// rounds identically, whatever the compiler would fuse in each context.
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// The same operations on the values of two lattice nodes at once: an f32x2
// register pair, one instruction for both (each half rounded to nearest, so
// a pair gives, half by half, what the scalar operation gives).
struct F2 {
    unsigned long long v;
};
__device__ __forceinline__ F2 f2(float lo, float hi) {
    F2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_split(F2 x, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x.v));
}
__device__ __forceinline__ F2 rmul(F2 a, F2 b) {
    F2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ F2 radd(F2 a, F2 b) {
    F2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ F2 rsub(F2 a, F2 b) {
    F2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ F2 rfma(F2 a, F2 b, F2 c) {
    F2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return d;
}
// A constant in either form.
template <class V> __device__ __forceinline__ V splat(float c);
template <> __device__ __forceinline__ float splat<float>(float c) { return c; }
template <> __device__ __forceinline__ F2 splat<F2>(float c) { return f2(c, c); }

// ---------------------------------------------------------------------------
// Raw moments m_pq = sum_i f_i c_ix^p c_iy^q (p, q in 0..2) of the nine
// populations.  D2Q9 is the tensor product of {-1, 0, 1} in x and y, so the
// transform is two passes of the 1-D map (a-, a0, a+) -> (a- + a0 + a+,
// a+ - a-, a+ + a-), whose inverse has only the coefficients 1 and 1/2: the
// round trip adds nothing but additions to the rounding.
template <class V> struct RawT {
    V m00, m10, m01, m20, m02, m11, m21, m12, m22;
};
using Raw = RawT<float>;

template <class V> __device__ __forceinline__ RawT<V> raw_moments(const V f[9]) {
    // rows c_y = -1: (f7, f4, f8); c_y = 0: (f3, f0, f1); c_y = +1: (f6, f2, f5)
    const V a0 = radd(radd(f[7], f[4]), f[8]), a1 = rsub(f[8], f[7]), a2 = radd(f[8], f[7]);
    const V b0 = radd(radd(f[3], f[0]), f[1]), b1 = rsub(f[1], f[3]), b2 = radd(f[1], f[3]);
    const V c0 = radd(radd(f[6], f[2]), f[5]), c1 = rsub(f[5], f[6]), c2 = radd(f[5], f[6]);
    RawT<V> m;
    m.m00 = radd(radd(a0, b0), c0);
    m.m01 = rsub(c0, a0);
    m.m02 = radd(c0, a0);
    m.m10 = radd(radd(a1, b1), c1);
    m.m11 = rsub(c1, a1);
    m.m12 = radd(c1, a1);
    m.m20 = radd(radd(a2, b2), c2);
    m.m21 = rsub(c2, a2);
    m.m22 = radd(c2, a2);
    return m;
}

// Inverse of the 1-D map: (s, d, p) -> (a-, a0, a+) = ((p - d)/2, s - p,
// (p + d)/2), with (p -/+ d)/2 formed as fma(-/+1/2, d, p/2): halving is exact,
// so this is the correctly rounded half of p -/+ d.
template <class V>
__device__ __forceinline__ void inverse3(V s, V d, V p, V &am, V &a0, V &ap) {
    const V h = rmul(splat<V>(0.5f), p);
    am = rfma(splat<V>(-0.5f), d, h);
    a0 = rsub(s, p);
    ap = rfma(splat<V>(0.5f), d, h);
}

template <class V> __device__ __forceinline__ void populations(const RawT<V> &m, V f[9]) {
    // inverse in y for each x-order p, then inverse in x for each row
    V a0, b0, c0, a1, b1, c1, a2, b2, c2;
    inverse3(m.m00, m.m01, m.m02, a0, b0, c0);
    inverse3(m.m10, m.m11, m.m12, a1, b1, c1);
    inverse3(m.m20, m.m21, m.m22, a2, b2, c2);
    inverse3(a0, a1, a2, f[7], f[4], f[8]);
    inverse3(b0, b1, b2, f[3], f[0], f[1]);
    inverse3(c0, c1, c2, f[6], f[2], f[5]);
}

// Moments of Eq. (moments) in deviation form: drho, m = sum f c (without S/2), P.
struct Mom {
    float dr, mx, my, pxx, pyy, pxy;
};

__device__ __forceinline__ Mom moments(const float f[9]) {
    const Raw r = raw_moments(f);
    return Mom{r.m00, r.m10, r.m01, r.m20, r.m02, r.m11};
}

// BGK collision with source (Eq. coll) carried out on the raw moments.  The
// map f -> f + omega (f^eq - f) + (1 - 1/(2 tau)) psi is the same linear map in
// any basis; in this one the raw moments of f^eq (Eq. fieq, c_s^2 = 1/3) are
//   rho, j, P                     (the moments the equilibrium reproduces)
//   m_xxy = j_y/3, m_xyy = j_x/3  (third moment c_s^2 (j d + j d + j d))
//   m_xxyy = (P_xx + P_yy)/3 - rho/9,
// and those of psi_i = 3 w_i c_i.S are S in the first and S/3 in the third
// moments.  rho and P pass through untouched and j gains exactly S, so the
// collision invariants are not disturbed by the rounding of 1/3 and 1/9.
// The relaxation on the raw moments; w = omega, s3 = (1 - 1/(2 tau))/3.
// Returns the momentum j = m + S/2 in jx, jy.  omega (f^eq - f) is formed as
// (-omega)(f - f^eq), which rounds to the same value.
template <class V>
__device__ __forceinline__ void relax_raw(RawT<V> &m, V sx, V sy, V w, V s3, V &jx, V &jy) {
    const V half = splat<V>(0.5f), third = splat<V>(1.0f / 3.0f);
    const V mthird = splat<V>(-1.0f / 3.0f), mninth = splat<V>(-1.0f / 9.0f);
    const V mw = rsub(splat<V>(0.0f), w);
    jx = rfma(half, sx, m.m10);
    jy = rfma(half, sy, m.m01);
    m.m10 = radd(m.m10, sx);
    m.m01 = radd(m.m01, sy);
    m.m21 = radd(m.m21, rfma(s3, sy, rmul(mw, rfma(jy, mthird, m.m21))));
    m.m12 = radd(m.m12, rfma(s3, sx, rmul(mw, rfma(jx, mthird, m.m12))));
    const V e = rfma(m.m00, mninth, rmul(radd(m.m20, m.m02), third));
    m.m22 = rfma(w, rsub(e, m.m22), m.m22);
}

// On return f holds f^col, jx/jy the momentum j = m + S/2, dr the density
// deviation; the same for one node (float) or two (F2).
template <class V>
__device__ __forceinline__ void collide_v(V f[9], V sx, V sy, V w, V s3, V &dr_out, V &jx_out,
                                          V &jy_out) {
    RawT<V> m = raw_moments(f);
    relax_raw(m, sx, sy, w, s3, jx_out, jy_out);
    dr_out = m.m00;
    populations(m, f);
}

__device__ __forceinline__ void collide(float f[9], float sx, float sy, const Lattice &L,
                                        float &dr_out, float &jx_out, float &jy_out) {
    collide_v<float>(f, sx, sy, L.omega, rmul(L.src, 1.0f / 3.0f), dr_out, jx_out, jy_out);
}

// u(t+1) = u(t) + j/rho with Kahan compensation per component; w holds
// (u_x, u_y, compensation_x, compensation_y).
__device__ __forceinline__ void integrate_u_value(float4 &w, float jx, float jy, float rho) {
    // v = j/rho as j times one approximate reciprocal (relative error about
    // 1e-7, far below the FP32 parity bound; no divisions)
    const float ir = __fdividef(1.0f, rho);
    const float vx = rmul(jx, ir), vy = rmul(jy, ir);
    float y = rsub(vx, w.z);
    float t = radd(w.x, y);
    w.z = rsub(rsub(t, w.x), y);
    w.x = t;
    y = rsub(vy, w.w);
    t = radd(w.y, y);
    w.w = rsub(rsub(t, w.y), y);
    w.y = t;
}

// 16-bit storage: u(t+1) = u(t) + j/rho without compensation; w holds
// (u_x, u_y).  The populations' own rounding (FP16: 2^-11 of their size, each
// step) is far larger than what the compensation recovers, and the record is
// half as many bytes in the bandwidth-bound step.
__device__ __forceinline__ void integrate_u_value(float2 &w, float jx, float jy, float rho) {
    const float ir = __fdividef(1.0f, rho);
    w.x = radd(w.x, rmul(jx, ir));
    w.y = radd(w.y, rmul(jy, ir));
}

// The displacement record of a storage type: FP32 populations keep the
// compensated float4, 16-bit populations a float2.
template <class T> struct URecOf { using type = float2; };
template <> struct URecOf<float> { using type = float4; };
template <class T> using URec = typename URecOf<T>::type;

// u of a record (the compensated sum without its compensation).
__device__ __forceinline__ float2 u_of(const float4 &w) {
    return make_float2(w.x - w.z, w.y - w.w);
}
__device__ __forceinline__ float2 u_of(const float2 &w) { return w; }

template <class W>
__device__ __forceinline__ void integrate_u(W *uc, float jx, float jy, float rho) {
    W w = *uc;
    integrate_u_value(w, jx, jy, rho);
    *uc = w;
}

// Raise the non-finite flag once: after the first, a plain read of the (cached)
// status word keeps a diverged lattice from serialising on the atomic.
__device__ __forceinline__ void flag_nonfinite(uint32_t *status, float a, float b, float c) {
    if (!isfinite(a + b + c) && !(*reinterpret_cast<volatile uint32_t *>(status) & 1u))
        atomicOr(status, 1u);
}

// Amplitude of a boundary value at (lattice) time t: step or ramp-then-hold.
__device__ __forceinline__ float amplitude(const BCDev &b, float t) {
    if (t < 0.0f) return 0.0f;
    if (b.profile == LBM_PROFILE_RAMP) return fminf(__fdiv_rn(t, b.t_ramp), 1.0f);
    return 1.0f;
}

// Traction t*(t) of a Neumann condition on a wall with outward normal n.
__device__ __forceinline__ void traction(const BCDev &b, float n0, float n1, float t, float &tx,
                                         float &ty) {
    const float a = amplitude(b, t);
    if (b.kind == LBM_BC_PRESSURE) {
        tx = rmul(rmul(-b.v0, n0), a);
        ty = rmul(rmul(-b.v0, n1), a);
    } else if (b.kind == LBM_BC_STRESS) {
        tx = rmul(rfma(b.v0, n0, rmul(b.v2, n1)), a);
        ty = rmul(rfma(b.v2, n0, rmul(b.v1, n1)), a);
    } else {
        tx = rmul(b.v0, a);
        ty = rmul(b.v1, a);
    }
}

// Interior pull: f_i(x, t) = f_i^col(x - c_i, t - 1).
template <class T>
__device__ __forceinline__ void pull_interior(const T *__restrict__ src, int64_t k, int pitch,
                                              int64_t plane, float inv_scale, float f[9]) {
    f[0] = Store<T>::ld(src + k, inv_scale);
    f[1] = Store<T>::ld(src + plane + k - 1, inv_scale);
    f[2] = Store<T>::ld(src + 2 * plane + k - pitch, inv_scale);
    f[3] = Store<T>::ld(src + 3 * plane + k + 1, inv_scale);
    f[4] = Store<T>::ld(src + 4 * plane + k + pitch, inv_scale);
    f[5] = Store<T>::ld(src + 5 * plane + k - pitch - 1, inv_scale);
    f[6] = Store<T>::ld(src + 6 * plane + k - pitch + 1, inv_scale);
    f[7] = Store<T>::ld(src + 7 * plane + k + pitch + 1, inv_scale);
    f[8] = Store<T>::ld(src + 8 * plane + k + pitch - 1, inv_scale);
}


// Where a step finds f_m^col(z, t-1) and puts f_m^col(x, t) (the stepping
// form).  kPull: two buffers; plane m at the node, read from one and written
// to the other.  kAAEven / kAAOdd: one buffer, updated in place in the AA
// pattern.  An even step reads every incoming population of x from x itself
// (f_m^col(z) sits at node z + c_m, plane m) and writes f_m^col(x) back into
// x, plane opp(m); an odd step reads f_m^col(z) from node z, plane opp(m), and
// writes f_m^col(x) to node x + c_m, plane m.  Each node then reads and writes
// the same nine locations, which no other node touches.  Population planes
// are L.fplane elements apart; with kAA the buffer has a ring of one node
// around the lattice for the populations leaving across the box edges.
enum : int { kPull = 0, kAAEven = 1, kAAOdd = 2 };

template <int LAY>
__device__ __forceinline__ int64_t col_at(int64_t kz, int m, const Lattice &L) {
    if (LAY == kAAEven) return m * L.fplane + kz + (int64_t)c_cy(m) * L.pitch + c_cx(m);
    if (LAY == kAAOdd) return opp(m) * L.fplane + kz;
    return m * L.fplane + kz;
}

template <int LAY>
__device__ __forceinline__ int64_t out_at(int64_t kx, int m, const Lattice &L) {
    if (LAY == kAAEven) return opp(m) * L.fplane + kx;
    if (LAY == kAAOdd) return m * L.fplane + kx + (int64_t)c_cy(m) * L.pitch + c_cx(m);
    return m * L.fplane + kx;
}

// Interior pull in any stepping form: f_i(x, t) = f_i^col(x - c_i, t - 1).
template <int LAY, class T>
__device__ __forceinline__ void pull_interior_at(const T *src, int64_t k, const Lattice &L,
                                                 float f[9]) {
#pragma unroll
    for (int i = 0; i < 9; ++i)
        f[i] = Store<T>::ld(src + col_at<LAY>(k - (int64_t)c_cy(i) * L.pitch - c_cx(i), i, L),
                            L.inv_scale);
}

// ---------------------------------------------------------------------------
// Cooperative boundary update: eight lanes per boundary node.  Lane j owns the
// population k = j + 1 and the link i = opp(k) through which it arrives.  Every
// lane reads the node's nine post-collision populations (the same addresses,
// a broadcast) and forms their moments with moments(); after the rules, the
// nine incoming populations are gathered with shuffles and every lane runs
// collide() on them.  The arithmetic is therefore that of a one-lane update
// (the same functions in the same order), whichever form a kernel uses.
__device__ __forceinline__ int lane_cx(int k) {
    return (k == 1 || k == 5 || k == 8) ? 1 : (k == 3 || k == 6 || k == 7) ? -1 : 0;
}
__device__ __forceinline__ int lane_cy(int k) {
    return (k == 2 || k == 5 || k == 6) ? 1 : (k == 4 || k == 7 || k == 8) ? -1 : 0;
}


// Pieces of the cut-link rules of Sec. 4, shared by every boundary path so
// that each evaluates the same expressions.
//
// kappa = (l - 2 s)/(l + 2 s) and 1 + kappa = 2 l/(l + 2 s) of the curved rules
// (Eqs. bbnoncon, abbnoncon) for q = s/l; q = 1/2 gives 0 and 1.
__device__ __forceinline__ void link_kappa(float q, float &kap, float &fac) {
    const float den = rfma(2.0f, q, 1.0f);
    kap = __fdiv_rn(rfma(-2.0f, q, 1.0f), den);
    fac = __fdiv_rn(2.0f, den);
}

// Dirichlet data j* = rho0 d(u*)/dt (Eq. bcchaindir); a corner link takes the
// mean of its two Dirichlet edges (bc2 = bc on a plain edge).
__device__ __forceinline__ void dirichlet_momentum(const BLink &lk, const BCDev *__restrict__ bcs,
                                                   float tb, const Lattice &L, float &jsx,
                                                   float &jsy) {
    const BCDev ba = bcs[lk.bc], bb = bcs[lk.bc2];
    const float aa = amplitude(ba, tb), ab = amplitude(bb, tb);
    const float h = rmul(L.rho0, 0.5f);
    jsx = rmul(h, rfma(ba.v0, aa, rmul(bb.v0, ab)));
    jsy = rmul(h, rfma(ba.v1, aa, rmul(bb.v1, ab)));
}

// Traction of a non-corner Neumann link in its boundary frame (e^n = n,
// e^t = (-n1, n0)): normal and tangential components (Eq. trafocauchy).
struct WallFrame {
    float n0, n1, t0, t1, tn, tt;
};

__device__ __forceinline__ WallFrame wall_frame(const BLink &lk, const BCDev *__restrict__ bcs,
                                                float tb) {
    WallFrame w;
    w.n0 = lk.n0;
    w.n1 = lk.n1;
    w.t0 = -w.n1;
    w.t1 = w.n0;
    float tx, ty;
    traction(bcs[lk.bc], w.n0, w.n1, tb, tx, ty);
    w.tn = rfma(tx, w.n0, rmul(ty, w.n1));
    w.tt = rfma(tx, w.t0, rmul(ty, w.t1));
    return w;
}

// Density deviation and Cauchy stress at the wall: the node's own values, or
// the linear extrapolation along the link (1 + q) a(x) - q a(x - c_i) when
// `neu_ex` (Sec. 4; q = 1/2 gives (3 a(x) - a(x - c_i))/2).
struct WallState {
    float drb, sxx, syy, sxy;
};

__device__ __forceinline__ WallState wall_state(bool neu_ex, float q, float dr_x, float pxx_x,
                                                float pyy_x, float pxy_x, float my_dr,
                                                float my_xx, float my_yy, float my_xy,
                                                const Lattice &L) {
    const float dvx = rmul(-L.lam_m_mu_r0, dr_x);
    const float sxx_x = radd(-pxx_x, dvx), syy_x = radd(-pyy_x, dvx), sxy_x = -pxy_x;
    WallState s{dr_x, sxx_x, syy_x, sxy_x};
    if (neu_ex) {
        const float dvy = rmul(-L.lam_m_mu_r0, my_dr);
        const float a1 = radd(1.0f, q);
        s.drb = rfma(a1, dr_x, -rmul(q, my_dr));
        s.sxx = rfma(a1, sxx_x, -rmul(q, radd(-my_xx, dvy)));
        s.syy = rfma(a1, syy_x, -rmul(q, radd(-my_yy, dvy)));
        s.sxy = rfma(a1, sxy_x, -rmul(q, -my_xy));
    }
    return s;
}

// sigma* = t_n n n + t_t (n t + t n) + sigma_tt t t with sigma_tt of the wall state.
__device__ __forceinline__ void wall_sigma(const WallFrame &w, const WallState &s, float &sxx,
                                           float &syy, float &sxy) {
    const float stt = rfma(rmul(w.t1, w.t1), s.syy,
                           rfma(rmul(rmul(2.0f, w.t0), w.t1), s.sxy, rmul(rmul(w.t0, w.t0), s.sxx)));
    sxx = rfma(rmul(stt, w.t0), w.t0,
               rfma(rmul(rmul(2.0f, w.tt), w.n0), w.t0, rmul(rmul(w.tn, w.n0), w.n0)));
    syy = rfma(rmul(stt, w.t1), w.t1,
               rfma(rmul(rmul(2.0f, w.tt), w.n1), w.t1, rmul(rmul(w.tn, w.n1), w.n1)));
    sxy = rfma(rmul(stt, w.t0), w.t1,
               rfma(w.tt, rfma(w.n0, w.t1, rmul(w.t0, w.n1)), rmul(rmul(w.tn, w.n0), w.n1)));
}

// Second moment of the wall equilibrium: P* = -sigma* + (lambda - mu) div u I,
// div u = (rho0 - rho^bd)/rho0 (Eqs. bcchainneum, approxdiv), in deviation form.
struct WallMoments {
    float drb, axx, ayy, pxy;
};

__device__ __forceinline__ WallMoments wall_moments(float drb, float sxx, float syy, float sxy,
                                                    const Lattice &L) {
    const float dv = rmul(-L.lam_m_mu_r0, drb);
    const float pxx = radd(-sxx, dv), pyy = radd(-syy, dv), pxy = -sxy;
    return WallMoments{drb, rfma(drb, -(1.0f / 3.0f), pxx), rfma(drb, -(1.0f / 3.0f), pyy), pxy};
}

// 2 w_i f_i^eq(rho^bd, P*) of the anti-bounce-back rule for link i = opp(k).
__device__ __forceinline__ float wall_equilibrium(int k, const WallMoments &m) {
    const int i = k <= 4 ? (k + 1) % 4 + 1 : (k - 3) % 4 + 5;  // opp(k)
    const float w = (i <= 4) ? (1.0f / 9.0f) : (1.0f / 36.0f);
    const float cix = (float)(-lane_cx(k)), ciy = (float)(-lane_cy(k));
    const float quad = rfma(rmul(ciy, ciy), m.ayy,
                            rfma(rmul(rmul(2.0f, cix), ciy), m.pxy, rmul(rmul(cix, cix), m.axx)));
    const float con = rmul(4.5f, rfma(-radd(m.axx, m.ayy), 1.0f / 3.0f, quad));
    return rmul(rmul(2.0f, w), radd(m.drb, con));
}

// Eq. (bbnoncon) for link i = opp(k) given j*; kappa = 0, 1 + kappa = 1 (q = 1/2)
// give Eq. (bbcon).
__device__ __forceinline__ float bounce_back(int k, float kap, float fac, float gk, float gi,
                                             float gy_i, float jsx, float jsy) {
    const int i = k <= 4 ? (k + 1) % 4 + 1 : (k - 3) % 4 + 5;
    const float w = (i <= 4) ? (1.0f / 9.0f) : (1.0f / 36.0f);
    const float cix = (float)(-lane_cx(k)), ciy = (float)(-lane_cy(k));
    const float cj = rfma(cix, jsx, rmul(ciy, jsy));
    return rfma(-rmul(fac, rmul(6.0f, w)), cj, rfma(kap, rsub(gy_i, gk), gi));
}

// Eq. (abbnoncon) for link i = opp(k) given its wall equilibrium term.
__device__ __forceinline__ float anti_bounce_back(float kap, float fac, float gk, float gi,
                                                  float gy_i, float eq) {
    return rfma(fac, eq, rfma(-kap, radd(gy_i, gk), -gi));
}

// f_k(x, t) arriving through the cut link i = opp(k) of a boundary node:
// Eq. (bbnoncon) for a Dirichlet link, Eq. (abbnoncon) for a Neumann one (both
// reduce to Eqs. bbcon/abbcon at q = 1/2).  gk, gi: f_k^col(x), f_i^col(x) at
// t-1; gy_i: f_i^col(x - c_i) (0 if the upstream node is unusable, `miss`);
// dr_x, p**_x: density deviation and P of f^col(x); my_*: the same moments at
// x - c_i, used when the Neumann wall values are extrapolated (`neu_ex`).
__device__ __forceinline__ float cut_link_value(int k, bool miss, bool dirich, bool corner,
                                                bool neu_ex, const BLink &lk, float gk, float gi,
                                                float gy_i, float dr_x, float pxx_x, float pyy_x,
                                                float pxy_x, float my_dr, float my_xx,
                                                float my_yy, float my_xy,
                                                const BCDev *__restrict__ bcs, float tb,
                                                const Lattice &L) {
    const float q = miss ? 0.5f : lk.q;
    float kap, fac;
    link_kappa(q, kap, fac);
    if (dirich) {
        float jsx, jsy;
        dirichlet_momentum(lk, bcs, tb, L, jsx, jsy);
        return bounce_back(k, kap, fac, gk, gi, gy_i, jsx, jsy);
    }
    const WallState st = wall_state(neu_ex, q, dr_x, pxx_x, pyy_x, pxy_x, my_dr, my_xx, my_yy,
                                    my_xy, L);
    float sxx, syy, sxy;  // sigma* (Eq. trafocauchy)
    if (corner) {
        float tax, tay, tbx, tby;
        traction(bcs[lk.bc], lk.n0, 0.0f, tb, tax, tay);
        traction(bcs[lk.bc2], 0.0f, lk.n1, tb, tbx, tby);
        sxx = rmul(tax, lk.n0);
        syy = rmul(tby, lk.n1);
        sxy = rmul(0.5f, rfma(tay, lk.n0, rmul(tbx, lk.n1)));
    } else {
        wall_sigma(wall_frame(lk, bcs, tb), st, sxx, syy, sxy);
    }
    const float eq = wall_equilibrium(k, wall_moments(st.drb, sxx, syy, sxy, L));
    return anti_bounce_back(kap, fac, gk, gi, gy_i, eq);
}

// Populations f(x, t) of a boundary node: pulled where the link is intact,
// otherwise given by Eqs. (bbnoncon)/(abbnoncon) (which reduce to Eqs. bbcon/
// abbcon at s = l/2) from f^col(., t-1), rho(., t-1), sigma(., t-1) and the
// boundary data at t-1.  rho and P are collision invariants, so their values
// at t-1 are the moments of the stored post-collision populations.
template <class T, int LAY = kPull>
__device__ __forceinline__ void pull_boundary(const T *src, const BNode &b,
                                              const BLink *__restrict__ links,
                                              const BCDev *__restrict__ bcs, float tb,
                                              const Lattice &L, float f[9]) {
    const int64_t k = (int64_t)b.y * L.pitch + b.x;
    // Phase 1: every load that depends only on the node record, issued before
    // any arithmetic so their latencies overlap.  Cut directions read the
    // node itself (a valid address whose value is not used).
    float gx[9], pl[9], gy1[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) gx[i] = Store<T>::ld(src + col_at<LAY>(k, i, L), L.inv_scale);
#pragma unroll
    for (int kk = 1; kk < 9; ++kk) {
        const int i = opp(kk);
        const bool cut = (b.cut >> i) & 1u;
        const int64_t sk = cut ? k : k - (int64_t)c_cy(kk) * L.pitch - c_cx(kk);
        pl[kk] = Store<T>::ld(src + col_at<LAY>(sk, kk, L), L.inv_scale);
        // f_i^col at the upstream node x - c_i of the cut link i (kappa term)
        const bool up = cut && !((b.miss >> i) & 1u);
        const int64_t ku = up ? k - (int64_t)c_cy(i) * L.pitch - c_cx(i) : k;
        gy1[i] = Store<T>::ld(src + col_at<LAY>(ku, i, L), L.inv_scale);
    }
    const Mom mx = moments(gx);
    f[0] = gx[0];
#pragma unroll
    for (int kk = 1; kk < 9; ++kk) {
        // population kk arrives through the link i = opp(kk), from x + c_i
        const int i = opp(kk);
        const uint32_t bit = 1u << i;
        if (!(b.cut & bit)) {
            f[kk] = pl[kk];
            continue;
        }
        const bool miss = (b.miss & bit) != 0;
        const bool dirich = (b.dirich & bit) != 0;
        const bool neu_ex = !miss && !L.wall_node && !dirich;
        float my_dr = 0.0f, my_xx = 0.0f, my_yy = 0.0f, my_xy = 0.0f;
        if (neu_ex) {
            const int64_t ku = k - (int64_t)c_cy(i) * L.pitch - c_cx(i);
            float gy[9];
#pragma unroll
            for (int m = 0; m < 9; ++m) gy[m] = Store<T>::ld(src + col_at<LAY>(ku, m, L), L.inv_scale);
            const Mom my = moments(gy);
            my_dr = my.dr;
            my_xx = my.pxx;
            my_yy = my.pyy;
            my_xy = my.pxy;
        }
        f[kk] = cut_link_value(kk, miss, dirich, (b.corner & bit) != 0, neu_ex, links[i - 1],
                               gx[kk], gx[i], miss ? 0.0f : gy1[i], mx.dr, mx.pxx, mx.pyy,
                               mx.pxy, my_dr, my_xx, my_yy, my_xy, bcs, tb, L);
    }
}

// f_k(x, t) for lane k of a boundary node: pulled where link opp(k) is intact,
// otherwise Eqs. (bbnoncon)/(abbnoncon).  Same rules and data as
// pull_boundary.  `ld(m, dx, dy)` returns f_m^col(t-1) at the node offset by
// (dx, dy); `link(i)` the link record of cut direction i; the masks are those
// of BNode.  g0 receives f_0^col(x), which is f_0(x, t).
template <class Ld, class Lk>
__device__ __forceinline__ float boundary8_pull(const Ld &ld, uint32_t cutm, uint32_t dirm,
                                                uint32_t corm, uint32_t missm, int k,
                                                const Lk &link, const BCDev *__restrict__ bcs,
                                                float tb, const Lattice &L, float &g0) {
    const int i = k <= 4 ? (k + 1) % 4 + 1 : (k - 3) % 4 + 5;  // opp(k)
    const int cxk = lane_cx(k), cyk = lane_cy(k);
    const uint32_t bit = 1u << i;
    const bool cut = (cutm & bit) != 0;
    const bool miss = (missm & bit) != 0;
    // loads, all independent
    float g[9];
#pragma unroll
    for (int m = 0; m < 9; ++m) g[m] = ld(m, 0, 0);  // f^col(x), the same on every lane
    g0 = g[0];
    const float gk = ld(k, 0, 0);                     // f_k^col(x)
    const float gi = ld(i, 0, 0);                     // f_i^col(x)
    const float pulled = cut ? gk : ld(k, -cxk, -cyk);
    const bool up = cut && !miss;                     // upstream node x - c_i = x + c_k usable
    const float gy_i = up ? ld(i, cxk, cyk) : 0.0f;
    const bool neu_ex = up && !L.wall_node && !(dirm & bit);
    float my_dr = 0.0f, my_xx = 0.0f, my_yy = 0.0f, my_xy = 0.0f;
    if (neu_ex) {
        float gy[9];
#pragma unroll
        for (int m = 0; m < 9; ++m) gy[m] = ld(m, cxk, cyk);
        const Mom my = moments(gy);
        my_dr = my.dr;
        my_xx = my.pxx;
        my_yy = my.pyy;
        my_xy = my.pxy;
    }
    if (!cut) return pulled;
    const Mom mx = moments(g);  // rho and P are collision invariants: those of f^col(x, t-1)
    return cut_link_value(k, miss, (dirm & bit) != 0, (corm & bit) != 0, neu_ex, link(i), gk, gi,
                          gy_i, mx.dr, mx.pxx, mx.pyy, mx.pxy, my_dr, my_xx, my_yy, my_xy, bcs, tb,
                          L);
}

// The same from the distributions in global memory.
template <class T, int LAY = kPull>
__device__ __forceinline__ float pull_boundary8(const T *src, const BNode &b, int k,
                                                const BLink *__restrict__ links,
                                                const BCDev *__restrict__ bcs, float tb,
                                                const Lattice &L, float &f0) {
    const int64_t kn = (int64_t)b.y * L.pitch + b.x;
    const int pitch = L.pitch;
    const float inv = L.inv_scale;
    auto ld = [&](int m, int dx, int dy) {
        return Store<T>::ld(src + col_at<LAY>(kn + (int64_t)dy * pitch + dx, m, L), inv);
    };
    auto link = [&](int i) { return links[i - 1]; };
    return boundary8_pull(ld, b.cut, b.dirich, b.corner, b.miss, k, link, bcs, tb, L, f0);
}

// Collision of a boundary node held one population per lane (group of eight
// lanes, direction kdir on lane kdir - 1; g0 = f_0): the nine populations are
// gathered on every lane and collide() runs on them.  Returns the
// post-collision population of the lane's direction; on every lane f0_out,
// jx, jy and dr are the node's rest population, momentum and density deviation.
__device__ __forceinline__ float boundary8_collide(float fk, float g0, int kdir, float sx,
                                                   float sy, const Lattice &L, float &f0_out,
                                                   float &jx, float &jy, float &dr) {
    const int base = threadIdx.x & 24;  // first lane of the group within the warp
    float f[9];
    f[0] = g0;
#pragma unroll
    for (int m = 1; m < 9; ++m) f[m] = __shfl_sync(0xffffffffu, fk, base + m - 1);
    collide(f, sx, sy, L, dr, jx, jy);
    float mine = f[1];
#pragma unroll
    for (int q = 2; q < 9; ++q)
        if (kdir == q) mine = f[q];
    f0_out = f[0];
    return mine;
}

// Density deviation rho - rho0 of nine populations, summed as raw_moments
// forms m00 (so it equals moments(f).dr bit for bit); one node or two.
template <class V> __device__ __forceinline__ V density_of(const V f[9]) {
    const V a0 = radd(radd(f[7], f[4]), f[8]);
    const V b0 = radd(radd(f[3], f[0]), f[1]);
    const V c0 = radd(radd(f[6], f[2]), f[5]);
    return radd(radd(a0, b0), c0);
}

// The source coefficient (mu - lambda)/rho = (mu - lambda) times an
// approximate reciprocal of rho0 + drho (relative error about 1e-7; the same
// value in every kernel).
__device__ __forceinline__ float source_coef(float r0, const Lattice &L) {
    return rmul(L.mu_m_lam, __fdividef(1.0f, radd(L.rho0, r0)));
}
__device__ __forceinline__ F2 source_coef(F2 r0, const Lattice &L) {
    float a, b;
    f2_split(radd(splat<F2>(L.rho0), r0), a, b);
    return rmul(splat<F2>(L.mu_m_lam), f2(__fdividef(1.0f, a), __fdividef(1.0f, b)));
}

// Source S = F + (mu - lambda)/rho grad rho (Eq. sourceterm) from the density
// deviations of the node (r0) and of its axis neighbours: central differences,
// one-sided where one neighbour of an axis is across a wall (open flags false),
// zero where both are.  Deviations, so the differences do not cancel against
// rho0.  Explicitly rounded, so every kernel forms the same S.
__device__ __forceinline__ void grad_source(float r0, float rxp, float rxm, float ryp, float rym,
                                            bool xp, bool xm, bool yp, bool ym, const Lattice &L,
                                            float &sx, float &sy) {
    float gx = 0.0f, gy = 0.0f;
    if (xp && xm) gx = rmul(0.5f, rsub(rxp, rxm));
    else if (xp) gx = rsub(rxp, r0);
    else if (xm) gx = rsub(r0, rxm);
    if (yp && ym) gy = rmul(0.5f, rsub(ryp, rym));
    else if (yp) gy = rsub(ryp, r0);
    else if (ym) gy = rsub(r0, rym);
    const float c = source_coef(r0, L);
    sx = rfma(c, gx, L.fx);
    sy = rfma(c, gy, L.fy);
}

// The same for two nodes whose four axis neighbours are all material: the
// operations of grad_source with every flag set, paired.
__device__ __forceinline__ void grad_source_open(F2 r0, F2 rxp, F2 rxm, F2 ryp, F2 rym,
                                                 const Lattice &L, F2 &sx, F2 &sy) {
    const F2 half = splat<F2>(0.5f);
    const F2 gx = rmul(half, rsub(rxp, rxm)), gy = rmul(half, rsub(ryp, rym));
    const F2 c = source_coef(r0, L);
    sx = rfma(c, gx, splat<F2>(L.fx));
    sy = rfma(c, gy, splat<F2>(L.fy));
}

// Source at an interior node from a dense array of density deviations.
__device__ __forceinline__ void source_interior(const float *__restrict__ drho, int64_t k, int pitch,
                                                float drho_k, const Lattice &L, float &sx,
                                                float &sy) {
    sx = L.fx;
    sy = L.fy;
    if (L.grad)
        grad_source(drho_k, __ldg(drho + k + 1), __ldg(drho + k - 1), __ldg(drho + k + pitch),
                    __ldg(drho + k - pitch), true, true, true, true, L, sx, sy);
}

// Same at a boundary node: one-sided where a neighbour is across a wall.
__device__ __forceinline__ void source_boundary(const float *__restrict__ rho, const BNode &b,
                                                int64_t k, float drho_k, const Lattice &L,
                                                float &sx, float &sy) {
    sx = L.fx;
    sy = L.fy;
    if (!L.grad) return;
    const bool xp = !(b.cut & (1u << 1)), xm = !(b.cut & (1u << 3));
    const bool yp = !(b.cut & (1u << 2)), ym = !(b.cut & (1u << 4));
    const float rxp = xp ? rho[k + 1] : 0.0f, rxm = xm ? rho[k - 1] : 0.0f;
    const float ryp = yp ? rho[k + L.pitch] : 0.0f, rym = ym ? rho[k - L.pitch] : 0.0f;
    grad_source(drho_k, rxp, rxm, ryp, rym, xp, xm, yp, ym, L, sx, sy);
}

// Density deviation at time t of material node k: from the boundary pass for a
// boundary node (rho holds it), the sum of the pulled populations otherwise.
template <class T>
__device__ __forceinline__ float node_drho(const T *__restrict__ src,
                                           const uint8_t *__restrict__ cls,
                                           const float *__restrict__ rho, int64_t k,
                                           const Lattice &L) {
    if (__ldg(cls + k) != kInterior) return rho[k];
    float f[9];
    pull_interior(src, k, L.pitch, L.fplane, L.inv_scale, f);
    return moments(f).dr;
}

// The nine incoming populations of a boundary node held one per lane (group
// of eight lanes, direction k on lane k - 1; g0 = f_0), on every lane.
__device__ __forceinline__ void gather8(float fk, float g0, float f[9]) {
    const int base = threadIdx.x & 24;  // first lane of the group within the warp
    f[0] = g0;
#pragma unroll
    for (int m = 1; m < 9; ++m) f[m] = __shfl_sync(0xffffffffu, fk, base + m - 1);
}

// Source S = F + (mu - lambda)/rho grad rho (Eq. sourceterm) at a boundary node,
// one-sided where an axis neighbour is across a wall.  Lanes 0..3 of the group
// fetch the density of the neighbour in direction j + 1; the lanes then agree
// on the gradient through shuffles.  rho holds the boundary pass's deviations.
template <class T>
__device__ __forceinline__ void source_boundary8(const T *__restrict__ src,
                                                 const uint8_t *__restrict__ cls,
                                                 const float *__restrict__ rho, const BNode &b,
                                                 int64_t kn, const Lattice &L, int j, float &sx,
                                                 float &sy) {
    const int d = j < 4 ? j + 1 : 1;  // axis direction handled by this lane
    const bool open = !((b.cut >> d) & 1u);
    float mine = 0.0f;
    if (j < 4 && open) {
        const int64_t kk = kn + (int64_t)c_cy(d) * L.pitch + c_cx(d);
        mine = node_drho(src, cls, rho, kk, L);
    }
    const int base = threadIdx.x & ~7;
    const float rxp = __shfl_sync(0xffffffffu, mine, base + 0);
    const float ryp = __shfl_sync(0xffffffffu, mine, base + 1);
    const float rxm = __shfl_sync(0xffffffffu, mine, base + 2);
    const float rym = __shfl_sync(0xffffffffu, mine, base + 3);
    const bool xp = !((b.cut >> 1) & 1u), yp = !((b.cut >> 2) & 1u);
    const bool xm = !((b.cut >> 3) & 1u), ym = !((b.cut >> 4) & 1u);
    grad_source(rho[kn], rxp, rxm, ryp, rym, xp, xm, yp, ym, L, sx, sy);
}

// ---------------------------------------------------------------------------
// One interior node: pull (Eq. stream), moments with the source, collision
// (Eq. coll), store, displacement.  Every load -- the nine pulled
// populations and the displacement record -- is issued before any arithmetic.
// With kAA src and dst are the same buffer: the node reads all nine of its
// locations before it writes any.
template <class T, int LAY = kPull>
__device__ __forceinline__ void interior_node(const T *src, T *dst, URec<T> *__restrict__ uc,
                                              const uint8_t *__restrict__ cls,
                                              const float *__restrict__ rho, const Lattice &L,
                                              int64_t k, uint32_t *__restrict__ status) {
    if (__ldg(cls + k) != kInterior) return;
    float f[9];
    pull_interior_at<LAY>(src, k, L, f);
    URec<T> w = uc[k];
    float sx = L.fx, sy = L.fy;
    if (L.grad) source_interior(rho, k, L.pitch, rho[k], L, sx, sy);
    float dr, jx, jy;
    collide(f, sx, sy, L, dr, jx, jy);
#pragma unroll
    for (int i = 0; i < 9; ++i) Store<T>::st(dst + out_at<LAY>(k, i, L), f[i], L.scale);
    if constexpr (std::is_same<T, __half>::value) {
        float m = 0.0f;
#pragma unroll
        for (int i = 0; i < 9; ++i) m = fmaxf(m, fabsf(f[i]));
        note_range<T>(L, m);
    }
    integrate_u_value(w, jx, jy, L.rho0 + dr);
    uc[k] = w;
    flag_nonfinite(status, dr, jx, jy);
}

constexpr int kB8 = 128;  // threads per block of the cooperative boundary kernels (16 nodes)

// One boundary node g (a valid index of the compacted list) handled by the
// 8-lane group that lane j belongs to.  A group with live == false computes and
// stores nothing visible, so every lane can take part in the shuffles.
// With a non-null `stage` the node's nine post-collision populations go to
// stage[9 g + m] (FP32) instead of the buffer: the in-place form stores them
// only after every boundary node has read its inputs.
template <class T, int LAY = kPull>
__device__ __forceinline__ void boundary8_node(const T *src, T *dst, URec<T> *__restrict__ uc,
                                               const BNode *__restrict__ bnodes,
                                               const BLink *__restrict__ blinks,
                                               const BCDev *__restrict__ bcs,
                                               const uint8_t *__restrict__ cls,
                                               const float *__restrict__ rho, const Lattice &L,
                                               int g, bool live, int j, float tb,
                                               uint32_t *__restrict__ status,
                                               float *__restrict__ stage = nullptr) {
    const bool lane0 = j == 0;
    const BNode b = bnodes[g];
    const int kdir = j + 1;
    float f0;
    const float fk =
        pull_boundary8<T, LAY>(src, b, kdir, blinks + (int64_t)g * 8, bcs, tb, L, f0);
    const int64_t kn = (int64_t)b.y * L.pitch + b.x;
    float sx = L.fx, sy = L.fy;
    if (L.grad) source_boundary8(src, cls, rho, b, kn, L, j, sx, sy);
    float fr, jx, jy, m00;
    const float mine = boundary8_collide(fk, f0, kdir, sx, sy, L, fr, jx, jy, m00);
    if (!live) return;
    if (stage) {
        stage[(int64_t)g * 9 + kdir] = mine;
        if (lane0) stage[(int64_t)g * 9] = fr;
    } else {
        Store<T>::st(dst + out_at<LAY>(kn, kdir, L), mine, L.scale);
        if (lane0) Store<T>::st(dst + out_at<LAY>(kn, 0, L), fr, L.scale);
        note_range<T>(L, fmaxf(fabsf(mine), lane0 ? fabsf(fr) : 0.0f));
    }
    if (lane0) {
        integrate_u(uc + kn, jx, jy, L.rho0 + m00);
        flag_nonfinite(status, m00, jx, jy);
    }
}

// Incoming populations f(x, t) of a "simple" boundary node (every cut link a
// mid-link wall, kappa = 0 and 1 + kappa = 1, of one BC and one axis-aligned
// normal: box edges and crack faces), one lane per node.  ld(i, dx, dy) is
// f_i^col(x + (dx, dy), t - 1); masks have bit i for direction i (cut: link i
// crosses the wall; dirich: it takes the bounce-back rule; miss: its upstream
// node x - c_i is unusable); sl is the link record shared by the cut links.
// The wall data that do not depend on the link are formed once; every value is
// computed by the same explicitly rounded functions as in cut_link_value, so
// the result is that of the cooperative form bit for bit.  With kGuard no
// population is read across a cut link (ld may only address the lattice);
// without it those reads are issued unconditionally and their values replaced
// (ld addresses rows with halo columns).
template <bool kGuard, class Ld>
__device__ __forceinline__ void simple_pull(const Ld &ld, uint32_t cut, uint32_t dirich,
                                            uint32_t miss, const BLink &sl,
                                            const BCDev *__restrict__ bcs, float tb,
                                            const Lattice &L, float f[9]) {
    float g[9];
#pragma unroll
    for (int m = 0; m < 9; ++m) g[m] = ld(m, 0, 0);
    f[0] = g[0];
#pragma unroll
    for (int k = 1; k < 9; ++k)  // intact links (the cut ones are replaced below)
        f[k] = kGuard && ((cut >> opp(k)) & 1u) ? 0.0f : ld(k, -c_cx(k), -c_cy(k));
    const Mom mx = moments(g);
    float kap, fac;
    link_kappa(0.5f, kap, fac);
    if (dirich) {
        float jsx, jsy;
        dirichlet_momentum(sl, bcs, tb, L, jsx, jsy);
#pragma unroll
        for (int k = 1; k < 9; ++k) {
            const int i = opp(k);
            const uint32_t bit = 1u << i;
            if (!(cut & bit)) continue;
            const float gy_i = (miss & bit) ? 0.0f : ld(i, c_cx(k), c_cy(k));
            f[k] = bounce_back(k, kap, fac, g[k], g[i], gy_i, jsx, jsy);
        }
        return;
    }
    const WallFrame wf = wall_frame(sl, bcs, tb);
    // wall values at the node: the wall-node option, or no usable upstream node
    const WallState st0 = wall_state(false, 0.5f, mx.dr, mx.pxx, mx.pyy, mx.pxy, 0.0f, 0.0f, 0.0f,
                                     0.0f, L);
    float sxx, syy, sxy;
    wall_sigma(wf, st0, sxx, syy, sxy);
    const WallMoments wm0 = wall_moments(st0.drb, sxx, syy, sxy, L);
#pragma unroll
    for (int k = 1; k < 9; ++k) {
        const int i = opp(k);
        const uint32_t bit = 1u << i;
        if (!(cut & bit)) continue;
        const int cxk = c_cx(k), cyk = c_cy(k);
        const bool ms = (miss & bit) != 0;
        const float gy_i = ms ? 0.0f : ld(i, cxk, cyk);
        WallMoments wm = wm0;
        if (!ms && !L.wall_node) {
            // extrapolation along the link from the upstream node x - c_i
            float gy[9];
#pragma unroll
            for (int m = 0; m < 9; ++m) gy[m] = ld(m, cxk, cyk);
            const Mom my = moments(gy);
            const WallState st = wall_state(true, 0.5f, mx.dr, mx.pxx, mx.pyy, mx.pxy, my.dr,
                                            my.pxx, my.pyy, my.pxy, L);
            float ax, ay, axy;
            wall_sigma(wf, st, ax, ay, axy);
            wm = wall_moments(st.drb, ax, ay, axy, L);
        }
        f[k] = anti_bounce_back(kap, fac, g[k], g[i], gy_i, wall_equilibrium(k, wm));
    }
}

// Populations f^col(x + (dx, dy), t - 1) of a two-buffer lattice in device memory.
template <class T>
struct GlobalRows {
    const T *src;
    int64_t k, pitch, fplane;
    float inv_scale;
    __device__ __forceinline__ float operator()(int i, int dx, int dy) const {
        return Store<T>::ld(src + i * fplane + k + dy * pitch + dx, inv_scale);
    }
};

// One simple boundary node g of the list (two buffers, lambda = mu), one lane:
// the update of boundary8_node, bit for bit.
template <class T>
__device__ __forceinline__ void simple_node(const T *src, T *dst, URec<T> *__restrict__ uc,
                                            const BNode *__restrict__ bnodes,
                                            const BLink *__restrict__ blinks,
                                            const BCDev *__restrict__ bcs, const Lattice &L, int g,
                                            float tb, uint32_t *__restrict__ status) {
    const BNode b = bnodes[g];
    const int64_t k = (int64_t)b.y * L.pitch + b.x;
    const uint32_t cut = b.cut;
    const int d0 = __ffs((int)(cut >> 1));  // first cut direction, 1..8
    const BLink sl = blinks[(int64_t)g * 8 + (d0 > 0 ? d0 - 1 : 0)];
    float f[9];
    simple_pull<true>(GlobalRows<T>{src, k, L.pitch, L.fplane, L.inv_scale}, cut, b.dirich,
                      b.miss, sl, bcs, tb, L, f);
    URec<T> w = uc[k];
    float dr, jx, jy;
    collide(f, L.fx, L.fy, L, dr, jx, jy);
#pragma unroll
    for (int i = 0; i < 9; ++i) Store<T>::st(dst + i * L.fplane + k, f[i], L.scale);
    if constexpr (std::is_same<T, __half>::value) {
        float m = 0.0f;
#pragma unroll
        for (int i = 0; i < 9; ++i) m = fmaxf(m, fabsf(f[i]));
        note_range<T>(L, m);
    }
    integrate_u_value(w, jx, jy, L.rho0 + dr);
    uc[k] = w;
    flag_nonfinite(status, dr, jx, jy);
}

}  // namespace lbm
