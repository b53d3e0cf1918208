// lbm_device.cuh -- device-side building blocks of the solid-LBM kernels:
// storage conversion, raw-moment collision, pull streaming and the boundary
// rules of Sec. 4.  Included by the single-solver kernels (lbm_kernels.cu) and
// the batched kernels (lbm_batch.cu), so both run the same arithmetic.
#pragma once

#include <cstdint>
#include <cstring>

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
// Raw moments m_pq = sum_i f_i c_ix^p c_iy^q (p, q in 0..2) of the nine
// populations.  D2Q9 is the tensor product of {-1, 0, 1} in x and y, so the
// transform is two passes of the 1-D map (a-, a0, a+) -> (a- + a0 + a+,
// a+ - a-, a+ + a-), whose inverse has only the coefficients 1 and 1/2: the
// round trip adds nothing but additions to the rounding.
struct Raw {
    float m00, m10, m01, m20, m02, m11, m21, m12, m22;
};

__device__ __forceinline__ Raw raw_moments(const float f[9]) {
    // rows c_y = -1: (f7, f4, f8); c_y = 0: (f3, f0, f1); c_y = +1: (f6, f2, f5)
    const float a0 = (f[7] + f[4]) + f[8], a1 = f[8] - f[7], a2 = f[8] + f[7];
    const float b0 = (f[3] + f[0]) + f[1], b1 = f[1] - f[3], b2 = f[1] + f[3];
    const float c0 = (f[6] + f[2]) + f[5], c1 = f[5] - f[6], c2 = f[5] + f[6];
    Raw m;
    m.m00 = (a0 + b0) + c0;
    m.m01 = c0 - a0;
    m.m02 = c0 + a0;
    m.m10 = (a1 + b1) + c1;
    m.m11 = c1 - a1;
    m.m12 = c1 + a1;
    m.m20 = (a2 + b2) + c2;
    m.m21 = c2 - a2;
    m.m22 = c2 + a2;
    return m;
}

__device__ __forceinline__ void populations(const Raw &m, float f[9]) {
    // inverse in y for each x-order p, then inverse in x for each row
    const float a0 = 0.5f * (m.m02 - m.m01), b0 = m.m00 - m.m02, c0 = 0.5f * (m.m02 + m.m01);
    const float a1 = 0.5f * (m.m12 - m.m11), b1 = m.m10 - m.m12, c1 = 0.5f * (m.m12 + m.m11);
    const float a2 = 0.5f * (m.m22 - m.m21), b2 = m.m20 - m.m22, c2 = 0.5f * (m.m22 + m.m21);
    f[7] = 0.5f * (a2 - a1);
    f[4] = a0 - a2;
    f[8] = 0.5f * (a2 + a1);
    f[3] = 0.5f * (b2 - b1);
    f[0] = b0 - b2;
    f[1] = 0.5f * (b2 + b1);
    f[6] = 0.5f * (c2 - c1);
    f[2] = c0 - c2;
    f[5] = 0.5f * (c2 + c1);
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
// On return f holds f^col, jx/jy the momentum j = m + S/2, dr the density deviation.
__device__ __forceinline__ void collide(float f[9], float sx, float sy, const Lattice &L,
                                        float &dr_out, float &jx_out, float &jy_out) {
    Raw m = raw_moments(f);
    const float jx = m.m10 + 0.5f * sx, jy = m.m01 + 0.5f * sy;
    const float w = L.omega;
    const float s3 = L.src * (1.0f / 3.0f);
    m.m10 += sx;
    m.m01 += sy;
    m.m21 += w * (jy * (1.0f / 3.0f) - m.m21) + s3 * sy;
    m.m12 += w * (jx * (1.0f / 3.0f) - m.m12) + s3 * sx;
    m.m22 += w * ((m.m20 + m.m02) * (1.0f / 3.0f) - m.m00 * (1.0f / 9.0f) - m.m22);
    dr_out = m.m00;
    jx_out = jx;
    jy_out = jy;
    populations(m, f);
}

// u(t+1) = u(t) + j/rho with Kahan compensation per component; w holds
// (u_x, u_y, compensation_x, compensation_y).
__device__ __forceinline__ void integrate_u_value(float4 &w, float jx, float jy, float rho) {
    const float vx = jx / rho, vy = jy / rho;
    float y = vx - w.z;
    float t = w.x + y;
    w.z = (t - w.x) - y;
    w.x = t;
    y = vy - w.w;
    t = w.y + y;
    w.w = (t - w.y) - y;
    w.y = t;
}

__device__ __forceinline__ void integrate_u(float4 *uc, float jx, float jy, float rho) {
    float4 w = *uc;
    const float vx = jx / rho, vy = jy / rho;
    float y = vx - w.z;
    float t = w.x + y;
    w.z = (t - w.x) - y;
    w.x = t;
    y = vy - w.w;
    t = w.y + y;
    w.w = (t - w.y) - y;
    w.y = t;
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
    if (b.profile == LBM_PROFILE_RAMP) return fminf(t / b.t_ramp, 1.0f);
    return 1.0f;
}

// Traction t*(t) of a Neumann condition on a wall with outward normal n.
__device__ __forceinline__ void traction(const BCDev &b, float n0, float n1, float t, float &tx,
                                         float &ty) {
    const float a = amplitude(b, t);
    if (b.kind == LBM_BC_PRESSURE) {
        tx = -b.v0 * n0 * a;
        ty = -b.v0 * n1 * a;
    } else if (b.kind == LBM_BC_STRESS) {
        tx = (b.v0 * n0 + b.v2 * n1) * a;
        ty = (b.v2 * n0 + b.v1 * n1) * a;
    } else {
        tx = b.v0 * a;
        ty = b.v1 * a;
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

// Populations f(x, t) of a boundary node: pulled where the link is intact,
// otherwise given by Eqs. (bbnoncon)/(abbnoncon) (which reduce to Eqs. bbcon/
// abbcon at s = l/2) from f^col(., t-1), rho(., t-1), sigma(., t-1) and the
// boundary data at t-1.  rho and P are collision invariants, so their values
// at t-1 are the moments of the stored post-collision populations.
template <class T>
__device__ __forceinline__ void pull_boundary(const T *__restrict__ src, const BNode &b,
                                              const BLink *__restrict__ links,
                                              const BCDev *__restrict__ bcs, float tb,
                                              const Lattice &L, float f[9]) {
    const int64_t k = (int64_t)b.y * L.pitch + b.x;
    const int64_t P = L.plane;
    // Phase 1: every load that depends only on the node record, issued before
    // any arithmetic so their latencies overlap.  Cut directions read the
    // node itself (a valid address whose value is not used).
    float gx[9], pl[9], gy1[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) gx[i] = Store<T>::ld(src + i * P + k, L.inv_scale);
#pragma unroll
    for (int kk = 1; kk < 9; ++kk) {
        const int i = opp(kk);
        const bool cut = (b.cut >> i) & 1u;
        const int64_t sk = cut ? k : k - (int64_t)c_cy(kk) * L.pitch - c_cx(kk);
        pl[kk] = Store<T>::ld(src + kk * P + sk, L.inv_scale);
        // f_i^col at the upstream node x - c_i of the cut link i (kappa term)
        const bool up = cut && !((b.miss >> i) & 1u);
        const int64_t ku = up ? k - (int64_t)c_cy(i) * L.pitch - c_cx(i) : k;
        gy1[i] = Store<T>::ld(src + i * P + ku, L.inv_scale);
    }
    const Mom mx = moments(gx);
    // Cauchy stress at x (Eq. poissonstress with Eq. approxdiv), deviation form
    const float dvx = -L.lam_m_mu_r0 * mx.dr;
    const float sxx_x = -mx.pxx + dvx, syy_x = -mx.pyy + dvx, sxy_x = -mx.pxy;

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
        const BLink lk = links[i - 1];
        const bool miss = (b.miss & bit) != 0;
        const float q = miss ? 0.5f : lk.q;
        const float kap = (1.0f - 2.0f * q) / (1.0f + 2.0f * q);
        const float fac = 2.0f / (1.0f + 2.0f * q);  // 1 + kappa = 2 l/(l + 2 s)
        const float w = (i <= 4) ? (1.0f / 9.0f) : (1.0f / 36.0f);
        const float cix = (float)c_cx(i), ciy = (float)c_cy(i);
        const float gy_i = miss ? 0.0f : gy1[i];
        if (b.dirich & bit) {
            const BCDev ba = bcs[lk.bc], bb = bcs[lk.bc2];
            const float aa = amplitude(ba, tb), ab = amplitude(bb, tb);
            // j* = rho0 d(u*)/dt (Eq. bcchaindir); corners: mean of the Dirichlet edges
            const float jsx = L.rho0 * 0.5f * (ba.v0 * aa + bb.v0 * ab);
            const float jsy = L.rho0 * 0.5f * (ba.v1 * aa + bb.v1 * ab);
            const float cj = cix * jsx + ciy * jsy;
            // Eq. (bbnoncon); kappa = 0 and 1 + kappa = 1 give Eq. (bbcon)
            f[kk] = gx[i] + kap * (gy_i - gx[kk]) - fac * (6.0f * w) * cj;
            continue;
        }
        // Neumann: density and stress at the wall by extrapolation along the link
        // (or the node's own values with the wall-node option)
        float drb = mx.dr, sbxx = sxx_x, sbyy = syy_x, sbxy = sxy_x;
        if (!miss && !L.wall_node) {
            const int64_t ku = k - (int64_t)c_cy(i) * L.pitch - c_cx(i);
            float gy[9];
#pragma unroll
            for (int m = 0; m < 9; ++m) gy[m] = Store<T>::ld(src + m * P + ku, L.inv_scale);
            const Mom my = moments(gy);
            const float dvy = -L.lam_m_mu_r0 * my.dr;
            const float a1 = 1.0f + q;
            drb = a1 * mx.dr - q * my.dr;
            sbxx = a1 * sxx_x - q * (-my.pxx + dvy);
            sbyy = a1 * syy_x - q * (-my.pyy + dvy);
            sbxy = a1 * sxy_x - q * (-my.pxy);
        }
        float sxx, syy, sxy;  // sigma* (Eq. trafocauchy)
        if (b.corner & bit) {
            float tax, tay, tbx, tby;
            traction(bcs[lk.bc], lk.n0, 0.0f, tb, tax, tay);
            traction(bcs[lk.bc2], 0.0f, lk.n1, tb, tbx, tby);
            sxx = tax * lk.n0;
            syy = tby * lk.n1;
            sxy = 0.5f * (tay * lk.n0 + tbx * lk.n1);
        } else {
            const float n0 = lk.n0, n1 = lk.n1, t0 = -n1, t1 = n0;  // e^n, e^t
            float tx, ty;
            traction(bcs[lk.bc], n0, n1, tb, tx, ty);
            const float tn = tx * n0 + ty * n1, tt = tx * t0 + ty * t1;
            const float stt = t0 * t0 * sbxx + 2.0f * t0 * t1 * sbxy + t1 * t1 * sbyy;
            sxx = tn * n0 * n0 + 2.0f * tt * n0 * t0 + stt * t0 * t0;
            syy = tn * n1 * n1 + 2.0f * tt * n1 * t1 + stt * t1 * t1;
            sxy = tn * n0 * n1 + tt * (n0 * t1 + t0 * n1) + stt * t0 * t1;
        }
        // P* = -sigma* + (lambda - mu) div u I, div u = (rho0 - rho^bd)/rho0 (Eq. bcchainneum)
        const float dv = -L.lam_m_mu_r0 * drb;
        const float pxx = -sxx + dv, pyy = -syy + dv, pxy = -sxy;
        const float axx = pxx - drb * (1.0f / 3.0f), ayy = pyy - drb * (1.0f / 3.0f);
        const float con = 4.5f * (cix * cix * axx + 2.0f * cix * ciy * pxy + ciy * ciy * ayy -
                                  (axx + ayy) * (1.0f / 3.0f));
        const float eq = 2.0f * w * (drb + con);
        // Eq. (abbnoncon); kappa = 0 and 1 + kappa = 1 give Eq. (abbcon)
        f[kk] = -gx[i] - kap * (gy_i + gx[kk]) + fac * eq;
    }
}

// ---------------------------------------------------------------------------
// Cooperative boundary update: eight lanes per boundary node.  Lane j owns the
// population k = j + 1 and the link i = opp(k) through which it arrives; lane
// 0 also carries the rest population.  Moments are formed with butterfly
// shuffles inside the 8-lane group (every lane ends with bit-identical sums,
// since each pairwise addition is commutative), so a node's loads are issued
// by eight lanes at once and its serial chain is an eighth of the single-thread
// form above.
__device__ __forceinline__ float grp8_sum(float v) {
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    return v;
}

__device__ __forceinline__ int lane_cx(int k) {
    return (k == 1 || k == 5 || k == 8) ? 1 : (k == 3 || k == 6 || k == 7) ? -1 : 0;
}
__device__ __forceinline__ int lane_cy(int k) {
    return (k == 2 || k == 5 || k == 6) ? 1 : (k == 4 || k == 7 || k == 8) ? -1 : 0;
}

// Raw moments of a node's populations held one per lane (+ f0 on lane 0).
__device__ __forceinline__ Raw grp8_raw(float fk, float f0, int cx, int cy, bool lane0) {
    const float cxx = (float)(cx * cx), cyy = (float)(cy * cy);
    Raw m;
    m.m00 = grp8_sum(fk + (lane0 ? f0 : 0.0f));
    m.m10 = grp8_sum(cx * fk);
    m.m01 = grp8_sum(cy * fk);
    m.m20 = grp8_sum(cxx * fk);
    m.m02 = grp8_sum(cyy * fk);
    m.m11 = grp8_sum((float)(cx * cy) * fk);
    m.m21 = grp8_sum(cxx * cy * fk);
    m.m12 = grp8_sum(cx * cyy * fk);
    m.m22 = grp8_sum(cxx * cyy * fk);
    return m;
}

// f_k(x, t) for lane k of a boundary node (and f_0 on lane 0): pulled where
// link opp(k) is intact, otherwise Eqs. (bbnoncon)/(abbnoncon).  Same rules
// and data as pull_boundary.
template <class T>
__device__ __forceinline__ float pull_boundary8(const T *__restrict__ src, const BNode &b, int k,
                                                const BLink *__restrict__ links,
                                                const BCDev *__restrict__ bcs, float tb,
                                                const Lattice &L, bool lane0, float &f0) {
    const int64_t kn = (int64_t)b.y * L.pitch + b.x;
    const int64_t P = L.plane;
    const int i = k <= 4 ? (k + 1) % 4 + 1 : (k - 3) % 4 + 5;  // opp(k)
    const int cxk = lane_cx(k), cyk = lane_cy(k);
    const int cxi = -cxk, cyi = -cyk;
    const uint32_t bit = 1u << i;
    const bool cut = (b.cut & bit) != 0;
    const bool miss = (b.miss & bit) != 0;
    // loads, all independent
    const float gk = Store<T>::ld(src + k * P + kn, L.inv_scale);      // f_k^col(x)
    const float gi = Store<T>::ld(src + i * P + kn, L.inv_scale);      // f_i^col(x)
    f0 = lane0 ? Store<T>::ld(src + kn, L.inv_scale) : 0.0f;           // f_0^col(x)
    const int64_t kpull = cut ? kn : kn - (int64_t)cyk * L.pitch - cxk;
    const float pulled = Store<T>::ld(src + k * P + kpull, L.inv_scale);
    const int64_t ku = (cut && !miss) ? kn - (int64_t)cyi * L.pitch - cxi : kn;
    const float gy_i = (cut && !miss) ? Store<T>::ld(src + i * P + ku, L.inv_scale) : 0.0f;
    const bool neu_ex = cut && !miss && !L.wall_node && !(b.dirich & bit);
    float my_dr = 0.0f, my_xx = 0.0f, my_yy = 0.0f, my_xy = 0.0f;
    if (neu_ex) {
        float gy[9];
#pragma unroll
        for (int m = 0; m < 9; ++m) gy[m] = Store<T>::ld(src + m * P + ku, L.inv_scale);
        const Mom my = moments(gy);
        my_dr = my.dr;
        my_xx = my.pxx;
        my_yy = my.pyy;
        my_xy = my.pxy;
    }
    BLink lk;
    if (cut) lk = links[i - 1];
    // moments of f^col(x, t-1) (rho and P are collision invariants)
    const float cxf = (float)cxk, cyf = (float)cyk;
    const float dr_x = grp8_sum(gk + f0);
    const float pxx_x = grp8_sum(cxf * cxf * gk);
    const float pyy_x = grp8_sum(cyf * cyf * gk);
    const float pxy_x = grp8_sum(cxf * cyf * gk);
    if (!cut) return pulled;
    const float q = miss ? 0.5f : lk.q;
    const float kap = (1.0f - 2.0f * q) / (1.0f + 2.0f * q);
    const float fac = 2.0f / (1.0f + 2.0f * q);
    const float w = (i <= 4) ? (1.0f / 9.0f) : (1.0f / 36.0f);
    const float cix = (float)cxi, ciy = (float)cyi;
    if (b.dirich & bit) {
        const BCDev ba = bcs[lk.bc], bb = bcs[lk.bc2];
        const float aa = amplitude(ba, tb), ab = amplitude(bb, tb);
        const float jsx = L.rho0 * 0.5f * (ba.v0 * aa + bb.v0 * ab);
        const float jsy = L.rho0 * 0.5f * (ba.v1 * aa + bb.v1 * ab);
        const float cj = cix * jsx + ciy * jsy;
        return gi + kap * (gy_i - gk) - fac * (6.0f * w) * cj;
    }
    const float dvx = -L.lam_m_mu_r0 * dr_x;
    const float sxx_x = -pxx_x + dvx, syy_x = -pyy_x + dvx, sxy_x = -pxy_x;
    float drb = dr_x, sbxx = sxx_x, sbyy = syy_x, sbxy = sxy_x;
    if (neu_ex) {
        const float dvy = -L.lam_m_mu_r0 * my_dr;
        const float a1 = 1.0f + q;
        drb = a1 * dr_x - q * my_dr;
        sbxx = a1 * sxx_x - q * (-my_xx + dvy);
        sbyy = a1 * syy_x - q * (-my_yy + dvy);
        sbxy = a1 * sxy_x - q * (-my_xy);
    }
    float sxx, syy, sxy;
    if (b.corner & bit) {
        float tax, tay, tbx, tby;
        traction(bcs[lk.bc], lk.n0, 0.0f, tb, tax, tay);
        traction(bcs[lk.bc2], 0.0f, lk.n1, tb, tbx, tby);
        sxx = tax * lk.n0;
        syy = tby * lk.n1;
        sxy = 0.5f * (tay * lk.n0 + tbx * lk.n1);
    } else {
        const float n0 = lk.n0, n1 = lk.n1, t0 = -n1, t1 = n0;
        float tx, ty;
        traction(bcs[lk.bc], n0, n1, tb, tx, ty);
        const float tn = tx * n0 + ty * n1, tt = tx * t0 + ty * t1;
        const float stt = t0 * t0 * sbxx + 2.0f * t0 * t1 * sbxy + t1 * t1 * sbyy;
        sxx = tn * n0 * n0 + 2.0f * tt * n0 * t0 + stt * t0 * t0;
        syy = tn * n1 * n1 + 2.0f * tt * n1 * t1 + stt * t1 * t1;
        sxy = tn * n0 * n1 + tt * (n0 * t1 + t0 * n1) + stt * t0 * t1;
    }
    const float dv = -L.lam_m_mu_r0 * drb;
    const float pxx = -sxx + dv, pyy = -syy + dv, pxy = -sxy;
    const float axx = pxx - drb * (1.0f / 3.0f), ayy = pyy - drb * (1.0f / 3.0f);
    const float con = 4.5f * (cix * cix * axx + 2.0f * cix * ciy * pxy + ciy * ciy * ayy -
                              (axx + ayy) * (1.0f / 3.0f));
    const float eq = 2.0f * w * (drb + con);
    return -gi - kap * (gy_i + gk) + fac * eq;
}

// Source S = F + (mu - lambda)/rho grad rho at an interior node (central
// differences).  `drho` holds density deviations rho - rho0, so the differences
// do not cancel against rho0.
__device__ __forceinline__ void source_interior(const float *__restrict__ drho, int64_t k, int pitch,
                                                float drho_k, const Lattice &L, float &sx,
                                                float &sy) {
    sx = L.fx;
    sy = L.fy;
    if (L.grad) {
        const float gx = 0.5f * (__ldg(drho + k + 1) - __ldg(drho + k - 1));
        const float gy = 0.5f * (__ldg(drho + k + pitch) - __ldg(drho + k - pitch));
        const float c = L.mu_m_lam / (L.rho0 + drho_k);
        sx += c * gx;
        sy += c * gy;
    }
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
    const float r0 = rho[k];
    float gx = 0.0f, gy = 0.0f;
    if (xp && xm) gx = 0.5f * (rho[k + 1] - rho[k - 1]);
    else if (xp) gx = rho[k + 1] - r0;
    else if (xm) gx = r0 - rho[k - 1];
    if (yp && ym) gy = 0.5f * (rho[k + L.pitch] - rho[k - L.pitch]);
    else if (yp) gy = rho[k + L.pitch] - r0;
    else if (ym) gy = r0 - rho[k - L.pitch];
    const float c = L.mu_m_lam / (L.rho0 + drho_k);
    sx += c * gx;
    sy += c * gy;
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
    pull_interior(src, k, L.pitch, L.plane, L.inv_scale, f);
    return moments(f).dr;
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
    const float r0 = rho[kn];
    float gx = 0.0f, gy = 0.0f;
    if (xp && xm) gx = 0.5f * (rxp - rxm);
    else if (xp) gx = rxp - r0;
    else if (xm) gx = r0 - rxm;
    if (yp && ym) gy = 0.5f * (ryp - rym);
    else if (yp) gy = ryp - r0;
    else if (ym) gy = r0 - rym;
    const float c = L.mu_m_lam / (L.rho0 + r0);
    sx += c * gx;
    sy += c * gy;
}

// ---------------------------------------------------------------------------
// One interior node: pull (Eq. stream), moments with the source, collision
// (Eq. coll), store, displacement.  Every load -- the nine pulled
// populations and the displacement record -- is issued before any arithmetic.
template <class T>
__device__ __forceinline__ void interior_node(const T *__restrict__ src, T *__restrict__ dst,
                                              float4 *__restrict__ uc,
                                              const uint8_t *__restrict__ cls,
                                              const float *__restrict__ rho, const Lattice &L,
                                              int64_t k, uint32_t *__restrict__ status) {
    if (__ldg(cls + k) != kInterior) return;
    float f[9];
    pull_interior(src, k, L.pitch, L.plane, L.inv_scale, f);
    float4 w = uc[k];
    float sx = L.fx, sy = L.fy;
    if (L.grad) source_interior(rho, k, L.pitch, rho[k], L, sx, sy);
    float dr, jx, jy;
    collide(f, sx, sy, L, dr, jx, jy);
#pragma unroll
    for (int i = 0; i < 9; ++i) Store<T>::st(dst + i * L.plane + k, f[i], L.scale);
    integrate_u_value(w, jx, jy, L.rho0 + dr);
    uc[k] = w;
    flag_nonfinite(status, dr, jx, jy);
}

constexpr int kB8 = 128;  // threads per block of the cooperative boundary kernels (16 nodes)

// One boundary node g (a valid index of the compacted list) handled by the
// 8-lane group that lane j belongs to.  A group with live == false computes and
// stores nothing visible, so every lane can take part in the shuffles.
template <class T>
__device__ __forceinline__ void boundary8_node(const T *__restrict__ src, T *__restrict__ dst,
                                               float4 *__restrict__ uc,
                                               const BNode *__restrict__ bnodes,
                                               const BLink *__restrict__ blinks,
                                               const BCDev *__restrict__ bcs,
                                               const uint8_t *__restrict__ cls,
                                               const float *__restrict__ rho, const Lattice &L,
                                               int g, bool live, int j, float tb,
                                               uint32_t *__restrict__ status) {
    const bool lane0 = j == 0;
    const BNode b = bnodes[g];
    const int kdir = j + 1;
    float f0;
    const float fk = pull_boundary8(src, b, kdir, blinks + (int64_t)g * 8, bcs, tb, L, lane0, f0);
    const int64_t kn = (int64_t)b.y * L.pitch + b.x;
    float sx = L.fx, sy = L.fy;
    if (L.grad) source_boundary8(src, cls, rho, b, kn, L, j, sx, sy);
    // collision on the raw moments (as collide())
    const int cx = lane_cx(kdir), cy = lane_cy(kdir);
    Raw m = grp8_raw(fk, f0, cx, cy, lane0);
    const float jx = m.m10 + 0.5f * sx, jy = m.m01 + 0.5f * sy;
    const float w = L.omega;
    const float s3 = L.src * (1.0f / 3.0f);
    m.m10 += sx;
    m.m01 += sy;
    m.m21 += w * (jy * (1.0f / 3.0f) - m.m21) + s3 * sy;
    m.m12 += w * (jx * (1.0f / 3.0f) - m.m12) + s3 * sx;
    m.m22 += w * ((m.m20 + m.m02) * (1.0f / 3.0f) - m.m00 * (1.0f / 9.0f) - m.m22);
    float f[9];
    populations(m, f);
    float mine = f[1];
#pragma unroll
    for (int q = 2; q < 9; ++q)
        if (kdir == q) mine = f[q];
    if (!live) return;
    Store<T>::st(dst + kdir * L.plane + kn, mine, L.scale);
    if (lane0) {
        Store<T>::st(dst + kn, f[0], L.scale);
        integrate_u(uc + kn, jx, jy, L.rho0 + m.m00);
        flag_nonfinite(status, m.m00, jx, jy);
    }
}

}  // namespace lbm
