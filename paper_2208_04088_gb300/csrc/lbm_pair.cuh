// Two horizontally adjacent interior nodes per thread with 16-bit storage, two
// buffers and lambda = mu (the one-step kernel of a single lattice and the
// batched interior kernel).  Part of the per-node code of the hot path: the
// pull of Eq. (stream), the collision of Eq. (coll) and the displacement
// update, for the nodes (x0, x0 + 1) with x0 even.
//
// Each population plane is read and written as aligned 32-bit pairs (the row
// pitch is a multiple of 64): the planes pulled straight up or down as one
// word, the others from two neighbouring words recombined with one byte
// permutation.  The pair collides with the f32x2 instructions.  Every value is
// the one interior_node forms for its node (the conversions, the power-of-two
// scalings and the paired arithmetic round each half as the scalar code does),
// and a node that is not interior reads nothing beyond its pair's own words and
// stores nothing.
#pragma once

#include <cstdint>
#include <cstring>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lbm_device.cuh"

namespace lbm {

template <class T> struct Pair16;
template <> struct Pair16<__half> {
    static __device__ __forceinline__ float2 to_f2(uint32_t w) {
        __half2 h;
        memcpy(&h, &w, 4);
        return __half22float2(h);
    }
    static __device__ __forceinline__ uint32_t from(float lo, float hi) {
        const __half2 h = __floats2half2_rn(lo, hi);
        uint32_t w;
        memcpy(&w, &h, 4);
        return w;
    }
};
template <> struct Pair16<__nv_bfloat16> {
    static __device__ __forceinline__ float2 to_f2(uint32_t w) {
        __nv_bfloat162 h;
        memcpy(&h, &w, 4);
        return __bfloat1622float2(h);
    }
    static __device__ __forceinline__ uint32_t from(float lo, float hi) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
        uint32_t w;
        memcpy(&w, &h, 4);
        return w;
    }
};

// The update of the pair at (x0, y), x0 even, x0 < nx, y < ny, with the
// step's scales in L.  Returns false, having read only the pair's node
// classes, when neither node is interior.
template <class T>
__device__ __forceinline__ bool interior_pair(const T *__restrict__ src, T *__restrict__ dst,
                                              float2 *__restrict__ uc,
                                              const uint8_t *__restrict__ cls, const Lattice &L,
                                              int x0, int y, uint32_t *__restrict__ status) {
    const int64_t k = (int64_t)y * L.pitch + x0;
    const uint32_t cc = __ldg(reinterpret_cast<const uint16_t *>(cls + k));
    const bool a = (cc & 0xffu) == kInterior;
    const bool b = x0 + 1 < L.nx && (cc >> 8) == kInterior;
    if (!a && !b) return false;
    // word of plane i at (x0 + 2 dw, y + dy): nodes x0 + 2 dw and x0 + 2 dw + 1
    auto word = [&](int i, int dw, int dy) {
        return __ldg(reinterpret_cast<const unsigned int *>(src + i * L.fplane + k +
                                                             (int64_t)dy * L.pitch) + dw);
    };
    uint32_t w[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int cx = c_cx(i), dy = -c_cy(i);
        const uint32_t w0 = word(i, 0, dy);
        if (cx == 0) {
            w[i] = w0;
        } else if (cx > 0) {  // from x - 1: (x0 - 1, x0)
            const uint32_t wm = a ? word(i, -1, dy) : 0u;
            w[i] = __byte_perm(wm, w0, 0x5432);
        } else {  // from x + 1: (x0 + 1, x0 + 2)
            const uint32_t wp = b ? word(i, 1, dy) : 0u;
            w[i] = __byte_perm(w0, wp, 0x5432);
        }
    }
    const float4 u2 = *reinterpret_cast<const float4 *>(uc + k);
    const F2 is2 = splat<F2>(L.inv_scale);
    F2 f[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const float2 v = Pair16<T>::to_f2(w[i]);
        f[i] = rmul(f2(v.x, v.y), is2);
    }
    F2 dr, jx, jy;
    collide_v(f, f2(L.fx, L.fx), f2(L.fy, L.fy), splat<F2>(L.omega),
              splat<F2>(rmul(L.src, 1.0f / 3.0f)), dr, jx, jy);
    const F2 sc2 = splat<F2>(L.scale);
    float m = 0.0f;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        float fa, fb;
        f2_split(f[i], fa, fb);
        if (a) m = fmaxf(m, fabsf(fa));
        if (b) m = fmaxf(m, fabsf(fb));
        float va, vb;
        f2_split(rmul(f[i], sc2), va, vb);
        T *o = dst + i * L.fplane + k;
        if (a && b) {
            *reinterpret_cast<uint32_t *>(o) = Pair16<T>::from(va, vb);
        } else if (a) {
            Store<T>::st(o, fa, L.scale);
        } else {
            Store<T>::st(o + 1, fb, L.scale);
        }
    }
    note_range<T>(L, m);
    float dra, drb, jxa, jxb, jya, jyb;
    f2_split(dr, dra, drb);
    f2_split(jx, jxa, jxb);
    f2_split(jy, jya, jyb);
    float2 ua = make_float2(u2.x, u2.y), ub = make_float2(u2.z, u2.w);
    if (a) {
        integrate_u_value(ua, jxa, jya, L.rho0 + dra);
        flag_nonfinite(status, dra, jxa, jya);
    }
    if (b) {
        integrate_u_value(ub, jxb, jyb, L.rho0 + drb);
        flag_nonfinite(status, drb, jxb, jyb);
    }
    if (a && b)
        *reinterpret_cast<float4 *>(uc + k) = make_float4(ua.x, ua.y, ub.x, ub.y);
    else if (a)
        uc[k] = ua;
    else
        uc[k + 1] = ub;
    return true;
}

}  // namespace lbm
