// lbm_kernels.cu -- sm_103a kernels of the solid lattice Boltzmann method
// (arXiv 2208.04088): one time step is
//   [density pass, lambda != mu only]  rho(t) at every material node
//   interior kernel   pull-stream + moments + BGK with source + store + u
//   boundary kernel   the same for the compacted list of boundary nodes, with
//                     the populations arriving across a wall replaced by the
//                     rules of Sec. 4
// Distributions are stored as deviations from the zero-stress rest state,
// delta f = f - f^eq(rho0, 0, 0), in structure-of-arrays planes
// [9][ny][pitch].  The buffer holds f^col(t-1); a step pulls f_i(x, t) =
// f_i^col(x - c_i, t-1) (Eq. stream), collides (Eq. coll) and writes f^col(x, t)
// to the other buffer, or, with in-place streaming, to the same buffer in the
// AA pattern (see col_at / out_at).
// All arithmetic is FP32.  The rest state is a fixed point of every rule, so
// each rule acts on the deviations with the same coefficients it has for f.
#include <cstdint>
#include <cstring>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "lbm_device.cuh"
#include "lbm_internal.h"
#include "lbm_pair.cuh"

namespace lbm {
// ---------------------------------------------------------------------------
// Kernels.
constexpr int kBX = 32, kBY = 8;
constexpr int kBB = 64;  // threads per block of the boundary-list kernels

// Interior kernel: one node per thread (NR rows per thread, kBY rows apart).
// Every load of a node -- the nine pulled populations and the displacement
// record -- is issued before any arithmetic, so all of them are in flight
// together.
// With FP16 storage the kernel takes its step's scales from the solver's
// record (step t = *time + toff), and its first thread publishes them.
template <class T>
__device__ __forceinline__ int64_t scales_of_step(Lattice &L, const int64_t *time, int toff,
                                                  bool publisher) {
    int64_t t = 0;
    if constexpr (std::is_same<T, __half>::value) {
        t = *time + toff;
        step_scales<T>(L, t);
        if (publisher) publish_scale<T>(L, t);
    }
    return t;
}

template <class T, int NR, int LAY = kPull>
__global__ void __launch_bounds__(kBX *kBY, 8) k_interior(const T *src, T *dst,
                                                       URec<T> *__restrict__ uc,
                                                       const uint8_t *__restrict__ cls,
                                                       const float *__restrict__ rho, Lattice L,
                                                       uint32_t *__restrict__ status,
                                                       const int64_t *__restrict__ time, int toff) {
    const int x = blockIdx.x * kBX + threadIdx.x;
    const int y0 = blockIdx.y * (kBY * NR) + threadIdx.y;
    scales_of_step<T>(L, time, toff, x == 0 && y0 == 0);
    if (x >= L.nx) return;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const int y = y0 + r * kBY;
        if (y < L.ny)
            interior_node<T, LAY>(src, dst, uc, cls, rho, L, (int64_t)y * L.pitch + x, status);
    }
}

// 16-bit storage, two buffers, lambda = mu: two adjacent nodes per thread
// (interior_pair).  Blocks per SM the register bound aims at: FP16 measured fastest at six (40
// registers: 93.9 against 90.4 GLUPS at four on the 2048^2 crack), BF16 at four
// (100.7 against 98.9 at six).
template <class T> constexpr int kPairMinBlocks = std::is_same<T, __half>::value ? 6 : 4;

template <class T>
__global__ void __launch_bounds__(kBX *kBY, kPairMinBlocks<T>) k_interior_pair(const T *__restrict__ src,
                                                            T *__restrict__ dst,
                                                            float2 *__restrict__ uc,
                                                            const uint8_t *__restrict__ cls,
                                                            Lattice L,
                                                            uint32_t *__restrict__ status,
                                                            const int64_t *__restrict__ time,
                                                            int toff) {
    const int x0 = 2 * (int)(blockIdx.x * kBX + threadIdx.x);
    const int y = blockIdx.y * kBY + threadIdx.y;
    // FP16: this step's scales.  The thread of node (0, 0), which is never
    // interior, publishes them after its node classes have been read, so that
    // no store sits between the loads of a thread and delays them.
    const int64_t t = scales_of_step<T>(L, time, toff, false);
    if (x0 >= L.nx || y >= L.ny) return;
    if (!interior_pair<T>(src, dst, uc, cls, L, x0, y, status) && x0 == 0 && y == 0)
        publish_scale<T>(L, t);
}

// Interior kernel for lambda != mu: the density deviations of the tile and a
// one-node ring around it are formed in shared memory (tile nodes from their
// own pulled populations, ring nodes by pulling theirs, boundary nodes from the
// boundary density pass), then the central differences of grad rho feed the
// source of Eq. (sourceterm).  No full-lattice density pass is needed.
constexpr int kGY = 8;  // rows of the lambda != mu tile (16 measured slower)

template <class T>
__global__ void __launch_bounds__(kBX *kGY) k_interior_grad(const T *__restrict__ src,
                                                            T *__restrict__ dst,
                                                            URec<T> *__restrict__ uc,
                                                            const uint8_t *__restrict__ cls,
                                                            const float *__restrict__ rho,
                                                            Lattice L,
                                                            uint32_t *__restrict__ status,
                                                            const int64_t *__restrict__ time,
                                                            int toff) {
    __shared__ float rs[kGY + 2][kBX + 2];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x0 = blockIdx.x * kBX, y0 = blockIdx.y * kGY;
    scales_of_step<T>(L, time, toff, x0 + tx == 0 && y0 + ty == 0);
    const int x = x0 + tx, y = y0 + ty;
    // the ring: top and bottom rows (kBX + 2 each), left and right columns (kGY each)
    const int tid = ty * kBX + tx;
    constexpr int kRing = 2 * (kBX + 2) + 2 * kGY;
    int hx = 0, hy = 0;
    int64_t kk = -1;  // lattice index of this thread's ring node, if any
    if (tid < kRing) {
        if (tid < kBX + 2) {
            hx = tid;
            hy = 0;
        } else if (tid < 2 * (kBX + 2)) {
            hx = tid - (kBX + 2);
            hy = kGY + 1;
        } else if (tid < 2 * (kBX + 2) + kGY) {
            hx = 0;
            hy = tid - 2 * (kBX + 2) + 1;
        } else {
            hx = kBX + 1;
            hy = tid - 2 * (kBX + 2) - kGY + 1;
        }
        const int gx = x0 - 1 + hx, gy = y0 - 1 + hy;
        if (gx >= 0 && gx < L.nx && gy >= 0 && gy < L.ny) kk = (int64_t)gy * L.pitch + gx;
    }
    // the node's and the ring node's loads are all issued before either
    // density is summed, so a ring thread waits for one memory round trip
    bool live = false, ring_int = false;
    float f[9], g[9];
    URec<T> w{};
    int64_t k = 0;
    float own = 0.0f, v = 0.0f;
    uint8_t c = kVoid, cr = kVoid;
    if (x < L.nx && y < L.ny) {
        k = (int64_t)y * L.pitch + x;
        c = __ldg(cls + k);
    }
    if (kk >= 0) cr = __ldg(cls + kk);
    if (c == kInterior) {
        live = true;
        pull_interior(src, k, L.pitch, L.fplane, L.inv_scale, f);
        w = uc[k];
    }
    if (cr == kInterior) {
        ring_int = true;
        pull_interior(src, kk, L.pitch, L.fplane, L.inv_scale, g);
    }
    if (live) own = moments(f).dr;
    else if (c == kBoundary) own = rho[k];
    if (ring_int) v = moments(g).dr;
    else if (cr == kBoundary) v = rho[kk];
    rs[ty + 1][tx + 1] = own;
    if (tid < kRing) rs[hy][hx] = v;
    __syncthreads();
    if (!live) return;
    // interior nodes have all four axis neighbours: central differences
    float sx, sy;
    grad_source(own, rs[ty + 1][tx + 2], rs[ty + 1][tx], rs[ty + 2][tx + 1], rs[ty][tx + 1], true,
                true, true, true, L, sx, sy);
    float dr, jx, jy;
    collide(f, sx, sy, L, dr, jx, jy);
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

template <class T, int LAY = kPull>
__global__ void __launch_bounds__(kB8) k_boundary8(const T *src, T *dst, URec<T> *__restrict__ uc,
                                                   const BNode *__restrict__ bnodes,
                                                   const BLink *__restrict__ blinks,
                                                   const BCDev *__restrict__ bcs,
                                                   const uint8_t *__restrict__ cls,
                                                   const float *__restrict__ rho, Lattice L,
                                                   const int64_t *__restrict__ time, int toff,
                                                   uint32_t *__restrict__ status,
                                                   float *__restrict__ stage) {
    const int g = (blockIdx.x * kB8 + threadIdx.x) >> 3;  // boundary node of this lane group
    const float tb = (float)(*time + toff - 1);           // boundary data at the time of f^col
    scales_of_step<T>(L, time, toff, false);
    // groups past the end of the list work on node 0 and store nothing
    const bool live = g < L.nb;
    boundary8_node<T, LAY>(src, dst, uc, bnodes, blinks, bcs, cls, rho, L, live ? g : 0, live,
                           threadIdx.x & 7, tb, status, stage);
}

// In-place streaming: the post-collision populations of the boundary nodes,
// staged by k_boundary8, into the buffer (one thread per node and direction).
template <class T, int LAY>
__global__ void __launch_bounds__(kBB) k_boundary_scatter(const float *__restrict__ stage,
                                                          T *dst,
                                                          const BNode *__restrict__ bnodes,
                                                          Lattice L,
                                                          const int64_t *__restrict__ time,
                                                          int toff) {
    scales_of_step<T>(L, time, toff, false);
    const int64_t e = (int64_t)blockIdx.x * kBB + threadIdx.x;
    if (e >= (int64_t)L.nb * 9) return;
    const int g = (int)(e / 9), m = (int)(e % 9);
    const BNode b = bnodes[g];
    const int64_t kn = (int64_t)b.y * L.pitch + b.x;
    int64_t o = 0;
    switch (m) {  // out_at for a run-time direction
#define LBM_OUT(mm) \
    case mm:        \
        o = out_at<LAY>(kn, mm, L); \
        break;
        LBM_OUT(0) LBM_OUT(1) LBM_OUT(2) LBM_OUT(3) LBM_OUT(4) LBM_OUT(5) LBM_OUT(6) LBM_OUT(7) LBM_OUT(8)
#undef LBM_OUT
    }
    Store<T>::st(dst + o, stage[e], L.scale);
    note_range<T>(L, fabsf(stage[e]));
}

// Density at time t of every material node (lambda != mu): pull, with the
// boundary rules at boundary nodes.  Writes the deviation rho - rho0 into a
// dense [ny][pitch] array.
template <class T>
__global__ void __launch_bounds__(kBX *kBY) k_density_interior(const T *__restrict__ src,
                                                               const uint8_t *__restrict__ cls,
                                                               float *__restrict__ rho, Lattice L,
                                                               const int64_t *__restrict__ time) {
    scales_of_step<T>(L, time, 0, false);
    const int x = blockIdx.x * kBX + threadIdx.x;
    const int y = blockIdx.y * kBY + threadIdx.y;
    if (x >= L.nx || y >= L.ny) return;
    const int64_t k = (int64_t)y * L.pitch + x;
    if (cls[k] != kInterior) return;
    float f[9];
    pull_interior(src, k, L.pitch, L.fplane, L.inv_scale, f);
    rho[k] = moments(f).dr;
}

template <class T>
__global__ void __launch_bounds__(kBB) k_density_boundary(const T *__restrict__ src,
                                                          const BNode *__restrict__ bnodes,
                                                          const BLink *__restrict__ blinks,
                                                          const BCDev *__restrict__ bcs,
                                                          float *__restrict__ rho, Lattice L,
                                                          const int64_t *__restrict__ time,
                                                          int toff) {
    scales_of_step<T>(L, time, toff, false);
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= L.nb) return;
    const BNode b = bnodes[m];
    const float tb = (float)(*time + toff - 1);
    float f[9];
    pull_boundary(src, b, blinks + (int64_t)m * 8, bcs, tb, L, f);
    rho[(int64_t)b.y * L.pitch + b.x] = moments(f).dr;
}

// Fields at the current time t (Eqs. moments, poissonstress, approxdiv).
template <class W>
__device__ __forceinline__ void write_fields(float *__restrict__ out, int64_t N, int64_t o,
                                             const float f[9], float sx, float sy, const W &w,
                                             const Lattice &L) {
    const Mom m = moments(f);
    const float jx = m.mx + 0.5f * sx, jy = m.my + 0.5f * sy;
    const float rho = L.rho0 + m.dr;
    const float dv = -L.lam_m_mu_r0 * m.dr;
    const float2 u = u_of(w);
    out[o] = u.x * L.out_u;
    out[N + o] = u.y * L.out_u;
    out[2 * N + o] = jx / rho * L.out_v;
    out[3 * N + o] = jy / rho * L.out_v;
    out[4 * N + o] = (-m.pxx + dv) * L.out_s;
    out[5 * N + o] = (-m.pyy + dv) * L.out_s;
    out[6 * N + o] = (-m.pxy) * L.out_s;
}

template <class T, int LAY = kPull>
__global__ void __launch_bounds__(kBX *kBY) k_fields_interior(const T *__restrict__ src,
                                                              const URec<T> *__restrict__ uc,
                                                              const uint8_t *__restrict__ cls,
                                                              const float *__restrict__ rho,
                                                              Lattice L, float *__restrict__ out,
                                                              const int64_t *__restrict__ time) {
    scales_of_step<T>(L, time, 0, false);  // the populations stored by the last step
    const int x = blockIdx.x * kBX + threadIdx.x;
    const int y = blockIdx.y * kBY + threadIdx.y;
    if (x >= L.nx || y >= L.ny) return;
    const int64_t k = (int64_t)y * L.pitch + x;
    const int64_t N = (int64_t)L.nx * L.ny, o = (int64_t)y * L.nx + x;
    const uint8_t c = cls[k];
    if (c == kBoundary) return;
    if (c == kVoid) {
#pragma unroll
        for (int a = 0; a < 7; ++a) out[a * N + o] = 0.0f;
        return;
    }
    float f[9];
    pull_interior_at<LAY>(src, k, L, f);
    float sx = L.fx, sy = L.fy;
    if (L.grad) source_interior(rho, k, L.pitch, rho[k], L, sx, sy);
    write_fields(out, N, o, f, sx, sy, uc[k], L);
}

template <class T, int LAY = kPull>
__global__ void __launch_bounds__(kBB) k_fields_boundary(const T *__restrict__ src,
                                                         const URec<T> *__restrict__ uc,
                                                         const BNode *__restrict__ bnodes,
                                                         const BLink *__restrict__ blinks,
                                                         const BCDev *__restrict__ bcs,
                                                         const float *__restrict__ rho, Lattice L,
                                                         const int64_t *__restrict__ time,
                                                         float *__restrict__ out) {
    scales_of_step<T>(L, time, 0, false);  // the populations stored by the last step
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= L.nb) return;
    const BNode b = bnodes[m];
    const float tb = (float)(*time - 1);
    float f[9];
    pull_boundary<T, LAY>(src, b, blinks + (int64_t)m * 8, bcs, tb, L, f);
    const int64_t k = (int64_t)b.y * L.pitch + b.x;
    float sx = L.fx, sy = L.fy;
    if (L.grad) source_boundary(rho, b, k, rho[k], L, sx, sy);
    const int64_t N = (int64_t)L.nx * L.ny, o = (int64_t)b.y * L.nx + b.x;
    write_fields(out, N, o, f, sx, sy, uc[k], L);
}

__global__ void k_advance(int64_t *time, int64_t n) { *time += n; }

// The scale record at rest: every step so far stored with the initial scale
// and no value passed the threshold.
__global__ void k_scale_reset(ScaleState *sc, float scale) {
    for (int i = 0; i < 3; ++i) {
        sc->s[i] = scale;
        sc->over[i] = 0u;
    }
}

__global__ void k_gather_probe(const float *__restrict__ stage, const int32_t *__restrict__ idx,
                               int count, int64_t N, float *__restrict__ out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= count) return;
    const int64_t o = idx[p];
#pragma unroll
    for (int a = 0; a < 7; ++a) out[(int64_t)p * 7 + a] = stage[a * N + o];
}

// ---------------------------------------------------------------------------
// Launchers.

// The boundary-list kernel runs beside the interior kernel; it is short and
// latency-bound, so it is launched at the highest stream priority: its blocks
// are placed before the interior kernel's pending blocks instead of waiting for
// the interior grid to drain.
static int high_priority() {
    static const int p = [] {
        int least = 0, greatest = 0;
        if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return greatest;
    }();
    return p;
}

template <class T, int LAY = kPull>
static cudaError_t launch_boundary(const T *src, T *dst, const DevState &S, const Lattice &L,
                                   int toff, cudaStream_t s, float *stage = nullptr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((L.nb + kB8 / 8 - 1) / (kB8 / 8));
    cfg.blockDim = dim3(kB8);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributePriority;
    attr[0].val.priority = high_priority();
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_boundary8<T, LAY>, src, dst, static_cast<URec<T> *>(S.ucomp),
                              (const BNode *)S.bnodes, (const BLink *)S.blinks,
                              (const BCDev *)S.bcs, (const uint8_t *)S.cls, (const float *)S.rho, L,
                              (const int64_t *)S.time, toff, S.status, stage);
}

template <class T>
static void launch_interior(const T *src, T *dst, const DevState &S, const Lattice &L, int toff,
                            cudaStream_t s) {
    if (L.grad) {
        const dim3 blk(kBX, kGY), grd((L.nx + kBX - 1) / kBX, (L.ny + kGY - 1) / kGY);
        k_interior_grad<T><<<grd, blk, 0, s>>>(src, dst, static_cast<URec<T> *>(S.ucomp), S.cls,
                                                S.rho, L, S.status,
                                                S.time, toff);
        return;
    }
    if constexpr (!std::is_same<T, float>::value) {
        // 16-bit storage: two nodes per thread
        const dim3 blk(kBX, kBY), grd((L.nx + 2 * kBX - 1) / (2 * kBX), (L.ny + kBY - 1) / kBY);
        k_interior_pair<T><<<grd, blk, 0, s>>>(src, dst, static_cast<float2 *>(S.ucomp), S.cls, L,
                                               S.status, S.time, toff);
        return;
    }
    // one row per thread measured fastest for every storage (2 and 4 rows cost
    // occupancy: 58+ registers)
    constexpr int NR = 1;
    const dim3 blk(kBX, kBY), grd((L.nx + kBX - 1) / kBX, (L.ny + kBY * NR - 1) / (kBY * NR));
    k_interior<T, NR><<<grd, blk, 0, s>>>(src, dst, static_cast<URec<T> *>(S.ucomp), S.cls, S.rho,
                                          L, S.status, S.time,
                                          toff);
}

// In-place step of parity LAY: every boundary node reads its inputs and
// stages its result before any population is overwritten (a boundary rule
// reads the node's own and upstream post-collision populations, which their
// pulling neighbours overwrite in place); then the interior kernel, and beside
// it the scatter of the staged boundary populations (the two touch disjoint
// locations).
template <class T, int LAY>
static cudaError_t step_in_place(const Lattice &L, const DevState &S, int toff,
                                 cudaStream_t s_main, cudaStream_t s_side, cudaEvent_t fork,
                                 cudaEvent_t join, const StepEvents *ev) {
    T *f = static_cast<T *>(S.f[0]);
    const bool split = s_side && fork && join && L.nb > 0;
    if (L.nb > 0) {
        if (ev) cudaEventRecord(ev->before_boundary, s_main);
        launch_boundary<T, LAY>(f, f, S, L, toff, s_main, S.stage);
        if (ev) cudaEventRecord(ev->after_boundary, s_main);
    }
    const int nsc = (int)(((int64_t)L.nb * 9 + kBB - 1) / kBB);
    if (split) {
        cudaEventRecord(fork, s_main);
        cudaStreamWaitEvent(s_side, fork, 0);
        k_boundary_scatter<T, LAY><<<nsc, kBB, 0, s_side>>>(S.stage, f, S.bnodes, L, S.time, toff);
        cudaEventRecord(join, s_side);
    }
    if (ev) cudaEventRecord(ev->before_interior, s_main);
    const dim3 blk(kBX, kBY), grd((L.nx + kBX - 1) / kBX, (L.ny + kBY - 1) / kBY);
    k_interior<T, 1, LAY><<<grd, blk, 0, s_main>>>(f, f, static_cast<URec<T> *>(S.ucomp), S.cls,
                                                   S.rho, L, S.status, S.time,
                                                   toff);
    if (ev) cudaEventRecord(ev->after_interior, s_main);
    if (split)
        cudaStreamWaitEvent(s_main, join, 0);
    else if (L.nb > 0)
        k_boundary_scatter<T, LAY><<<nsc, kBB, 0, s_main>>>(S.stage, f, S.bnodes, L, S.time, toff);
    return cudaGetLastError();
}

template <class T>
static cudaError_t step_t(const Lattice &L, const DevState &S, int cur, int toff,
                          cudaStream_t s_main, cudaStream_t s_side, cudaEvent_t fork,
                          cudaEvent_t join, const StepEvents *ev) {
    if (L.in_place)  // the parity of the step is that of `cur`
        return cur ? step_in_place<T, kAAOdd>(L, S, toff, s_main, s_side, fork, join, ev)
                   : step_in_place<T, kAAEven>(L, S, toff, s_main, s_side, fork, join, ev);
    const T *src = static_cast<const T *>(S.f[cur]);
    T *dst = static_cast<T *>(S.f[cur ^ 1]);
    const dim3 blk(kBX, kBY), grd((L.nx + kBX - 1) / kBX, (L.ny + kBY - 1) / kBY);
    const int nbb = (L.nb + kBB - 1) / kBB;
    // lambda != mu: densities of the boundary nodes first (the interior kernel
    // forms all other densities it needs in shared memory)
    if (L.grad && L.nb > 0)
        k_density_boundary<T><<<nbb, kBB, 0, s_main>>>(src, S.bnodes, S.blinks, S.bcs, S.rho, L,
                                                       S.time, toff);
    const bool split = s_side && fork && join && L.nb > 0;
    cudaStream_t s_b = split ? s_side : s_main;
    if (split) {
        cudaEventRecord(fork, s_main);
        cudaStreamWaitEvent(s_side, fork, 0);
        if (ev) cudaEventRecord(ev->before_boundary, s_side);
        launch_boundary<T>(src, dst, S, L, toff, s_side);
        if (ev) cudaEventRecord(ev->after_boundary, s_side);
        cudaEventRecord(join, s_side);
    }
    if (ev) cudaEventRecord(ev->before_interior, s_main);
    launch_interior<T>(src, dst, S, L, toff, s_main);
    if (ev) cudaEventRecord(ev->after_interior, s_main);
    if (split) {
        cudaStreamWaitEvent(s_main, join, 0);
    } else {
        if (ev) cudaEventRecord(ev->before_boundary, s_b);
        if (L.nb > 0) launch_boundary<T>(src, dst, S, L, toff, s_b);
        if (ev) cudaEventRecord(ev->after_boundary, s_b);
    }
    return cudaGetLastError();
}

cudaError_t launch_step(int storage, const Lattice &L, const DevState &S, int cur, int toff,
                        cudaStream_t s_main, cudaStream_t s_side, cudaEvent_t fork,
                        cudaEvent_t join, const StepEvents *ev) {
    switch (storage) {
        case LBM_F16_DEV:
            return step_t<__half>(L, S, cur, toff, s_main, s_side, fork, join, ev);
        case LBM_BF16_DEV:
            return step_t<__nv_bfloat16>(L, S, cur, toff, s_main, s_side, fork, join, ev);
        default:
            return step_t<float>(L, S, cur, toff, s_main, s_side, fork, join, ev);
    }
}

int kernels_per_step(const Lattice &L) {
    return (L.grad && L.nb > 0 ? 1 : 0) + 1 + (L.nb > 0 ? (L.in_place ? 2 : 1) : 0);
}
int kernels_per_fields(const Lattice &L) { return (L.grad ? (L.nb > 0 ? 2 : 1) : 0) + 1 + (L.nb > 0 ? 1 : 0); }

cudaError_t launch_advance(const DevState &S, int64_t n, cudaStream_t s) {
    k_advance<<<1, 1, 0, s>>>(S.time, n);
    return cudaGetLastError();
}

template <class T, int LAY>
static void fields_in_place(const Lattice &L, const DevState &S, cudaStream_t s) {
    const T *src = static_cast<const T *>(S.f[0]);
    const dim3 blk(kBX, kBY), grd((L.nx + kBX - 1) / kBX, (L.ny + kBY - 1) / kBY);
    k_fields_interior<T, LAY><<<grd, blk, 0, s>>>(src, static_cast<const URec<T> *>(S.ucomp), S.cls,
                                                  S.rho, L, S.stage, S.time);
    if (L.nb > 0)
        k_fields_boundary<T, LAY><<<(L.nb + kBB - 1) / kBB, kBB, 0, s>>>(
            src, static_cast<const URec<T> *>(S.ucomp), S.bnodes, S.blinks, S.bcs, S.rho, L, S.time,
            S.stage);
}

template <class T>
static cudaError_t fields_t(const Lattice &L, const DevState &S, int cur, cudaStream_t s) {
    if (L.in_place) {  // lambda = mu only: no density pass
        if (cur)
            fields_in_place<T, kAAOdd>(L, S, s);
        else
            fields_in_place<T, kAAEven>(L, S, s);
        return cudaGetLastError();
    }
    const T *src = static_cast<const T *>(S.f[cur]);
    const dim3 blk(kBX, kBY), grd((L.nx + kBX - 1) / kBX, (L.ny + kBY - 1) / kBY);
    const int nbb = (L.nb + kBB - 1) / kBB;
    if (L.grad) {
        k_density_interior<T><<<grd, blk, 0, s>>>(src, S.cls, S.rho, L, S.time);
        if (L.nb > 0)
            k_density_boundary<T><<<nbb, kBB, 0, s>>>(src, S.bnodes, S.blinks, S.bcs, S.rho, L,
                                                      S.time, 0);
    }
    k_fields_interior<T><<<grd, blk, 0, s>>>(src, static_cast<const URec<T> *>(S.ucomp), S.cls,
                                             S.rho, L, S.stage, S.time);
    if (L.nb > 0)
        k_fields_boundary<T><<<nbb, kBB, 0, s>>>(src, static_cast<const URec<T> *>(S.ucomp),
                                                 S.bnodes, S.blinks, S.bcs, S.rho,
                                                 L, S.time, S.stage);
    return cudaGetLastError();
}

cudaError_t launch_fields(int storage, const Lattice &L, const DevState &S, int cur, float *u,
                          float *v, float *sigma, cudaStream_t s) {
    cudaError_t e;
    switch (storage) {
        case LBM_F16_DEV:
            e = fields_t<__half>(L, S, cur, s);
            break;
        case LBM_BF16_DEV:
            e = fields_t<__nv_bfloat16>(L, S, cur, s);
            break;
        default:
            e = fields_t<float>(L, S, cur, s);
    }
    if (e != cudaSuccess) return e;
    const int64_t N = (int64_t)L.nx * L.ny;
    if (u) e = cudaMemcpyAsync(u, S.stage, 2 * N * sizeof(float), cudaMemcpyDefault, s);
    if (e == cudaSuccess && v)
        e = cudaMemcpyAsync(v, S.stage + 2 * N, 2 * N * sizeof(float), cudaMemcpyDefault, s);
    if (e == cudaSuccess && sigma)
        e = cudaMemcpyAsync(sigma, S.stage + 4 * N, 3 * N * sizeof(float), cudaMemcpyDefault, s);
    return e;
}

cudaError_t launch_gather_probe(const Lattice &L, const DevState &S, int count, cudaStream_t s) {
    const int64_t N = (int64_t)L.nx * L.ny;
    k_gather_probe<<<(count + 127) / 128, 128, 0, s>>>(S.stage, S.probe_idx, count, N, S.probe);
    return cudaGetLastError();
}

cudaError_t launch_reset(int storage, const Lattice &L, const DevState &S, cudaStream_t s) {
    const size_t esz = storage == LBM_F32 ? 4 : 2;
    const size_t fbytes = (size_t)9 * L.fplane * esz;
    // in place: the planes start one row and one column before node (0, 0)
    char *f0 = static_cast<char *>(S.f[0]) - (L.in_place ? (size_t)(L.pitch + 1) * esz : 0);
    cudaError_t e = cudaMemsetAsync(f0, 0, fbytes, s);
    if (e == cudaSuccess && S.f[1]) e = cudaMemsetAsync(S.f[1], 0, fbytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(S.ucomp, 0, (size_t)L.plane * urec_bytes(storage), s);
    if (e == cudaSuccess && S.rho) e = cudaMemsetAsync(S.rho, 0, (size_t)L.plane * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(S.status, 0, sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(S.time, 0, sizeof(int64_t), s);
    if (e == cudaSuccess && L.sc) {
        k_scale_reset<<<1, 1, 0, s>>>(L.sc, L.scale);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace lbm
