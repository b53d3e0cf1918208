// lbm_wave.cu -- temporally blocked time stepping: kWaveK steps of the solid
// LBM (Eqs. stream, moments, fieq, coll and the boundary rules of Sec. 4) per
// kernel launch, FP32 storage, lambda = mu (k_wave); kGradK steps per launch
// when lambda != mu and the source needs the density gradient (k_wave_grad).
//
// One step reads and writes every population once, so the one-step kernels
// are bound by HBM at 104 B per lattice update.  Here a block owns a strip of
// kWaveC columns (kWaveW core columns plus kWaveK halo columns on each side)
// and a segment of rows, and sweeps the segment bottom-up.  Time level l
// (1..kWaveK) of row y is computed at sweep step y + 2(l - 1): the levels run
// side by side, two rows apart, so every level reads rows y - 1 .. y + 1 of
// the level below that are complete by the previous sweep step.  Level l - 1
// keeps its last four rows in a shared-memory ring; level 0 (the populations
// f^col(t0 - 1) in HBM) arrives by TMA into an eight-row ring, together with
// the per-node words and the displacement of each row, kWaveD rows ahead of
// use.  Level kWaveK writes f^col(t0 + kWaveK - 1) and u of the core nodes to
// HBM.  The halo shrinks by one node per level, so the core of every strip is
// exact; strips and segments overlap only in what they read.
//
// Per node and level the arithmetic is that of the one-step kernels: the
// incoming populations (pulled, or given by the rules of Sec. 4) go through
// the same collision (collide_v), two nodes per lane as paired f32x2
// operations.  Box edges and crack faces ("simple" boundary nodes) are pulled
// one lane per node; other boundary nodes are updated by eight lanes, as in
// the cooperative boundary kernel.  The rules are explicitly rounded and the
// moments formed in one order, so every stored value is bit-identical to the
// one-step path.  The blocks of a launch are planned on the host
// (lbm_plan.cpp).
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <vector>

#include <cuda.h>
#include <cuda_runtime.h>

#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

namespace {

constexpr int kC = kWaveC, kK = kWaveK, kW = kWaveW;
constexpr int kNI = 8;                // rows of the level-0 ring (and mbarriers)
constexpr int kD = kNI - 3;           // rows issued ahead of the row level 1 needs
constexpr int kNU = 2 * kK + kD;      // rows of the node-word and displacement rings
constexpr int kThreads = kK * kC / 2;  // two columns per thread
constexpr int kRowF = 9 * kC;         // floats per ring row (nine planes of kC)
constexpr uint32_t kFRowBytes = kRowF * 4;
constexpr uint32_t kNwRowBytes = kC * 8;
constexpr uint32_t kURowBytes = kW * 16;
constexpr uint32_t kTxBytes = kFRowBytes + kNwRowBytes + kURowBytes;
constexpr size_t kOffIn = 0;
constexpr size_t kOffLev = kOffIn + (size_t)kNI * kFRowBytes;
constexpr size_t kOffU = kOffLev + (size_t)(kK - 1) * 4 * kFRowBytes;
constexpr size_t kOffNw = kOffU + (size_t)kNU * kURowBytes;
constexpr size_t kOffBar = kOffNw + (size_t)kNU * kNwRowBytes;
constexpr size_t kSmem = kOffBar + (size_t)kNI * 8;
static_assert(kSmem <= 232448, "shared memory of one block");
static_assert(kThreads <= 1024 && kC % 32 == 0, "block shape");
static_assert(kOffLev % 128 == 0 && kOffU % 128 == 0 && kOffNw % 128 == 0 &&
                  kURowBytes % 128 == 0 && kNwRowBytes % 128 == 0 && kFRowBytes % 128 == 0,
              "TMA destinations 128-byte aligned");
static_assert(kW % 4 == 0 && kK % 2 == 0, "TMA x coordinates on 16-byte boundaries");

// Node word: bits 0-1 class; 2-9 cut, 10-17 Dirichlet, 18-25 corner, 26-33
// upstream-missing masks (bit d - 1 for direction d); bit 34 "simple": every
// cut link is a mid-link wall with the same BC and the same axis-aligned
// normal, given by bits 35-50 (BC index) and 51-52 (normal +x, -x, +y, -y);
// otherwise bits 35-63 hold the node's index in the boundary list.
__device__ __forceinline__ uint32_t nw_mask(uint64_t w, int shift) {
    return (uint32_t)((w >> shift) & 0xffu) << 1;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_inval(uint32_t bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for a phase of an mbarrier, giving up after about limit_ns nanoseconds.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (int outer = 0; outer < (1 << 24); ++outer) {
        for (int i = 0; i < 32; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > (uint64_t)limit_ns) return false;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            int z, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

// Indices taken from a node word are clamped into their tables.  A node word
// is only wrong when a block reads a ring row whose copy has not landed (after
// a wait has run out, the block finishes its sweep on stale rows and reports
// LBM_ERR_TIMEOUT); the clamps keep every access of such a sweep in bounds.
//
// The common link record of a simple node (node-word bits 35-52).
__device__ __forceinline__ BLink simple_link(uint32_t hi, const Lattice &L) {
    const uint32_t code = (hi >> 16) & 3u;
    const uint32_t bc = hi & 0xffffu;
    BLink sl;
    sl.q = 0.5f;
    sl.n0 = code == 0 ? 1.0f : (code == 1 ? -1.0f : 0.0f);
    sl.n1 = code == 2 ? 1.0f : (code == 3 ? -1.0f : 0.0f);
    sl.bc = (uint16_t)(bc < (uint32_t)L.nbcs ? bc : 0u);
    sl.bc2 = sl.bc;
    return sl;
}

// The boundary-list index of a node word (bits 35-63).
__device__ __forceinline__ int64_t boundary_index(uint64_t w, const Lattice &L) {
    const uint32_t g = (uint32_t)(w >> 35);
    return g < (uint32_t)L.nb ? g : 0;
}

// Three consecutive ring rows of the level below and the node's column.
struct Rows {
    const float *rm, *r0, *rp;
    int c;
    __device__ __forceinline__ float operator()(int i, int dx, int dy) const {
        const float *r = dy < 0 ? rm : (dy > 0 ? rp : r0);
        return r[i * kC + c + dx];
    }
};

// Stores the post-collision populations of a lane's two nodes (columns c and
// c + 32; plane stride `stride`), those that were updated.
__device__ __forceinline__ void store_pair(float *out, int64_t stride, const F2 f[9], bool a,
                                           bool b) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        float va, vb;
        f2_split(f[i], va, vb);
        if (a) out[i * stride] = va;
        if (b) out[i * stride + 32] = vb;
    }
}

// One region of a blocked launch: kWaveK steps of every material node of the
// region (X0, Y0, rows, has_boundary): core columns [X0, X0 + kWaveW), core
// rows [Y0, Y0 + rows); has_boundary says whether a boundary node lies in the
// region or its halo.  Each warp computes one level of one 64-column half of
// the ring, two columns per lane, c and c + 32 (ring column c is lattice
// column X0 - kWaveK + c): their collisions run as one stream of paired
// (f32x2) operations, and every shared-memory access of a warp stays on
// consecutive words.  tf, tnw and tu are the tensor maps of the input
// populations, the node words and the displacement records; `sm` is the
// block's dynamic shared memory.  The block's earlier use of `sm` must be over
// (a barrier) before the call.  *cycle_out, if given, receives the region's SM
// cycles.
__device__ __forceinline__ void wave_region(
    const CUtensorMap *tf, const CUtensorMap *tnw, const CUtensorMap *tu, float *__restrict__ dst,
    float4 *__restrict__ uc, const BLink *__restrict__ blinks, const BCDev *__restrict__ bcs,
    const Lattice &L, const int64_t *__restrict__ time, int toff, const int4 region,
    uint32_t *__restrict__ status, long long *cycle_out, unsigned char *sm) {
    const long long t_start = clock64();
    float *in = reinterpret_cast<float *>(sm + kOffIn);
    float *lev = reinterpret_cast<float *>(sm + kOffLev);
    float4 *ur = reinterpret_cast<float4 *>(sm + kOffU);
    const uint64_t *nwr = reinterpret_cast<const uint64_t *>(sm + kOffNw);
    const uint32_t bar0 = smem_addr(sm + kOffBar);

    // Warp w runs on sub-partition w % 4 of the SM.  Warp w = 2 l' + h' takes
    // level l' + 1 and half h = h' xor (l' / 2) % 2: the two halves of a level
    // sit on two sub-partitions, and one half across the levels on all four,
    // so neither a wall row nor a wall column piles its boundary updates onto
    // one of them.
    static_assert(kC == 128 && kThreads == kK * 64, "two halves of 64 columns per level");
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int lv = (warp >> 1) + 1;  // time level of this thread (warp-uniform)
    const int half = (warp ^ (warp >> 2)) & 1;
    const int c = (half << 6) | lane;  // the lane's columns c, c + 32
    const int X0 = region.x, Y0 = region.y, Hs = region.z;
    const int xin = X0 - kK;     // lattice column of ring column 0
    const int y_in0 = Y0 - kK;   // lattice row of input row index 0
    const int j_last = Hs - 1 + 2 * kK;
    const int nsweep = Hs + 3 * kK - 3;
    const float tb = (float)(*time + toff + lv - 2);  // boundary data at the time of f^col
    const F2 sx2 = f2(L.fx, L.fx), sy2 = f2(L.fy, L.fy);
    const F2 w2 = splat<F2>(L.omega), s32 = splat<F2>(rmul(L.src, 1.0f / 3.0f));

    auto issue = [&](int j) {
        const uint32_t bar = bar0 + 8u * (uint32_t)(j & (kNI - 1));
        const int y = y_in0 + j;
        mbar_expect_tx(bar, kTxBytes);
        tma_load_3d(smem_addr(in + (size_t)(j & (kNI - 1)) * kRowF), tf, xin, y, 0, bar);
        tma_load_2d(smem_addr(sm + kOffNw + (size_t)(j % kNU) * kNwRowBytes), tnw, xin, y, bar);
        tma_load_3d(smem_addr(sm + kOffU + (size_t)(j % kNU) * kURowBytes), tu, 0, X0, y, bar);
    };
    auto wait_row = [&](int j, int64_t limit) {
        return mbar_wait(bar0 + 8u * (uint32_t)(j & (kNI - 1)), (uint32_t)((j / kNI) & 1), limit);
    };

    bool ok = true;       // thread 0: every wait so far completed
    int j_issued = -1;    // thread 0: last input row issued
    int last_waited = -1; // thread 0: last input row known to have landed
    if (tid == 0) {
        for (int s = 0; s < kNI; ++s) mbar_init(bar0 + 8u * s, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
        for (int j = 0; j <= kD + 1 && j <= j_last; ++j) {
            issue(j);
            j_issued = j;
        }
        // a limit of 0 gives up at once, whether or not the copies have landed
        for (int j = 0; j <= 2 && j <= j_last && ok; ++j) {
            ok = L.wait_ns > 0 && wait_row(j, L.wait_ns);
            last_waited = ok ? j : j - 1;
        }
    }
    __syncthreads();

    // a lane's node counts only inside the level's live columns and inside the
    // lattice: every global store of the block then goes to a node of its
    // region, whatever its shared-memory rows hold (after a wait has run out
    // the sweep reads rows that never landed)
    const bool live_a = c >= lv && c < kC - lv && (unsigned)(xin + c) < (unsigned)L.nx;
    const bool live_b =
        c + 32 >= lv && c + 32 < kC - lv && (unsigned)(xin + c + 32) < (unsigned)L.nx;
    const int lo = Y0 - (kK - lv), hi = Y0 + Hs - 1 + (kK - lv);
    const float *prev_base = lv == 1 ? in : lev + (size_t)(lv - 2) * 4 * kRowF;
    const int pmask = lv == 1 ? kNI - 1 : 3;
    float *own_base = lev + (size_t)(lv - 1) * 4 * kRowF;  // unused by level kWaveK
    const bool core_a = c >= kK && c < kC - kK, core_b = c + 32 >= kK && c + 32 < kC - kK;

    // The sweep, compiled twice: with the boundary updates, and without them
    // for regions that hold no boundary node (their interior update is then
    // scheduled on its own).
    float nonfinite = 0.0f;  // the last level's moments, summed: non-finite if any one is
    auto sweep = [&](auto with_boundary) {
        constexpr bool kB = decltype(with_boundary)::value;
        int ju_next = ((1 - 2 * (lv - 1)) % kNU + kNU) % kNU;
        // node words of the row of the next step, loaded a step ahead (their
        // rows landed at least one step earlier)
        uint64_t pf_a, pf_b;
        {
            const int y0 = y_in0 + 1 - 2 * (lv - 1);
            const bool in = y0 >= lo && y0 <= hi;
            pf_a = (in && live_a) ? nwr[ju_next * kC + c] : 0ull;
            pf_b = (in && live_b) ? nwr[ju_next * kC + c + 32] : 0ull;
        }
        for (int n = 0; n < nsweep; ++n) {
            if (tid == 0 && n + kD + 2 <= j_last && ok) {
                // order the block's earlier shared-memory accesses before the copy
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue(n + kD + 2);
                j_issued = n + kD + 2;
            }
            const int y = y_in0 + 1 + n - 2 * (lv - 1);
            const int j = y - y_in0;
            // ring rows of this step, advanced from the previous one: node-word and
            // displacement rings (mod kNU), level rings (mod 4 or kNI)
            const int ju = ju_next;
            ju_next = ju + 1 == kNU ? 0 : ju + 1;
            if (y >= lo && y <= hi) {  // warp-uniform: one level per warp
                const uint64_t nwa = pf_a, nwb = pf_b;
                const uint32_t cla = (uint32_t)(nwa & 3u), clb = (uint32_t)(nwb & 3u);
                const float *rm = prev_base + ((j - 1) & pmask) * kRowF + c;
                const float *r0 = prev_base + (j & pmask) * kRowF + c;
                const float *rp = prev_base + ((j + 1) & pmask) * kRowF + c;
                float *own = own_base + (j & 3) * kRowF + c;
                const bool core_row = y >= Y0 && y < Y0 + Hs;
                const int64_t grow = (int64_t)y * L.pitch + xin + c;  // lattice index of column c
                // the row's update, compiled with and without the boundary
                // updates; a warp takes the second unless its row holds a
                // boundary node, so rows inside the material run the plain
                // interior update
                auto row = [&](auto with_boundary_row) {
                    constexpr bool kR = decltype(with_boundary_row)::value;
                    const bool sim_a = kR && cla == kBoundary && ((nwa >> 34) & 1u);
                    const bool sim_b = kR && clb == kBoundary && ((nwb >> 34) & 1u);
                    const bool do_a = cla == kInterior || sim_a, do_b = clb == kInterior || sim_b;
                    // the other boundary nodes of the warp (curved walls, corners): eight
                    // lanes each, the update of the cooperative boundary kernel (four
                    // nodes per pass); node m of the 64 is column m of the half.  They
                    // go first: their long dependent chains then overlap the other
                    // warps' updates instead of delaying the row's barrier.
                    if (kR) {
                        const bool cx_a = cla == kBoundary && !sim_a, cx_b = clb == kBoundary && !sim_b;
                        const unsigned ma = __ballot_sync(0xffffffffu, cx_a);
                        const unsigned mb = __ballot_sync(0xffffffffu, cx_b);
                        if (ma | mb) {  // warp-uniform
                            const int grp = lane >> 3, kdir = (lane & 7) + 1;
                            const bool lane0 = kdir == 1;  // lane 0 of the group stores f_0 and u
                            unsigned long long rem = ((unsigned long long)mb << 32) | ma;
                            while (rem) {
                                // group g takes the g-th remaining node; spare groups redo
                                // the first one and store nothing
                                unsigned long long r = rem;
                                for (int q = 0; q < grp; ++q) r &= r - 1;
                                const bool live = r != 0;
                                const int m = __ffsll((long long)(live ? r : rem)) - 1;
                                for (int q = 0; q < 4; ++q) rem &= rem - 1;
                                const int src = m & 31, hb = m >> 5;
                                const uint64_t wa = __shfl_sync(0xffffffffu, nwa, src);
                                const uint64_t wbb = __shfl_sync(0xffffffffu, nwb, src);
                                const uint64_t wb = hb ? wbb : wa;
                                const int cb = (half << 6) + m;
                                const bool simple = (wb >> 34) & 1u;
                                const BLink sl = simple_link((uint32_t)(wb >> 35), L);
                                const BLink *lrec = blinks + boundary_index(wb, L) * 8;
                                auto link = [&](int i) { return simple ? sl : lrec[i - 1]; };
                                float f0;
                                const float fk = boundary8_pull(
                                    Rows{rm - c, r0 - c, rp - c, cb}, nw_mask(wb, 2), nw_mask(wb, 10),
                                    nw_mask(wb, 18), nw_mask(wb, 26), kdir, link, bcs, tb, L, f0);
                                float fr, jx, jy, m00;
                                const float mine =
                                    boundary8_collide(fk, f0, kdir, L.fx, L.fy, L, fr, jx, jy, m00);
                                if (live) {
                                    const int64_t gb = (int64_t)y * L.pitch + xin + cb;
                                    if (lv < kK) {
                                        own[kdir * kC + cb - c] = mine;
                                        if (lane0) own[cb - c] = fr;
                                    } else {
                                        dst[kdir * L.fplane + gb] = mine;
                                        if (lane0) dst[gb] = fr;
                                    }
                                    if (lane0 && core_row && cb >= kK && cb < kC - kK) {
                                        float4 *up = ur + ju * kW + (cb - kK);
                                        float4 w = *up;
                                        integrate_u_value(w, jx, jy, L.rho0 + m00);
                                        if (lv < kK) {
                                            *up = w;
                                        } else {
                                            uc[gb] = w;
                                            nonfinite = radd(nonfinite, radd(radd(m00, jx), jy));
                                        }
                                    }
                                }
                            }
                        }
                    }
                    if (do_a || do_b) {
                        F2 f[9];
                        if (!kR || (cla == kInterior && clb == kInterior)) {
                            // pulls of both nodes (a node of the pair that is not
                            // updated reads in-bounds values it never stores)
                            auto ld2 = [](const float *r) { return f2(r[0], r[32]); };
                            f[0] = ld2(r0);
                            f[1] = ld2(r0 + kC - 1);
                            f[2] = ld2(rm + 2 * kC);
                            f[3] = ld2(r0 + 3 * kC + 1);
                            f[4] = ld2(rp + 4 * kC);
                            f[5] = ld2(rm + 5 * kC - 1);
                            f[6] = ld2(rm + 6 * kC + 1);
                            f[7] = ld2(rp + 7 * kC + 1);
                            f[8] = ld2(rp + 8 * kC - 1);
                        } else {
                            // one of the pair is a simple boundary node: each node
                            // pulled on its own (one copy of the code), then the
                            // pair collides together
#pragma unroll
                            for (int i = 0; i < 9; ++i) f[i] = f2(0.0f, 0.0f);
#pragma unroll 1
                            for (int h = 0; h < 2; ++h) {
                                float g[9];
                                const int dc = h << 5;
                                if (h ? sim_b : sim_a) {
                                    const uint64_t wn = h ? nwb : nwa;
                                    simple_pull<false>(
                                        Rows{rm - c, r0 - c, rp - c, c + dc}, nw_mask(wn, 2),
                                        nw_mask(wn, 10), nw_mask(wn, 26),
                                        simple_link((uint32_t)(wn >> 35), L), bcs, tb, L, g);
                                } else {
                                    g[0] = r0[dc];
                                    g[1] = r0[kC + dc - 1];
                                    g[2] = rm[2 * kC + dc];
                                    g[3] = r0[3 * kC + dc + 1];
                                    g[4] = rp[4 * kC + dc];
                                    g[5] = rm[5 * kC + dc - 1];
                                    g[6] = rm[6 * kC + dc + 1];
                                    g[7] = rp[7 * kC + dc + 1];
                                    g[8] = rp[8 * kC + dc - 1];
                                }
#pragma unroll
                                for (int i = 0; i < 9; ++i) {
                                    float va, vb;
                                    f2_split(f[i], va, vb);
                                    f[i] = h ? f2(va, g[i]) : f2(g[i], vb);
                                }
                            }
                        }
                        F2 dr, jx, jy;
                        collide_v(f, sx2, sy2, w2, s32, dr, jx, jy);
                        if (lv < kK)
                            store_pair(own, kC, f, do_a, do_b);
                        else
                            store_pair(dst + grow, L.fplane, f, do_a, do_b);
                        if (core_row) {
                            float dra, drb, jxa, jxb, jya, jyb;
                            f2_split(dr, dra, drb);
                            f2_split(jx, jxa, jxb);
                            f2_split(jy, jya, jyb);
                            auto u_one = [&](int dc, float d, float mx, float my) {
                                float4 *up = ur + ju * kW + (c + dc - kK);
                                float4 w = *up;
                                integrate_u_value(w, mx, my, L.rho0 + d);
                                if (lv < kK) {
                                    *up = w;
                                } else {
                                    uc[grow + dc] = w;
                                    nonfinite = radd(nonfinite, radd(radd(d, mx), my));
                                }
                            };
                            if (do_a && core_a) u_one(0, dra, jxa, jya);
                            if (do_b && core_b) u_one(32, drb, jxb, jyb);
                        }
                    }
                };
                if (kB && __ballot_sync(0xffffffffu, cla == kBoundary || clb == kBoundary))
                    row(std::true_type{});
                else
                    row(std::false_type{});
            }
            {
                const int yn = y + 1;
                const bool in = yn >= lo && yn <= hi;
                pf_a = (in && live_a) ? nwr[ju_next * kC + c] : 0ull;
                pf_b = (in && live_b) ? nwr[ju_next * kC + c + 32] : 0ull;
            }
            if (tid == 0 && n + 3 <= j_last && ok) {
                ok = wait_row(n + 3, L.wait_ns);
                if (!ok) last_waited = n + 2;
            }
            __syncthreads();
        }
    };
    if (region.w)
        sweep(std::true_type{});
    else
        sweep(std::false_type{});
    if (!isfinite(nonfinite)) flag_nonfinite(status, nonfinite, 0.0f, 0.0f);
    if (cycle_out && tid == 0) *cycle_out = clock64() - t_start;
    if (tid == 0 && !ok) {
        // a copy did not land within the limit (the rest of the sweep ran on
        // stale rows; thread 0 issued no copy after that): flag it, then wait
        // for every copy issued after the last completed wait, each with the
        // default limit, so that none is still writing this block's shared
        // memory when the block exits
        atomicOr(status, 2u);
        for (int j = last_waited + 1; j <= j_issued; ++j) wait_row(j, kDefaultWaitNs);
    }
    // every copy has been waited for: the barriers are released, so that the
    // block can initialise them again for its next region
    if (tid == 0)
        for (int q = 0; q < kNI; ++q) mbar_inval(bar0 + 8u * q);
}

// One launch over the regions of many lattices (a batch): a persistent grid
// whose blocks take regions from an atomic counter; each region's instance
// record supplies its tensor maps and buffers, and its lattice parameters are
// staged in shared memory.
__global__ void __launch_bounds__(kThreads, 1)
    k_wave_batch(const WaveInst *__restrict__ insts, const int4 *__restrict__ regions,
                 const int32_t *__restrict__ region_inst, int nregions,
                 int32_t *__restrict__ counter, int cur, int toff) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ int s_r;
    __shared__ __align__(16) Lattice s_L;
    for (;;) {
        if (threadIdx.x == 0) s_r = atomicAdd(counter, 1);
        __syncthreads();
        const int r = s_r;
        if (r >= nregions) break;
        const WaveInst *I = insts + region_inst[r];
        if (threadIdx.x == 0) s_L = I->L;
        __syncthreads();
        wave_region(&I->tf[cur], &I->tnw, &I->tu, I->f[cur ^ 1], I->uc, I->blinks, I->bcs, s_L,
                    I->time, toff, regions[r], I->status, nullptr, sm);
        __syncthreads();  // the next region reuses the shared memory
    }
}

// One launch: kWaveK steps of every material node of one lattice; block b
// handles the region tab[b].
__global__ void __launch_bounds__(kThreads, 1)
    k_wave(const __grid_constant__ CUtensorMap tf, const __grid_constant__ CUtensorMap tnw,
           const __grid_constant__ CUtensorMap tu, float *__restrict__ dst,
           float4 *__restrict__ uc, const BLink *__restrict__ blinks,
           const BCDev *__restrict__ bcs, Lattice L, const int64_t *__restrict__ time, int toff,
           const int4 *__restrict__ tab, uint32_t *__restrict__ status,
           long long *__restrict__ cycles) {
    extern __shared__ __align__(1024) unsigned char sm[];
    wave_region(&tf, &tnw, &tu, dst, uc, blinks, bcs, L, time, toff, tab[blockIdx.x], status,
                cycles ? cycles + blockIdx.x : nullptr, sm);
}

// ---------------------------------------------------------------------------
// lambda != mu: the source S = F + (mu - lambda)/rho grad rho needs the
// densities of the four axis neighbours at the same time level.  Each level l
// therefore runs two tasks per sweep step, on two sets of warps: the density of
// row y + 2 (from the pulled, or rule-given, populations of level l - 1, into a
// four-row density ring of its own) and the collision of row y (pulled
// populations, the densities of rows y - 1 .. y + 1, Eq. sourceterm, Eq. coll).
// Row y + 2 of level l - 1 must be complete a step earlier, so the levels run
// four rows apart; the level rings hold eight rows, and the halo shrinks by two
// nodes per level.  With kGradK = 4 levels the core is the same 112 columns.
constexpr int kGradK = kWaveGradK;        // time steps per launch
constexpr int kGradSkew = 4;              // rows between consecutive levels
constexpr int kGradNI = 8, kGradD = 3;    // level-0 ring rows; rows issued ahead
constexpr int kGradNL = 8, kGradND = 4;   // level ring rows; density ring rows
constexpr int kGradNU = 19;               // node-word and displacement ring rows
constexpr int kGradThreads = 2 * kGradK * kC / 2;  // collision warps, then density warps
constexpr size_t kGOffIn = 0;
constexpr size_t kGOffLev = kGOffIn + (size_t)kGradNI * kFRowBytes;
constexpr size_t kGOffDen = kGOffLev + (size_t)(kGradK - 1) * kGradNL * kFRowBytes;
constexpr size_t kGOffU = kGOffDen + (size_t)kGradK * kGradND * kC * 4;
constexpr size_t kGOffNw = kGOffU + (size_t)kGradNU * kURowBytes;
constexpr size_t kGOffBar = kGOffNw + (size_t)kGradNU * kNwRowBytes;
constexpr size_t kGSmem = kGOffBar + (size_t)kGradNI * 8;
static_assert(kGSmem <= 232448, "shared memory of one block");
static_assert(kGradThreads <= 1024, "block shape");
static_assert(kC - 4 * kGradK == kW, "the same strips as the lambda = mu kernel");
static_assert(kGOffLev % 128 == 0 && kGOffDen % 128 == 0 && kGOffU % 128 == 0 &&
                  kGOffNw % 128 == 0,
              "TMA destinations 128-byte aligned");

// The incoming populations of an interior node from three ring rows, column
// dc of rows rm, r0, rp.
__device__ __forceinline__ void pull_rows(const float *rm, const float *r0, const float *rp,
                                          int dc, float f[9]) {
    f[0] = r0[dc];
    f[1] = r0[kC + dc - 1];
    f[2] = rm[2 * kC + dc];
    f[3] = r0[3 * kC + dc + 1];
    f[4] = rp[4 * kC + dc];
    f[5] = rm[5 * kC + dc - 1];
    f[6] = rm[6 * kC + dc + 1];
    f[7] = rp[7 * kC + dc + 1];
    f[8] = rp[8 * kC + dc - 1];
}

// Axis directions 1..4 open (not cut) from a node word's cut mask.
__device__ __forceinline__ void open_axes(uint64_t nw, bool &xp, bool &yp, bool &xm, bool &ym) {
    const uint32_t cut = nw_mask(nw, 2);
    xp = !((cut >> 1) & 1u);
    yp = !((cut >> 2) & 1u);
    xm = !((cut >> 3) & 1u);
    ym = !((cut >> 4) & 1u);
}

// One launch: kGradK steps of every material node, lambda != mu.  Blocks and
// regions are those of k_wave.  Warps 0..7 run the collisions, warps 8..15
// the densities; within each set warp 2 l' + h' takes level l' + 1 and the
// 64-column half h' xor (l' / 2) % 2, and lane t its columns c = 64 h + t and
// c + 32, as in k_wave.  Each sub-partition holds two warps of each set.
__global__ void __launch_bounds__(kGradThreads, 1)
    k_wave_grad(const __grid_constant__ CUtensorMap tf, const __grid_constant__ CUtensorMap tnw,
                const __grid_constant__ CUtensorMap tu, float *__restrict__ dst,
                float4 *__restrict__ uc, const BLink *__restrict__ blinks,
                const BCDev *__restrict__ bcs, Lattice L, const int64_t *__restrict__ time,
                int toff, const int4 *__restrict__ tab, uint32_t *__restrict__ status,
                long long *__restrict__ cycles) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const long long t_start = clock64();
    float *in = reinterpret_cast<float *>(sm + kGOffIn);
    float *lev = reinterpret_cast<float *>(sm + kGOffLev);
    float *den = reinterpret_cast<float *>(sm + kGOffDen);
    float4 *ur = reinterpret_cast<float4 *>(sm + kGOffU);
    const uint64_t *nwr = reinterpret_cast<const uint64_t *>(sm + kGOffNw);
    const uint32_t bar0 = smem_addr(sm + kGOffBar);

    static_assert(kGradThreads == 2 * kGradK * 64, "two sets of warps, two columns per lane");
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const bool density_warp = (tid >> 5) >= 2 * kGradK;  // warp-uniform
    const int w = (tid >> 5) & (2 * kGradK - 1);
    const int lv = (w >> 1) + 1;  // time level of this thread (warp-uniform)
    const int half = (w ^ (w >> 2)) & 1;
    const int c = (half << 6) | lane;  // the lane's columns c, c + 32
    const int4 region = tab[blockIdx.x];
    const int X0 = region.x, Y0 = region.y, Hs = region.z;
    const int xin = X0 - 2 * kGradK;    // lattice column of ring column 0
    const int y_in0 = Y0 - 2 * kGradK;  // lattice row of input row index 0
    const int j_last = Hs + 4 * kGradK - 1;
    const int nsweep = Hs + 6 * kGradK - 3;
    const float tb = (float)(*time + toff + lv - 2);  // boundary data at the time of f^col
    const F2 w2 = splat<F2>(L.omega), s32 = splat<F2>(rmul(L.src, 1.0f / 3.0f));

    auto issue = [&](int j) {
        const uint32_t bar = bar0 + 8u * (uint32_t)(j & (kGradNI - 1));
        const int y = y_in0 + j;
        mbar_expect_tx(bar, kTxBytes);
        tma_load_3d(smem_addr(in + (size_t)(j & (kGradNI - 1)) * kRowF), &tf, xin, y, 0, bar);
        tma_load_2d(smem_addr(sm + kGOffNw + (size_t)(j % kGradNU) * kNwRowBytes), &tnw, xin, y,
                    bar);
        tma_load_3d(smem_addr(sm + kGOffU + (size_t)(j % kGradNU) * kURowBytes), &tu, 0, X0, y,
                    bar);
    };
    auto wait_row = [&](int j, int64_t limit) {
        return mbar_wait(bar0 + 8u * (uint32_t)(j & (kGradNI - 1)),
                         (uint32_t)((j / kGradNI) & 1), limit);
    };

    bool ok = true;        // thread 0: every wait so far completed
    int j_issued = -1;     // thread 0: last input row issued
    int last_waited = -1;  // thread 0: last input row known to have landed
    if (tid == 0) {
        for (int q = 0; q < kGradNI; ++q) mbar_init(bar0 + 8u * q, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
        for (int j = 0; j <= kGradD + 1 && j <= j_last; ++j) {
            issue(j);
            j_issued = j;
        }
        // a limit of 0 gives up at once, whether or not the copies have landed
        for (int j = 0; j <= 2 && j <= j_last && ok; ++j) {
            ok = L.wait_ns > 0 && wait_row(j, L.wait_ns);
            last_waited = ok ? j : j - 1;
        }
    }
    __syncthreads();

    // collision columns shrink by two per level, density columns by one less
    const int m0 = density_warp ? 2 * lv - 1 : 2 * lv;
    // inside the live columns and the lattice (see k_wave)
    const bool live_a = c >= m0 && c < kC - m0 && (unsigned)(xin + c) < (unsigned)L.nx;
    const bool live_b =
        c + 32 >= m0 && c + 32 < kC - m0 && (unsigned)(xin + c + 32) < (unsigned)L.nx;
    const bool core_a = c >= 2 * kGradK && c < kC - 2 * kGradK;
    const bool core_b = c + 32 >= 2 * kGradK && c + 32 < kC - 2 * kGradK;
    const int lo = Y0 - 2 * (kGradK - lv), hi = Y0 + Hs - 1 + 2 * (kGradK - lv);
    const float *prev_base = lv == 1 ? in : lev + (size_t)(lv - 2) * kGradNL * kRowF;
    float *own_base = lev + (size_t)(lv - 1) * kGradNL * kRowF;  // unused by the last level
    float *den_base = den + (size_t)(lv - 1) * kGradND * kC;
    const int grp = lane >> 3, kdir = (lane & 7) + 1;

    // Populations of the lane's two nodes pulled from ring rows rm, r0, rp
    // (offset to column c): paired loads when both are interior (or when the
    // row holds no boundary node), else each node on its own, a simple
    // boundary node by its rules (one copy of the code).
    auto pull_pair = [&](auto with_boundary_row, const float *rm, const float *r0, const float *rp,
                         uint32_t cla, uint32_t clb, bool sim_a, bool sim_b, uint64_t nwa,
                         uint64_t nwb, F2 f[9]) {
        constexpr bool kR = decltype(with_boundary_row)::value;
        if (!kR || (cla == kInterior && clb == kInterior)) {
            auto ld2 = [](const float *r) { return f2(r[0], r[32]); };
            f[0] = ld2(r0);
            f[1] = ld2(r0 + kC - 1);
            f[2] = ld2(rm + 2 * kC);
            f[3] = ld2(r0 + 3 * kC + 1);
            f[4] = ld2(rp + 4 * kC);
            f[5] = ld2(rm + 5 * kC - 1);
            f[6] = ld2(rm + 6 * kC + 1);
            f[7] = ld2(rp + 7 * kC + 1);
            f[8] = ld2(rp + 8 * kC - 1);
        } else {
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i] = f2(0.0f, 0.0f);
#pragma unroll 1
            for (int h = 0; h < 2; ++h) {
                float g[9];
                const int dc = h << 5;
                if (h ? sim_b : sim_a) {
                    const uint64_t wn = h ? nwb : nwa;
                    simple_pull<false>(Rows{rm - c, r0 - c, rp - c, c + dc}, nw_mask(wn, 2),
                                       nw_mask(wn, 10), nw_mask(wn, 26),
                                       simple_link((uint32_t)(wn >> 35), L), bcs, tb, L, g);
                } else {
                    pull_rows(rm, r0, rp, dc, g);
                }
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    float va, vb;
                    f2_split(f[i], va, vb);
                    f[i] = h ? f2(va, g[i]) : f2(g[i], vb);
                }
            }
        }
    };
    // The 8-lane passes over the row's other boundary nodes (node m of the 64
    // is column m of the half): `use` gets the gathered populations of the
    // group's node, its column and word, and whether the group holds a node.
    auto passes = [&](const float *rm, const float *r0, const float *rp, bool cx_a, bool cx_b,
                      uint64_t nwa, uint64_t nwb, auto use) {
        const unsigned ma = __ballot_sync(0xffffffffu, cx_a);
        const unsigned mb = __ballot_sync(0xffffffffu, cx_b);
        unsigned long long rem = ((unsigned long long)mb << 32) | ma;
        while (rem) {  // warp-uniform
            unsigned long long r = rem;
            for (int q = 0; q < grp; ++q) r &= r - 1;
            const bool live = r != 0;
            const int m = __ffsll((long long)(live ? r : rem)) - 1;
            for (int q = 0; q < 4; ++q) rem &= rem - 1;
            const int src = m & 31;
            const uint64_t wa = __shfl_sync(0xffffffffu, nwa, src);
            const uint64_t wbb = __shfl_sync(0xffffffffu, nwb, src);
            const uint64_t wb = (m >> 5) ? wbb : wa;
            const int cb = (half << 6) + m;
            const BLink *lrec = blinks + boundary_index(wb, L) * 8;
            auto link = [&](int i) { return lrec[i - 1]; };
            float g0, f[9];
            const float fk = boundary8_pull(Rows{rm - c, r0 - c, rp - c, cb}, nw_mask(wb, 2),
                                            nw_mask(wb, 10), nw_mask(wb, 18), nw_mask(wb, 26),
                                            kdir, link, bcs, tb, L, g0);
            gather8(fk, g0, f);
            use(f, cb, wb, live);
        }
    };

    auto sweep = [&](auto with_boundary) {
        constexpr bool kB = decltype(with_boundary)::value;
        for (int n = 0; n < nsweep; ++n) {
            if (tid == 0 && n + kGradD + 2 <= j_last && ok) {
                // order the block's earlier shared-memory accesses before the copy
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue(n + kGradD + 2);
                j_issued = n + kGradD + 2;
            }
            const int y = y_in0 - 1 + n - kGradSkew * (lv - 1);
            const int j = y - y_in0;
            if (density_warp) {
                // density deviations of row y + 2 at this level
                if (y + 2 >= lo - 1 && y + 2 <= hi + 1) {
                    const int jd = j + 2;
                    const int ju = jd % kGradNU;
                    const uint64_t nwa = live_a ? nwr[ju * kC + c] : 0ull;
                    const uint64_t nwb = live_b ? nwr[ju * kC + c + 32] : 0ull;
                    const uint32_t cla = (uint32_t)(nwa & 3u), clb = (uint32_t)(nwb & 3u);
                    const float *rm = prev_base + ((jd - 1) & (kGradNL - 1)) * kRowF + c;
                    const float *r0 = prev_base + (jd & (kGradNL - 1)) * kRowF + c;
                    const float *rp = prev_base + ((jd + 1) & (kGradNL - 1)) * kRowF + c;
                    float *drow = den_base + (jd & (kGradND - 1)) * kC;
                    auto row = [&](auto with_boundary_row) {
                        constexpr bool kR = decltype(with_boundary_row)::value;
                        const bool sim_a = kR && cla == kBoundary && ((nwa >> 34) & 1u);
                        const bool sim_b = kR && clb == kBoundary && ((nwb >> 34) & 1u);
                        if (kR)
                            passes(rm, r0, rp, cla == kBoundary && !sim_a, clb == kBoundary && !sim_b,
                                   nwa, nwb, [&](const float *f, int cb, uint64_t, bool live) {
                                       if (live && kdir == 1) drow[cb] = density_of(f);
                                   });
                        const bool do_a = cla == kInterior || sim_a, do_b = clb == kInterior || sim_b;
                        if (do_a || do_b) {
                            F2 f[9];
                            pull_pair(with_boundary_row, rm, r0, rp, cla, clb, sim_a, sim_b, nwa,
                                      nwb, f);
                            float da, db;
                            f2_split(density_of(f), da, db);
                            if (do_a) drow[c] = da;
                            if (do_b) drow[c + 32] = db;
                        }
                    };
                    if (kB && __ballot_sync(0xffffffffu, cla == kBoundary || clb == kBoundary))
                        row(std::true_type{});
                    else
                        row(std::false_type{});
                }
            } else if (y >= lo && y <= hi) {
                // collision of row y at this level
                const int ju = j % kGradNU;
                const uint64_t nwa = live_a ? nwr[ju * kC + c] : 0ull;
                const uint64_t nwb = live_b ? nwr[ju * kC + c + 32] : 0ull;
                const uint32_t cla = (uint32_t)(nwa & 3u), clb = (uint32_t)(nwb & 3u);
                const float *rm = prev_base + ((j - 1) & (kGradNL - 1)) * kRowF + c;
                const float *r0 = prev_base + (j & (kGradNL - 1)) * kRowF + c;
                const float *rp = prev_base + ((j + 1) & (kGradNL - 1)) * kRowF + c;
                const float *dm = den_base + ((j - 1) & (kGradND - 1)) * kC;
                const float *d0 = den_base + (j & (kGradND - 1)) * kC;
                const float *dp = den_base + ((j + 1) & (kGradND - 1)) * kC;
                float *own = own_base + (j & (kGradNL - 1)) * kRowF;
                const int64_t krow = (int64_t)y * L.pitch + xin;  // lattice index of ring column 0
                const bool core_row = y >= Y0 && y < Y0 + Hs;
                float4 *urow = ur + ju * kW;
                auto advance_u = [&](int col, float jx, float jy, float dr) {
                    float4 *up = urow + (col - 2 * kGradK);
                    float4 wu = *up;
                    integrate_u_value(wu, jx, jy, L.rho0 + dr);
                    if (lv < kGradK) {
                        *up = wu;
                    } else {
                        uc[krow + col] = wu;
                        flag_nonfinite(status, dr, jx, jy);
                    }
                };
                // the scalar source of one node of the pair from its pulled populations
                auto source_one = [&](const float *g, int col, uint64_t nw, bool open, float &sx,
                                      float &sy) {
                    bool xp = true, yp = true, xm = true, ym = true;
                    if (!open) open_axes(nw, xp, yp, xm, ym);
                    grad_source(density_of(g), d0[col + 1], d0[col - 1], dp[col], dm[col], xp, xm,
                                yp, ym, L, sx, sy);
                };
                auto row = [&](auto with_boundary_row) {
                    constexpr bool kR = decltype(with_boundary_row)::value;
                    const bool sim_a = kR && cla == kBoundary && ((nwa >> 34) & 1u);
                    const bool sim_b = kR && clb == kBoundary && ((nwb >> 34) & 1u);
                    if (kR)
                        passes(rm, r0, rp, cla == kBoundary && !sim_a, clb == kBoundary && !sim_b,
                               nwa, nwb, [&](float *f, int cb, uint64_t wb, bool live) {
                                   float sx, sy, dr, jx, jy;
                                   source_one(f, cb, wb, false, sx, sy);
                                   collide(f, sx, sy, L, dr, jx, jy);
                                   float mine = f[1];
#pragma unroll
                                   for (int q = 2; q < 9; ++q)
                                       if (kdir == q) mine = f[q];
                                   if (!live) return;
                                   if (lv < kGradK) own[kdir * kC + cb] = mine;
                                   else dst[kdir * L.fplane + krow + cb] = mine;
                                   if (kdir == 1) {
                                       if (lv < kGradK) own[cb] = f[0];
                                       else dst[krow + cb] = f[0];
                                       if (core_row && cb >= 2 * kGradK && cb < kC - 2 * kGradK)
                                           advance_u(cb, jx, jy, dr);
                                   }
                               });
                    const bool do_a = cla == kInterior || sim_a, do_b = clb == kInterior || sim_b;
                    if (do_a || do_b) {
                        F2 f[9];
                        pull_pair(with_boundary_row, rm, r0, rp, cla, clb, sim_a, sim_b, nwa, nwb, f);
                        F2 sx, sy;
                        if (!kR || (cla == kInterior && clb == kInterior)) {
                            const float *d0c = d0 + c, *dpc = dp + c, *dmc = dm + c;
                            grad_source_open(density_of(f), f2(d0c[1], d0c[33]), f2(d0c[-1], d0c[31]),
                                             f2(dpc[0], dpc[32]), f2(dmc[0], dmc[32]), L, sx, sy);
                        } else {
                            float sxa = 0.0f, sya = 0.0f, sxb = 0.0f, syb = 0.0f;
#pragma unroll 1
                            for (int h = 0; h < 2; ++h) {
                                float g[9];
#pragma unroll
                                for (int i = 0; i < 9; ++i) {
                                    float va, vb;
                                    f2_split(f[i], va, vb);
                                    g[i] = h ? vb : va;
                                }
                                float hx, hy;
                                source_one(g, c + (h << 5), h ? nwb : nwa, (h ? clb : cla) == kInterior,
                                           hx, hy);
                                if (h) {
                                    sxb = hx;
                                    syb = hy;
                                } else {
                                    sxa = hx;
                                    sya = hy;
                                }
                            }
                            sx = f2(sxa, sxb);
                            sy = f2(sya, syb);
                        }
                        F2 dr, jx, jy;
                        collide_v(f, sx, sy, w2, s32, dr, jx, jy);
                        if (lv < kGradK)
                            store_pair(own + c, kC, f, do_a, do_b);
                        else
                            store_pair(dst + krow + c, L.fplane, f, do_a, do_b);
                        if (core_row) {
                            float dra, drb, jxa, jxb, jya, jyb;
                            f2_split(dr, dra, drb);
                            f2_split(jx, jxa, jxb);
                            f2_split(jy, jya, jyb);
                            if (do_a && core_a) advance_u(c, jxa, jya, dra);
                            if (do_b && core_b) advance_u(c + 32, jxb, jyb, drb);
                        }
                    }
                };
                if (kB && __ballot_sync(0xffffffffu, cla == kBoundary || clb == kBoundary))
                    row(std::true_type{});
                else
                    row(std::false_type{});
            }
            if (tid == 0 && n + 3 <= j_last && ok) {
                ok = wait_row(n + 3, L.wait_ns);
                if (!ok) last_waited = n + 2;
            }
            __syncthreads();
        }
    };
    if (region.w)
        sweep(std::true_type{});
    else
        sweep(std::false_type{});
    if (cycles && tid == 0) cycles[blockIdx.x] = clock64() - t_start;
    if (tid == 0 && !ok) {
        // a copy did not land within the limit (the rest of the sweep ran on
        // stale rows; thread 0 issued no copy after that): flag it, then wait
        // for every copy issued after the last completed wait, each with the
        // default limit, so that none is still writing this block's shared
        // memory when the block exits
        atomicOr(status, 2u);
        for (int j = last_waited + 1; j <= j_issued; ++j) wait_row(j, kDefaultWaitNs);
    }
}

// Node words: the class of every node, then the boundary records.
__global__ void k_nw_fill(const uint8_t *__restrict__ cls, uint64_t *__restrict__ nw, int64_t n) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) nw[k] = cls[k];
}

__device__ __forceinline__ int normal_code(float n0, float n1) {
    if (n1 == 0.0f && n0 == 1.0f) return 0;
    if (n1 == 0.0f && n0 == -1.0f) return 1;
    if (n0 == 0.0f && n1 == 1.0f) return 2;
    if (n0 == 0.0f && n1 == -1.0f) return 3;
    return -1;
}

__global__ void k_nw_boundary(const BNode *__restrict__ bnodes, const BLink *__restrict__ blinks,
                              int nb, int pitch, uint64_t *__restrict__ nw) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nb) return;
    const BNode b = bnodes[g];
    bool simple = b.corner == 0;
    int bc = -1, code = -1;
    for (int i = 1; i < 9; ++i) {
        if (!((b.cut >> i) & 1u)) continue;
        const BLink lk = blinks[(int64_t)g * 8 + i - 1];
        const int cd = normal_code(lk.n0, lk.n1);
        if (lk.q != 0.5f || lk.bc != lk.bc2 || cd < 0) simple = false;
        if (bc < 0) {
            bc = lk.bc;
            code = cd;
        } else if (lk.bc != bc || cd != code) {
            simple = false;
        }
    }
    uint64_t w = (uint64_t)kBoundary | ((uint64_t)((b.cut >> 1) & 0xffu) << 2) |
                 ((uint64_t)((b.dirich >> 1) & 0xffu) << 10) |
                 ((uint64_t)((b.corner >> 1) & 0xffu) << 18) |
                 ((uint64_t)((b.miss >> 1) & 0xffu) << 26);
    if (simple && bc >= 0)
        w |= (1ull << 34) | ((uint64_t)bc << 35) | ((uint64_t)code << 51);
    else
        w |= (uint64_t)g << 35;
    nw[(int64_t)b.y * pitch + b.x] = w;
}

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                 const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                 const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
    static EncodeTiled fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return (EncodeTiled) nullptr;
        }
        return reinterpret_cast<EncodeTiled>(p);
    }();
    return fn;
}

bool encode(CUtensorMap *map, CUtensorMapDataType type, cuuint32_t rank, void *base,
            const cuuint64_t *dims, const cuuint64_t *strides, const cuuint32_t *box) {
    EncodeTiled fn = encoder();
    if (!fn) return false;
    const cuuint32_t es[3] = {1, 1, 1};
    return fn(map, type, rank, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

size_t wave_smem_bytes() { return kSmem; }

bool wave_supported(const Lattice &L) {
    return L.nx >= kC && L.ny >= 1 && L.nb < (1 << 28) && encoder() != nullptr;
}

cudaError_t wave_prepare(const Tables &t, const Lattice &L, const DevState &S, WaveMaps *m,
                         cudaStream_t s, int plan_blocks) {
    const int64_t n = L.plane;
    k_nw_fill<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(S.cls, S.nw, n);
    if (L.nb > 0)
        k_nw_boundary<<<(L.nb + 127) / 128, 128, 0, s>>>(S.bnodes, S.blinks, L.nb, L.pitch, S.nw);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const cuuint64_t fdims[3] = {(cuuint64_t)L.nx, (cuuint64_t)L.ny, 9};
    const cuuint64_t fstr[2] = {(cuuint64_t)L.pitch * 4, (cuuint64_t)L.fplane * 4};
    const cuuint32_t fbox[3] = {(cuuint32_t)kC, 1, 9};
    for (int b = 0; b < 2; ++b)
        if (!encode(&m->f[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, S.f[b], fdims, fstr, fbox))
            return cudaErrorInvalidValue;
    const cuuint64_t ndims[2] = {(cuuint64_t)L.nx, (cuuint64_t)L.ny};
    const cuuint64_t nstr[1] = {(cuuint64_t)L.pitch * 8};
    const cuuint32_t nbox[2] = {(cuuint32_t)kC, 1};
    if (!encode(&m->nw, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, S.nw, ndims, nstr, nbox))
        return cudaErrorInvalidValue;
    const cuuint64_t udims[3] = {4, (cuuint64_t)L.nx, (cuuint64_t)L.ny};
    const cuuint64_t ustr[2] = {16, (cuuint64_t)L.pitch * 16};
    const cuuint32_t ubox[3] = {4, (cuuint32_t)kW, 1};
    if (!encode(&m->u, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, S.ucomp, udims, ustr, ubox))
        return cudaErrorInvalidValue;
    e = L.grad ? cudaFuncSetAttribute(k_wave_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)kGSmem)
               : cudaFuncSetAttribute(k_wave, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)kSmem);
    if (e != cudaSuccess) return e;
    const std::vector<int4> plan = wave_plan(t, plan_blocks > 0 ? plan_blocks : device_sms());
    m->nblocks = (int)plan.size();
    if (plan.empty() || plan.size() > wave_table_entries(t.nx, t.ny)) return cudaErrorInvalidValue;
    // pageable source: the copy is staged before the call returns
    return cudaMemcpyAsync(S.wave_tab, plan.data(), plan.size() * sizeof(int4),
                           cudaMemcpyHostToDevice, s);
}

cudaError_t launch_wave_batch(const WaveInst *insts, const int4 *regions, const int32_t *region_inst,
                              int nregions, int32_t *counter, int cur, int toff, int sms,
                              cudaStream_t s) {
    static const cudaError_t attr =
        cudaFuncSetAttribute(k_wave_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
    if (attr != cudaSuccess) return attr;
    if (nregions <= 0) return cudaSuccess;
    k_wave_batch<<<(unsigned)std::min(sms, nregions), kThreads, kSmem, s>>>(
        insts, regions, region_inst, nregions, counter, cur, toff);
    return cudaGetLastError();
}

cudaError_t launch_wave(const Lattice &L, const DevState &S, const WaveMaps &m, int cur, int toff,
                        cudaStream_t s, long long *cycles) {
    if (L.grad)
        k_wave_grad<<<(unsigned)m.nblocks, kGradThreads, kGSmem, s>>>(
            m.f[cur], m.nw, m.u, static_cast<float *>(S.f[cur ^ 1]),
            static_cast<float4 *>(S.ucomp), S.blinks, S.bcs, L,
            S.time, toff, S.wave_tab, S.status, cycles);
    else
        k_wave<<<(unsigned)m.nblocks, kThreads, kSmem, s>>>(
            m.f[cur], m.nw, m.u, static_cast<float *>(S.f[cur ^ 1]),
            static_cast<float4 *>(S.ucomp), S.blinks, S.bcs, L,
            S.time, toff, S.wave_tab, S.status, cycles);
    return cudaGetLastError();
}

}  // namespace lbm
