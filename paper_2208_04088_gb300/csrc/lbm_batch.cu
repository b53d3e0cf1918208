// lbm_batch.cu -- many independent solver instances advanced by one persistent
// launch per step: the lockstep batch (lbm_batch_*) and the continuous-batching
// server (lbm_server_*) of include/lbm.h.
//
// Each instance is an ordinary lbm_solver whose workspace is carved from one
// device arena.  Per step, a persistent interior kernel walks a table of
// (instance, tile) pairs and a persistent cooperative boundary kernel walks a
// table of (instance, boundary node) pairs; both run the per-node device code
// of the single-solver kernels (lbm_device.cuh), so an instance computes
// bit-identical fields alone and in a batch.  The table sizes and every
// instance's clock live in device memory, so one captured CUDA graph stays
// valid while instances come and go.
//
// In the lockstep batch, FP32 instances with two population buffers and at
// least kWaveC columns are stepped by the temporally blocked kernel instead:
// one persistent launch per kWaveK steps over the strip segments (regions) of
// all of them, longest first, each block taking the next region from a
// counter.  Its per-node arithmetic is that of the one-step kernels too.
#include <algorithm>
#include <chrono>
#include <climits>
#include <cstring>
#include <future>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "lbm_device.cuh"
#include "lbm_internal.h"
#include "lbm_pair.cuh"

namespace lbm {

// Device descriptor of one instance.
struct InstDev {
    Lattice L;
    void *f[2];      // two buffers, or f[0] alone with in-place streaming (L.in_place)
    float *stage;    // in place: the boundary nodes' staged populations
    void *uc;        // displacement records (URec of the storage type)
    const uint8_t *cls;
    const BNode *bn;
    const BLink *bl;
    const BCDev *bcs;
    uint32_t *status;
    int64_t *time;   // completed steps (the instance's own clock)
    int64_t target;  // the instance stops stepping at this time
    int32_t tiles_x;
    int32_t blocked;  // stepped by the temporally blocked batch kernel
};

// Sizes of the work tables and the dynamic-schedule counters (device memory).
struct BatchCounts {
    int32_t ntiles, nbnodes, ninst;
    int32_t nbx;  // entries [0, nbx) of the boundary map take the eight-lane update, the rest one lane
    int32_t tile_counter, pad2[3];
};

namespace {

constexpr int kChunk = 16;  // steps per replayed graph

// Batched interior kernel.  The descriptor of the tile's instance is staged in
// shared memory when a block turns to a tile of another instance, so the
// per-node code reads its lattice parameters from shared memory (as the
// single-solver kernel reads them from the parameter bank).  Schedules: 0
// persistent grid stride, 1 persistent with tiles handed out by an atomic
// counter, 2 one tile per block, 3 one block per kTileRun consecutive tiles
// (an instance's tiles are consecutive in the table, so most runs stage the
// descriptor once).  kMixed: the
// batch holds in-place instances, so each tile branches on its instance's
// streaming; without them the pull-only form is launched (the three inlined
// node updates of the mixed form cost registers: 88 bytes of spills against 24).
constexpr int kTileRun = 4;

// With 16-bit storage and only two-buffer instances each thread updates two
// adjacent nodes (interior_pair), and a tile of TX x TY threads covers
// 2 TX x TY nodes.  Threads per SM the register bound allows: on 256 plates
// with a hole, FP16 measured 79.6 GLUPS at 1536 (40 registers), 79.4 at 1280,
// 76.4 at 1024; BF16 78.7, 81.7 and 78.5.
template <class T, bool kMixed>
constexpr bool kBatchPair = !kMixed && !std::is_same<T, float>::value;
template <class T, bool kMixed>
constexpr int kBatchThreadsPerSm =
    !kBatchPair<T, kMixed> ? 2048 : (std::is_same<T, __half>::value ? 1536 : 1280);

template <class T, int TX, int TY, bool kMixed>
__global__ void __launch_bounds__(TX *TY, kBatchThreadsPerSm<T, kMixed> / (TX * TY)) k_batch_interior(const InstDev *__restrict__ insts,
                                                           const int2 *__restrict__ tiles,
                                                           BatchCounts *__restrict__ counts,
                                                           int schedule) {
    constexpr int kWords = (int)(sizeof(InstDev) / 4);
    static_assert(sizeof(InstDev) % 4 == 0, "InstDev is copied as 32-bit words");
    __shared__ __align__(16) uint32_t s_inst[kWords];
    __shared__ int s_tile, s_local;
    __shared__ long long s_time;
    const int tid = threadIdx.y * TX + threadIdx.x;
    const int ntiles = counts->ntiles;
    int tile = schedule == 1 ? -1 : (schedule == 3 ? (int)blockIdx.x * kTileRun : (int)blockIdx.x);
    int staged = -1;  // instance whose descriptor is in s_inst
    for (;;) {
        if (tid == 0) {
            if (schedule == 1) tile = atomicAdd(&counts->tile_counter, 1);
            s_tile = tile;
            if (tile < ntiles) {
                const int2 t = tiles[tile];
                s_local = t.y;
                s_time = (long long)*insts[t.x].time;
            }
        }
        __syncthreads();
        tile = s_tile;
        if (tile >= ntiles) break;
        const int inst = tiles[tile].x;
        const int64_t time = s_time;
        if (inst != staged) {  // uniform over the block
            // copy the descriptor (a few hundred bytes) with the whole block
            const uint32_t *src_words = reinterpret_cast<const uint32_t *>(insts + inst);
            for (int w = tid; w < kWords; w += TX * TY) s_inst[w] = __ldg(src_words + w);
            __syncthreads();
            if constexpr (std::is_same<T, __half>::value) {
                // the instance's scales of this step (FP16)
                if (tid == 0 && time < reinterpret_cast<const InstDev *>(s_inst)->target)
                    step_scales<T>(reinterpret_cast<InstDev *>(s_inst)->L, time);
                __syncthreads();
            }
            staged = inst;
        }
        const InstDev &I = *reinterpret_cast<const InstDev *>(s_inst);
        if constexpr (std::is_same<T, __half>::value) {
            // the tile of local index 0 publishes the instance's scales
            if (tid == 0 && time < I.target && s_local == 0) publish_scale<T>(I.L, time);
        }
        if (time < I.target) {
            const int local = s_local;
            const int tx = local % I.tiles_x, ty = local / I.tiles_x;
            const int x = tx * TX + threadIdx.x, y = ty * TY + threadIdx.y;
            if constexpr (kBatchPair<T, kMixed>) {
                const int x0 = tx * (2 * TX) + 2 * (int)threadIdx.x;
                const int cur = (int)(time & 1);
                if (x0 < I.L.nx && y < I.L.ny)
                    interior_pair<T>(static_cast<const T *>(I.f[cur]),
                                     static_cast<T *>(I.f[cur ^ 1]), static_cast<float2 *>(I.uc),
                                     I.cls, I.L, x0, y, I.status);
            } else if (x < I.L.nx && y < I.L.ny) {
                const int cur = (int)(time & 1);
                const int64_t k = (int64_t)y * I.L.pitch + x;
                if (kMixed && I.L.in_place) {  // one buffer: the AA step of the instance's parity
                    T *f = static_cast<T *>(I.f[0]);
                    if (cur)
                        interior_node<T, kAAOdd>(f, f, static_cast<URec<T> *>(I.uc), I.cls, nullptr, I.L, k, I.status);
                    else
                        interior_node<T, kAAEven>(f, f, static_cast<URec<T> *>(I.uc), I.cls, nullptr, I.L, k, I.status);
                } else {
                    interior_node<T>(static_cast<const T *>(I.f[cur]),
                                     static_cast<T *>(I.f[cur ^ 1]), static_cast<URec<T> *>(I.uc), I.cls, nullptr, I.L, k,
                                     I.status);
                }
            }
        }
        if (schedule == 2) break;
        if (schedule == 3) {
            if ((tile + 1) % kTileRun == 0) break;
            tile += 1;
        }
        if (schedule == 0) tile += gridDim.x;
        __syncthreads();  // the next tile may overwrite the staged descriptor and s_tile
    }
}

template <class T>
__global__ void __launch_bounds__(kB8) k_batch_boundary(const InstDev *__restrict__ insts,
                                                        const int2 *__restrict__ bmap,
                                                        const BatchCounts *__restrict__ counts) {
    const int nb = counts->nbx;  // map entries [0, nbx): eight lanes to a node
    constexpr int kGroups = kB8 / 8;
    const int j = threadIdx.x & 7;
    // the loop bound is uniform over the block, so all lanes reach the shuffles
    for (int base = blockIdx.x * kGroups; base < nb; base += gridDim.x * kGroups) {
        const int g = base + (threadIdx.x >> 3);
        const bool in_list = g < nb;
        const int2 m = bmap[in_list ? g : base];
        const InstDev &I = insts[m.x];
        const int64_t time = *I.time;
        const bool live = in_list && time < I.target;
        const int cur = (int)(time & 1);
        Lattice L = I.L;
        step_scales<T>(L, time);
        if (I.L.in_place) {
            // stage: the instance's populations are stored by k_batch_scatter
            // once every boundary node has read its inputs
            T *f = static_cast<T *>(I.f[0]);
            if (cur)
                boundary8_node<T, kAAOdd>(f, f, static_cast<URec<T> *>(I.uc), I.bn, I.bl, I.bcs, I.cls, nullptr, L, m.y,
                                          live, j, (float)(time - 1), I.status, I.stage);
            else
                boundary8_node<T, kAAEven>(f, f, static_cast<URec<T> *>(I.uc), I.bn, I.bl, I.bcs, I.cls, nullptr, L, m.y,
                                           live, j, (float)(time - 1), I.status, I.stage);
        } else {
            boundary8_node<T>(static_cast<const T *>(I.f[cur]), static_cast<T *>(I.f[cur ^ 1]),
                              static_cast<URec<T> *>(I.uc), I.bn, I.bl, I.bcs, I.cls, nullptr, L, m.y, live, j,
                              (float)(time - 1), I.status);
        }
    }
}

// Map entries [nbx, nbnodes): the simple boundary nodes of two-buffer
// instances (box edges, crack faces), one lane each, bit-identical to the
// eight-lane update.
template <class T>
__global__ void __launch_bounds__(128) k_batch_simple(const InstDev *__restrict__ insts,
                                                      const int2 *__restrict__ bmap,
                                                      const BatchCounts *__restrict__ counts) {
    for (int g = counts->nbx + blockIdx.x * 128 + threadIdx.x; g < counts->nbnodes;
         g += gridDim.x * 128) {
        const int2 m = bmap[g];
        const InstDev &I = insts[m.x];
        const int64_t time = *I.time;
        if (time >= I.target) continue;
        const int cur = (int)(time & 1);
        Lattice L = I.L;
        step_scales<T>(L, time);
        simple_node<T>(static_cast<const T *>(I.f[cur]), static_cast<T *>(I.f[cur ^ 1]), static_cast<URec<T> *>(I.uc),
                       I.bn, I.bl, I.bcs, L, m.y, (float)(time - 1), I.status);
    }
}

// In-place instances: the staged boundary populations into the buffer (one
// thread per boundary node and direction), beside the interior kernel.
template <class T>
__global__ void __launch_bounds__(256) k_batch_scatter(const InstDev *__restrict__ insts,
                                                       const int2 *__restrict__ bmap,
                                                       const BatchCounts *__restrict__ counts) {
    const int64_t n = (int64_t)counts->nbnodes * 9;
    for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < n; e += (int64_t)gridDim.x * 256) {
        const int2 m = bmap[e / 9];
        const int d = (int)(e % 9);
        const InstDev &I = insts[m.x];
        if (!I.L.in_place) continue;
        const int64_t time = *I.time;
        if (time >= I.target) continue;
        Lattice L = I.L;
        step_scales<T>(L, time);
        const BNode b = I.bn[m.y];
        const int64_t kn = (int64_t)b.y * I.L.pitch + b.x;
        int64_t o = 0;
        const bool odd = time & 1;
        switch (d) {  // out_at for a run-time direction and parity
#define LBM_OUT(mm) \
    case mm:        \
        o = odd ? out_at<kAAOdd>(kn, mm, I.L) : out_at<kAAEven>(kn, mm, I.L); \
        break;
            LBM_OUT(0) LBM_OUT(1) LBM_OUT(2) LBM_OUT(3) LBM_OUT(4) LBM_OUT(5) LBM_OUT(6) LBM_OUT(7)
            LBM_OUT(8)
#undef LBM_OUT
        }
        const float v = I.stage[(int64_t)m.y * 9 + d];
        Store<T>::st(static_cast<T *>(I.f[0]) + o, v, L.scale);
        note_range<T>(L, fabsf(v));
    }
}

__global__ void k_batch_advance(const InstDev *__restrict__ insts,
                                BatchCounts *__restrict__ counts) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) counts->tile_counter = 0;
    if (i < counts->ninst && !insts[i].blocked) {
        int64_t *t = insts[i].time;
        if (*t < insts[i].target) *t += 1;
    }
}

// The clocks of the instances stepped by the blocked kernel, n steps on.
__global__ void k_batch_advance_blocked(const InstDev *__restrict__ insts,
                                        const BatchCounts *__restrict__ counts, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < counts->ninst && insts[i].blocked) *insts[i].time += n;
}

lbm_status fail_cuda(cudaError_t e, const char *where) {
    set_error(std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) +
              ")");
    return LBM_ERR_CUDA;
}

// First-fit arena over one device allocation (256-byte granules).
class Arena {
   public:
    lbm_status init(uint64_t bytes) {
        bytes_ = (bytes + 255) / 256 * 256;
        cudaError_t e = cudaMalloc(&base_, bytes_);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("arena: cudaMalloc of " + std::to_string(bytes_) + " bytes failed");
            return LBM_ERR_NOMEM;
        }
        free_[0] = bytes_;
        return LBM_OK;
    }
    ~Arena() {
        if (base_) cudaFree(base_);
    }
    // returns offset or UINT64_MAX
    uint64_t alloc(uint64_t bytes) {
        bytes = (bytes + 255) / 256 * 256;
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= bytes) {
                const uint64_t off = it->first, len = it->second;
                free_.erase(it);
                if (len > bytes) free_[off + bytes] = len - bytes;
                used_ += bytes;
                return off;
            }
        return UINT64_MAX;
    }
    void release(uint64_t off, uint64_t bytes) {
        bytes = (bytes + 255) / 256 * 256;
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    char *base() const { return static_cast<char *>(base_); }
    uint64_t capacity() const { return bytes_; }
    uint64_t used() const { return used_; }

   private:
    void *base_ = nullptr;
    uint64_t bytes_ = 0, used_ = 0;
    std::map<uint64_t, uint64_t> free_;
};

// Deep copy of an lbm_desc (the caller may free its arrays after submitting).
struct DescCopy {
    lbm_desc d;
    std::vector<uint8_t> node_type;
    std::vector<lbm_link> links;
    std::vector<lbm_bc> bcs;
    explicit DescCopy(const lbm_desc &src) : d(src) {
        node_type.assign(src.node_type, src.node_type + (size_t)src.nx * src.ny);
        links.assign(src.links, src.links + src.nlinks);
        bcs.assign(src.bcs, src.bcs + src.nbcs);
        d.node_type = node_type.data();
        d.links = links.data();
        d.bcs = bcs.data();
    }
};

struct Instance {
    int64_t id = -1;
    bool blocked = false;  // stepped by the blocked batch kernel
    int plan_blocks = 0;   // its regions (strip segments)
    lbm_solver *h = nullptr;
    uint64_t off = 0, bytes = 0;
    int64_t steps = 0;   // requested steps
    int64_t done = 0;    // steps completed (host mirror)
    int64_t nodes = 0;
};

// A server request's tables, validated and classified on a worker thread
// from the moment it is submitted.
struct Prepared {
    lbm_status st = LBM_OK;
    std::string err;
    lbm_desc d;
    Tables t;
    Units u;
};

struct Request {
    int64_t id;
    std::unique_ptr<DescCopy> desc;
    int64_t steps;
    int state = 0;  // 0 queued, 1 active, 2 done, 3 failed
    bool unstable = false;      // done, but a non-finite moment was produced
    std::vector<float> result;  // u(2N), v(2N), sigma(3N) when done
    std::string error;
    std::shared_ptr<Prepared> prep;
    std::future<void> ready;    // the worker that fills prep (destroyed first)
};

// A finished server instance whose fields are on their way to the host: its
// workspace stays reserved until the copy has completed.
struct Retiring {
    Instance I;
    cudaEvent_t done = nullptr;
    float *buf = nullptr;  // pinned: u(2N), v(2N), sigma(3N), then the status word
    size_t cap = 0;        // floats
};

}  // namespace
}  // namespace lbm

using namespace lbm;

struct lbm_engine {
    int storage = LBM_F32;
    bool server = false;
    cudaStream_t stream = nullptr, cap_main = nullptr, cap_side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr, ev0 = nullptr, ev1 = nullptr;
    Arena arena;
    std::vector<Instance> inst;          // active instances (table order)
    std::map<int64_t, Request> requests; // server requests by id
    std::vector<int64_t> queue;          // queued request ids (FIFO)
    int64_t next_id = 0;
    // device tables
    InstDev *d_inst = nullptr;
    int2 *d_tiles = nullptr, *d_bmap = nullptr;
    BatchCounts *d_counts = nullptr;
    int cap_inst = 0;
    int64_t cap_tiles = 0, cap_bnodes = 0;
    int64_t ntiles = 0;  // tiles in the current table (grid of schedule 2)
    bool tables_dirty = true;
    lbm_launch_shape shape{32, 8, 8, 0};
    int sms = 0;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};  // by the blocked instances' buffer
    bool graph_in_place = false;  // the captured graph orders the boundary kernel first
    // instances stepped by the blocked kernel: their records and regions
    WaveInst *d_winst = nullptr;
    int4 *d_regions = nullptr;
    int32_t *d_region_inst = nullptr, *d_wcounter = nullptr;
    int cap_winst = 0, cap_regions = 0, nregions = 0, nblocked = 0;
    int wcur = 0;  // the buffer that holds their populations
    // pinned staging of the table uploads (reused once the last upload is done)
    char *h_stage = nullptr;
    size_t h_stage_cap = 0;
    cudaEvent_t stage_done = nullptr;
    bool stage_pending = false;
    // server: finishing instances, pinned result buffers, queued ticks
    std::vector<Retiring> retiring;
    std::vector<std::pair<float *, size_t>> pinned;  // free result buffers (floats)
    std::vector<cudaEvent_t> spare_events;
    cudaEvent_t tick_done[2] = {nullptr, nullptr};
    int64_t ticks = 0;
    int n_in_place = 0;           // instances with in-place streaming
    int64_t launches = 0;
    int64_t step_count = 0;  // steps run by the engine
    ~lbm_engine();
};

namespace {

void drop_graphs(lbm_engine *E) {
    for (auto &g : E->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

lbm_status ensure_capacity(lbm_engine *E, int ninst, int64_t ntiles, int64_t nbnodes) {
    bool realloc = false;
    cudaError_t e = cudaSuccess;
    if (ninst > E->cap_inst) {
        if (E->d_inst) cudaFree(E->d_inst);
        E->cap_inst = std::max(ninst, 2 * E->cap_inst);
        e = cudaMalloc(&E->d_inst, sizeof(InstDev) * E->cap_inst);
        realloc = true;
    }
    if (e == cudaSuccess && ntiles > E->cap_tiles) {
        if (E->d_tiles) cudaFree(E->d_tiles);
        E->cap_tiles = std::max<int64_t>(ntiles, 2 * E->cap_tiles);
        e = cudaMalloc(&E->d_tiles, sizeof(int2) * E->cap_tiles);
        realloc = true;
    }
    if (e == cudaSuccess && nbnodes > E->cap_bnodes) {
        if (E->d_bmap) cudaFree(E->d_bmap);
        E->cap_bnodes = std::max<int64_t>(std::max<int64_t>(nbnodes, 1), 2 * E->cap_bnodes);
        e = cudaMalloc(&E->d_bmap, sizeof(int2) * E->cap_bnodes);
        realloc = true;
    }
    if (e == cudaSuccess && !E->d_counts) {
        e = cudaMalloc(&E->d_counts, sizeof(BatchCounts));
        if (e == cudaSuccess) e = cudaMemset(E->d_counts, 0, sizeof(BatchCounts));
        realloc = true;
    }
    if (e != cudaSuccess) return fail_cuda(e, "batch: table allocation");
    if (realloc) drop_graphs(E);
    return LBM_OK;
}

// Regions of the blocked instances: per instance, the strip segments of a
// plan for plan_blocks blocks; all of them ordered by the planner's modelled
// cost (row sweeps, boundary updates included), the most expensive first, so
// that the blocks that take them from the counter end close together.
lbm_status rebuild_wave_tables(lbm_engine *E) {
    bool any = E->nblocked > 0;
    for (const Instance &I : E->inst) any = any || I.blocked;
    if (!any) return LBM_OK;
    std::vector<WaveInst> wi;
    std::vector<std::pair<int, int4>> reg;  // (record, region)
    std::vector<double> cost;
    for (size_t i = 0; i < E->inst.size(); ++i) {
        const Instance &I = E->inst[i];
        if (!I.blocked) continue;
        const lbm_solver *h = I.h;
        WaveInst w;
        std::memset(&w, 0, sizeof w);
        w.tf[0] = h->wave.f[0];
        w.tf[1] = h->wave.f[1];
        w.tnw = h->wave.nw;
        w.tu = h->wave.u;
        w.f[0] = static_cast<float *>(h->S.f[0]);
        w.f[1] = static_cast<float *>(h->S.f[1]);
        w.uc = static_cast<float4 *>(h->S.ucomp);
        w.blinks = h->S.blinks;
        w.bcs = h->S.bcs;
        w.time = h->S.time;
        w.status = h->S.status;
        w.L = h->L;
        const std::vector<int4> plan = wave_plan(h->tab, I.plan_blocks);
        const std::vector<double> c = wave_plan_costs(h->tab, plan);
        for (size_t r = 0; r < plan.size(); ++r) {
            reg.emplace_back((int)wi.size(), plan[r]);
            cost.push_back(c[r]);
        }
        wi.push_back(w);
    }
    std::vector<size_t> order(reg.size());
    for (size_t r = 0; r < order.size(); ++r) order[r] = r;
    std::stable_sort(order.begin(), order.end(),
                     [&cost](size_t a, size_t b) { return cost[a] > cost[b]; });
    std::vector<int4> regions(reg.size());
    std::vector<int32_t> rinst(reg.size());
    for (size_t r = 0; r < reg.size(); ++r) {
        regions[r] = reg[order[r]].second;
        rinst[r] = reg[order[r]].first;
    }
    cudaError_t e = cudaSuccess;
    if ((int)wi.size() > E->cap_winst) {
        if (E->d_winst) cudaFree(E->d_winst);
        E->cap_winst = std::max((int)wi.size(), 2 * E->cap_winst);
        e = cudaMalloc(&E->d_winst, sizeof(WaveInst) * E->cap_winst);
        drop_graphs(E);
    }
    if (e == cudaSuccess && (int)regions.size() > E->cap_regions) {
        if (E->d_regions) cudaFree(E->d_regions);
        if (E->d_region_inst) cudaFree(E->d_region_inst);
        E->cap_regions = std::max((int)regions.size(), 2 * E->cap_regions);
        e = cudaMalloc(&E->d_regions, sizeof(int4) * E->cap_regions);
        if (e == cudaSuccess) e = cudaMalloc(&E->d_region_inst, sizeof(int32_t) * E->cap_regions);
        drop_graphs(E);
    }
    if (e == cudaSuccess && !E->d_wcounter) e = cudaMalloc(&E->d_wcounter, sizeof(int32_t));
    // sets the kernel's shared-memory limit (outside any capture); launches nothing
    if (e == cudaSuccess && !wi.empty())
        e = launch_wave_batch(nullptr, nullptr, nullptr, 0, nullptr, 0, 0, E->sms, E->stream);
    if (e != cudaSuccess) return fail_cuda(e, "batch: blocked tables");
    if ((int)regions.size() != E->nregions || (int)wi.size() != E->nblocked) drop_graphs(E);
    E->nregions = (int)regions.size();
    E->nblocked = (int)wi.size();
    if (!wi.empty())
        e = cudaMemcpyAsync(E->d_winst, wi.data(), sizeof(WaveInst) * wi.size(),
                            cudaMemcpyHostToDevice, E->stream);
    if (e == cudaSuccess && !regions.empty())
        e = cudaMemcpyAsync(E->d_regions, regions.data(), sizeof(int4) * regions.size(),
                            cudaMemcpyHostToDevice, E->stream);
    if (e == cudaSuccess && !rinst.empty())
        e = cudaMemcpyAsync(E->d_region_inst, rinst.data(), sizeof(int32_t) * rinst.size(),
                            cudaMemcpyHostToDevice, E->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(E->stream);  // the host vectors die here
    if (e != cudaSuccess) return fail_cuda(e, "batch: blocked tables upload");
    return LBM_OK;
}

// Rebuild the instance, tile and boundary-node tables on the device.
lbm_status rebuild_tables(lbm_engine *E) {
    const int TX = E->shape.tile_x, TY = E->shape.tile_y;
    // nodes per tile row: two per thread when the pull-only 16-bit form runs
    bool any_in_place = false;
    for (const auto &I : E->inst) any_in_place = any_in_place || (!I.blocked && I.h->L.in_place);
    const int TXN = (E->storage != LBM_F32 && !any_in_place) ? 2 * TX : TX;
    std::vector<InstDev> hi(E->inst.size());
    std::vector<int2> tiles, bmap, simple;
    for (size_t i = 0; i < E->inst.size(); ++i) {
        const lbm_solver *h = E->inst[i].h;
        InstDev &d = hi[i];
        std::memset(&d, 0, sizeof d);
        d.L = h->L;
        d.f[0] = h->S.f[0];
        d.f[1] = h->S.f[1];
        d.stage = h->S.stage;
        d.uc = h->S.ucomp;
        d.cls = h->S.cls;
        d.bn = h->S.bnodes;
        d.bl = h->S.blinks;
        d.bcs = h->S.bcs;
        d.status = h->S.status;
        d.time = h->S.time;
        d.target = E->server ? E->inst[i].steps : INT64_MAX;
        d.tiles_x = (h->L.nx + TXN - 1) / TXN;
        d.blocked = E->inst[i].blocked ? 1 : 0;
        if (d.blocked) continue;  // not in the one-step tables
        const int tiles_y = (h->L.ny + TY - 1) / TY;
        for (int t = 0; t < d.tiles_x * tiles_y; ++t) tiles.push_back(make_int2((int)i, t));
        // the simple boundary nodes (after the others in the list) of a two-buffer
        // instance take one lane each; in place, every node takes eight
        const int nbx = h->L.in_place ? h->L.nb : (int)h->tab.nbx;
        for (int b = 0; b < nbx; ++b) bmap.push_back(make_int2((int)i, b));
        for (int b = nbx; b < h->L.nb; ++b) simple.push_back(make_int2((int)i, b));
    }
    const int32_t nbx = (int32_t)bmap.size();
    bmap.insert(bmap.end(), simple.begin(), simple.end());
    lbm_status st = ensure_capacity(E, (int)hi.size(), (int64_t)tiles.size(), (int64_t)bmap.size());
    if (st != LBM_OK) return st;
    E->n_in_place = 0;
    for (const InstDev &d : hi) E->n_in_place += d.L.in_place ? 1 : 0;
    if (E->graph_in_place != (E->n_in_place > 0)) drop_graphs(E);  // the kernels' order changes
    if (E->shape.dynamic >= 2 && (int64_t)tiles.size() != E->ntiles) {
        drop_graphs(E);  // one block per tile: the captured grid must match the table
    }
    lbm_status wst = rebuild_wave_tables(E);
    if (wst != LBM_OK) return wst;
    E->ntiles = (int64_t)tiles.size();
    BatchCounts c;
    std::memset(&c, 0, sizeof c);
    c.ntiles = (int32_t)tiles.size();
    c.nbnodes = (int32_t)bmap.size();
    c.nbx = nbx;
    c.ninst = (int32_t)hi.size();
    // the uploads go through pinned staging, queued on the stream behind the
    // steps already queued (which still read the old tables); the staging is
    // written again only once the previous upload has been done
    const size_t b_inst = sizeof(InstDev) * hi.size(), b_tiles = sizeof(int2) * tiles.size();
    const size_t b_bmap = sizeof(int2) * bmap.size(), need = b_inst + b_tiles + b_bmap + sizeof c;
    cudaError_t e = cudaSuccess;
    if (E->stage_pending) {
        e = cudaEventSynchronize(E->stage_done);
        E->stage_pending = false;
    }
    if (e == cudaSuccess && need > E->h_stage_cap) {
        if (E->h_stage) cudaFreeHost(E->h_stage);
        E->h_stage = nullptr;
        E->h_stage_cap = std::max(need, 2 * E->h_stage_cap);
        e = cudaMallocHost(&E->h_stage, E->h_stage_cap);
    }
    if (e == cudaSuccess && !E->stage_done)
        e = cudaEventCreateWithFlags(&E->stage_done, cudaEventDisableTiming);
    if (e != cudaSuccess) return fail_cuda(e, "batch: table staging");
    char *p = E->h_stage;
    std::memcpy(p, hi.data(), b_inst);
    std::memcpy(p + b_inst, tiles.data(), b_tiles);
    std::memcpy(p + b_inst + b_tiles, bmap.data(), b_bmap);
    std::memcpy(p + b_inst + b_tiles + b_bmap, &c, sizeof c);
    if (b_inst) e = cudaMemcpyAsync(E->d_inst, p, b_inst, cudaMemcpyHostToDevice, E->stream);
    if (e == cudaSuccess && b_tiles)
        e = cudaMemcpyAsync(E->d_tiles, p + b_inst, b_tiles, cudaMemcpyHostToDevice, E->stream);
    if (e == cudaSuccess && b_bmap)
        e = cudaMemcpyAsync(E->d_bmap, p + b_inst + b_tiles, b_bmap, cudaMemcpyHostToDevice,
                            E->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(E->d_counts, p + b_inst + b_tiles + b_bmap, sizeof c,
                            cudaMemcpyHostToDevice, E->stream);
    if (e == cudaSuccess) e = cudaEventRecord(E->stage_done, E->stream);
    if (e != cudaSuccess) return fail_cuda(e, "batch: table upload");
    E->stage_pending = true;
    E->tables_dirty = false;
    return LBM_OK;
}

int high_priority_value() {
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return greatest;
}

template <class T, int TX, int TY>
cudaError_t launch_interior_shape(lbm_engine *E, cudaStream_t s) {
    const int sched = E->shape.dynamic;
    const unsigned blocks =
        sched == 2   ? (unsigned)std::max<int64_t>(1, E->ntiles)
        : sched == 3 ? (unsigned)std::max<int64_t>(1, (E->ntiles + kTileRun - 1) / kTileRun)
                     : (unsigned)(E->shape.blocks_per_sm * E->sms);
    const dim3 blk(TX, TY), grd(blocks);
    if (E->n_in_place > 0)
        k_batch_interior<T, TX, TY, true><<<grd, blk, 0, s>>>(E->d_inst, E->d_tiles, E->d_counts, sched);
    else
        k_batch_interior<T, TX, TY, false><<<grd, blk, 0, s>>>(E->d_inst, E->d_tiles, E->d_counts, sched);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_batch_step_t(lbm_engine *E, cudaStream_t s_main, cudaStream_t s_side) {
    // boundary nodes beside the interior tiles, at the highest priority; with
    // in-place instances the boundary kernel goes first (it stages their
    // boundary populations before their neighbours are overwritten) and the
    // scatter of the staged populations runs beside the interior tiles
    const bool in_place = E->n_in_place > 0;
    cudaStream_t s_b = in_place ? s_main : s_side;
    if (!in_place) {
        cudaEventRecord(E->fork, s_main);
        cudaStreamWaitEvent(s_side, E->fork, 0);
    }
    cudaLaunchConfig_t cfg = {};
    // four blocks per SM: the boundary kernel is bound by the latency of its
    // dependent loads (list entry, instance record, populations); two blocks per
    // SM left 12 % of the warp slots active, and four measured 1-2 % faster
    // steps on 256 plates with holes (it overlaps the interior tiles)
    cfg.gridDim = dim3(4 * E->sms);
    cfg.blockDim = dim3(kB8);
    cfg.stream = s_b;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributePriority;
    attr[0].val.priority = high_priority_value();
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_batch_boundary<T>, (const InstDev *)E->d_inst,
                                       (const int2 *)E->d_bmap,
                                       (const BatchCounts *)E->d_counts);
    if (e != cudaSuccess) return e;
    if (in_place) {
        cudaEventRecord(E->fork, s_main);
        cudaStreamWaitEvent(s_side, E->fork, 0);
        k_batch_scatter<T><<<2 * E->sms, 256, 0, s_side>>>(
            (const InstDev *)E->d_inst, (const int2 *)E->d_bmap, (const BatchCounts *)E->d_counts);
    }
    // the simple boundary nodes of the two-buffer instances, beside the interior tiles
    cfg.gridDim = dim3(2 * E->sms);
    cfg.blockDim = dim3(128);
    cfg.stream = s_side;
    e = cudaLaunchKernelEx(&cfg, k_batch_simple<T>, (const InstDev *)E->d_inst,
                           (const int2 *)E->d_bmap, (const BatchCounts *)E->d_counts);
    if (e != cudaSuccess) return e;
    cudaEventRecord(E->join, s_side);
    const int TX = E->shape.tile_x, TY = E->shape.tile_y;
    if (TX == 32 && TY == 8)
        e = launch_interior_shape<T, 32, 8>(E, s_main);
    else if (TX == 32 && TY == 4)
        e = launch_interior_shape<T, 32, 4>(E, s_main);
    else if (TX == 64 && TY == 4)
        e = launch_interior_shape<T, 64, 4>(E, s_main);
    else
        e = launch_interior_shape<T, 32, 16>(E, s_main);
    if (e != cudaSuccess) return e;
    cudaStreamWaitEvent(s_main, E->join, 0);
    k_batch_advance<<<(std::max(1, E->cap_inst) + 255) / 256, 256, 0, s_main>>>(E->d_inst,
                                                                               E->d_counts);
    return cudaGetLastError();
}

cudaError_t launch_batch_step(lbm_engine *E, cudaStream_t s_main, cudaStream_t s_side) {
    switch (E->storage) {
        case LBM_F16_DEV:
            return launch_batch_step_t<__half>(E, s_main, s_side);
        case LBM_BF16_DEV:
            return launch_batch_step_t<__nv_bfloat16>(E, s_main, s_side);
        default:
            return launch_batch_step_t<float>(E, s_main, s_side);
    }
}

// kChunk steps of the instances stepped by the blocked kernel: kChunk/kWaveK
// launches from buffer `wcur` (an even number, so they end in it), then their
// clocks.  They read the clocks at the start of the chunk (toff = the launch's
// first step within it).
static_assert(kChunk % (2 * kWaveK) == 0, "blocked launches per chunk");

cudaError_t launch_blocked_chunk(lbm_engine *E, cudaStream_t s) {
    if (E->nblocked == 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    int cur = E->wcur;
    for (int toff = 0; toff < kChunk && e == cudaSuccess; toff += kWaveK) {
        e = cudaMemsetAsync(E->d_wcounter, 0, sizeof(int32_t), s);
        if (e == cudaSuccess)
            e = launch_wave_batch(E->d_winst, E->d_regions, E->d_region_inst, E->nregions,
                                  E->d_wcounter, cur, toff, E->sms, s);
        cur ^= 1;
    }
    if (e != cudaSuccess) return e;
    k_batch_advance_blocked<<<(std::max(1, E->cap_inst) + 255) / 256, 256, 0, s>>>(
        E->d_inst, E->d_counts, kChunk);
    return cudaGetLastError();
}

// Launches of one chunk beyond the blocked part: the one-step steps of the
// other instances (none when every instance is blocked).
int64_t one_step_instances(const lbm_engine *E) {
    return (int64_t)E->inst.size() - E->nblocked;
}

lbm_status build_batch_graph(lbm_engine *E) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(E->cap_main, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return fail_cuda(e, "batch: begin capture");
    e = launch_blocked_chunk(E, E->cap_main);
    if (one_step_instances(E) > 0)
        for (int s = 0; s < kChunk && e == cudaSuccess; ++s)
            e = launch_batch_step(E, E->cap_main, E->cap_side);
    cudaError_t e2 = cudaStreamEndCapture(E->cap_main, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail_cuda(e != cudaSuccess ? e : e2, "batch: capture");
    }
    e = cudaGraphInstantiate(&E->graph[E->wcur], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail_cuda(e, "batch: instantiate");
    E->graph_in_place = E->n_in_place > 0;
    return LBM_OK;
}

// Advance every active instance by nsteps (instances past their target idle).
lbm_status engine_steps(lbm_engine *E, int64_t nsteps) {
    if (E->tables_dirty) {
        lbm_status st = rebuild_tables(E);
        if (st != LBM_OK) return st;
    }
    if (E->inst.empty() || nsteps <= 0) return LBM_OK;
    cudaError_t e = cudaSuccess;
    int64_t done = 0;
    // boundary, simple boundary nodes, interior, advance (+ scatter with in-place instances)
    const int per_step = one_step_instances(E) > 0 ? (E->n_in_place > 0 ? 5 : 4) : 0;
    if (nsteps >= kChunk) {
        if (!E->graph[E->wcur]) {
            lbm_status st = build_batch_graph(E);
            if (st != LBM_OK) return st;
        }
        for (; done + kChunk <= nsteps; done += kChunk) {
            e = cudaGraphLaunch(E->graph[E->wcur], E->stream);
            if (e != cudaSuccess) return fail_cuda(e, "batch: graph launch");
            E->launches += per_step * kChunk + (E->nblocked > 0 ? kChunk / kWaveK + 1 : 0);
        }
    }
    const int64_t rest = nsteps - done;
    if (rest > 0) {
        if (one_step_instances(E) > 0)
            for (int64_t k = 0; k < rest; ++k) {
                e = launch_batch_step(E, E->stream, E->cap_side);
                if (e != cudaSuccess) return fail_cuda(e, "batch: launch");
            }
        E->launches += per_step * rest;
        // the blocked instances take the rest of the steps with their own
        // launches, as lbm_step would: blocked launches, then one-step ones
        for (auto &I : E->inst) {
            if (!I.blocked) continue;
            lbm_solver *h = I.h;
            for (int64_t k = 0; k < rest && e == cudaSuccess;) {
                if (rest - k >= kWaveK) {
                    e = launch_wave(h->L, h->S, h->wave, h->cur, (int)k, E->stream);
                    k += kWaveK;
                    E->launches += 1;
                } else {
                    e = launch_step(h->storage, h->L, h->S, h->cur, (int)k, E->stream, nullptr,
                                    nullptr, nullptr, nullptr);
                    k += 1;
                    E->launches += kernels_per_step(h->L);
                }
                h->cur ^= 1;
            }
            if (e == cudaSuccess) e = launch_advance(h->S, rest, E->stream);
            if (e != cudaSuccess) return fail_cuda(e, "batch: blocked instance launch");
            E->launches += 1;
            E->wcur = h->cur;  // the same for every blocked instance
        }
    }
    E->step_count += nsteps;
    for (auto &I : E->inst) {
        I.done = E->server ? std::min(I.steps, I.done + nsteps) : I.done + nsteps;
        I.h->time = I.done;
        if (!I.blocked) I.h->cur = (int)(I.done & 1);
    }
    return LBM_OK;
}

lbm_status engine_init(lbm_engine *E, int storage, void *stream) {
    E->storage = storage;
    E->stream = static_cast<cudaStream_t>(stream);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&E->sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&E->cap_main, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&E->cap_side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&E->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&E->join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&E->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&E->ev1);
    if (e != cudaSuccess) return fail_cuda(e, "engine: init");
    return LBM_OK;
}

// The batched kernels step every instance one step per launch, so instances
// are created without the tables of the temporally blocked kernel; each keeps
// the streaming form its descriptor asks for.
lbm_desc one_step(const lbm_desc &d) {
    lbm_desc o = d;
    o.time_block = 1;
    return o;
}

// Rows of the strip segments a blocked batch instance is cut into: long
// enough that the 3 kWaveK - 3 rows of a segment's pipeline fill and drain
// stay a small part of it, short enough that a batch holds many more segments
// than the device has SMs.
constexpr int kBatchSegmentRows = 768;

// Whether an instance of the lockstep batch takes the temporally blocked
// kernel: FP32 storage, two population buffers and at least kWaveC columns.
bool batch_blocked(const lbm_engine *E, const lbm_desc &d) {
    return !E->server && d.storage == LBM_F32 && d.streaming == LBM_STREAM_TWO_BUFFERS &&
           d.nx >= kWaveC;
}

// The descriptor an instance is created from: the blocked form for the
// instances batch_blocked() picks, one step per launch for the others.
lbm_desc instance_desc(const lbm_engine *E, const lbm_desc &d_in) {
    lbm_desc o = one_step(d_in);
    if (batch_blocked(E, d_in)) o.time_block = LBM_TIME_BLOCK;
    return o;
}

// Admit one instance, from tables already validated and classified (d is the
// instance's descriptor, instance_desc()), into the arena; LBM_ERR_NOMEM if it
// does not fit now, and the tables are then left as they were.  Server
// instances are created deferred: their uploads are queued behind the steps
// already queued, with no wait on the host.
lbm_status admit_prepared(lbm_engine *E, const lbm_desc &d, Tables &t, const Units &u, int64_t id,
                          int64_t steps) {
    // the batched kernels implement the lambda = mu path (no density pass)
    if (u.lam != u.mu) {
        set_error("batch/server: instances must have lambda = mu (the density pass of the "
                  "lambda != mu source is single-solver only)");
        return LBM_ERR_ARG;
    }
    if (d.storage != E->storage) {
        set_error("batch/server: every instance must use the engine's storage");
        return LBM_ERR_ARG;
    }
    const uint64_t bytes = workspace_bytes_for(d, t, u);
    if (bytes == 0) {
        set_error("batch/server: the instance's stepping form is not supported");
        return LBM_ERR_ARG;
    }
    lbm_status st = LBM_OK;
    const uint64_t off = E->arena.alloc(bytes);
    if (off == UINT64_MAX) {
        set_error("batch/server: not enough room in the device budget");
        return LBM_ERR_NOMEM;
    }
    lbm_handle h = nullptr;
    int plan_blocks = 0;
    if (d.time_block == LBM_TIME_BLOCK) {
        const int strips = (d.nx + kWaveW - 1) / kWaveW;
        const int segments = std::max(1, (d.ny + kBatchSegmentRows / 2) / kBatchSegmentRows);
        plan_blocks = strips * segments;
    }
    CreateOptions opt;
    opt.plan_blocks = plan_blocks;
    opt.deferred = E->server;
    st = create_prepared(&d, std::move(t), u, E->stream, E->arena.base() + off, bytes, opt, &h);
    if (st != LBM_OK) {
        E->arena.release(off, bytes);
        return st;
    }
    Instance I;
    I.id = id;
    I.blocked = h->block == kWaveK;
    I.plan_blocks = plan_blocks;
    I.h = h;
    I.off = off;
    I.bytes = bytes;
    I.steps = steps;
    I.nodes = h->tab.interior + h->L.nb;
    E->inst.push_back(I);
    E->tables_dirty = true;
    return LBM_OK;
}

// Admit one instance from its descriptor (the lockstep batch).
lbm_status admit(lbm_engine *E, const lbm_desc &d_in, int64_t id, int64_t steps) {
    const lbm_desc d = instance_desc(E, d_in);
    Tables t;
    Units u;
    lbm_status st = prepare(&d, &t, &u);
    if (st != LBM_OK) return st;
    return admit_prepared(E, d, t, u, id, steps);
}

// A pinned result buffer of at least n floats from the pool.
float *take_pinned(lbm_engine *E, size_t n, size_t *cap) {
    size_t best = SIZE_MAX;
    for (size_t k = 0; k < E->pinned.size(); ++k)
        if (E->pinned[k].second >= n && (best == SIZE_MAX || E->pinned[k].second < E->pinned[best].second))
            best = k;
    if (best != SIZE_MAX) {
        float *p = E->pinned[best].first;
        *cap = E->pinned[best].second;
        E->pinned.erase(E->pinned.begin() + (long)best);
        return p;
    }
    float *p = nullptr;
    if (cudaMallocHost(&p, n * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    *cap = n;
    return p;
}

cudaEvent_t take_event(lbm_engine *E) {
    if (!E->spare_events.empty()) {
        cudaEvent_t ev = E->spare_events.back();
        E->spare_events.pop_back();
        return ev;
    }
    cudaEvent_t ev = nullptr;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return ev;
}

// Server: instance k has reached its step count.  Its fields and status word
// are queued for the host (fields kernels into the workspace's staging, then
// copies into a pinned buffer); it leaves the tables now and its workspace is
// released once the copies have completed (finish_retired).
lbm_status start_retire(lbm_engine *E, size_t k) {
    Retiring R;
    R.I = E->inst[k];
    lbm_solver *h = R.I.h;
    const size_t N = (size_t)h->L.nx * h->L.ny;
    R.buf = take_pinned(E, 7 * N + 1, &R.cap);
    R.done = take_event(E);
    if (!R.buf || !R.done) {
        set_error("server: pinned result buffer or event allocation failed");
        return LBM_ERR_NOMEM;
    }
    cudaError_t e = launch_fields(h->storage, h->L, h->S, h->cur, nullptr, nullptr, nullptr, E->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(R.buf, h->S.stage, 7 * N * sizeof(float), cudaMemcpyDeviceToHost,
                            E->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(R.buf + 7 * N, h->S.status, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                            E->stream);
    if (e == cudaSuccess) e = cudaEventRecord(R.done, E->stream);
    if (e != cudaSuccess) return fail_cuda(e, "server: retire");
    E->launches += kernels_per_fields(h->L);
    E->retiring.push_back(R);
    E->inst.erase(E->inst.begin() + (long)k);
    E->tables_dirty = true;
    return LBM_OK;
}

// Server: the retiring instances whose copies have completed deliver their
// results and give back their workspace; returns how many did.
int finish_retired(lbm_engine *E) {
    int n = 0;
    for (size_t k = 0; k < E->retiring.size();) {
        Retiring &R = E->retiring[k];
        const cudaError_t q = cudaEventQuery(R.done);
        if (q == cudaErrorNotReady) {
            cudaGetLastError();
            ++k;
            continue;
        }
        Request &r = E->requests.at(R.I.id);
        lbm_solver *h = R.I.h;
        const size_t N = (size_t)h->L.nx * h->L.ny;
        if (q == cudaSuccess) {
            uint32_t status = 0;
            std::memcpy(&status, R.buf + 7 * N, sizeof status);
            r.result.assign(R.buf, R.buf + 7 * N);
            r.unstable = (status & 1u) != 0;
            r.state = (status & 2u) ? 3 : 2;
            if (status & 2u) r.error = "a bounded wait for a tile copy expired on the device";
        } else {
            r.state = 3;
            r.error = std::string("server: ") + cudaGetErrorString(q);
        }
        r.desc.reset();
        destroy_deferred(h);
        E->arena.release(R.I.off, R.I.bytes);
        E->pinned.emplace_back(R.buf, R.cap);
        E->spare_events.push_back(R.done);
        E->retiring.erase(E->retiring.begin() + (long)k);
        ++n;
    }
    return n;
}

}  // namespace

lbm_engine::~lbm_engine() {
    if (stream) cudaStreamSynchronize(stream);
    for (auto &I : inst) lbm_destroy(I.h);
    inst.clear();
    for (auto &R : retiring) {
        destroy_deferred(R.I.h);
        if (R.buf) cudaFreeHost(R.buf);
        if (R.done) cudaEventDestroy(R.done);
    }
    retiring.clear();
    for (auto &p : pinned) cudaFreeHost(p.first);
    for (auto ev : spare_events) cudaEventDestroy(ev);
    for (auto ev : tick_done)
        if (ev) cudaEventDestroy(ev);
    if (stage_done) cudaEventDestroy(stage_done);
    if (h_stage) cudaFreeHost(h_stage);
    requests.clear();  // waits for the workers of requests never admitted
    for (auto &g : graph)
        if (g) cudaGraphExecDestroy(g);
    if (d_winst) cudaFree(d_winst);
    if (d_regions) cudaFree(d_regions);
    if (d_region_inst) cudaFree(d_region_inst);
    if (d_wcounter) cudaFree(d_wcounter);
    if (d_inst) cudaFree(d_inst);
    if (d_tiles) cudaFree(d_tiles);
    if (d_bmap) cudaFree(d_bmap);
    if (d_counts) cudaFree(d_counts);
    if (cap_main) cudaStreamDestroy(cap_main);
    if (cap_side) cudaStreamDestroy(cap_side);
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
}

// ---------------------------------------------------------------------------
// Lockstep batch.

extern "C" lbm_status lbm_batch_create(const lbm_desc *descs, int32_t count, void *stream,
                                       lbm_batch *out) {
    set_error("");
    if (!descs || count < 1 || !out) {
        set_error("lbm_batch_create: bad arguments");
        return LBM_ERR_ARG;
    }
    *out = nullptr;
    std::unique_ptr<lbm_engine> E(new lbm_engine());
    lbm_status st = engine_init(E.get(), descs[0].storage, stream);
    if (st != LBM_OK) return st;
    uint64_t total = 0;
    for (int32_t i = 0; i < count; ++i) {
        uint64_t b = 0;
        const lbm_desc di = instance_desc(E.get(), descs[i]);
        st = lbm_workspace_size(&di, &b);
        if (st != LBM_OK) return st;
        total += (b + 255) / 256 * 256;
    }
    st = E->arena.init(total);
    if (st != LBM_OK) return st;
    for (int32_t i = 0; i < count; ++i) {
        st = admit(E.get(), descs[i], i, INT64_MAX);
        if (st != LBM_OK) return st;
    }
    st = rebuild_tables(E.get());
    if (st != LBM_OK) return st;
    *out = E.release();
    return LBM_OK;
}

extern "C" lbm_status lbm_batch_step(lbm_batch b, int64_t nsteps) {
    set_error("");
    if (!b || nsteps < 0) {
        set_error("lbm_batch_step: bad arguments");
        return LBM_ERR_ARG;
    }
    return engine_steps(b, nsteps);
}

extern "C" lbm_status lbm_batch_get_fields(lbm_batch b, int32_t index, float *u, float *v,
                                           float *sigma, int32_t on_device) {
    set_error("");
    if (!b || index < 0 || index >= (int32_t)b->inst.size()) {
        set_error("lbm_batch_get_fields: bad instance index");
        return LBM_ERR_ARG;
    }
    return lbm_get_fields(b->inst[index].h, u, v, sigma, on_device);
}

extern "C" lbm_status lbm_batch_set_shape(lbm_batch b, const lbm_launch_shape *shape) {
    set_error("");
    if (!b || !shape) {
        set_error("lbm_batch_set_shape: bad arguments");
        return LBM_ERR_ARG;
    }
    const bool ok_tile = (shape->tile_x == 32 && (shape->tile_y == 4 || shape->tile_y == 8 ||
                                                  shape->tile_y == 16)) ||
                         (shape->tile_x == 64 && shape->tile_y == 4);
    if (!ok_tile || shape->blocks_per_sm < 1 || shape->blocks_per_sm > 64 ||
        shape->dynamic < 0 || shape->dynamic > 3) {
        set_error("lbm_batch_set_shape: tiles 32x4, 32x8, 32x16 or 64x4; 1..64 blocks per SM; "
                  "schedule 0, 1 or 2");
        return LBM_ERR_ARG;
    }
    b->shape = *shape;
    b->tables_dirty = true;
    drop_graphs(b);
    return LBM_OK;
}

extern "C" lbm_status lbm_batch_reset(lbm_batch b) {
    set_error("");
    if (!b) {
        set_error("lbm_batch_reset: NULL batch");
        return LBM_ERR_ARG;
    }
    for (auto &I : b->inst) {
        lbm_status st = lbm_reset(I.h);
        if (st != LBM_OK) return st;
        I.done = 0;
    }
    b->wcur = 0;  // lbm_reset puts every instance's populations in buffer 0
    return LBM_OK;
}

extern "C" lbm_status lbm_batch_sync(lbm_batch b) {
    set_error("");
    if (!b) {
        set_error("lbm_batch_sync: NULL batch");
        return LBM_ERR_ARG;
    }
    for (auto &I : b->inst) {
        lbm_status st = lbm_sync(I.h);
        if (st != LBM_OK) return st;
    }
    return LBM_OK;
}

extern "C" lbm_status lbm_batch_tune(lbm_batch b, int32_t steps_per_trial,
                                     lbm_launch_shape *chosen) {
    set_error("");
    if (!b || steps_per_trial < 1) {
        set_error("lbm_batch_tune: bad arguments");
        return LBM_ERR_ARG;
    }
    const lbm_launch_shape cands[] = {
        {32, 8, 8, 2},  {32, 4, 16, 2}, {64, 4, 8, 2},  {32, 16, 4, 2}, {32, 8, 8, 0},
        {32, 8, 8, 1},  {32, 8, 4, 0},  {32, 4, 16, 0}, {32, 4, 16, 1}, {64, 4, 8, 0},
        {64, 4, 8, 1},  {32, 16, 4, 0}, {32, 16, 4, 1}, {32, 4, 16, 3}, {32, 8, 8, 3},
        {64, 4, 8, 3}};
    float best = 1e30f;
    lbm_launch_shape best_shape = b->shape;
    for (const auto &c : cands) {
        lbm_status st = lbm_batch_set_shape(b, &c);
        if (st == LBM_OK) st = engine_steps(b, 2);  // warm-up (tables, caches)
        if (st != LBM_OK) return st;
        cudaEventRecord(b->ev0, b->stream);
        st = engine_steps(b, steps_per_trial);
        if (st != LBM_OK) return st;
        cudaEventRecord(b->ev1, b->stream);
        cudaError_t e = cudaEventSynchronize(b->ev1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, b->ev0, b->ev1);
        if (e != cudaSuccess) return fail_cuda(e, "lbm_batch_tune");
        if (ms < best) {
            best = ms;
            best_shape = c;
        }
    }
    lbm_status st = lbm_batch_set_shape(b, &best_shape);
    if (st == LBM_OK) st = lbm_batch_reset(b);
    if (st == LBM_OK && chosen) *chosen = best_shape;
    return st;
}

extern "C" lbm_status lbm_batch_info(lbm_batch b, lbm_batch_stats *stats) {
    set_error("");
    if (!b || !stats) {
        set_error("lbm_batch_info: bad arguments");
        return LBM_ERR_ARG;
    }
    std::memset(stats, 0, sizeof *stats);
    stats->instances = (int32_t)b->inst.size();
    for (auto &I : b->inst) {
        const lbm_status st = lbm_sync(I.h);
        if (st == LBM_ERR_UNSTABLE)
            ++stats->unstable;
        else if (st != LBM_OK)
            return st;
    }
    set_error("");
    for (auto &I : b->inst) stats->nodes += I.nodes;
    stats->steps = b->step_count;
    stats->device_bytes = b->arena.used();
    stats->kernel_launches = b->launches;
    stats->shape = b->shape;
    stats->blocked_instances = b->nblocked;
    return LBM_OK;
}

extern "C" lbm_status lbm_batch_destroy(lbm_batch b) {
    delete b;
    return LBM_OK;
}

// ---------------------------------------------------------------------------
// Continuous-batching server.

extern "C" lbm_status lbm_server_create(uint64_t hbm_budget_bytes, int32_t storage, void *stream,
                                        lbm_server *out) {
    set_error("");
    if (!out || hbm_budget_bytes < (1u << 20) || storage < LBM_F32 || storage > LBM_BF16_DEV) {
        set_error("lbm_server_create: bad arguments (budget >= 1 MiB, known storage)");
        return LBM_ERR_ARG;
    }
    *out = nullptr;
    std::unique_ptr<lbm_engine> E(new lbm_engine());
    E->server = true;
    lbm_status st = engine_init(E.get(), storage, stream);
    if (st == LBM_OK) st = E->arena.init(hbm_budget_bytes);
    if (st != LBM_OK) return st;
    *out = E.release();
    return LBM_OK;
}

extern "C" lbm_status lbm_server_submit(lbm_server s, const lbm_desc *desc, int64_t nsteps,
                                        int64_t *id) {
    set_error("");
    if (!s || !desc || nsteps < 1 || !id) {
        set_error("lbm_server_submit: bad arguments");
        return LBM_ERR_ARG;
    }
    // a request that can never fit is refused now: one population buffer and
    // the displacement records alone exceed the budget
    const uint64_t esz = desc->storage == LBM_F32 ? 4 : 2;
    const uint64_t nodes = (uint64_t)std::max(desc->nx, 0) * (uint64_t)std::max(desc->ny, 0);
    if (nodes * (9 * esz + 16) > s->arena.capacity()) {
        set_error("lbm_server_submit: the request alone exceeds the device budget");
        return LBM_ERR_NOMEM;
    }
    Request r;
    r.id = s->next_id++;
    r.desc.reset(new DescCopy(*desc));
    r.steps = nsteps;
    // validation and classification run on a worker thread from now on; a
    // request that fails them fails at admission
    auto prep = std::make_shared<Prepared>();
    const DescCopy *dc = r.desc.get();
    r.prep = prep;
    r.ready = std::async(std::launch::async, [prep, dc]() {
        prep->d = one_step(dc->d);
        prep->st = prepare(&prep->d, &prep->t, &prep->u);
        if (prep->st != LBM_OK) prep->err = lbm_last_error();
    });
    *id = r.id;
    s->queue.push_back(r.id);
    s->requests.emplace(r.id, std::move(r));
    return LBM_OK;
}

extern "C" lbm_status lbm_server_tick(lbm_server s, int32_t max_steps, lbm_server_stats *stats) {
    set_error("");
    if (!s || max_steps < 1) {
        set_error("lbm_server_tick: bad arguments");
        return LBM_ERR_ARG;
    }
    int32_t admitted = 0;
    // results whose copies have landed
    int32_t finished = finish_retired(s);
    // admit queued requests in arrival order while they are classified and fit
    while (!s->queue.empty()) {
        Request &r = s->requests.at(s->queue.front());
        if (r.ready.valid()) {
            // with instances running, an unclassified request waits for a
            // later tick; with none, there is nothing else to do than wait
            if (!s->inst.empty() &&
                r.ready.wait_for(std::chrono::seconds(0)) != std::future_status::ready)
                break;
            r.ready.get();
        }
        Prepared &P = *r.prep;
        lbm_status st = P.st;
        std::string err = P.err;
        if (st == LBM_OK && workspace_bytes_for(P.d, P.t, P.u) > s->arena.capacity()) {
            st = LBM_ERR_NOMEM;
            err = "the request alone exceeds the device budget";
        } else if (st == LBM_OK) {
            st = admit_prepared(s, P.d, P.t, P.u, r.id, r.steps);
            if (st == LBM_ERR_NOMEM) break;  // room frees up as requests finish
            if (st != LBM_OK) err = lbm_last_error();
        }
        s->queue.erase(s->queue.begin());
        r.prep.reset();
        if (st != LBM_OK) {
            r.state = 3;
            r.error = err;
            continue;
        }
        r.state = 1;
        ++admitted;
    }
    // advance: at most max_steps, and no further than the nearest completion.
    // At most two ticks are queued on the device: the host prepares the next
    // while the device runs the previous one.
    int64_t adv = max_steps;
    for (auto &I : s->inst) adv = std::min(adv, I.steps - I.done);
    if (!s->inst.empty()) {
        if (adv < 1) adv = 1;
        cudaEvent_t &slot = s->tick_done[s->ticks & 1];
        if (!slot && cudaEventCreateWithFlags(&slot, cudaEventDisableTiming) != cudaSuccess)
            return fail_cuda(cudaGetLastError(), "server: tick event");
        if (s->ticks >= 2) {
            const cudaError_t e = cudaEventSynchronize(slot);
            if (e != cudaSuccess) return fail_cuda(e, "server: tick wait");
        }
        lbm_status st = engine_steps(s, adv);
        if (st != LBM_OK) return st;
        // instances that reach their step count in this tick start retiring
        for (size_t k = 0; k < s->inst.size();) {
            if (s->inst[k].done < s->inst[k].steps) {
                ++k;
                continue;
            }
            st = start_retire(s, k);
            if (st != LBM_OK) return st;
        }
        const cudaError_t e = cudaEventRecord(slot, s->stream);
        if (e != cudaSuccess) return fail_cuda(e, "server: tick event");
        ++s->ticks;
    } else if (!s->retiring.empty()) {
        // nothing to step: wait for the results in flight instead of spinning
        const cudaError_t e = cudaEventSynchronize(s->retiring.front().done);
        if (e != cudaSuccess) return fail_cuda(e, "server: result wait");
        finished += finish_retired(s);
    }
    if (stats) {
        std::memset(stats, 0, sizeof *stats);
        stats->active = (int32_t)s->inst.size();
        stats->queued = (int32_t)s->queue.size();
        stats->admitted = admitted;
        stats->finished = finished;
        stats->steps = s->inst.empty() ? 0 : adv;
        for (auto &I : s->inst) stats->active_nodes += I.nodes;
        stats->device_bytes = s->arena.used();
        stats->kernel_launches = s->launches;
    }
    return LBM_OK;
}

extern "C" lbm_status lbm_server_result(lbm_server s, int64_t id, int32_t *state, float *u,
                                        float *v, float *sigma) {
    set_error("");
    if (!s || !state) {
        set_error("lbm_server_result: bad arguments");
        return LBM_ERR_ARG;
    }
    auto it = s->requests.find(id);
    if (it == s->requests.end()) {
        set_error("lbm_server_result: unknown or already collected request");
        return LBM_ERR_ARG;
    }
    Request &r = it->second;
    *state = r.state;
    if (r.state == 3) {
        set_error("lbm_server_result: request failed: " + r.error);
        s->requests.erase(it);
        return LBM_ERR_ARG;
    }
    if (r.state != 2) return LBM_OK;
    const size_t N = r.result.size() / 7;
    if (u) std::memcpy(u, r.result.data(), 2 * N * sizeof(float));
    if (v) std::memcpy(v, r.result.data() + 2 * N, 2 * N * sizeof(float));
    if (sigma) std::memcpy(sigma, r.result.data() + 4 * N, 3 * N * sizeof(float));
    const bool unstable = r.unstable;
    s->requests.erase(it);
    if (unstable) {
        set_error("lbm_server_result: the run produced a non-finite moment (unstable)");
        return LBM_ERR_UNSTABLE;
    }
    return LBM_OK;
}

extern "C" lbm_status lbm_server_destroy(lbm_server s) {
    delete s;
    return LBM_OK;
}
