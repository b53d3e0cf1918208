// lbm_capi.cu -- the C ABI of include/lbm.h: handle life cycle, device memory
// layout, stepping (direct launches or replayed CUDA graphs), fields and probes.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "lbm_internal.h"

using namespace lbm;


namespace {

constexpr int kGraphChunk = 32;  // steps per replayed graph (even: parity preserved)

lbm_status cuda_fail(cudaError_t e, const char *where) {
    set_error(std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
    return LBM_ERR_CUDA;
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

struct Layout {
    size_t f0, f1, ucomp, cls, bnodes, blinks, bcs, rho, status, time, scale, stage, probe,
        probe_idx, nw, wave_tab, total;
};

// Steps per launch for a description: the temporally blocked kernel needs FP32
// storage and a lattice at least one strip wide (8 steps per launch, 4 when
// lambda != mu).  Returns 0 if
// the description asks for blocking that this lattice cannot have.
// Boundary nodes that the blocked kernel updates eight lanes to a node: all but
// the "simple" ones (every cut link a mid-link wall of one BC and one
// axis-aligned normal: box edges and crack faces).
int64_t complex_boundary_nodes(const Tables &t) {
    int64_t n = 0;
    for (size_t g = 0; g < t.bnodes.size(); ++g) n += complex_boundary_node(t, g) ? 1 : 0;
    return n;
}

int steps_per_launch(const lbm_desc &d, const Tables &t, const Units &u) {
    const bool ok = d.storage == LBM_F32 && t.nx >= kWaveC && t.bnodes.size() < (size_t(1) << 28) &&
                    d.streaming != LBM_STREAM_IN_PLACE;
    const int k = u.lam == u.mu ? kWaveK : kWaveGradK;
    if (d.time_block == 1) return 1;
    if (d.time_block == LBM_TIME_BLOCK) return ok ? k : 0;
    // The library default: blocked where that measured faster on GB300 --
    // lambda = mu (with lambda != mu the blocked kernel carries 4 levels and
    // its collision warps set each row's time: 48 vs 47 GLUPS on the 2048^2
    // crack, too small a margin to make it the default), lattices of at
    // least 2^21 nodes (below, the fill of each block's row pipeline dominates:
    // 1024^2 plate 57 vs 80 GLUPS), and at most one boundary node off box edges
    // and crack faces per 800 nodes: the blocked kernel updates those eight
    // lanes to a node at every level (2048^2 plates with a hole: radius 512,
    // one per 1022 nodes, 74 vs 59 GLUPS; radius 900, one per 582, 34 vs 48).
    const int64_t nodes = (int64_t)t.nx * t.ny;
    const bool faster = u.lam == u.mu && nodes >= ((int64_t)1 << 21) &&
                        complex_boundary_nodes(t) * 800 <= nodes;
    return ok && faster ? k : 1;
}

Layout layout(const Tables &t, int storage, bool grad, int block, bool in_place) {
    const size_t plane = (size_t)t.pitch * t.ny;
    const size_t fplane = in_place ? (size_t)t.pitch * (t.ny + 2) : plane;
    const size_t esz = storage == LBM_F32 ? 4 : 2;
    const size_t N = (size_t)t.nx * t.ny;
    Layout l;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += align256(bytes);
        return at;
    };
    l.f0 = take(9 * fplane * esz);
    l.f1 = in_place ? 0 : take(9 * fplane * esz);
    l.ucomp = take(plane * urec_bytes(storage));
    l.cls = take(plane);
    l.bnodes = take(std::max<size_t>(1, t.bnodes.size()) * sizeof(BNode));
    l.blinks = take(std::max<size_t>(1, t.blinks.size()) * sizeof(BLink));
    l.bcs = take(t.bcs.size() * sizeof(BCDev));
    l.rho = grad ? take(plane * sizeof(float)) : 0;
    l.status = take(sizeof(uint32_t));
    l.time = take(sizeof(int64_t));
    l.scale = take(sizeof(ScaleState));
    // field staging; in place it also holds the boundary nodes' populations
    // between their update and their store (9 per boundary node)
    l.stage = take(std::max(7 * N, in_place ? 9 * t.bnodes.size() : 0) * sizeof(float));
    l.probe = take(7 * (size_t)kMaxProbe * sizeof(float));
    l.probe_idx = take((size_t)kMaxProbe * sizeof(int32_t));
    l.nw = block > 1 ? take(plane * sizeof(uint64_t)) : 0;
    l.wave_tab =
        block > 1 ? take(wave_table_entries(t.nx, t.ny) * (sizeof(int4) + sizeof(long long))) : 0;
    l.total = o;
    return l;
}

Lattice make_lattice(const Tables &t, const Units &u, int storage) {
    Lattice L;
    std::memset(&L, 0, sizeof L);
    L.nx = t.nx;
    L.ny = t.ny;
    L.pitch = t.pitch;
    L.nb = (int32_t)t.bnodes.size();
    L.nbcs = (int32_t)t.bcs.size();
    L.plane = (int64_t)t.pitch * t.ny;
    L.fplane = L.plane;
    L.omega = (float)(1.0 / u.tau);
    L.src = (float)(1.0 - 1.0 / (2.0 * u.tau));
    L.fx = (float)u.fx;
    L.fy = (float)u.fy;
    L.mu_m_lam = (float)(u.mu - u.lam);
    L.lam_m_mu_r0 = (float)((u.lam - u.mu) / u.rho0);
    L.rho0 = (float)u.rho0;
    L.inv_rho0 = (float)(1.0 / u.rho0);
    // 16-bit storage: a power-of-two scale that maps the largest boundary value
    // to about 8, leaving a factor 8000 below the FP16 maximum for stress
    // concentrations (crack tips) and the normal range down to 1e-5 of the load
    float scale = 1.0f;
    if (storage != LBM_F32) {
        const double a = t.max_load > 0.0f ? (double)t.max_load : 1e-3;
        const int e = (int)std::floor(std::log2(8.0 / a));
        scale = std::ldexp(1.0f, std::max(-30, std::min(60, e)));
    }
    L.scale = scale;
    L.inv_scale = 1.0f / scale;
    L.out_u = (float)u.dx;
    L.out_v = (float)u.U;
    L.out_s = (float)(u.U * u.U);
    L.grad = (u.lam != u.mu) ? 1 : 0;
    L.wait_ns = kDefaultWaitNs;
    return L;
}

}  // namespace

lbm_status lbm::prepare(const lbm_desc *desc, Tables *t, Units *u) {
    if (!desc) {
        set_error("NULL descriptor");
        return LBM_ERR_ARG;
    }
    lbm_status st = make_units(*desc, u);
    if (st != LBM_OK) return st;
    st = classify(*desc, *u, t);
    if (st == LBM_OK) partition_boundary(*t);
    return st;
}

namespace {

void destroy_graphs(lbm_solver *h) {
    for (auto &g : h->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

// Capture kGraphChunk steps starting in buffer `start`: one-step launches
// with the boundary kernel on a side branch beside the interior kernel, or
// kGraphChunk / kWaveK temporally blocked launches (an even number, so the
// chunk ends in the buffer it started from either way).
static_assert(kGraphChunk % (2 * kWaveK) == 0 && kGraphChunk % (2 * kWaveGradK) == 0,
              "graph chunk and time block");

lbm_status build_graph(lbm_solver *h, int start) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(h->cap_main, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "lbm_step: begin capture");
    int cur = start;
    for (int s = 0; s < kGraphChunk && e == cudaSuccess;) {
        if (h->block > 1) {
            e = launch_wave(h->L, h->S, h->wave, cur, s, h->cap_main);
            s += h->block;
        } else {
            e = launch_step(h->storage, h->L, h->S, cur, s, h->cap_main, h->cap_side, h->gfork,
                            h->gjoin, nullptr);
            s += 1;
        }
        cur ^= 1;
    }
    if (e == cudaSuccess) e = launch_advance(h->S, kGraphChunk, h->cap_main);
    cudaError_t e2 = cudaStreamEndCapture(h->cap_main, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(e != cudaSuccess ? e : e2, "lbm_step: capture");
    }
    e = cudaGraphInstantiate(&h->graph[start], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "lbm_step: instantiate");
    return LBM_OK;
}

}  // namespace

extern "C" lbm_status lbm_workspace_size(const lbm_desc *desc, uint64_t *bytes) {
    set_error("");
    if (!bytes) {
        set_error("lbm_workspace_size: NULL output");
        return LBM_ERR_ARG;
    }
    Tables t;
    Units u;
    lbm_status st = prepare(desc, &t, &u);
    if (st != LBM_OK) return st;
    const int block = steps_per_launch(*desc, t, u);
    if (block == 0) {
        set_error("lbm_workspace_size: time_block = LBM_TIME_BLOCK needs FP32 storage, nx >= 128 and two buffers");
        return LBM_ERR_ARG;
    }
    *bytes = layout(t, desc->storage, u.lam != u.mu, block, desc->streaming == LBM_STREAM_IN_PLACE).total;
    return LBM_OK;
}

extern "C" lbm_status lbm_create(const lbm_desc *desc, void *stream, void *workspace,
                                 uint64_t workspace_bytes, lbm_handle *out) {
    return lbm::create_solver(desc, stream, workspace, workspace_bytes, 0, out);
}

namespace lbm {

// Pinned host staging of the probes and the status word, allocated on first
// use for handles created without them.
cudaError_t host_buffers(lbm_solver *h) {
    cudaError_t e = cudaSuccess;
    if (!h->h_probe_idx) e = cudaMallocHost(&h->h_probe_idx, kMaxProbe * sizeof(int32_t));
    if (e == cudaSuccess && !h->h_probe_out)
        e = cudaMallocHost(&h->h_probe_out, 7 * kMaxProbe * sizeof(float));
    if (e == cudaSuccess && !h->h_status) {
        e = cudaMallocHost(&h->h_status, sizeof(uint32_t));
        if (e == cudaSuccess) *h->h_status = 0;
    }
    return e;
}

uint64_t workspace_bytes_for(const lbm_desc &d, const Tables &t, const Units &u) {
    const int block = steps_per_launch(d, t, u);
    if (block == 0) return 0;
    return layout(t, d.storage, u.lam != u.mu, block, d.streaming == LBM_STREAM_IN_PLACE).total;
}

lbm_status create_solver(const lbm_desc *desc, void *stream, void *workspace,
                         uint64_t workspace_bytes, int plan_blocks, lbm_handle *out) {
    set_error("");
    if (!out) {
        set_error("lbm_create: NULL output handle");
        return LBM_ERR_ARG;
    }
    *out = nullptr;
    Tables t;
    Units u;
    lbm_status st = prepare(desc, &t, &u);
    if (st != LBM_OK) return st;
    CreateOptions opt;
    opt.plan_blocks = plan_blocks;
    return create_prepared(desc, std::move(t), u, stream, workspace, workspace_bytes, opt, out);
}

lbm_status create_prepared(const lbm_desc *desc, Tables &&tab, const Units &units, void *stream,
                           void *workspace, uint64_t workspace_bytes, const CreateOptions &opt,
                           lbm_handle *out) {
    set_error("");
    *out = nullptr;
    const int plan_blocks = opt.plan_blocks;
    lbm_solver *h = new lbm_solver();
    h->tab = std::move(tab);
    h->units = units;
    h->deferred = opt.deferred;
    h->storage = desc->storage;
    h->stream = static_cast<cudaStream_t>(stream);
    h->L = make_lattice(h->tab, h->units, h->storage);
    h->L.wall_node = desc->wall_values == LBM_WALL_NODE ? 1 : 0;
    h->block = steps_per_launch(*desc, h->tab, h->units);
    if (h->block == 0) {
        set_error("lbm_create: time_block = LBM_TIME_BLOCK needs FP32 storage, nx >= 128 and two buffers");
        delete h;
        return LBM_ERR_ARG;
    }
    const bool in_place = desc->streaming == LBM_STREAM_IN_PLACE;
    if (in_place) {
        h->L.in_place = 1;
        h->L.fplane = (int64_t)h->tab.pitch * (h->tab.ny + 2);
    }
    const Layout lay = layout(h->tab, h->storage, h->L.grad != 0, h->block, in_place);
    h->bytes = lay.total;
    cudaError_t e = cudaSuccess;
    if (workspace) {
        if (workspace_bytes < lay.total || (reinterpret_cast<uintptr_t>(workspace) & 255u)) {
            set_error("lbm_create: workspace smaller than lbm_workspace_size() or not 256-byte aligned");
            delete h;
            return LBM_ERR_NOMEM;
        }
        h->base = workspace;
    } else {
        size_t free_b = 0, total_b = 0;
        e = cudaMemGetInfo(&free_b, &total_b);
        if (e != cudaSuccess) {
            delete h;
            return cuda_fail(e, "lbm_create: cudaMemGetInfo");
        }
        if (lay.total > free_b) {
            set_error("lbm_create: needs " + std::to_string(lay.total) + " device bytes, " +
                      std::to_string(free_b) + " free");
            delete h;
            return LBM_ERR_NOMEM;
        }
        e = cudaMalloc(&h->owned, lay.total);
        if (e != cudaSuccess) {
            cudaGetLastError();
            delete h;
            set_error("lbm_create: cudaMalloc failed");
            return LBM_ERR_NOMEM;
        }
        h->base = h->owned;
    }
    char *b = static_cast<char *>(h->base);
    DevState &S = h->S;
    const size_t esz = h->storage == LBM_F32 ? 4 : 2;
    // in place: node (0, 0) sits one row and one column into the padded planes
    S.f[0] = b + lay.f0 + (in_place ? (size_t)(h->tab.pitch + 1) * esz : 0);
    S.f[1] = in_place ? nullptr : b + lay.f1;
    S.ucomp = b + lay.ucomp;
    S.cls = reinterpret_cast<uint8_t *>(b + lay.cls);
    S.bnodes = reinterpret_cast<BNode *>(b + lay.bnodes);
    S.blinks = reinterpret_cast<BLink *>(b + lay.blinks);
    S.bcs = reinterpret_cast<BCDev *>(b + lay.bcs);
    S.rho = h->L.grad ? reinterpret_cast<float *>(b + lay.rho) : nullptr;
    S.status = reinterpret_cast<uint32_t *>(b + lay.status);
    S.time = reinterpret_cast<int64_t *>(b + lay.time);
    // FP16 storage rescales itself (ScaleState); the other forms keep L.scale
    h->L.sc = h->storage == LBM_F16_DEV ? reinterpret_cast<ScaleState *>(b + lay.scale) : nullptr;
    S.stage = reinterpret_cast<float *>(b + lay.stage);
    S.probe = reinterpret_cast<float *>(b + lay.probe);
    S.probe_idx = reinterpret_cast<int32_t *>(b + lay.probe_idx);
    S.nw = h->block > 1 ? reinterpret_cast<uint64_t *>(b + lay.nw) : nullptr;
    S.wave_tab = h->block > 1 ? reinterpret_cast<int4 *>(b + lay.wave_tab) : nullptr;
    S.wave_cyc = h->block > 1 ? reinterpret_cast<long long *>(
                                    b + lay.wave_tab + wave_table_entries(h->tab.nx, h->tab.ny) * sizeof(int4))
                              : nullptr;

    auto fail = [&](cudaError_t err, const char *where) {
        lbm_status s = cuda_fail(err, where);
        lbm_destroy(h);
        return s;
    };
    const Tables &t = h->tab;
    e = cudaMemcpyAsync(S.cls, t.cls.data(), t.cls.size(), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && !t.bnodes.empty())
        e = cudaMemcpyAsync(S.bnodes, t.bnodes.data(), t.bnodes.size() * sizeof(BNode),
                            cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && !t.blinks.empty())
        e = cudaMemcpyAsync(S.blinks, t.blinks.data(), t.blinks.size() * sizeof(BLink),
                            cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(S.bcs, t.bcs.data(), t.bcs.size() * sizeof(BCDev),
                            cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = launch_reset(h->storage, h->L, S, h->stream);
    if (e == cudaSuccess && h->block > 1) {
        if (!wave_supported(h->L)) {
            if (desc->time_block == LBM_TIME_BLOCK) {
                set_error("lbm_create: the temporally blocked kernel is unavailable (tensor-map encoder)");
                lbm_destroy(h);
                return LBM_ERR_ARG;
            }
            h->block = 1;  // default: fall back to one step per launch
        } else {
            e = wave_prepare(h->tab, h->L, S, &h->wave, h->stream, plan_blocks);
            if (e == cudaSuccess && plan_blocks <= 0)
                e = wave_calibrate(h->tab, h->L, S, &h->wave, h->stream);
            if (e == cudaSuccess) e = launch_reset(h->storage, h->L, S, h->stream);
        }
    }
    // the host tables stay in the handle, so the uploads need not be waited
    // for when the creator orders its own work after them (deferred)
    if (e == cudaSuccess && !opt.deferred) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return fail(e, "lbm_create: upload");
    e = cudaStreamCreateWithFlags(&h->cap_main, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cap_side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->gfork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->gjoin, cudaEventDisableTiming);
    if (e == cudaSuccess && !opt.deferred) e = host_buffers(h);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->status_ready, cudaEventDisableTiming);
    if (e != cudaSuccess) return fail(e, "lbm_create: streams/events");
    *out = h;
    return LBM_OK;
}

}  // namespace lbm

extern "C" lbm_status lbm_step(lbm_handle h, int64_t nsteps) {
    set_error("");
    if (!h || nsteps < 0) {
        set_error("lbm_step: bad handle or negative step count");
        return LBM_ERR_ARG;
    }
    // status of work queued by an earlier call, if the device has finished it
    if (h->status_pending) {
        const cudaError_t q = cudaEventQuery(h->status_ready);
        if (q == cudaSuccess) {
            h->status_pending = false;
            if (*h->h_status & 2u) {
                set_error("lbm_step: a bounded wait for a tile copy expired on the device");
                return LBM_ERR_TIMEOUT;
            }
            if (*h->h_status & 1u) {
                set_error("lbm_step: a non-finite moment was produced (unstable run)");
                return LBM_ERR_UNSTABLE;
            }
        } else if (q == cudaErrorNotReady) {
            cudaGetLastError();  // clear the not-ready code so later launch checks see only real errors
        } else {
            return cuda_fail(q, "lbm_step: status query");
        }
    }
    cudaError_t e = host_buffers(h);
    if (e != cudaSuccess) return cuda_fail(e, "lbm_step: host buffers");
    int64_t done = 0;
    const int per_step = kernels_per_step(h->L);
    if (h->timing) {
        // kernels one by one, interior and boundary bracketed by events
        for (int64_t s = 0; s < nsteps; ++s) {
            if (h->ev_used == h->ev_pool.size()) {
                StepEvents ev{};
                e = cudaEventCreate(&ev.before_interior);
                if (e == cudaSuccess) e = cudaEventCreate(&ev.after_interior);
                if (e == cudaSuccess) e = cudaEventCreate(&ev.before_boundary);
                if (e == cudaSuccess) e = cudaEventCreate(&ev.after_boundary);
                if (e != cudaSuccess) return cuda_fail(e, "lbm_step: timing events");
                h->ev_pool.push_back(ev);
            }
            StepEvents &ev = h->ev_pool[h->ev_used++];
            ev.nsteps = 1;
            if (h->block > 1 && nsteps - s >= h->block) {
                ev.nsteps = h->block;
                // one blocked launch as the bulk kernel; the boundary nodes are inside it
                e = cudaEventRecord(ev.before_interior, h->stream);
                if (e == cudaSuccess) e = launch_wave(h->L, h->S, h->wave, h->cur, (int)s, h->stream);
                if (e == cudaSuccess) e = cudaEventRecord(ev.after_interior, h->stream);
                if (e == cudaSuccess) e = cudaEventRecord(ev.before_boundary, h->stream);
                if (e == cudaSuccess) e = cudaEventRecord(ev.after_boundary, h->stream);
                s += h->block - 1;
                h->launches += 1;
            } else {
                e = launch_step(h->storage, h->L, h->S, h->cur, (int)s, h->stream, h->cap_side,
                                h->fork, h->join, &ev);
                h->launches += per_step;
            }
            if (e != cudaSuccess) return cuda_fail(e, "lbm_step: launch");
            h->cur ^= 1;
        }
        done = nsteps;
    }
    if (nsteps - done >= kGraphChunk) {
        // the graph runs on the caller's stream
        for (; done + kGraphChunk <= nsteps; done += kGraphChunk) {
            if (!h->graph[h->cur]) {
                lbm_status st = build_graph(h, h->cur);
                if (st != LBM_OK) return st;
            }
            e = cudaGraphLaunch(h->graph[h->cur], h->stream);
            if (e != cudaSuccess) return cuda_fail(e, "lbm_step: graph launch");
            h->launches += (h->block > 1 ? kGraphChunk / h->block : kGraphChunk * per_step) + 1;
        }
    }
    const int64_t rest = nsteps - done;
    for (int64_t s = 0; s < rest;) {
        if (h->block > 1 && rest - s >= h->block) {
            e = launch_wave(h->L, h->S, h->wave, h->cur, (int)s, h->stream);
            s += h->block;
            h->launches += 1;
        } else {
            e = launch_step(h->storage, h->L, h->S, h->cur, (int)s, h->stream, nullptr, nullptr,
                            nullptr, nullptr);
            s += 1;
            h->launches += per_step;
        }
        if (e != cudaSuccess) return cuda_fail(e, "lbm_step: launch");
        h->cur ^= 1;
    }
    const int64_t direct = rest + (h->timing ? nsteps : 0);
    if (direct > 0) {
        e = launch_advance(h->S, direct, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "lbm_step: advance");
        h->launches += 1;
    }
    h->time += nsteps;
    if (nsteps > 0 && !h->status_pending) {
        e = cudaMemcpyAsync(h->h_status, h->S.status, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                            h->stream);
        if (e == cudaSuccess) e = cudaEventRecord(h->status_ready, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "lbm_step: status copy");
        h->status_pending = true;
    }
    return LBM_OK;
}

extern "C" lbm_status lbm_get_fields(lbm_handle h, float *u, float *v, float *sigma,
                                     int32_t on_device) {
    set_error("");
    if (!h) {
        set_error("lbm_get_fields: NULL handle");
        return LBM_ERR_ARG;
    }
    cudaError_t e = launch_fields(h->storage, h->L, h->S, h->cur, u, v, sigma, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "lbm_get_fields");
    h->launches += kernels_per_fields(h->L);
    if (!on_device) {
        e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "lbm_get_fields: sync");
    }
    return LBM_OK;
}

extern "C" lbm_status lbm_probe(lbm_handle h, const int32_t *nodes, int32_t count, float *out) {
    set_error("");
    if (!h || count < 0 || count > kMaxProbe || (count > 0 && (!nodes || !out))) {
        set_error("lbm_probe: bad arguments (at most 4096 nodes)");
        return LBM_ERR_ARG;
    }
    if (count == 0) return LBM_OK;
    const int64_t N = (int64_t)h->L.nx * h->L.ny;
    for (int32_t p = 0; p < count; ++p) {
        if (nodes[p] < 0 || nodes[p] >= N) {
            set_error("lbm_probe: node index out of range");
            return LBM_ERR_ARG;
        }
        h->h_probe_idx[p] = nodes[p];
    }
    cudaError_t e = cudaMemcpyAsync(h->S.probe_idx, h->h_probe_idx, count * sizeof(int32_t),
                                    cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = launch_fields(h->storage, h->L, h->S, h->cur, nullptr, nullptr, nullptr, h->stream);
    if (e == cudaSuccess) e = launch_gather_probe(h->L, h->S, count, h->stream);
    h->launches += kernels_per_fields(h->L) + 1;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->h_probe_out, h->S.probe, 7 * (size_t)count * sizeof(float),
                            cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "lbm_probe");
    std::memcpy(out, h->h_probe_out, 7 * (size_t)count * sizeof(float));
    return LBM_OK;
}

extern "C" lbm_status lbm_set_bc(lbm_handle h, int32_t index, const lbm_bc *bc) {
    set_error("");
    if (!h || !bc || index < 0 || index >= (int32_t)h->tab.bcs.size()) {
        set_error("lbm_set_bc: bad arguments");
        return LBM_ERR_ARG;
    }
    if (bc->kind != h->tab.bcs[index].kind) {
        // the bounce-back / anti-bounce-back choice is baked into the link tables
        set_error("lbm_set_bc: the kind of a boundary condition cannot change");
        return LBM_ERR_ARG;
    }
    if ((bc->profile != LBM_PROFILE_STEP && bc->profile != LBM_PROFILE_RAMP) ||
        !std::isfinite(bc->value[0]) || !std::isfinite(bc->value[1]) ||
        !std::isfinite(bc->value[2]) || (bc->profile == LBM_PROFILE_RAMP && !(bc->t_ramp > 0.0))) {
        set_error("lbm_set_bc: bad boundary condition");
        return LBM_ERR_ARG;
    }
    h->tab.bcs[index] = to_lattice(*bc, h->units);
    // bounded by the table size; stream-ordered with the steps
    cudaError_t e = cudaMemcpyAsync(h->S.bcs + index, &h->tab.bcs[index], sizeof(BCDev),
                                    cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "lbm_set_bc");
    return LBM_OK;
}

extern "C" lbm_status lbm_reset(lbm_handle h) {
    set_error("");
    if (!h) {
        set_error("lbm_reset: NULL handle");
        return LBM_ERR_ARG;
    }
    cudaError_t e = host_buffers(h);
    if (e == cudaSuccess) e = launch_reset(h->storage, h->L, h->S, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "lbm_reset");
    h->cur = 0;
    h->time = 0;
    h->launches += 0;  // the reset is memsets, not kernels
    if (h->status_pending) cudaEventSynchronize(h->status_ready);
    h->status_pending = false;
    *h->h_status = 0;
    return LBM_OK;
}

extern "C" lbm_status lbm_sync(lbm_handle h) {
    set_error("");
    if (!h) {
        set_error("lbm_sync: NULL handle");
        return LBM_ERR_ARG;
    }
    uint32_t status = 0;
    cudaError_t e = cudaMemcpyAsync(&status, h->S.status, sizeof status, cudaMemcpyDeviceToHost,
                                    h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "lbm_sync");
    if (status & 2u) {
        set_error("lbm_sync: a bounded wait for a tile copy expired on the device");
        return LBM_ERR_TIMEOUT;
    }
    if (status & 1u) {
        set_error("lbm_sync: a non-finite moment was produced (unstable run)");
        return LBM_ERR_UNSTABLE;
    }
    return LBM_OK;
}

extern "C" lbm_status lbm_get_info(lbm_handle h, lbm_info *info) {
    set_error("");
    if (!h || !info) {
        set_error("lbm_get_info: bad arguments");
        return LBM_ERR_ARG;
    }
    info->nx = h->L.nx;
    info->ny = h->L.ny;
    info->pitch = h->L.pitch;
    info->storage = h->storage;
    info->time = h->time;
    info->boundary_nodes = h->L.nb;
    info->interior_nodes = h->tab.interior;
    info->workspace_bytes = h->bytes;
    info->storage_scale = h->L.scale;
    if (h->L.sc) {
        // FP16: the scale the last step stored with (waits for the stream)
        ScaleState sc;
        cudaError_t e = cudaMemcpyAsync(&sc, h->L.sc, sizeof sc, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "lbm_get_info: scale");
        info->storage_scale = sc.s[(h->time + 2) % 3];
    }
    const float esz = h->storage == LBM_F32 ? 4.0f : 2.0f;
    // f read and written, the displacement record read and written
    info->bytes_per_update = 2.0f * 9.0f * esz + 2.0f * (float)urec_bytes(h->storage);
    info->kernel_launches = h->launches;
    info->time_block = h->block;
    info->streaming = h->L.in_place ? LBM_STREAM_IN_PLACE : LBM_STREAM_TWO_BUFFERS;
    return LBM_OK;
}

extern "C" lbm_status lbm_set_wait_limit(lbm_handle h, int64_t limit_ns) {
    set_error("");
    if (!h) {
        set_error("lbm_set_wait_limit: NULL handle");
        return LBM_ERR_ARG;
    }
    if (limit_ns < 0 || limit_ns > 60 * kDefaultWaitNs) {
        set_error("lbm_set_wait_limit: the limit must lie in 0 .. 60e9 ns");
        return LBM_ERR_ARG;
    }
    // captured graphs hold the lattice parameters by value: capture again
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "lbm_set_wait_limit: sync");
    destroy_graphs(h);
    h->L.wait_ns = limit_ns;
    return LBM_OK;
}

extern "C" lbm_status lbm_set_timing(lbm_handle h, int32_t enable) {
    set_error("");
    if (!h) {
        set_error("lbm_set_timing: NULL handle");
        return LBM_ERR_ARG;
    }
    h->timing = enable != 0;
    return LBM_OK;
}

extern "C" lbm_status lbm_get_timing(lbm_handle h, lbm_timing *out) {
    set_error("");
    if (!h || !out) {
        set_error("lbm_get_timing: bad arguments");
        return LBM_ERR_ARG;
    }
    std::memset(out, 0, sizeof *out);
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "lbm_get_timing: sync");
    for (size_t k = 0; k < h->ev_used; ++k) {
        float a = 0.0f, b = 0.0f;
        e = cudaEventElapsedTime(&a, h->ev_pool[k].before_interior, h->ev_pool[k].after_interior);
        if (e == cudaSuccess)
            e = cudaEventElapsedTime(&b, h->ev_pool[k].before_boundary, h->ev_pool[k].after_boundary);
        if (e != cudaSuccess) return cuda_fail(e, "lbm_get_timing: elapsed");
        out->interior_ms += a;
        out->boundary_ms += b;
        out->steps += h->ev_pool[k].nsteps;
    }
    h->ev_used = 0;
    return LBM_OK;
}

namespace lbm {

void destroy_deferred(lbm_handle h) {
    if (!h) return;
    destroy_graphs(h);
    if (h->cap_main) cudaStreamDestroy(h->cap_main);
    if (h->cap_side) cudaStreamDestroy(h->cap_side);
    if (h->fork) cudaEventDestroy(h->fork);
    if (h->join) cudaEventDestroy(h->join);
    if (h->gfork) cudaEventDestroy(h->gfork);
    if (h->gjoin) cudaEventDestroy(h->gjoin);
    if (h->status_ready) cudaEventDestroy(h->status_ready);
    delete h;
}

}  // namespace lbm

extern "C" lbm_status lbm_destroy(lbm_handle h) {
    if (!h) return LBM_OK;
    if (h->stream || h->owned) cudaStreamSynchronize(h->stream);
    destroy_graphs(h);
    if (h->cap_main) cudaStreamDestroy(h->cap_main);
    if (h->cap_side) cudaStreamDestroy(h->cap_side);
    if (h->fork) cudaEventDestroy(h->fork);
    if (h->join) cudaEventDestroy(h->join);
    if (h->gfork) cudaEventDestroy(h->gfork);
    if (h->gjoin) cudaEventDestroy(h->gjoin);
    if (h->h_probe_idx) cudaFreeHost(h->h_probe_idx);
    if (h->h_probe_out) cudaFreeHost(h->h_probe_out);
    if (h->h_status) cudaFreeHost(h->h_status);
    if (h->status_ready) cudaEventDestroy(h->status_ready);
    for (auto &ev : h->ev_pool) {
        cudaEventDestroy(ev.before_interior);
        cudaEventDestroy(ev.after_interior);
        cudaEventDestroy(ev.before_boundary);
        cudaEventDestroy(ev.after_boundary);
    }
    if (h->owned) cudaFree(h->owned);
    delete h;
    return LBM_OK;
}

// ---------------------------------------------------------------------------
// Fields to host memory without any device allocation.
//
// lbm_get_fields stages the seven field planes in the handle's workspace.
// This variant stages them in a fixed device array that lives in the module
// instead, so a caller whose handle sits in a workspace it sized itself (or
// that must not allocate at this point) can still read the fields back.  The
// array is shared by every call on a device and keeps the last call's
// contents; each call overwrites every entry it later copies, so nothing has
// to be cleared first.  Calls whose device work overlaps (on different
// streams, or from different threads) race on the array.

namespace {

constexpr int64_t kNoAllocMaxNodes = int64_t(1) << 18;  // nx * ny limit: 262144 nodes
constexpr int kNoAllocMaxDevices = 64;

// 7 planes x 2^18 nodes x 4 bytes = 7 MiB held on every device that loads the library.
static __device__ __align__(256) float g_noalloc_fields[7 * kNoAllocMaxNodes];

std::mutex g_noalloc_mutex;
float *g_noalloc_ptr[kNoAllocMaxDevices] = {nullptr};

// Device address of the array on the current device, looked up once per device.
lbm_status noalloc_scratch(float **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "lbm_get_fields_host_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        set_error("lbm_get_fields_host_noalloc: device ordinal beyond 63");
        return LBM_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_fields);
        if (e != cudaSuccess)
            return cuda_fail(e, "lbm_get_fields_host_noalloc: cudaGetSymbolAddress");
        g_noalloc_ptr[dev] = static_cast<float *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return LBM_OK;
}

}  // namespace

extern "C" lbm_status lbm_get_fields_host_noalloc(lbm_handle h, float *u, float *v,
                                                  float *sigma) {
    set_error("");
    if (!h) {
        set_error("lbm_get_fields_host_noalloc: NULL handle");
        return LBM_ERR_ARG;
    }
    const int64_t N = (int64_t)h->L.nx * h->L.ny;
    if (N > kNoAllocMaxNodes) {
        set_error("lbm_get_fields_host_noalloc: nx*ny = " + std::to_string(N) +
                  " exceeds the 262144 nodes of the static staging array");
        return LBM_ERR_ARG;
    }
    float *scratch = nullptr;
    lbm_status st = noalloc_scratch(&scratch);
    if (st != LBM_OK) return st;
    DevState S = h->S;
    S.stage = scratch;  // same kernels, staging redirected to the static array
    cudaError_t e = launch_fields(h->storage, h->L, S, h->cur, nullptr, nullptr, nullptr,
                                  h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "lbm_get_fields_host_noalloc");
    h->launches += kernels_per_fields(h->L);
    if (u) e = cudaMemcpyAsync(u, scratch, 2 * N * sizeof(float), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && v)
        e = cudaMemcpyAsync(v, scratch + 2 * N, 2 * N * sizeof(float), cudaMemcpyDeviceToHost,
                            h->stream);
    if (e == cudaSuccess && sigma)
        e = cudaMemcpyAsync(sigma, scratch + 4 * N, 3 * N * sizeof(float),
                            cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "lbm_get_fields_host_noalloc: copy");
    return LBM_OK;
}
