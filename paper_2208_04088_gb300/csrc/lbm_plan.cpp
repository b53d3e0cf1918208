// lbm_plan.cpp -- host side of the temporally blocked stepping: the blocks of
// one launch (strip segments), cut first from a cost model and then balanced
// by measuring the blocks' SM cycles (wave_calibrate), and the per-process
// cache of measured plans.  The kernels are in lbm_wave.cu.
#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>

#include "lbm_internal.h"

namespace lbm {

namespace {
constexpr int kPK = kWaveK, kPW = kWaveW;  // halo rows and core columns of a strip
}  // namespace

size_t wave_table_entries(int nx, int ny) {
    // the plan makes at most max(number of SMs, strips) blocks; 4096 bounds the
    // SMs of any device
    (void)ny;
    const size_t strips = (size_t)(nx + kPW - 1) / kPW;
    return std::max<size_t>(strips, 4096) + strips;
}

// The blocks of one launch.  Every strip of kWaveW columns is cut into row
// segments; a segment sweeps 3 kWaveK - 3 rows more than it owns.  The cost of
// a block is modelled in row sweeps, from per-block cycle counts measured on
// GB300 (edge and centre cracks, plates with holes of radius 64 to 512):
//   - each row of the sweep costs 1, and the block kBlockCost more;
//   - a row's 64-column half of the region (one warp per level) that holds a
//     boundary node takes the boundary update: kHalfRowCost, counted also in
//     the segment's halo rows;
//   - curved-wall, corner and crack-mouth nodes (the 8-lane update, four nodes
//     per pass in each half) add kPassCost per pass.
// Segments are cut greedily against a target cost, and the smallest target for
// which all blocks fit one wave on `sms` SMs (one block per SM) is found by
// bisection.  Each entry also says whether a boundary node lies in the
// block's region or halo.
constexpr double kBlockCost = 6.0;
constexpr double kHalfRowCost = 1.0;
constexpr double kPassCost = 5.5;

// A boundary node the blocked kernel updates eight lanes to a node (curved
// walls, corners, crack mouth): not every cut link is a mid-link wall of one
// BC and one axis-aligned normal (the node words' "simple" flag).
bool complex_boundary_node(const Tables &t, size_t g) {
    const BNode &b = t.bnodes[g];
    if (b.corner) return true;
    int bc = -1;
    float n0 = 0.0f, n1 = 0.0f;
    for (int i = 1; i < kQ; ++i) {
        if (!((b.cut >> i) & 1u)) continue;
        const BLink &lk = t.blinks[g * 8 + i - 1];
        const bool axis = (lk.n0 == 0.0f && (lk.n1 == 1.0f || lk.n1 == -1.0f)) ||
                          (lk.n1 == 0.0f && (lk.n0 == 1.0f || lk.n0 == -1.0f));
        if (lk.q != 0.5f || lk.bc != lk.bc2 || !axis) return true;
        if (bc < 0) {
            bc = lk.bc;
            n0 = lk.n0;
            n1 = lk.n1;
        } else if (lk.bc != bc || lk.n0 != n0 || lk.n1 != n1) {
            return true;
        }
    }
    return bc < 0;
}

void partition_boundary(Tables &t) {
    const size_t nb = t.bnodes.size();
    std::vector<BNode> bn;
    std::vector<BLink> bl;
    bn.reserve(nb);
    bl.reserve(nb * 8);
    for (int pass = 0; pass < 2; ++pass)
        for (size_t g = 0; g < nb; ++g)
            if (complex_boundary_node(t, g) == (pass == 0)) {
                bn.push_back(t.bnodes[g]);
                bl.insert(bl.end(), t.blinks.begin() + g * 8, t.blinks.begin() + g * 8 + 8);
            }
    t.nbx = 0;
    for (size_t g = 0; g < nb; ++g) t.nbx += complex_boundary_node(t, g) ? 1 : 0;
    t.bnodes.swap(bn);
    t.blinks.swap(bl);
}

namespace {

// Modelled extra cost (row sweeps) of each row of every strip: the boundary
// update of each 64-column half holding a boundary node, and the passes of
// the 8-lane update.  Rows sorted, with prefix sums.
struct StripRows {
    std::vector<std::vector<int>> row;
    std::vector<std::vector<double>> pre;
};

StripRows strip_rows(const Tables &t, int nstrips) {
    // boundary nodes seen by each strip's region (core and halo columns), as
    // keys row * 4 + half * 2 + curved
    std::vector<std::vector<int64_t>> keys(nstrips);
    for (size_t g = 0; g < t.bnodes.size(); ++g) {
        const BNode &b = t.bnodes[g];
        const int64_t cx = complex_boundary_node(t, g) ? 1 : 0;
        const int s_lo = std::max(0, (b.x - kPK) / kPW), s_hi = std::min(nstrips - 1, (b.x + kPK) / kPW);
        for (int sx = s_lo; sx <= s_hi; ++sx) {
            const int X0 = sx * kPW;
            if (b.x >= X0 - kPK && b.x < X0 + kPW + kPK)
                keys[sx].push_back((int64_t)b.y * 4 + ((b.x - X0 + kPK) >> 6) * 2 + cx);
        }
    }
    StripRows r;
    r.row.resize(nstrips);
    r.pre.resize(nstrips);
    for (int sx = 0; sx < nstrips; ++sx) {
        auto &k = keys[sx];
        std::sort(k.begin(), k.end());
        r.pre[sx].push_back(0.0);
        for (size_t a = 0; a < k.size();) {
            const int64_t y = k[a] >> 2;
            double extra = 0.0;
            while (a < k.size() && (k[a] >> 2) == y) {  // one half of row y
                const int64_t hk = k[a] >> 1;
                int curved = 0;
                for (; a < k.size() && (k[a] >> 1) == hk; ++a) curved += (int)(k[a] & 1);
                extra += kHalfRowCost + kPassCost * (double)((curved + 3) / 4);
            }
            r.row[sx].push_back((int)y);
            r.pre[sx].push_back(r.pre[sx].back() + extra);
        }
    }
    return r;
}

// Cuts every strip into segments greedily against a target cost (cost(sx, a,
// b) of the segment owning rows [a, b)); the smallest target for which the
// blocks fit `budget` is found by bisection.
template <class Cost>
std::vector<int4> cut_strips(const StripRows &br, int nstrips, int ny, int budget, Cost cost) {
    auto cut = [&](int sx, double T, std::vector<int> *ends) {
        int count = 0;
        for (int a = 0; a < ny;) {
            int lo = a + 1, hi = ny;  // the largest b in [a + 1, ny] with cost(a, b) <= T
            if (cost(sx, a, lo) <= T) {
                while (lo < hi) {
                    const int mid = lo + (hi - lo + 1) / 2;
                    if (cost(sx, a, mid) <= T) lo = mid;
                    else hi = mid - 1;
                }
            }
            if (ends) ends->push_back(lo);
            a = lo;
            ++count;
        }
        return count;
    };
    auto blocks_for = [&](double T) {
        int n = 0;
        for (int sx = 0; sx < nstrips; ++sx) n += cut(sx, T, nullptr);
        return n;
    };
    double hi_T = 0.0, lo_T = 0.0;
    for (int sx = 0; sx < nstrips; ++sx) hi_T = std::max(hi_T, cost(sx, 0, ny));
    for (int it = 0; it < 48; ++it) {
        const double mid = 0.5 * (lo_T + hi_T);
        if (blocks_for(mid) <= budget) hi_T = mid;
        else lo_T = mid;
    }
    std::vector<int4> out;
    for (int sx = 0; sx < nstrips; ++sx) {
        std::vector<int> ends;
        cut(sx, hi_T, &ends);
        int Y0 = 0;
        for (int e : ends) {
            const int Hs = e - Y0;
            const auto &r = br.row[sx];
            const auto it = std::lower_bound(r.begin(), r.end(), Y0 - kPK);
            const int has = (it != r.end() && *it < Y0 + Hs + kPK) ? 1 : 0;
            out.push_back(make_int4(sx * kPW, Y0, Hs, has));
            Y0 = e;
        }
    }
    // heavy blocks first
    std::stable_sort(out.begin(), out.end(), [](const int4 &a, const int4 &b) { return a.w > b.w; });
    return out;
}

}  // namespace

int device_sms() {
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaGetLastError();
    return sms;
}

std::vector<int4> wave_plan(const Tables &t, int sms) {
    const int nx = t.nx, ny = t.ny;
    const int nstrips = (nx + kPW - 1) / kPW;
    const StripRows br = strip_rows(t, nstrips);
    auto cost = [&](int sx, int a, int b) {
        const auto &r = br.row[sx];
        const size_t lo = std::lower_bound(r.begin(), r.end(), a - kPK) - r.begin();
        const size_t hi = std::lower_bound(r.begin(), r.end(), b + kPK) - r.begin();
        return (double)(b - a + 3 * kPK - 3) + kBlockCost + (br.pre[sx][hi] - br.pre[sx][lo]);
    };
    return cut_strips(br, nstrips, ny, std::max(sms, nstrips), cost);
}

std::vector<double> wave_plan_costs(const Tables &t, const std::vector<int4> &plan) {
    const int nstrips = (t.nx + kPW - 1) / kPW;
    const StripRows br = strip_rows(t, nstrips);
    std::vector<double> out;
    out.reserve(plan.size());
    for (const int4 &b : plan) {
        const int sx = b.x / kPW, a = b.y, e = b.y + b.z;
        const auto &r = br.row[sx];
        const size_t lo = std::lower_bound(r.begin(), r.end(), a - kPK) - r.begin();
        const size_t hi = std::lower_bound(r.begin(), r.end(), e + kPK) - r.begin();
        out.push_back((double)(e - a + 3 * kPK - 3) + kBlockCost + (br.pre[sx][hi] - br.pre[sx][lo]));
    }
    return out;
}

namespace {

// Measured plans of this process, by lattice: a lattice created again (same
// size, boundary tables, kernel and device) takes its plan without the
// calibration launches.  Any plan gives the same results; only the balance
// depends on it.
struct PlanKey {
    int nx, ny, grad, wall_node, sms;
    uint64_t tables;
    bool operator<(const PlanKey &o) const {
        return std::tie(nx, ny, grad, wall_node, sms, tables) <
               std::tie(o.nx, o.ny, o.grad, o.wall_node, o.sms, o.tables);
    }
};
std::mutex g_plan_mu;
std::map<PlanKey, std::vector<int4>> g_plans;

// FNV-1a over the boundary tables (nodes, links, BC kinds and profiles).
uint64_t tables_hash(const Tables &t) {
    uint64_t h = 1469598103934665603ull;
    auto add = [&h](const void *p, size_t n) {
        const unsigned char *b = static_cast<const unsigned char *>(p);
        for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
    };
    add(t.bnodes.data(), t.bnodes.size() * sizeof(BNode));
    add(t.blinks.data(), t.blinks.size() * sizeof(BLink));
    for (const BCDev &b : t.bcs) {
        add(&b.kind, sizeof b.kind);
        add(&b.profile, sizeof b.profile);
    }
    return h;
}

}  // namespace

cudaError_t wave_calibrate(const Tables &t, const Lattice &L, const DevState &S, WaveMaps *m,
                           cudaStream_t s) {
    const int nx = t.nx, ny = t.ny;
    const int nstrips = (nx + kPW - 1) / kPW;
    const int sms = device_sms();
    const int budget = std::max(sms, nstrips);
    const PlanKey key{nx, ny, L.grad, L.wall_node, sms, tables_hash(t)};
    {
        std::lock_guard<std::mutex> lock(g_plan_mu);
        const auto it = g_plans.find(key);
        if (it != g_plans.end()) {
            m->nblocks = (int)it->second.size();
            // pageable source: the copy is staged before the call returns
            return cudaMemcpyAsync(S.wave_tab, it->second.data(), it->second.size() * sizeof(int4),
                                   cudaMemcpyHostToDevice, s);
        }
    }
    const StripRows br = strip_rows(t, nstrips);
    // per strip and row: the modelled extra cost, and the measured/modelled
    // ratio of the block that owned the row (1 before any measurement)
    std::vector<std::vector<double>> extra(nstrips, std::vector<double>(ny, 0.0));
    for (int sx = 0; sx < nstrips; ++sx)
        for (size_t i = 0; i < br.row[sx].size(); ++i) {
            const int y = br.row[sx][i];
            if (y >= 0 && y < ny) extra[sx][y] = br.pre[sx][i + 1] - br.pre[sx][i];
        }
    std::vector<std::vector<double>> ratio(nstrips, std::vector<double>(ny, 1.0));
    std::vector<std::vector<double>> p1(nstrips), pe(nstrips);
    auto prefix = [&]() {
        for (int sx = 0; sx < nstrips; ++sx) {
            p1[sx].assign(ny + 1, 0.0);
            pe[sx].assign(ny + 1, 0.0);
            for (int y = 0; y < ny; ++y) {
                p1[sx][y + 1] = p1[sx][y] + ratio[sx][y];
                pe[sx][y + 1] = pe[sx][y] + extra[sx][y] * ratio[sx][y];
            }
        }
    };
    // the modelled cost of a segment with every row scaled by its ratio (the
    // fixed sweep of 3 kWaveK - 3 rows and kBlockCost by the segment's mean)
    auto cost = [&](int sx, int a, int b) {
        const double rows = p1[sx][b] - p1[sx][a];
        const double halo = pe[sx][std::min(ny, b + kPK)] - pe[sx][std::max(0, a - kPK)];
        return rows + halo + (3 * kPK - 3 + kBlockCost) * rows / (double)(b - a);
    };
    std::vector<long long> cyc;
    auto measure = [&](const std::vector<int4> &plan) -> cudaError_t {
        if (plan.empty() || plan.size() > wave_table_entries(nx, ny)) return cudaErrorInvalidValue;
        m->nblocks = (int)plan.size();
        cudaError_t e = cudaMemcpyAsync(S.wave_tab, plan.data(), plan.size() * sizeof(int4),
                                        cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = launch_wave(L, S, *m, 0, 0, s, S.wave_cyc);
        cyc.assign(plan.size(), 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(cyc.data(), S.wave_cyc, plan.size() * sizeof(long long),
                                cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        return e;
    };
    prefix();
    std::vector<int4> plan = cut_strips(br, nstrips, ny, budget, cost);
    std::vector<int4> best;
    long long best_max = 0;
    for (int round = 0; round < 3; ++round) {
        cudaError_t e = measure(plan);
        if (e != cudaSuccess) return e;
        const long long mx = *std::max_element(cyc.begin(), cyc.end());
        if (best.empty() || mx < best_max) {
            best = plan;
            best_max = mx;
        }
        if (round == 2) break;
        // scale the rows of every block by its measured/modelled ratio
        for (size_t b = 0; b < plan.size(); ++b) {
            const int sx = plan[b].x / kPW, a = plan[b].y, e2 = plan[b].y + plan[b].z;
            const double modelled = cost(sx, a, e2);
            if (!(modelled > 0.0) || cyc[b] <= 0) continue;
            const double f = (double)cyc[b] / modelled;
            for (int y = a; y < e2; ++y) ratio[sx][y] *= f;
        }
        prefix();
        plan = cut_strips(br, nstrips, ny, budget, cost);
    }
    m->nblocks = (int)best.size();
    {
        std::lock_guard<std::mutex> lock(g_plan_mu);
        if (g_plans.size() >= 64) g_plans.clear();
        g_plans[key] = best;
    }
    // pageable source: the copy is staged before the call returns
    return cudaMemcpyAsync(S.wave_tab, best.data(), best.size() * sizeof(int4),
                           cudaMemcpyHostToDevice, s);
}

}  // namespace lbm
