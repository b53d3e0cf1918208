// lbm_geometry.cpp -- host side of the solid-LBM library: analytic geometry
// builder, unit conversion, and validation/classification of the node mask and
// cut-link table into the compacted boundary list the kernels consume.
//
// Geometry follows Sec. 4 (Fig. bound, Fig. boundnoncon): boundary lattice
// sites are the material nodes with at least one link crossing the wall; each
// cut link carries its wall distance s_i/l_i (Eqs. bbnoncon, abbnoncon).
// Compiled with -ffp-contract=off so the double-precision wall distances are
// reproducible bit for bit on every host.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "lbm_internal.h"

namespace lbm {

namespace {

thread_local std::string g_error;

bool is_finite(double v) { return std::isfinite(v); }

struct Cut {
    int32_t node, dir;
    lbm_link link;
};

}  // namespace

void set_error(const std::string &msg) { g_error = msg; }

}  // namespace lbm

extern "C" const char *lbm_last_error(void) { return lbm::g_error.c_str(); }

namespace lbm {

// ---------------------------------------------------------------------------
// Analytic geometry.  Built feature by feature (box edges, crack faces, hole
// rim), then merged into canonical (node, direction) order.
static lbm_status build_geometry(const lbm_geom &g, uint8_t *node_type, std::vector<Cut> *cuts) {
    const int32_t nx = g.nx, ny = g.ny;
    if (nx < 1 || ny < 1 || nx > 65535 || ny > 65535) {
        set_error("lbm_geom_build: nx and ny must be in 1..65535");
        return LBM_ERR_ARG;
    }
    for (int e = 0; e < 4; ++e)
        if (g.edge_bc[e] < 0) {
            set_error("lbm_geom_build: edge_bc entries must be >= 0 (periodic edges are not supported)");
            return LBM_ERR_ARG;
        }
    const bool hole = g.hole_r > 0.0;
    const bool crack = g.crack_len > 0;
    if (hole && crack) {
        set_error("lbm_geom_build: a geometry has either a hole or a crack");
        return LBM_ERR_ARG;
    }
    if (crack && (ny % 2 != 0 || ny < 2)) {
        set_error("lbm_geom_build: an edge crack needs an even ny");
        return LBM_ERR_ARG;
    }
    if (g.crack_x0 < 0) {
        set_error("lbm_geom_build: crack_x0 must be >= 0");
        return LBM_ERR_ARG;
    }
    if (hole && !(is_finite(g.hole_cx) && is_finite(g.hole_cy) && is_finite(g.hole_r))) {
        set_error("lbm_geom_build: hole parameters must be finite");
        return LBM_ERR_ARG;
    }

    // node mask: void strictly inside the circle (rows in chunks on host threads)
    const double R = g.hole_r;
    {
        auto rows = [&](int32_t ya, int32_t yb) {
            for (int32_t y = ya; y < yb; ++y) {
                uint8_t *row = node_type + (int64_t)y * nx;
                std::memset(row, 1, (size_t)nx);
                if (!hole) continue;
                const double dy = y - g.hole_cy;
                if (dy * dy >= R * R) continue;
                for (int32_t x = 0; x < nx; ++x) {
                    const double dx = x - g.hole_cx;
                    if (dx * dx + dy * dy < R * R) row[x] = 0;
                }
            }
        };
        const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
        const int nparts = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)hw, 16, ny / 64}));
        std::vector<std::thread> workers;
        for (int part = 1; part < nparts; ++part)
            workers.emplace_back(rows, (int32_t)((int64_t)ny * part / nparts),
                                 (int32_t)((int64_t)ny * (part + 1) / nparts));
        rows(0, (int32_t)((int64_t)ny / nparts));
        for (auto &w : workers) w.join();
    }

    // crack plane between rows yb and yb + 1; tip at x = crack_len - 1/2
    const int32_t yb = ny / 2 - 1;
    auto crosses_crack = [&](int32_t x, int32_t y, int i) {
        if (!crack || kCy[i] == 0) return false;
        const int32_t ty = y + kCy[i];
        if (!((y == yb && ty == yb + 1) || (y == yb + 1 && ty == yb))) return false;
        // abscissa of the crossing, doubled: 2x + c_x; the crack spans
        // (2 crack_x0 - 1, 2 (crack_x0 + crack_len) - 1), open at both tips,
        // and reaches the left edge when crack_x0 = 0
        const int32_t xm2 = 2 * x + kCx[i];
        const bool right_of_start = g.crack_x0 == 0 || xm2 > 2 * g.crack_x0 - 1;
        return right_of_start && xm2 < 2 * (g.crack_x0 + g.crack_len) - 1;
    };

    // (1) box edges and crack faces: walls at mid-link
    auto add_midlink = [&](int32_t x, int32_t y, int i) {
        const int32_t tx = x + kCx[i], ty = y + kCy[i];
        const bool ox = tx < 0 || tx >= nx;
        const bool oy = ty < 0 || ty >= ny;
        const bool oc = crosses_crack(x, y, i);
        if (!(ox || oy || oc)) return;
        if (!node_type[(int64_t)y * nx + x]) return;
        lbm_link L;
        std::memset(&L, 0, sizeof L);
        L.node = y * nx + x;
        L.dir = i;
        L.q = 0.5;
        L.bc2 = -1;
        const double sx = (tx < 0) ? -1.0 : 1.0;
        const int32_t bx = (tx < 0) ? g.edge_bc[0] : g.edge_bc[1];
        double sy;
        int32_t by;
        if (oy) {
            sy = (ty < 0) ? -1.0 : 1.0;
            by = (ty < 0) ? g.edge_bc[2] : g.edge_bc[3];
        } else {
            sy = (kCy[i] > 0) ? 1.0 : -1.0;  // crack face: normal points across the crack
            by = g.crack_bc;
        }
        if (ox && (oy || oc)) {
            L.bc = bx;
            L.bc2 = by;
            L.n[0] = sx;
            L.n[1] = sy;
        } else if (ox) {
            L.bc = bx;
            L.n[0] = sx;
            L.n[1] = 0.0;
        } else {
            L.bc = by;
            L.n[0] = 0.0;
            L.n[1] = sy;
        }
        cuts->push_back({L.node, i, L});
    };
    for (int32_t x = 0; x < nx; ++x)
        for (int i = 1; i < kQ; ++i) {
            add_midlink(x, 0, i);
            if (ny > 1) add_midlink(x, ny - 1, i);
        }
    for (int32_t y = 1; y < ny - 1; ++y)
        for (int i = 1; i < kQ; ++i) {
            add_midlink(0, y, i);
            if (nx > 1) add_midlink(nx - 1, y, i);
        }
    if (crack)
        for (int32_t y : {yb, yb + 1})
            if (y > 0 && y < ny - 1)  // rows 0 and ny-1 were visited with the box
                for (int32_t x = std::max(1, g.crack_x0 - 1);
                     x < std::min(nx - 1, g.crack_x0 + g.crack_len + 1); ++x)
                    for (int i = 1; i < kQ; ++i) add_midlink(x, y, i);

    // (2) hole rim: links from a material node to a void node
    if (hole) {
        const int32_t x0 = std::max(0, (int32_t)std::floor(g.hole_cx - R) - 1);
        const int32_t x1 = std::min(nx - 1, (int32_t)std::ceil(g.hole_cx + R) + 1);
        const int32_t y0 = std::max(0, (int32_t)std::floor(g.hole_cy - R) - 1);
        const int32_t y1 = std::min(ny - 1, (int32_t)std::ceil(g.hole_cy + R) + 1);
        for (int32_t y = y0; y <= y1; ++y)
            for (int32_t x = x0; x <= x1; ++x) {
                if (!node_type[(int64_t)y * nx + x]) continue;
                for (int i = 1; i < kQ; ++i) {
                    const int32_t tx = x + kCx[i], ty = y + kCy[i];
                    if (tx < 0 || tx >= nx || ty < 0 || ty >= ny) continue;
                    if (node_type[(int64_t)ty * nx + tx]) continue;
                    const double dx = x - g.hole_cx, dy = y - g.hole_cy;
                    const double b = kCx[i] * dx + kCy[i] * dy;
                    const double c0 = dx * dx + dy * dy - R * R;
                    const double a = (double)(kCx[i] * kCx[i] + kCy[i] * kCy[i]);
                    const double disc = b * b - a * c0;
                    const double q = (-b - std::sqrt(disc)) / a;
                    lbm_link L;
                    std::memset(&L, 0, sizeof L);
                    L.node = y * nx + x;
                    L.dir = i;
                    L.bc = g.hole_bc;
                    L.bc2 = -1;
                    L.q = q;
                    const double wx = x + q * kCx[i], wy = y + q * kCy[i];
                    L.n[0] = (g.hole_cx - wx) / R;
                    L.n[1] = (g.hole_cy - wy) / R;
                    cuts->push_back({L.node, i, L});
                }
            }
    }
    std::sort(cuts->begin(), cuts->end(), [](const Cut &a, const Cut &b) {
        return a.node != b.node ? a.node < b.node : a.dir < b.dir;
    });
    // a box corner node may have been visited twice (row and column sweeps)
    cuts->erase(std::unique(cuts->begin(), cuts->end(),
                            [](const Cut &a, const Cut &b) { return a.node == b.node && a.dir == b.dir; }),
                cuts->end());
    return LBM_OK;
}

}  // namespace lbm

extern "C" lbm_status lbm_geom_build(const lbm_geom *geom, uint8_t *node_type, lbm_link *links,
                                     int64_t cap, int64_t *nlinks) {
    using namespace lbm;
    set_error("");
    if (!geom || !node_type || !nlinks) {
        set_error("lbm_geom_build: NULL argument");
        return LBM_ERR_ARG;
    }
    std::vector<Cut> cuts;
    lbm_status st = build_geometry(*geom, node_type, &cuts);
    if (st != LBM_OK) return st;
    *nlinks = (int64_t)cuts.size();
    if (!links) return LBM_OK;
    if (cap < (int64_t)cuts.size()) {
        set_error("lbm_geom_build: link capacity too small");
        return LBM_ERR_NOMEM;
    }
    for (size_t k = 0; k < cuts.size(); ++k) links[k] = cuts[k].link;
    return LBM_OK;
}

namespace lbm {

// ---------------------------------------------------------------------------
// Units: the isotropy condition dx/(sqrt(3) dt) = sqrt(mu/rho0) of Sec. 5.1
// fixes c_s^2 = 1/3 in lattice units.
lbm_status make_units(const lbm_desc &d, Units *u) {
    if (!(d.rho0 > 0.0) || !(d.mu > 0.0) || !(d.dx > 0.0) || !(d.dt > 0.0) ||
        !is_finite(d.lambda) || !is_finite(d.rho0) || !is_finite(d.mu)) {
        set_error("lbm_create: rho0, mu, dx, dt must be positive and finite");
        return LBM_ERR_ARG;
    }
    if (!(d.tau > 0.5) || !is_finite(d.tau)) {
        set_error("lbm_create: tau (tau_bar/dt) must exceed 1/2");
        return LBM_ERR_ARG;
    }
    const double U = d.dx / d.dt;
    const double cs2 = d.mu / (d.rho0 * U * U);
    if (std::fabs(cs2 * 3.0 - 1.0) > 1e-3) {
        set_error("lbm_create: dx/(sqrt(3) dt) must equal sqrt(mu/rho0) (isotropy condition)");
        return LBM_ERR_ARG;
    }
    if (!(d.lambda / d.mu > -1.0)) {
        set_error("lbm_create: lambda/mu must exceed -1 (positive bulk modulus in plane strain)");
        return LBM_ERR_ARG;
    }
    u->U = U;
    u->dx = d.dx;
    u->dt = d.dt;
    u->rho0 = d.rho0;
    u->mu = d.rho0 / 3.0;
    u->lam = (d.lambda / d.mu) * d.rho0 / 3.0;
    u->tau = d.tau;
    u->fx = d.force[0] * d.dt / U;
    u->fy = d.force[1] * d.dt / U;
    if (!is_finite(u->fx) || !is_finite(u->fy)) {
        set_error("lbm_create: body force must be finite");
        return LBM_ERR_ARG;
    }
    return LBM_OK;
}

BCDev to_lattice(const lbm_bc &b, const Units &u) {
    BCDev o;
    o.kind = b.kind;
    o.profile = b.profile;
    const double s = (b.kind == LBM_BC_DIRICHLET) ? 1.0 / u.U : 1.0 / (u.U * u.U);
    o.v0 = (float)(b.value[0] * s);
    o.v1 = (float)(b.value[1] * s);
    o.v2 = (float)(b.value[2] * s);
    o.t_ramp = (float)(b.t_ramp / u.dt);
    return o;
}

// ---------------------------------------------------------------------------
// Validation and classification of a node mask + cut-link table.
lbm_status classify(const lbm_desc &d, const Units &u, Tables *t) {
    const int32_t nx = d.nx, ny = d.ny;
    if (nx < 2 || ny < 2 || nx > 65535 || ny > 65535) {
        set_error("lbm_create: nx and ny must be in 2..65535");
        return LBM_ERR_ARG;
    }
    if (!d.node_type || (d.nlinks > 0 && !d.links) || d.nlinks < 0 || !d.bcs || d.nbcs < 1 ||
        d.nbcs > 65535) {
        set_error("lbm_create: node_type, links, bcs (1..65535 entries) are required");
        return LBM_ERR_ARG;
    }
    if (d.storage < LBM_F32 || d.storage > LBM_BF16_DEV) {
        set_error("lbm_create: unknown storage");
        return LBM_ERR_ARG;
    }
    if ((d.wall_values != LBM_WALL_EXTRAPOLATE && d.wall_values != LBM_WALL_NODE) ||
        (d.time_block != 0 && d.time_block != 1 && d.time_block != LBM_TIME_BLOCK)) {
        set_error("lbm_create: unknown wall_values, or time_block not 0, 1 or LBM_TIME_BLOCK");
        return LBM_ERR_ARG;
    }
    if (d.streaming != LBM_STREAM_TWO_BUFFERS && d.streaming != LBM_STREAM_IN_PLACE) {
        set_error("lbm_create: unknown streaming");
        return LBM_ERR_ARG;
    }
    if (d.streaming == LBM_STREAM_IN_PLACE && u.lam != u.mu) {
        // the source's density gradient would read neighbours' populations
        // that the in-place step overwrites
        set_error("lbm_create: in-place streaming needs lambda = mu");
        return LBM_ERR_ARG;
    }
    const int64_t N = (int64_t)nx * ny;
    // boundary conditions
    t->bcs.resize(d.nbcs);
    t->max_load = 0.0f;
    for (int32_t k = 0; k < d.nbcs; ++k) {
        const lbm_bc &b = d.bcs[k];
        if (b.kind < LBM_BC_DIRICHLET || b.kind > LBM_BC_STRESS ||
            (b.profile != LBM_PROFILE_STEP && b.profile != LBM_PROFILE_RAMP) ||
            !is_finite(b.value[0]) || !is_finite(b.value[1]) || !is_finite(b.value[2]) ||
            (b.profile == LBM_PROFILE_RAMP && !(b.t_ramp > 0.0))) {
            set_error("lbm_create: bad boundary condition " + std::to_string(k));
            return LBM_ERR_ARG;
        }
        t->bcs[k] = to_lattice(b, u);
        const BCDev &c = t->bcs[k];
        t->max_load = std::max({t->max_load, std::fabs(c.v0), std::fabs(c.v1), std::fabs(c.v2)});
    }
    // sorted copy of the links
    std::vector<const lbm_link *> L((size_t)d.nlinks);
    for (int64_t k = 0; k < d.nlinks; ++k) {
        const lbm_link &l = d.links[k];
        if (l.node < 0 || l.node >= N || l.dir < 1 || l.dir > 8 || l.bc < 0 || l.bc >= d.nbcs ||
            l.bc2 < -1 || l.bc2 >= d.nbcs || !(l.q > 0.0 && l.q <= 1.0) || !is_finite(l.n[0]) ||
            !is_finite(l.n[1])) {
            set_error("lbm_create: bad cut link " + std::to_string(k));
            return LBM_ERR_ARG;
        }
        if (!d.node_type[l.node]) {
            set_error("lbm_create: cut link " + std::to_string(k) + " starts at a void node");
            return LBM_ERR_ARG;
        }
        L[k] = &l;
    }
    std::sort(L.begin(), L.end(), [](const lbm_link *a, const lbm_link *b) {
        return a->node != b->node ? a->node < b->node : a->dir < b->dir;
    });
    for (size_t k = 1; k < L.size(); ++k)
        if (L[k]->node == L[k - 1]->node && L[k]->dir == L[k - 1]->dir) {
            set_error("lbm_create: duplicate cut link at node " + std::to_string(L[k]->node));
            return LBM_ERR_ARG;
        }

    t->nx = nx;
    t->ny = ny;
    // in-place streaming keeps a ring of one node around the population planes
    t->pitch = (nx + (d.streaming == LBM_STREAM_IN_PLACE ? 2 : 0) + 63) / 64 * 64;
    t->cls.assign((size_t)t->pitch * ny, kVoid);
    t->bnodes.clear();
    t->blinks.clear();
    t->interior = 0;
    // Rows are classified in contiguous chunks on host threads; each chunk
    // keeps its own boundary lists, merged in row order, so the tables are
    // those of a single pass.  Errors are reported for the first offending
    // node in row-major order (the error text is set by the calling thread).
    struct Part {
        std::vector<BNode> bn;
        std::vector<BLink> bl;
        int64_t interior = 0;
        std::string err;
    };
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int nparts = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)hw, 16, ny / 64}));
    std::vector<Part> parts((size_t)nparts);
    auto classify_rows = [&](int part) {
        Part &out = parts[(size_t)part];
        const int32_t ya = (int32_t)((int64_t)ny * part / nparts);
        const int32_t yb = (int32_t)((int64_t)ny * (part + 1) / nparts);
        // first cut link of the chunk
        size_t p = (size_t)(std::lower_bound(L.begin(), L.end(), (int64_t)ya * nx,
                                             [](const lbm_link *l, int64_t node) {
                                                 return l->node < node;
                                             }) -
                            L.begin());
        // full[x] of row y: the node and its eight neighbours are all material.
        // Formed as the AND of three horizontal 3-ANDs (rows y - 1, y, y + 1;
        // outside the box counts as void), so most nodes are classified interior
        // without the per-link checks below.
        std::vector<uint8_t> h0((size_t)nx, 0), h1((size_t)nx, 0), h2((size_t)nx, 0),
            full((size_t)nx, 0);
        auto hrow = [&](int32_t yy, std::vector<uint8_t> &h) {
            if (yy < 0 || yy >= ny) {
                std::fill(h.begin(), h.end(), (uint8_t)0);
                return;
            }
            const uint8_t *__restrict__ r = d.node_type + (int64_t)yy * nx;
            uint8_t *__restrict__ o = h.data();
            o[0] = 0;
            o[nx - 1] = 0;
            for (int32_t x = 1; x < nx - 1; ++x)
                o[x] = (uint8_t)((r[x - 1] != 0) & (r[x] != 0) & (r[x + 1] != 0));
        };
        hrow(ya - 1, h0);
        hrow(ya, h1);
        for (int32_t y = ya; y < yb; ++y) {
            hrow(y + 1, h2);
            {
                const uint8_t *__restrict__ a = h0.data(), *__restrict__ b = h1.data(),
                                           *__restrict__ c = h2.data();
                uint8_t *__restrict__ o = full.data();
                for (int32_t x = 0; x < nx; ++x) o[x] = (uint8_t)(a[x] & b[x] & c[x]);
            }
            std::swap(h0, h1);
            std::swap(h1, h2);
            const int64_t row0 = (int64_t)y * nx;
            uint8_t *crow = t->cls.data() + (size_t)y * t->pitch;
            static_assert(kInterior == 1, "a full node's class is its flag");
            for (int32_t x = 0; x < nx; ++x) {
                // the run of nodes up to the next one with cut links: its full
                // nodes are interior (one branch-free pass); any other material
                // node of the run goes through the checks below (which reject it:
                // it lacks a cut link towards a void or outside neighbour)
                const int32_t xl = (p < L.size() && L[p]->node < row0 + nx)
                                       ? (int32_t)(L[p]->node - row0) : nx;
                if (x < xl) {
                    const uint8_t *__restrict__ fr = full.data();
                    uint8_t *__restrict__ cr = crow;
                    uint32_t cnt = 0;
                    for (int32_t q = x; q < xl; ++q) {
                        cr[q] = fr[q];
                        cnt += fr[q];
                    }
                    out.interior += cnt;
                    int32_t bad = xl;
                    for (int32_t q = x; q < xl; ++q)
                        if (!full[q] && d.node_type[row0 + q]) {
                            bad = q;
                            break;
                        }
                    if (bad == xl) {
                        x = xl - 1;
                        continue;
                    }
                    x = bad;
                    crow[x] = kVoid;
                }
                const int64_t node = row0 + x;
                const lbm_link *mine[kQ] = {nullptr};
                uint16_t cut = 0;
                while (p < L.size() && L[p]->node == node) {
                    mine[L[p]->dir] = L[p];
                    cut |= (uint16_t)(1u << L[p]->dir);
                    ++p;
                }
                if (!d.node_type[node]) continue;
                // every link to a void or outside node must be cut
                for (int i = 1; i < kQ; ++i) {
                    const int32_t tx = x + kCx[i], ty = y + kCy[i];
                    const bool outside = tx < 0 || tx >= nx || ty < 0 || ty >= ny;
                    if ((outside || !d.node_type[(int64_t)ty * nx + tx]) && !(cut & (1u << i))) {
                        out.err = "lbm_create: node (" + std::to_string(x) + "," + std::to_string(y) +
                                  ") links to a void or outside node in direction " +
                                  std::to_string(i) + " without a cut link";
                        return;
                    }
                }
                if (!cut) {
                    crow[x] = kInterior;
                    ++out.interior;
                    continue;
                }
                crow[x] = kBoundary;
                BNode bn;
                std::memset(&bn, 0, sizeof bn);
                bn.x = x;
                bn.y = y;
                bn.cut = cut;
                BLink slots[8];
                std::memset(slots, 0, sizeof slots);
                for (int i = 1; i < kQ; ++i) {
                    if (!(cut & (1u << i))) continue;
                    const lbm_link &l = *mine[i];
                    BLink &s = slots[i - 1];
                    s.q = (float)l.q;
                    s.n0 = (float)l.n[0];
                    s.n1 = (float)l.n[1];
                    // upstream node x - c_i usable?
                    const int32_t ux = x - kCx[i], uy = y - kCy[i];
                    const bool up_ok = ux >= 0 && ux < nx && uy >= 0 && uy < ny &&
                                       d.node_type[(int64_t)uy * nx + ux] && !(cut & (1u << kOpp[i]));
                    if (!up_ok) bn.miss |= (uint16_t)(1u << i);
                    const bool da = d.bcs[l.bc].kind == LBM_BC_DIRICHLET;
                    const bool db = l.bc2 >= 0 && d.bcs[l.bc2].kind == LBM_BC_DIRICHLET;
                    if (da || db) {
                        bn.dirich |= (uint16_t)(1u << i);
                        const int32_t first = da ? l.bc : l.bc2;
                        const int32_t second = (da && db) ? l.bc2 : first;
                        s.bc = (uint16_t)first;
                        s.bc2 = (uint16_t)second;
                    } else if (l.bc2 >= 0) {
                        bn.corner |= (uint16_t)(1u << i);
                        s.bc = (uint16_t)l.bc;
                        s.bc2 = (uint16_t)l.bc2;
                    } else {
                        s.bc = (uint16_t)l.bc;
                        s.bc2 = (uint16_t)l.bc;
                    }
                }
                out.bn.push_back(bn);
                for (int i = 0; i < 8; ++i) out.bl.push_back(slots[i]);
            }
        }
    };
    std::vector<std::thread> workers;
    for (int part = 1; part < nparts; ++part) workers.emplace_back(classify_rows, part);
    classify_rows(0);
    for (auto &w : workers) w.join();
    size_t nb = 0;
    for (const Part &q : parts) {
        if (!q.err.empty()) {  // the first chunk with an error holds the first offending node
            set_error(q.err);
            return LBM_ERR_ARG;
        }
        nb += q.bn.size();
    }
    t->bnodes.reserve(nb);
    t->blinks.reserve(nb * 8);
    for (const Part &q : parts) {
        t->bnodes.insert(t->bnodes.end(), q.bn.begin(), q.bn.end());
        t->blinks.insert(t->blinks.end(), q.bl.begin(), q.bl.end());
        t->interior += q.interior;
    }
    return LBM_OK;
}

}  // namespace lbm
