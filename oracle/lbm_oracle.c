/*
 * lbm_oracle.c -- plain, slow FP64 CPU oracle of the solid lattice Boltzmann
 * method with local Dirichlet and Neumann boundary rules (Faust, Schlueter,
 * Mueller, Mueller 2022, arXiv 2208.04088).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference for the
 * CUDA library in paper_2208_04088_gb300/.  Only tests/, the smoke check in
 * __graft_entry__.py and the CPU-baseline leg of bench.py may load it.  It
 * shares no code, header, table or constant with the CUDA path.
 *
 * Everything is double precision, absolute distribution functions (not
 * deviations), push streaming, one node at a time, in the order the paper
 * states the algorithm:
 *
 *   Sec. 3   D2Q9 lattice; equilibrium Eq. (fieq); source Eq. (sourceterm)
 *            with S = F + (mu - lambda)/rho grad rho; BGK collision
 *            Eq. (coll); streaming Eq. (stream); moments Eq. (moments).
 *   Sec. 2.2 Dirichlet data j* = rho d_t u*  (Eq. bcchaindir);  Neumann data
 *            by rotation to the boundary frame (Eq. trafocauchy) and the
 *            Poisson stress P* (Eq. bcchainneum) with div u from Eq. (approxdiv).
 *   Sec. 4   modified bounce-back Eq. (bbcon), modified anti-bounce-back
 *            Eq. (abbcon), and their curved forms Eq. (bbnoncon), Eq. (abbnoncon).
 *
 * Conventions where the paper is silent (each one is a stated reading):
 *   - D2Q9 numbering 0 rest, 1 +x, 2 +y, 3 -x, 4 -y, 5 (+,+), 6 (-,+),
 *     7 (-,-), 8 (+,-); weights 4/9, 1/9, 1/36; c_s^2 = 1/3 in lattice units
 *     (Sec. 5.1 isotropy condition dx/(sqrt(3) dt) = c_s), dx = dt = 1.
 *   - grad rho: central difference over the axis neighbours, one-sided when
 *     one neighbour is void or across a cut link, zero when both are.
 *   - displacement: u(t+1) = u(t) + j(t)/rho(t)   (j includes S/2).
 *   - boundary data j*(t), t*(t) are evaluated at the time of f^col(t).
 *   - j* = rho0 * d(u*)/dt.
 *   - sigma_tt^n in the boundary frame is extrapolated along the link like
 *     rho^bd; div u at the wall is (rho0 - rho^bd)/rho0.
 *   - the rotation of Sec. 2.2 is the orthogonal change of basis with the
 *     rows of T equal to e^n and e^t: sigma^n = T sigma T^T, sigma = T^T sigma^n T.
 *   - a link whose wall point is the corner of two edges is Dirichlet if
 *     either edge is (j* = mean of the Dirichlet edges), otherwise Neumann
 *     with sigma* assembled from both edges (xx from the x-normal edge, yy
 *     from the y-normal edge, xy the mean of both), no extrapolation.
 *   - if the upstream node x - c_i is void or across a cut link, the
 *     lattice-conforming form is used with rho^bd = rho(x), sigma^bd = sigma(x).
 *   - option wall_node (not the paper's rule, off by default): rho^bd and
 *     sigma^bd are the boundary node's own values instead of the extrapolation
 *     along the link; the kappa terms of the curved rules are unchanged.
 *   - geometry: nodes at integer (i, j); the box is [-1/2, nx-1/2] x
 *     [-1/2, ny-1/2]; a node is void iff strictly inside the hole circle; a
 *     link is cut by the hole iff its end node is void, with s/l the smaller
 *     root of |x + q c_i - centre| = R; the edge crack lies on
 *     y = ny/2 - 1/2 for x < crack_len - 1/2 (edge crack), or between the tips
 *     crack_x0 - 1/2 and crack_x0 + crack_len - 1/2 (crack_x0 > 0).
 *
 * Parity: pinned by tests/test_oracle_*.py (moment identities, conservation,
 * wave speeds, exact uniform states, 1-D impact closed forms, hand-derived
 * first-step populations, Freund's K_I^0).
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (see oracle/__init__.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* D2Q9 lattice (Sec. 3)                                               */
/* ------------------------------------------------------------------ */
enum { Q = 9 };
static const int CX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[Q] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double W[Q] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                            1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2 = 1.0 / 3.0;

/* ------------------------------------------------------------------ */
/* Public records (mirrored by ctypes in oracle/__init__.py)           */
/* ------------------------------------------------------------------ */
typedef struct {
    int32_t node;   /* y*nx + x of the material node holding the link */
    int32_t dir;    /* i in 1..8: the link towards x + c_i crosses the wall */
    int32_t bc;     /* boundary-condition index (x-normal edge for corners) */
    int32_t bc2;    /* -1, or the y-normal edge of a corner link */
    double q;       /* s_i / l_i, wall distance over link length, in (0, 1] */
    double n0, n1;  /* outward unit normal of the material at the wall point;
                       for a corner link the signs of the two edge normals */
    int32_t curved; /* 1: non-lattice-conforming wall (Eqs. bbnoncon/abbnoncon) */
    int32_t pad;
} ora_link;

typedef struct {
    int32_t kind;    /* 0 Dirichlet: value = d(u*)/dt (x, y)
                        1 Neumann:   value = traction t* (x, y)
                        2 Neumann:   value[0] = pressure p, t* = -p n
                        3 Neumann:   value = stress (xx, yy, xy), t* = sigma n */
    int32_t profile; /* 0 Heaviside step at t = 0, 1 linear ramp then hold */
    double value[3];
    double t_ramp;   /* ramp length in time steps */
} ora_bc;

/* ------------------------------------------------------------------ */
/* Equilibrium, Eq. (fieq)                                             */
/* ------------------------------------------------------------------ */
void ora_feq(double rho, double jx, double jy, double pxx, double pyy, double pxy,
             double *feq) {
    const double j[2] = {jx, jy};
    const double P[2][2] = {{pxx, pxy}, {pxy, pyy}};
    for (int i = 0; i < Q; ++i) {
        const double c[2] = {(double)CX[i], (double)CY[i]};
        double cj = 0.0;
        for (int a = 0; a < 2; ++a) cj += c[a] * j[a];
        double second = 0.0;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                const double d = (a == b) ? 1.0 : 0.0;
                second += (P[a][b] - rho * CS2 * d) * (c[a] * c[b] - CS2 * d);
            }
        feq[i] = W[i] * (rho + cj / CS2 + second / (2.0 * CS2 * CS2));
    }
}

/* Source term psi_i of Eq. (sourceterm). */
static void source_psi(double Sx, double Sy, double *psi) {
    for (int i = 0; i < Q; ++i) psi[i] = W[i] * (CX[i] * Sx + CY[i] * Sy) / CS2;
}

/* Moments of Eq. (moments): rho, j (with the S/2 term), P. */
static void moments(const double *f, double Sx, double Sy, double *rho, double *jx,
                    double *jy, double *pxx, double *pyy, double *pxy) {
    double r = 0, mx = 0, my = 0, xx = 0, yy = 0, xy = 0;
    for (int i = 0; i < Q; ++i) {
        r += f[i];
        mx += f[i] * CX[i];
        my += f[i] * CY[i];
        xx += f[i] * CX[i] * CX[i];
        yy += f[i] * CY[i] * CY[i];
        xy += f[i] * CX[i] * CY[i];
    }
    *rho = r;
    *jx = mx + 0.5 * Sx;
    *jy = my + 0.5 * Sy;
    *pxx = xx;
    *pyy = yy;
    *pxy = xy;
}

/* BGK collision with source, Eq. (coll), dt = 1, tau = tau_bar/dt.
 * Exported for the moment pins; j receives the moment used in f^eq. */
void ora_collide(const double *f, double Sx, double Sy, double tau, double *fcol, double *j) {
    double rho, jx, jy, pxx, pyy, pxy, feq[Q], psi[Q];
    moments(f, Sx, Sy, &rho, &jx, &jy, &pxx, &pyy, &pxy);
    ora_feq(rho, jx, jy, pxx, pyy, pxy, feq);
    source_psi(Sx, Sy, psi);
    for (int i = 0; i < Q; ++i)
        fcol[i] = f[i] - (f[i] - feq[i]) / tau + (1.0 - 1.0 / (2.0 * tau)) * psi[i];
    if (j) {
        j[0] = jx;
        j[1] = jy;
    }
}

/* ------------------------------------------------------------------ */
/* Geometry classification                                             */
/* ------------------------------------------------------------------ */
/* edge_bc = {left, right, bottom, top}; -1 on both sides of an axis makes
 * that axis periodic.  Returns the number of cut links, or -1 if cap is too
 * small (links may be NULL to count only), or -2 on a bad argument. */
int64_t ora_geometry(int32_t nx, int32_t ny, const int32_t *edge_bc, double hole_cx,
                     double hole_cy, double hole_r, int32_t hole_bc, int32_t crack_len,
                     int32_t crack_bc, int32_t crack_x0, uint8_t *node_type, ora_link *links,
                     int64_t cap) {
    if (nx < 1 || ny < 1) return -2;
    const int per_x = (edge_bc[0] < 0), per_y = (edge_bc[2] < 0);
    if (per_x != (edge_bc[1] < 0) || per_y != (edge_bc[3] < 0)) return -2;
    const int has_hole = hole_r > 0.0, has_crack = crack_len > 0;
    if (has_crack && (ny % 2 != 0 || per_y || crack_x0 < 0)) return -2;
    const double ycrack = 0.5 * ny - 0.5; /* crack plane y* */

    /* material iff outside the hole circle */
    for (int32_t y = 0; y < ny; ++y)
        for (int32_t x = 0; x < nx; ++x) {
            int mat = 1;
            if (has_hole) {
                const double dx = x - hole_cx, dy = y - hole_cy;
                if (dx * dx + dy * dy < hole_r * hole_r) mat = 0;
            }
            node_type[(int64_t)y * nx + x] = (uint8_t)mat;
        }

    int64_t n = 0;
    for (int32_t y = 0; y < ny; ++y)
        for (int32_t x = 0; x < nx; ++x) {
            if (!node_type[(int64_t)y * nx + x]) continue;
            for (int i = 1; i < Q; ++i) {
                const int32_t tx = x + CX[i], ty = y + CY[i];
                const int out_x = !per_x && (tx < 0 || tx >= nx);
                const int out_y = !per_y && (ty < 0 || ty >= ny);
                /* a link crossing y* between rows ny/2-1 and ny/2 at abscissa
                 * x + c_ix/2 is cut by the crack iff that abscissa lies on the
                 * crack: left of the tip at crack_x0 + crack_len - 1/2 and, for
                 * a crack away from the left edge (crack_x0 > 0), right of its
                 * other tip at crack_x0 - 1/2; crossings at a tip are not cut */
                int on_crack = 0;
                if (has_crack && CY[i] != 0) {
                    const double ymid = y + 0.5 * CY[i];
                    const double xmid = x + 0.5 * CX[i];
                    const int right_of_start = (crack_x0 == 0) || (xmid > crack_x0 - 0.5);
                    if (ymid == ycrack && right_of_start && xmid < crack_x0 + crack_len - 0.5)
                        on_crack = 1;
                }
                ora_link L;
                memset(&L, 0, sizeof L);
                L.node = y * nx + x;
                L.dir = i;
                L.bc2 = -1;
                L.q = 0.5;
                if (out_x || out_y || on_crack) {
                    /* walls at mid-link: box edges and crack faces */
                    const int xedge = out_x;
                    const int yedge = out_y || on_crack;
                    double sx = 0.0, sy = 0.0;
                    int32_t bx = -1, by = -1;
                    if (xedge) {
                        sx = (tx < 0) ? -1.0 : 1.0;
                        bx = (tx < 0) ? edge_bc[0] : edge_bc[1];
                    }
                    if (yedge) {
                        if (out_y) {
                            sy = (ty < 0) ? -1.0 : 1.0;
                            by = (ty < 0) ? edge_bc[2] : edge_bc[3];
                        } else {
                            /* crack face: the material lies on the node's side,
                             * the outward normal points across the crack */
                            sy = (CY[i] > 0) ? 1.0 : -1.0;
                            by = crack_bc;
                        }
                    }
                    if (xedge && yedge) { /* wall point is a corner */
                        L.bc = bx;
                        L.bc2 = by;
                        L.n0 = sx;
                        L.n1 = sy;
                    } else if (xedge) {
                        L.bc = bx;
                        L.n0 = sx;
                        L.n1 = 0.0;
                    } else {
                        L.bc = by;
                        L.n0 = 0.0;
                        L.n1 = sy;
                    }
                    L.curved = 0;
                } else {
                    /* wrap periodic targets, then test for a void end node */
                    const int32_t wx = (tx + nx) % nx, wy = (ty + ny) % ny;
                    if (node_type[(int64_t)wy * nx + wx]) continue; /* not cut */
                    /* smaller root in (0, 1] of |x + q c_i - centre|^2 = R^2 */
                    const double dx = x - hole_cx, dy = y - hole_cy;
                    const double b = CX[i] * dx + CY[i] * dy;
                    const double c0 = dx * dx + dy * dy - hole_r * hole_r;
                    const double a = (double)(CX[i] * CX[i] + CY[i] * CY[i]);
                    const double disc = b * b - a * c0;
                    const double qq = (-b - sqrt(disc)) / a;
                    const double wxp = x + qq * CX[i], wyp = y + qq * CY[i];
                    L.bc = hole_bc;
                    L.q = qq;
                    /* outward normal of the material points into the hole */
                    L.n0 = (hole_cx - wxp) / hole_r;
                    L.n1 = (hole_cy - wyp) / hole_r;
                    L.curved = 1;
                }
                if (links) {
                    if (n >= cap) return -1;
                    links[n] = L;
                }
                ++n;
            }
        }
    return n;
}

/* ------------------------------------------------------------------ */
/* Solver                                                              */
/* ------------------------------------------------------------------ */
typedef struct {
    int32_t nx, ny, per_x, per_y;
    int64_t N;
    double lambda, mu, rho0, tau, Fx, Fy;
    int64_t t;
    uint8_t *mat;
    double *f, *fnew, *fcol;  /* [N][9] absolute distributions */
    double *u;                /* [N][2] displacement */
    double *rho, *jm, *pm;    /* rho [N], j [N][2], P [N][3] (xx, yy, xy) at time t */
    int64_t *cut;             /* [N][9] link index or -1 */
    ora_link *links;
    int64_t nlinks;
    ora_bc *bcs;
    int32_t nbcs;
    int32_t wall_node; /* 1: rho^bd, sigma^bd taken at the boundary node */
} ora_solver;

static int64_t neighbour(const ora_solver *s, int64_t k, int i) {
    int32_t x = (int32_t)(k % s->nx) + CX[i], y = (int32_t)(k / s->nx) + CY[i];
    if (s->per_x) x = (x + s->nx) % s->nx;
    if (s->per_y) y = (y + s->ny) % s->ny;
    if (x < 0 || x >= s->nx || y < 0 || y >= s->ny) return -1;
    return (int64_t)y * s->nx + x;
}

/* Amplitude of a boundary value at time t (Sec. 5: step, or ramp then hold). */
static double amplitude(const ora_bc *b, double t) {
    if (t < 0.0) return 0.0;
    if (b->profile == 1) return (t >= b->t_ramp) ? 1.0 : t / b->t_ramp;
    return 1.0;
}

/* Prescribed traction t*(t) of a Neumann condition on a wall with outward
 * unit normal n (Eq. bcneu). */
static void traction(const ora_bc *b, double n0, double n1, double t, double *ts) {
    const double amp = amplitude(b, t);
    if (b->kind == 2) {
        ts[0] = -b->value[0] * n0 * amp;
        ts[1] = -b->value[0] * n1 * amp;
    } else if (b->kind == 3) {
        ts[0] = (b->value[0] * n0 + b->value[2] * n1) * amp;
        ts[1] = (b->value[2] * n0 + b->value[1] * n1) * amp;
    } else {
        ts[0] = b->value[0] * amp;
        ts[1] = b->value[1] * amp;
    }
}

void *ora_create(int32_t nx, int32_t ny, double lambda, double mu, double rho0, double tau,
                 double Fx, double Fy, int32_t per_x, int32_t per_y, const uint8_t *node_type,
                 const ora_link *links, int64_t nlinks, const ora_bc *bcs, int32_t nbcs,
                 int32_t wall_node) {
    ora_solver *s = (ora_solver *)calloc(1, sizeof *s);
    s->wall_node = wall_node;
    s->nx = nx;
    s->ny = ny;
    s->per_x = per_x;
    s->per_y = per_y;
    s->N = (int64_t)nx * ny;
    s->lambda = lambda;
    s->mu = mu;
    s->rho0 = rho0;
    s->tau = tau;
    s->Fx = Fx;
    s->Fy = Fy;
    s->mat = (uint8_t *)malloc(s->N);
    memcpy(s->mat, node_type, s->N);
    s->f = (double *)calloc(s->N * Q, sizeof(double));
    s->fnew = (double *)calloc(s->N * Q, sizeof(double));
    s->fcol = (double *)calloc(s->N * Q, sizeof(double));
    s->u = (double *)calloc(s->N * 2, sizeof(double));
    s->rho = (double *)calloc(s->N, sizeof(double));
    s->jm = (double *)calloc(s->N * 2, sizeof(double));
    s->pm = (double *)calloc(s->N * 3, sizeof(double));
    s->cut = (int64_t *)malloc(s->N * Q * sizeof(int64_t));
    for (int64_t k = 0; k < s->N * Q; ++k) s->cut[k] = -1;
    s->links = (ora_link *)malloc((nlinks > 0 ? nlinks : 1) * sizeof(ora_link));
    if (nlinks > 0) memcpy(s->links, links, nlinks * sizeof(ora_link));
    s->nlinks = nlinks;
    for (int64_t l = 0; l < nlinks; ++l) s->cut[(int64_t)links[l].node * Q + links[l].dir] = l;
    s->bcs = (ora_bc *)malloc((nbcs > 0 ? nbcs : 1) * sizeof(ora_bc));
    if (nbcs > 0) memcpy(s->bcs, bcs, nbcs * sizeof(ora_bc));
    s->nbcs = nbcs;
    /* zero-stress rest state (footnote to Eq. poissonstress): P = 0, j = 0 */
    double frest[Q];
    ora_feq(rho0, 0.0, 0.0, 0.0, 0.0, 0.0, frest);
    for (int64_t k = 0; k < s->N; ++k)
        if (s->mat[k]) memcpy(s->f + k * Q, frest, sizeof frest);
    return s;
}

void ora_destroy(void *h) {
    ora_solver *s = (ora_solver *)h;
    if (!s) return;
    free(s->mat);
    free(s->f);
    free(s->fnew);
    free(s->fcol);
    free(s->u);
    free(s->rho);
    free(s->jm);
    free(s->pm);
    free(s->cut);
    free(s->links);
    free(s->bcs);
    free(s);
}

void ora_set_state(void *h, const double *f, const double *u, int64_t t) {
    ora_solver *s = (ora_solver *)h;
    if (f) memcpy(s->f, f, s->N * Q * sizeof(double));
    if (u) memcpy(s->u, u, s->N * 2 * sizeof(double));
    s->t = t;
}

void ora_get_state(void *h, double *f, double *u, int64_t *t) {
    ora_solver *s = (ora_solver *)h;
    if (f) memcpy(f, s->f, s->N * Q * sizeof(double));
    if (u) memcpy(u, s->u, s->N * 2 * sizeof(double));
    if (t) *t = s->t;
}

/* rho(x,t) = sum_i f_i for every material node (Eq. moments). */
static void densities(ora_solver *s) {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < s->N; ++k) {
        double r = 0.0;
        if (s->mat[k])
            for (int i = 0; i < Q; ++i) r += s->f[k * Q + i];
        s->rho[k] = r;
    }
}

/* Source S = F + (mu - lambda)/rho grad rho (Eq. sourceterm), with the
 * one-sided fallback for missing axis neighbours. */
static void source_at(const ora_solver *s, int64_t k, double *Sx, double *Sy) {
    double g[2] = {0.0, 0.0};
    const int plus[2] = {1, 2}, minus[2] = {3, 4};
    for (int a = 0; a < 2; ++a) {
        const int64_t kp = (s->cut[k * Q + plus[a]] < 0) ? neighbour(s, k, plus[a]) : -1;
        const int64_t km = (s->cut[k * Q + minus[a]] < 0) ? neighbour(s, k, minus[a]) : -1;
        if (kp >= 0 && km >= 0)
            g[a] = 0.5 * (s->rho[kp] - s->rho[km]);
        else if (kp >= 0)
            g[a] = s->rho[kp] - s->rho[k];
        else if (km >= 0)
            g[a] = s->rho[k] - s->rho[km];
    }
    const double coef = (s->mu - s->lambda) / s->rho[k];
    *Sx = s->Fx + coef * g[0];
    *Sy = s->Fy + coef * g[1];
}

/* Cauchy stress from the Poisson stress, Eq. (poissonstress) with the
 * divergence of Eq. (approxdiv): sigma = -P + (lambda - mu)(rho0 - rho)/rho0 I. */
static void cauchy(const ora_solver *s, double rho, const double *P, double sig[2][2]) {
    const double divu = (s->rho0 - rho) / s->rho0;
    sig[0][0] = -P[0] + (s->lambda - s->mu) * divu;
    sig[1][1] = -P[1] + (s->lambda - s->mu) * divu;
    sig[0][1] = sig[1][0] = -P[2];
}

/* The missing population f_{opp(i)}(x, t+1) for the cut link (x, i),
 * Eqs. (bbcon), (abbcon), (bbnoncon), (abbnoncon). */
static double boundary_rule(const ora_solver *s, int64_t k, int i, const ora_link *L) {
    const int ib = OPP[i];
    const double *fc = s->fcol + k * Q;
    const ora_bc *ba = &s->bcs[L->bc];
    const ora_bc *bb = (L->bc2 >= 0) ? &s->bcs[L->bc2] : NULL;
    const double t = (double)s->t;

    /* upstream node x - c_i, usable only if material and not across a cut link */
    int64_t ku = -1;
    if (s->cut[k * Q + ib] < 0) ku = neighbour(s, k, ib);
    if (ku >= 0 && !s->mat[ku]) ku = -1;
    const int curved = L->curved && ku >= 0;
    const double q = L->q;

    int dirichlet = (ba->kind == 0) || (bb && bb->kind == 0);
    if (dirichlet) {
        /* j* = rho0 d(u*)/dt (Eq. bcchaindir); corners: mean of the Dirichlet edges */
        double js[2] = {0.0, 0.0};
        int nd = 0;
        const ora_bc *edges[2] = {ba, bb};
        for (int e = 0; e < 2; ++e) {
            if (!edges[e] || edges[e]->kind != 0) continue;
            const double amp = amplitude(edges[e], t);
            js[0] += s->rho0 * edges[e]->value[0] * amp;
            js[1] += s->rho0 * edges[e]->value[1] * amp;
            ++nd;
        }
        js[0] /= nd;
        js[1] /= nd;
        const double cj = CX[i] * js[0] + CY[i] * js[1];
        if (!curved) /* Eq. (bbcon) */
            return fc[i] - (2.0 / CS2) * W[i] * cj;
        /* Eq. (bbnoncon) with l_i - 2 s_i over l_i + 2 s_i = (1 - 2q)/(1 + 2q) */
        const double kappa = (1.0 - 2.0 * q) / (1.0 + 2.0 * q);
        const double fac = 2.0 / (1.0 + 2.0 * q); /* 2 l_i/(l_i + 2 s_i) */
        return fc[i] + kappa * (s->fcol[ku * Q + i] - fc[ib]) - fac * (2.0 / CS2) * W[i] * cj;
    }

    /* Neumann.  Density and stress at the wall, extrapolated along the link:
     * (3 a(x) - a(x - c_i))/2 lattice-conforming, (1+q) a(x) - q a(x - c_i) curved. */
    double sx[2][2], su[2][2], sbd[2][2];
    cauchy(s, s->rho[k], s->pm + k * 3, sx);
    double rbd;
    if (ku < 0 || s->wall_node) {
        /* no usable upstream node, or wall values taken at the boundary node */
        rbd = s->rho[k];
        memcpy(sbd, sx, sizeof sx);
    } else {
        cauchy(s, s->rho[ku], s->pm + ku * 3, su);
        if (!curved) {
            rbd = 0.5 * (3.0 * s->rho[k] - s->rho[ku]);
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b) sbd[a][b] = 0.5 * (3.0 * sx[a][b] - su[a][b]);
        } else {
            rbd = (1.0 + q) * s->rho[k] - q * s->rho[ku];
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b) sbd[a][b] = (1.0 + q) * sx[a][b] - q * su[a][b];
        }
    }

    double sig[2][2]; /* sigma* */
    if (bb) {
        /* corner of an x-normal edge (sign n0) and a y-normal edge (sign n1) */
        double ta[2], tb[2];
        traction(ba, L->n0, 0.0, t, ta);
        traction(bb, 0.0, L->n1, t, tb);
        sig[0][0] = ta[0] * L->n0;
        sig[1][1] = tb[1] * L->n1;
        sig[0][1] = sig[1][0] = 0.5 * (ta[1] * L->n0 + tb[0] * L->n1);
    } else {
        /* rotation to the boundary frame: rows of T are e^n and e^t */
        double ts[2];
        traction(ba, L->n0, L->n1, t, ts);
        const double T[2][2] = {{L->n0, L->n1}, {-L->n1, L->n0}};
        double tn[2] = {0.0, 0.0}; /* t*^n = T t* */
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) tn[a] += T[a][b] * ts[b];
        double stt = 0.0; /* (T sigma^bd T^T)_tt */
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) stt += T[1][a] * sbd[a][b] * T[1][b];
        const double sn[2][2] = {{tn[0], tn[1]}, {tn[1], stt}};
        /* Eq. (trafocauchy): back to the lattice frame, sigma* = T^T sigma^n T */
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                double acc = 0.0;
                for (int g = 0; g < 2; ++g)
                    for (int z = 0; z < 2; ++z) acc += T[g][a] * sn[g][z] * T[z][b];
                sig[a][b] = acc;
            }
    }
    /* Eq. (bcchainneum) with div u from Eq. (approxdiv) at the wall */
    const double divu = (s->rho0 - rbd) / s->rho0;
    double Ps[2][2];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            Ps[a][b] = -sig[a][b] + ((a == b) ? (s->lambda - s->mu) * divu : 0.0);
    const double c[2] = {(double)CX[i], (double)CY[i]};
    double second = 0.0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            const double d = (a == b) ? 1.0 : 0.0;
            second += (Ps[a][b] - rbd * CS2 * d) * (c[a] * c[b] - CS2 * d);
        }
    const double eqpart = 2.0 * W[i] * (rbd + second / (2.0 * CS2 * CS2));
    if (!curved) /* Eq. (abbcon) */
        return -fc[i] + eqpart;
    /* Eq. (abbnoncon) */
    const double kappa = (1.0 - 2.0 * q) / (1.0 + 2.0 * q);
    const double fac = 2.0 / (1.0 + 2.0 * q);
    return -fc[i] - kappa * (s->fcol[ku * Q + i] + fc[ib]) + fac * eqpart;
}

/* One time step t -> t+1. */
static void step_once(ora_solver *s) {
    const int64_t N = s->N;
    densities(s);
    /* collision (Eq. coll) at every material node, displacement update */
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < N; ++k) {
        if (!s->mat[k]) continue;
        double Sx, Sy, fc[Q], j[2], rho, jx, jy, pxx, pyy, pxy;
        source_at(s, k, &Sx, &Sy);
        moments(s->f + k * Q, Sx, Sy, &rho, &jx, &jy, &pxx, &pyy, &pxy);
        s->pm[k * 3 + 0] = pxx;
        s->pm[k * 3 + 1] = pyy;
        s->pm[k * 3 + 2] = pxy;
        s->jm[k * 2 + 0] = jx;
        s->jm[k * 2 + 1] = jy;
        ora_collide(s->f + k * Q, Sx, Sy, s->tau, fc, j);
        memcpy(s->fcol + k * Q, fc, sizeof fc);
        s->u[k * 2 + 0] += jx / rho;
        s->u[k * 2 + 1] += jy / rho;
    }
    /* streaming (Eq. stream) and boundary rules: each destination population
     * is written by exactly one source, so the loop runs in parallel */
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < N; ++k) {
        if (!s->mat[k]) continue;
        s->fnew[k * Q + 0] = s->fcol[k * Q + 0];
        for (int i = 1; i < Q; ++i) {
            const int64_t l = s->cut[k * Q + i];
            if (l >= 0) {
                s->fnew[k * Q + OPP[i]] = boundary_rule(s, k, i, &s->links[l]);
            } else {
                const int64_t kn = neighbour(s, k, i);
                s->fnew[kn * Q + i] = s->fcol[k * Q + i];
            }
        }
    }
    double *tmp = s->f;
    s->f = s->fnew;
    s->fnew = tmp;
    s->t += 1;
}

void ora_step(void *h, int32_t n) {
    ora_solver *s = (ora_solver *)h;
    for (int32_t k = 0; k < n; ++k) step_once(s);
}

/* Fields at the current time: u, v = j/rho, sigma (Eqs. moments,
 * poissonstress, approxdiv).  Planes: u[2][N], v[2][N], sigma[3][N]
 * (xx, yy, xy); void nodes are zero.  Any pointer may be NULL. */
void ora_fields(void *h, double *u, double *v, double *sigma, double *rho_out) {
    ora_solver *s = (ora_solver *)h;
    const int64_t N = s->N;
    densities(s);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < N; ++k) {
        double uu[2] = {0, 0}, vv[2] = {0, 0}, sg[2][2] = {{0, 0}, {0, 0}}, r = 0.0;
        if (s->mat[k]) {
            double Sx, Sy, rho, jx, jy, P[3];
            source_at(s, k, &Sx, &Sy);
            moments(s->f + k * Q, Sx, Sy, &rho, &jx, &jy, &P[0], &P[1], &P[2]);
            uu[0] = s->u[k * 2];
            uu[1] = s->u[k * 2 + 1];
            vv[0] = jx / rho;
            vv[1] = jy / rho;
            cauchy(s, rho, P, sg);
            r = rho;
        }
        if (u) {
            u[k] = uu[0];
            u[N + k] = uu[1];
        }
        if (v) {
            v[k] = vv[0];
            v[N + k] = vv[1];
        }
        if (sigma) {
            sigma[k] = sg[0][0];
            sigma[N + k] = sg[1][1];
            sigma[2 * N + k] = sg[0][1];
        }
        if (rho_out) rho_out[k] = r;
    }
}

int64_t ora_time(void *h) { return ((ora_solver *)h)->t; }

int32_t ora_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void ora_set_threads(int32_t n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
