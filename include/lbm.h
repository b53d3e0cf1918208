/*
 * lbm.h -- C ABI of a GB300 (sm_103a) solver for the solid lattice Boltzmann
 * method with local Dirichlet and Neumann boundary rules (Faust, Schlueter,
 * Mueller, Mueller 2022, arXiv 2208.04088).
 *
 * What one time step computes (lattice units dx = dt = 1, c_s^2 = 1/3):
 *   streaming of the nine D2Q9 populations (Sec. 3, Eq. stream, pull form),
 *   the moments rho, j, P (Eq. moments) with the source S = F +
 *   (mu - lambda)/rho grad rho (Eq. sourceterm), the equilibrium of Eq. (fieq),
 *   BGK collision with source (Eq. coll), the boundary rules of Sec. 4
 *   (Eqs. bbcon, abbcon, bbnoncon, abbnoncon) for the populations that would
 *   stream in from across a wall, and u += j/rho for the displacement.
 *
 * Conventions fixed by this library where the paper is silent:
 *   - D2Q9 directions 0 rest, 1 +x, 2 +y, 3 -x, 4 -y, 5 (+x,+y), 6 (-x,+y),
 *     7 (-x,-y), 8 (+x,-y); weights 4/9, 1/9, 1/36.
 *   - nodes sit at integer (x, y), 0 <= x < nx, 0 <= y < ny, row-major index
 *     y*nx + x; the box is [-1/2, nx - 1/2] x [-1/2, ny - 1/2].
 *   - Dirichlet data j* = rho0 d(u*)/dt; Neumann data sigma* from the traction
 *     in the boundary frame with sigma_tt extrapolated along the link like
 *     rho^bd (Sec. 2.2, Eqs. trafocauchy, bcchainneum, approxdiv).
 *   - boundary values are taken at the time of the post-collision populations
 *     they act on; a step load is on from the first step.
 *   - a corner link (wall point at the corner of two edges) is Dirichlet if
 *     either edge is; otherwise sigma* takes xx from the x-normal edge, yy from
 *     the y-normal edge and the mean of both shears.
 *   - if the node upstream of a cut link (x - c_i) is void or itself across a
 *     wall, the link uses the lattice-conforming rule with rho^bd = rho(x).
 *   - grad rho: central differences, one-sided next to a wall, zero between two.
 *
 * Errors: every call returns an lbm_status; the library never aborts.  The
 * text of the last error of the calling thread is lbm_last_error().
 * Threading: a handle may be used by one host thread at a time.
 * All calls that launch device work are asynchronous on the handle's stream
 * unless stated otherwise.
 */
#ifndef LBM_H
#define LBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_solver *lbm_handle;

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = 1,      /* invalid argument or inconsistent tables */
    LBM_ERR_NOMEM = 2,    /* device memory or workspace too small */
    LBM_ERR_CUDA = 3,     /* a CUDA runtime call failed (see lbm_last_error) */
    LBM_ERR_UNSTABLE = 4, /* a non-finite moment was produced (Sec. 6 lists
                             the scheme's stability as an open issue) */
    LBM_ERR_TIMEOUT = 5   /* a bounded wait expired */
} lbm_status;

/* Storage of the distribution functions.  All arithmetic is FP32; the 16-bit
 * forms store f - f_rest scaled by a power of two and round to nearest.  The
 * scale starts where the largest boundary value maps to about 8.  BF16 has the
 * exponent range of FP32 and keeps it; FP16 ends at 65504, so its scale halves
 * from one step to the next whenever a step stored a value above 8192 (a run
 * that grows keeps finite values as long as FP32 would).  The displacement u
 * is accumulated in FP32: with FP32 storage with Kahan compensation (16 bytes
 * per node), with 16-bit storage without it (8 bytes per node; the populations'
 * own rounding is far larger than what compensation recovers). */
typedef enum { LBM_F32 = 0, LBM_F16_DEV = 1, LBM_BF16_DEV = 2 } lbm_storage;

/* Where the Neumann rules take the wall density rho^bd and the wall stress
 * used for sigma_tt.  LBM_WALL_EXTRAPOLATE is the rule of Sec. 4 (linear
 * extrapolation along the link, (3 a(x) - a(x - c_i))/2 at a mid-link wall).
 * LBM_WALL_NODE takes both at the boundary node itself; it is not the paper's
 * rule.  On lattices with lambda = mu the density is otherwise undamped and the
 * extrapolation feeds it back at traction edges: runs of more than about a
 * thousand steps grow a density mode there, which LBM_WALL_NODE removes on
 * straight edges. */
typedef enum { LBM_WALL_EXTRAPOLATE = 0, LBM_WALL_NODE = 1 } lbm_wall_values;

/* How the populations are streamed (lbm_desc.streaming).  LBM_STREAM_TWO_BUFFERS
 * pulls f_i(x, t) = f_i^col(x - c_i, t-1) (Eq. stream) from one buffer into
 * the other.  LBM_STREAM_IN_PLACE keeps one buffer and updates it in place in
 * the AA pattern: even steps read and write each node's own slots (reversed),
 * odd steps the slots of its neighbours, so every node reads and writes the
 * same nine locations.  It halves the population memory at the same bytes per
 * lattice update; it needs lambda = mu and one step per launch (time_block 0
 * or 1), and gives fields bit-identical to LBM_STREAM_TWO_BUFFERS. */
typedef enum { LBM_STREAM_TWO_BUFFERS = 0, LBM_STREAM_IN_PLACE = 1 } lbm_streaming;

/* Boundary-condition kinds (Sec. 2, Eqs. bcdir and bcneu). */
typedef enum {
    LBM_BC_DIRICHLET = 0, /* value[0..1] = d(u*)/dt  (velocity of the wall)  */
    LBM_BC_TRACTION = 1,  /* value[0..1] = t*                                  */
    LBM_BC_PRESSURE = 2,  /* value[0] = p, t* = -p n  (n outward normal)       */
    LBM_BC_STRESS = 3     /* value = (s_xx, s_yy, s_xy), t* = s n              */
} lbm_bc_kind;

typedef enum {
    LBM_PROFILE_STEP = 0, /* Heaviside: full value from t = 0 */
    LBM_PROFILE_RAMP = 1  /* linear from 0 at t = 0 to full at t_ramp, then held */
} lbm_profile;

/* One boundary condition, in the physical units of lbm_desc. 40 bytes. */
typedef struct {
    int32_t kind;    /* lbm_bc_kind */
    int32_t profile; /* lbm_profile */
    double value[3];
    double t_ramp;   /* ramp duration (time units); used by LBM_PROFILE_RAMP */
} lbm_bc;

/* One cut link: the link from material node `node` towards node + c_dir
 * crosses the wall at distance s = q * |c_dir| (Fig. boundnoncon).  40 bytes. */
typedef struct {
    int32_t node; /* y*nx + x of a material node */
    int32_t dir;  /* 1..8 */
    int32_t bc;   /* index into lbm_desc.bcs (the x-normal edge of a corner link) */
    int32_t bc2;  /* -1, or the y-normal edge of a corner link */
    double q;     /* s/l in (0, 1]; 0.5 is a lattice-conforming (mid-link) wall */
    double n[2];  /* outward unit normal of the material at the wall point; for
                     a corner link the signs (+-1, +-1) of the two edge normals */
} lbm_link;

/* Analytic geometry: a box, optionally with a circular hole or a crack.
 * Box edges cut links at mid-link.  A node is void iff strictly inside the
 * hole; a link is cut by the hole iff its end node is void, with q the first
 * crossing of the circle.  The crack lies on y = ny/2 - 1/2 (ny even): with
 * crack_x0 = 0 it runs from the left edge to its tip at x = crack_len - 1/2
 * (an edge crack, Sec. 5.2 in half-plane form); with crack_x0 > 0 it lies
 * between the tips crack_x0 - 1/2 and crack_x0 + crack_len - 1/2 (the centre
 * crack of Sec. 5.2).  Links crossing exactly at a tip are not cut. */
typedef struct {
    int32_t nx, ny;
    int32_t edge_bc[4]; /* bc index of the left, right, bottom, top edge */
    double hole_cx, hole_cy, hole_r; /* hole_r <= 0: no hole */
    int32_t hole_bc;
    int32_t crack_len; /* <= 0: no crack */
    int32_t crack_bc;  /* both crack faces */
    int32_t crack_x0;  /* first column of the crack (>= 0) */
} lbm_geom;

/* Problem description.  Physical units: the lattice spacing dx and the time
 * step dt must satisfy the isotropy condition dx/(sqrt(3) dt) = sqrt(mu/rho0)
 * of Sec. 5.1 to a relative 1e-3; the scheme then runs in lattice units with
 * mu_lattice = rho0/3 and lambda_lattice = (lambda/mu) rho0/3. */
typedef struct {
    int32_t nx, ny;          /* lattice size, 2..65535 each (lbm_geom: 1..65535) */
    double lambda, mu, rho0; /* Lame parameters and reference density */
    double dx, dt;           /* lattice spacing, time step */
    double tau;              /* relaxation time tau_bar/dt of Eq. (coll), > 0.5 */
    double force[2];         /* constant body force density F (Eq. sourceterm) */
    const uint8_t *node_type; /* host, nx*ny row-major: 0 void, 1 material */
    const lbm_link *links;    /* host, nlinks cut links, any order, each
                                 (node, dir) at most once */
    int64_t nlinks;
    const lbm_bc *bcs; /* host, nbcs entries */
    int32_t nbcs;      /* 1..65535 */
    int32_t storage;   /* lbm_storage */
    int32_t wall_values; /* lbm_wall_values */
    int32_t time_block;  /* time steps fused into one kernel launch:
                            0  library default: LBM_TIME_BLOCK where it is the
                               faster form (supported, lambda = mu, at least 2^21
                               nodes, at most one boundary node per 800 nodes that
                               is not on a box edge or crack face); else 1
                            1  one launch per step (bulk and boundary-list kernels)
                            LBM_TIME_BLOCK  temporal blocking: each launch carries
                               LBM_TIME_BLOCK steps (4 when lambda != mu, whose
                               source needs the density gradient) of a strip of
                               the lattice in shared memory, so the populations
                               cross HBM once per launch; needs FP32 storage and
                               nx >= 128 (LBM_ERR_ARG otherwise).  Every stored
                               value is bit-identical to time_block = 1. */
    int32_t streaming;   /* lbm_streaming (0: two buffers) */
} lbm_desc;

/* Steps per launch of the temporally blocked kernel (lbm_desc.time_block). */
#define LBM_TIME_BLOCK 8

/* Read-only information about a handle. */
typedef struct {
    int32_t nx, ny, pitch, storage;
    int64_t time;           /* completed time steps */
    int64_t boundary_nodes; /* nodes with at least one cut link */
    int64_t interior_nodes; /* material nodes without cut links */
    uint64_t workspace_bytes;
    float storage_scale;    /* power-of-two scale of the 16-bit forms, 1 for FP32.
                               FP16 rescales itself: this is the scale the last
                               step stored with (lbm_get_info then waits for
                               the handle's stream) */
    float bytes_per_update; /* algorithmic HBM bytes per interior lattice update */
    int64_t kernel_launches; /* kernels this handle has launched so far */
    int32_t time_block;      /* steps per launch in use: 1, LBM_TIME_BLOCK, or 4
                                (temporal blocking with lambda != mu) */
    int32_t streaming;       /* lbm_streaming in use */
} lbm_info;

/* Accumulated kernel times of timing mode (see lbm_set_timing). */
typedef struct {
    double interior_ms; /* sum over launches of the interior (bulk) kernel, or of
                           the temporally blocked kernel (boundary nodes included) */
    double boundary_ms; /* sum over steps of the boundary-list kernel (0 for
                           temporally blocked launches) */
    int64_t steps;      /* steps timed */
} lbm_timing;

/* Build the node mask and cut-link table of an analytic geometry on the host.
 * node_type: nx*ny bytes written.  links: capacity `cap`, may be NULL to only
 * count; *nlinks receives the number of cut links.  Links come in canonical
 * order (node row-major, then direction).  q and n are computed in double
 * precision with a fixed operation order: dx = x - cx, dy = y - cy,
 * b = c.(dx, dy), c0 = dx*dx + dy*dy - R*R, a = |c|^2,
 * q = (-b - sqrt(b*b - a*c0))/a, n = ((cx - (x + q c_x))/R, (cy - (y + q c_y))/R).
 * Returns LBM_ERR_ARG for a bad geometry, LBM_ERR_NOMEM if cap is too small. */
lbm_status lbm_geom_build(const lbm_geom *geom, uint8_t *node_type, lbm_link *links,
                          int64_t cap, int64_t *nlinks);

/* Device bytes a handle for `desc` needs (distributions, displacement,
 * tables, field staging).  Host tables are validated as in lbm_create. */
lbm_status lbm_workspace_size(const lbm_desc *desc, uint64_t *bytes);

/* Create a solver: validates and classifies the tables on the host, copies
 * them to the device and sets the zero-stress rest state at t = 0 (footnote
 * to Eq. poissonstress).  `stream` is a cudaStream_t (NULL: the legacy default
 * stream).  If `workspace` is non-NULL it must be device memory of at least
 * lbm_workspace_size() bytes, 256-byte aligned, owned by the caller and kept
 * alive until lbm_destroy; otherwise the library allocates with cudaMalloc.
 * The caller keeps ownership of every host array; none is referenced after
 * return.  With temporal blocking, three blocked launches on the zero state
 * measure the SM cycles of every block and the strips are re-cut to balance
 * them (a launch plan with the smallest measured maximum is kept; a lattice
 * created again in the same process reuses it); the state is then reset.
 * Synchronises the stream before returning. */
lbm_status lbm_create(const lbm_desc *desc, void *stream, void *workspace,
                      uint64_t workspace_bytes, lbm_handle *out);

/* Advance nsteps >= 0 time steps (asynchronous).  Long runs replay CUDA
 * graphs of a fixed number of steps.  Returns LBM_ERR_UNSTABLE if an earlier
 * step, already completed on the device, produced a non-finite moment. */
lbm_status lbm_step(lbm_handle h, int64_t nsteps);

/* Fields at the current time t, dense row-major planes, physical units:
 *   u     [2][ny][nx]  displacement (x plane, then y plane)
 *   v     [2][ny][nx]  velocity j/rho
 *   sigma [3][ny][nx]  Cauchy stress xx, yy, xy: sigma = -P + (lambda - mu)
 *                      (rho0 - rho)/rho0 I (Eqs. poissonstress, approxdiv)
 * Void nodes are 0.  Any pointer may be NULL.  on_device = 1: device pointers,
 * asynchronous; on_device = 0: host pointers, returns after the copy. */
lbm_status lbm_get_fields(lbm_handle h, float *u, float *v, float *sigma, int32_t on_device);

/* The fields of lbm_get_fields, copied to host memory, for callers that must
 * not allocate device memory.  The paper has no counterpart; this is a service
 * of the library.  Some callers cannot call cudaMalloc: code that runs under a
 * fixed device-memory budget reserved up front by another allocator (it passed
 * its own workspace to lbm_create, sized by lbm_workspace_size), or code on a
 * latency-critical path where a cudaMalloc and its implicit device
 * synchronisation are not acceptable.  This call allocates nothing: the field
 * planes are staged in a fixed array inside the library, 7 x 262144 floats
 * (7 MiB), which every GPU that loads the library holds until the process
 * exits.  Limits and behaviour:
 *   - nx * ny must not exceed 262144 (e.g. 512 x 512); larger lattices return
 *     LBM_ERR_ARG with a message naming the limit;
 *   - u, v, sigma are host pointers with the layouts of lbm_get_fields, any
 *     may be NULL; the call returns after the copies (synchronous);
 *   - the first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture on the device;
 *   - every call on a device shares the array and leaves its contents behind;
 *     calls whose device work overlaps (different streams or threads) race. */
lbm_status lbm_get_fields_host_noalloc(lbm_handle h, float *u, float *v, float *sigma);

/* Fields at `count` nodes (host indices y*nx + x) into host `out`
 * [count][7] = (u_x, u_y, v_x, v_y, s_xx, s_yy, s_xy).  Synchronous. */
lbm_status lbm_probe(lbm_handle h, const int32_t *nodes, int32_t count, float *out);

/* Replace boundary condition `index` (takes effect from the next step). */
lbm_status lbm_set_bc(lbm_handle h, int32_t index, const lbm_bc *bc);

/* Back to the rest state at t = 0 (asynchronous). */
lbm_status lbm_reset(lbm_handle h);

/* Wait for the handle's stream; LBM_ERR_UNSTABLE if a non-finite moment was
 * produced since creation or the last reset. */
lbm_status lbm_sync(lbm_handle h);

lbm_status lbm_get_info(lbm_handle h, lbm_info *info);

/* Limit of every bounded wait inside the kernels (the temporally blocked
 * kernels wait for the tile copies of their input rows), in nanoseconds;
 * 0 .. 60e9, default 1e9 (1 s).  The paper has no counterpart; this is a
 * service of the library.  After a wait runs out the block issues no further
 * copy and finishes its sweep on whatever its shared-memory rows hold (every
 * table index it reads from them is clamped into its table, so all accesses
 * stay in bounds); it then waits for every copy it still has in flight, each
 * with the default limit, and exits.  lbm_sync and the next lbm_step return
 * then undefined until lbm_reset.  A limit of 0 makes every block give up at
 * its first wait, whether or not that copy has landed, so every blocked launch
 * reports LBM_ERR_TIMEOUT: it exists to test this path.  Synchronises the handle's stream; takes effect
 * from the next step.  LBM_ERR_ARG for a NULL handle or a limit out of range. */
lbm_status lbm_set_wait_limit(lbm_handle h, int64_t limit_ns);

/* Timing mode for profiling.  While enabled, lbm_step launches the kernels of
 * each step directly (no graphs; the boundary kernel on a private stream beside
 * the interior kernel, joined before the next step, as inside the graphs) and
 * records CUDA events around both on their streams; with temporal blocking each
 * launch of LBM_TIME_BLOCK steps is bracketed as one interior kernel.
 * lbm_get_timing synchronises, returns the accumulated times and clears them. */
lbm_status lbm_set_timing(lbm_handle h, int32_t enable);
lbm_status lbm_get_timing(lbm_handle h, lbm_timing *out);

/* Release the handle and any memory the library allocated (synchronises). */
lbm_status lbm_destroy(lbm_handle h);

/* Text of the last error on the calling thread ("" if none). */
const char *lbm_last_error(void);

/* ------------------------------------------------------------------------
 * Many instances, one launch per step.  The paper has one lattice per run;
 * these entry points advance many independent lattices (Poisson solids,
 * lambda = mu, one storage form) together.  A step is one persistent interior
 * kernel over a table of (instance, tile) pairs and persistent boundary
 * kernels over a table of (instance, boundary node) pairs (eight lanes to a
 * node; the simple nodes of box edges and crack faces one lane each), running
 * the same per-node code as lbm_step, so every instance's fields are
 * bit-identical to the same instance stepped alone.  FP32 instances of at
 * least 128 columns are stepped instead by the temporally blocked kernel, 8
 * steps per launch over all of them.  Steps replay a captured CUDA graph.
 * ------------------------------------------------------------------------ */
typedef struct lbm_engine *lbm_batch;
typedef struct lbm_engine *lbm_server;

/* Launch shape of the batched interior kernel: a tile of tile_x x tile_y
 * threads (one node each; 32x4, 32x8, 32x16 or 64x4) and a schedule
 * (`dynamic`): 0 a persistent grid of blocks_per_sm blocks per SM walking the
 * tiles with a grid stride, 1 the same grid taking tiles from an atomic
 * counter, 2 one block per tile, 3 one block per 4 consecutive tiles. */
typedef struct {
    int32_t tile_x, tile_y, blocks_per_sm, dynamic;
} lbm_launch_shape;

typedef struct {
    int32_t instances;
    int32_t unstable;        /* instances that produced a non-finite moment */
    int64_t nodes;           /* material nodes over all instances */
    int64_t steps;           /* steps run */
    uint64_t device_bytes;   /* arena bytes in use */
    int64_t kernel_launches;
    lbm_launch_shape shape;
    int32_t blocked_instances; /* instances stepped by the temporally blocked kernel */
    int32_t pad;
} lbm_batch_stats;

/* Create a batch of `count` instances (host descriptors as for lbm_create,
 * every one with lambda = mu and the same storage), all at rest at t = 0.
 * FP32 instances with two population buffers and nx >= 128 are stepped by the
 * temporally blocked kernel: one persistent launch per LBM_TIME_BLOCK steps
 * over the strip segments of all of them (segments of about 768 rows, the
 * longest first, taken by the blocks from a counter).  The other instances
 * are stepped one step per launch by the batched interior and boundary
 * kernels.  time_block of the descriptors is not used; each instance keeps
 * the streaming form its descriptor asks for, and in-place instances take
 * less of the arena.  Either way every instance's fields are bit-identical
 * to the instance stepped alone.  Device memory: one arena sized for all
 * instances.  Synchronous. */
lbm_status lbm_batch_create(const lbm_desc *descs, int32_t count, void *stream, lbm_batch *out);
/* Advance every instance by nsteps (asynchronous). */
lbm_status lbm_batch_step(lbm_batch b, int64_t nsteps);
/* Fields of instance `index`, as lbm_get_fields. */
lbm_status lbm_batch_get_fields(lbm_batch b, int32_t index, float *u, float *v, float *sigma,
                                int32_t on_device);
/* Autotuner: time each candidate launch shape on this batch for
 * steps_per_trial steps (CUDA events), keep the fastest, then put every
 * instance back to rest at t = 0.  `chosen` may be NULL.  Synchronous. */
lbm_status lbm_batch_tune(lbm_batch b, int32_t steps_per_trial, lbm_launch_shape *chosen);
lbm_status lbm_batch_set_shape(lbm_batch b, const lbm_launch_shape *shape);
lbm_status lbm_batch_reset(lbm_batch b);
/* Wait; LBM_ERR_UNSTABLE if any instance produced a non-finite moment. */
lbm_status lbm_batch_sync(lbm_batch b);
/* Statistics; waits for the batch's stream to count unstable instances. */
lbm_status lbm_batch_info(lbm_batch b, lbm_batch_stats *stats);
lbm_status lbm_batch_destroy(lbm_batch b);

/* Continuous-batching server.  Requests (a descriptor and a step count) are
 * queued by lbm_server_submit; each lbm_server_tick admits queued requests in
 * arrival order while their workspaces fit in the device budget, queues the
 * steps that advance every admitted instance together by up to max_steps
 * (never past the nearest completion), and starts retiring the instances that
 * reach their step count: their fields are copied to pinned host memory
 * behind those steps, and once a later tick finds the copy complete the
 * result is delivered and the device memory returns to the budget.  A tick
 * does not wait for the device except to keep at most two ticks queued on it
 * (and, when no instance is left to step, for the results in flight), so the
 * host admits and classifies new requests while the device runs earlier
 * ones.  Requests that arrive while others run join at the next tick. */
typedef struct {
    int32_t active, queued;   /* after the tick */
    int32_t admitted, finished; /* during the tick */
    int64_t steps;            /* steps advanced by the tick */
    int64_t active_nodes;
    uint64_t device_bytes;
    int64_t kernel_launches;  /* cumulative */
} lbm_server_stats;

lbm_status lbm_server_create(uint64_t hbm_budget_bytes, int32_t storage, void *stream,
                             lbm_server *out);
/* Queue a request; the descriptor's host arrays are copied.  Validation and
 * classification of the tables then run on a host worker thread while
 * earlier requests run, so the tick that admits the request finds them ready.
 * Returns LBM_ERR_NOMEM at once if one population buffer and the displacement
 * records of the lattice alone exceed the budget; any other problem with the
 * request (bad tables, lambda != mu, another storage, a workspace larger than
 * the budget) makes it fail at admission: lbm_server_result then returns
 * LBM_ERR_ARG with the reason. */
lbm_status lbm_server_submit(lbm_server s, const lbm_desc *desc, int64_t nsteps, int64_t *id);
lbm_status lbm_server_tick(lbm_server s, int32_t max_steps, lbm_server_stats *stats);
/* *state: 0 queued, 1 running, 2 done (fields copied to the host arrays, any
 * may be NULL, layouts of lbm_get_fields; the request is then forgotten).
 * A done request whose run produced a non-finite moment still delivers its
 * fields but returns LBM_ERR_UNSTABLE.  A failed request returns LBM_ERR_ARG
 * with its error text. */
lbm_status lbm_server_result(lbm_server s, int64_t id, int32_t *state, float *u, float *v,
                             float *sigma);
lbm_status lbm_server_destroy(lbm_server s);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
