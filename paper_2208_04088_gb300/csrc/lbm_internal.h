// lbm_internal.h -- layouts shared by the host classifier, the kernels and the
// C ABI of the GB300 solid-LBM library.  Not part of the public interface
// (include/lbm.h is).
#pragma once

#include <cstdint>

#include <cuda.h>
#include <cuda_runtime.h>
#include <string>
#include <vector>

#include "lbm.h"

namespace lbm {

// D2Q9 numbering (0 rest, 1 +x, 2 +y, 3 -x, 4 -y, 5 (+,+), 6 (-,+), 7 (-,-),
// 8 (+,-)) -- the same numbering the public header states.
constexpr int kQ = 9;
constexpr int kCx[kQ] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
constexpr int kCy[kQ] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
constexpr int kOpp[kQ] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

// Node classes in the per-node class array.
enum : uint8_t { kVoid = 0, kInterior = 1, kBoundary = 2 };

// One boundary node of the compacted list.  Bit i (1..8) of each mask refers
// to the link from the node towards node + c_i.
struct BNode {
    int32_t x, y;
    uint16_t cut;     // link i crosses a wall
    uint16_t dirich;  // cut link i takes the bounce-back rule (Dirichlet)
    uint16_t corner;  // cut link i is a Neumann corner link
    uint16_t miss;    // upstream node x - c_i of cut link i is unusable
};
static_assert(sizeof(BNode) == 16, "BNode layout");

// Per (boundary node, direction 1..8) slot; meaningful where the cut bit is set.
struct BLink {
    float q;        // s/l
    float n0, n1;   // outward unit normal (corner: the two edge-normal signs)
    uint16_t bc;    // Dirichlet: first Dirichlet edge; Neumann: x-normal edge
    uint16_t bc2;   // Dirichlet: second Dirichlet edge (or bc); corner: y-normal edge
};
static_assert(sizeof(BLink) == 16, "BLink layout");

// Boundary condition in lattice units.
struct BCDev {
    int32_t kind, profile;
    float v0, v1, v2;
    float t_ramp;  // steps
};
static_assert(sizeof(BCDev) == 24, "BCDev layout");

// FP16 storage: the power-of-two scale of the populations stored by each of
// the last three steps (step t in entry t mod 3) and whether a value stored by
// that step exceeded kScaleOver.  Step t loads with the scale of step t - 1
// and stores with it, halved if that step's flag is set (FP16 ends at 65504,
// so a value can grow eightfold in one step before it overflows).
struct ScaleState {
    float s[3];
    uint32_t over[3];
};
constexpr float kScaleOver = 8192.0f;
// The smallest scale, 2^-126 (the smallest normal FP32 number; its inverse,
// 2^126, is finite): scaled FP16 values then reach 65504 * 2^126, beyond the
// FP32 range, so FP16 storage never overflows before an FP32 solve would.
constexpr float kScaleMin = 1.17549435e-38f;

// Scalar parameters of one lattice, passed by value to every kernel.
struct Lattice {
    int32_t nx, ny, pitch, nb;  // nb: number of boundary nodes
    int64_t plane;              // elements per population plane (pitch * ny)
    float omega;                // 1/tau
    float src;                  // 1 - 1/(2 tau), Eq. (coll)
    float fx, fy;               // body force, lattice units
    float mu_m_lam;             // mu - lambda (lattice units), Eq. (sourceterm)
    float lam_m_mu_r0;          // (lambda - mu)/rho0, Eqs. (poissonstress), (approxdiv)
    float rho0, inv_rho0;
    float scale, inv_scale;     // 16-bit storage scale (1 for FP32)
    float out_u, out_v, out_s;  // lattice -> physical units for the fields
    int32_t grad;               // lambda != mu: the source needs grad rho
    int32_t wall_node;          // Neumann wall values at the boundary node (no extrapolation)
    int64_t fplane;             // elements per population plane: plane, or with
                                // in-place streaming pitch * (ny + 2) (a ring of one node)
    int32_t in_place;           // one population buffer, AA pattern (lbm_desc.streaming)
    int32_t nbcs;               // entries of the boundary-condition table
    int64_t wait_ns;            // limit of a kernel's wait for a tile copy (lbm_set_wait_limit)
    ScaleState *sc;             // FP16 storage: the adaptive scale (null otherwise)
    uint32_t *over;             // FP16: this step's flag in *sc (set per step by step_scales)
};

// Bytes of one node's displacement record: the compensated (u, kahan) float4
// with FP32 storage, (u_x, u_y) with 16-bit storage.
inline size_t urec_bytes(int storage) { return storage == LBM_F32 ? 16 : 8; }

// Default of Lattice::wait_ns, and the limit of the waits that drain the
// copies still in flight after a wait has run out: 1 s.
constexpr int64_t kDefaultWaitNs = 1000000000;

// Host-side result of validating and classifying an lbm_desc.
struct Tables {
    int32_t nx = 0, ny = 0, pitch = 0;
    std::vector<uint8_t> cls;    // [ny][pitch]
    std::vector<BNode> bnodes;   // row-major; partition_boundary puts the simple ones last
    std::vector<BLink> blinks;   // [nb][8]
    std::vector<BCDev> bcs;
    int64_t nbx = 0;             // boundary nodes before the simple ones (partition_boundary)
    int64_t interior = 0;
    float max_load = 0.0f;       // largest boundary-value magnitude (lattice units)
};

// Unit conversion from lbm_desc to lattice units.
struct Units {
    double U = 1.0;       // dx/dt
    double dx = 1.0, dt = 1.0;
    double lam = 0.0, mu = 0.0, rho0 = 1.0, tau = 0.55;
    double fx = 0.0, fy = 0.0;
};

// lbm_create with a choice of launch plan for the temporally blocked kernel:
// plan_blocks <= 0 plans for the device's SMs and balances the plan by
// measurement (lbm_create); plan_blocks > 0 plans that many blocks from the
// cost model alone (the regions a batch schedules itself).
lbm_status create_solver(const lbm_desc *desc, void *stream, void *workspace,
                         uint64_t workspace_bytes, int plan_blocks, lbm_handle *out);

// Creation from tables already validated and classified (prepare()).
// deferred: the uploads are queued on the stream and not waited for (the
// creator orders its later work on the same stream), and the pinned host
// staging of probes and status is allocated on first use.
struct CreateOptions {
    int plan_blocks = 0;
    bool deferred = false;
};
lbm_status prepare(const lbm_desc *desc, Tables *t, Units *u);
uint64_t workspace_bytes_for(const lbm_desc &d, const Tables &t, const Units &u);
lbm_status create_prepared(const lbm_desc *desc, Tables &&t, const Units &u, void *stream,
                           void *workspace, uint64_t workspace_bytes, const CreateOptions &opt,
                           lbm_handle *out);
// Releases a handle's host-side resources without synchronising: only for a
// handle none of whose device work is still pending or will be queued again
// (its workspace belongs to its creator).
void destroy_deferred(lbm_handle h);

// Thread-local error text for lbm_last_error().
void set_error(const std::string &msg);

lbm_status make_units(const lbm_desc &d, Units *u);
BCDev to_lattice(const lbm_bc &b, const Units &u);
lbm_status classify(const lbm_desc &d, const Units &u, Tables *t);

// ---------------------------------------------------------------------------
// Kernel launchers (lbm_kernels.cu).  `cur` holds f^col(t-1), `nxt` receives
// f^col(t).  d_time holds the number of completed steps; a launch with offset
// `toff` computes f at time t = *d_time + toff.
struct DevState {
    void *f[2] = {nullptr, nullptr};  // two distribution buffers (9 planes each); with
                                      // in-place streaming f[0] only, at node (0, 0) of
                                      // its padded planes
    void *ucomp = nullptr;            // per node: FP32 storage (u_x, u_y, kahan_x, kahan_y)
                                      // float4; 16-bit storage (u_x, u_y) float2
    uint8_t *cls = nullptr;
    BNode *bnodes = nullptr;
    BLink *blinks = nullptr;
    BCDev *bcs = nullptr;
    float *rho = nullptr;             // density deviation at the current time (lambda != mu)
    uint32_t *status = nullptr;       // bit 0: non-finite moment seen
    int64_t *time = nullptr;
    float *stage = nullptr;           // field staging [7][ny][nx]
    float *probe = nullptr;           // probe staging [7][max_probe]
    int32_t *probe_idx = nullptr;
    uint64_t *nw = nullptr;           // per-node words of the temporally blocked kernel
    int4 *wave_tab = nullptr;         // blocks of a temporally blocked launch
    long long *wave_cyc = nullptr;    // per-block SM cycles of a calibration launch
};

constexpr int kMaxProbe = 4096;

// Events recorded around the interior and boundary kernels of one step (timing
// mode).  With a side stream the boundary kernel runs beside the interior one,
// as in the replayed graphs.
struct StepEvents {
    cudaEvent_t before_interior, after_interior;  // on the main stream
    cudaEvent_t before_boundary, after_boundary;  // on the stream of the boundary kernel
    int nsteps = 1;                               // steps the bracketed launch carries
};

cudaError_t launch_step(int storage, const Lattice &L, const DevState &S, int cur, int toff,
                        cudaStream_t s_main, cudaStream_t s_side, cudaEvent_t fork,
                        cudaEvent_t join, const StepEvents *ev);
int kernels_per_step(const Lattice &L);
int kernels_per_fields(const Lattice &L);
cudaError_t launch_advance(const DevState &S, int64_t n, cudaStream_t s);
cudaError_t launch_fields(int storage, const Lattice &L, const DevState &S, int cur,
                          float *u, float *v, float *sigma, cudaStream_t s);
cudaError_t launch_gather_probe(const Lattice &L, const DevState &S, int count,
                                cudaStream_t s);
cudaError_t launch_reset(int storage, const Lattice &L, const DevState &S, cudaStream_t s);

// Temporally blocked stepping (kernels in lbm_wave.cu, launch plans in
// lbm_plan.cpp): kWaveK steps per launch (kWaveGradK when lambda != mu), FP32
// storage.  A block owns kWaveC columns, of which the middle kWaveW are its
// core.
constexpr int kWaveK = 8;
constexpr int kWaveC = 128;
constexpr int kWaveW = kWaveC - 2 * kWaveK;

struct WaveMaps {
    CUtensorMap f[2];  // the two distribution buffers, [9][ny][pitch] FP32
    CUtensorMap nw;    // node words [ny][pitch]
    CUtensorMap u;     // displacement records [ny][pitch] float4
    int nblocks = 0;
};

bool wave_supported(const Lattice &L);
// Steps carried by one temporally blocked launch: kWaveK, or kWaveGradK when
// the source needs the density gradient (lambda != mu).
constexpr int kWaveGradK = 4;
size_t wave_smem_bytes();
// SMs of the current device (148 if it cannot be queried).
int device_sms();
// Upper bound of the blocks of one launch (entries of S.wave_tab and S.wave_cyc).
size_t wave_table_entries(int nx, int ny);
// Whether boundary node g takes the blocked kernel's eight-lane update (curved
// walls, corners, crack mouth) rather than the one-lane update of a mid-link
// wall with one BC and one axis-aligned normal.
bool complex_boundary_node(const Tables &t, size_t g);
// Reorders the boundary list (nodes and their link records) so that the nodes
// that are not simple come first, each part in its original order; sets t.nbx.
void partition_boundary(Tables &t);
// The blocks of one launch for a device with `sms` SMs: (X0, Y0, rows, has_boundary).
std::vector<int4> wave_plan(const Tables &t, int sms);
// The modelled cost (in row sweeps) of each block of a plan of this lattice.
std::vector<double> wave_plan_costs(const Tables &t, const std::vector<int4> &plan);
// Builds the node words from the class and boundary tables, the TMA
// descriptors and the block table (planned for the device's SMs, or for
// plan_blocks blocks if it is positive); S.nw (8 bytes per node of the
// pitched plane) and S.wave_tab must be allocated.
cudaError_t wave_prepare(const Tables &t, const Lattice &L, const DevState &S, WaveMaps *m,
                         cudaStream_t s, int plan_blocks = 0);
// Balances the blocks of a launch by measurement: blocked launches from
// buffer 0 record each block's SM cycles, the modelled cost of every row is
// scaled by its block's measured/modelled ratio and the strips are cut again
// (twice); the plan with the smallest measured maximum is kept in
// S.wave_tab.  Leaves f[1], the displacements and the status word modified:
// the caller resets the state.  A lattice created again in the same process
// (same size, boundary tables, kernel and device) reuses its measured plan.
cudaError_t wave_calibrate(const Tables &t, const Lattice &L, const DevState &S, WaveMaps *m,
                           cudaStream_t s);
// kWaveK steps from buffer `cur` into buffer cur ^ 1; the first of them is
// step `toff` after *S.time.  With `cycles`, block b stores its SM cycles in
// cycles[b].
// Device record of one instance of a batch stepped by the blocked kernel:
// its tensor maps (input populations from buffer 0 or 1, node words,
// displacement records), buffers, tables and lattice parameters.
struct WaveInst {
    CUtensorMap tf[2];
    CUtensorMap tnw, tu;
    float *f[2];
    float4 *uc;
    const BLink *blinks;
    const BCDev *bcs;
    const int64_t *time;
    uint32_t *status;
    Lattice L;
};
// One blocked launch over the regions of many instances: kWaveK steps of
// every region; region r = (X0, Y0, rows, has_boundary) of instance
// region_inst[r], read from buffer `cur` into cur ^ 1, its first step `toff`
// after the instance's *time.  The blocks take regions in table order from
// *counter, which must be 0 at the launch.
cudaError_t launch_wave_batch(const WaveInst *insts, const int4 *regions, const int32_t *region_inst,
                              int nregions, int32_t *counter, int cur, int toff, int sms,
                              cudaStream_t s);
cudaError_t launch_wave(const Lattice &L, const DevState &S, const WaveMaps &m, int cur, int toff,
                        cudaStream_t s, long long *cycles = nullptr);

}  // namespace lbm

// One solver instance (the object behind lbm_handle).
struct lbm_solver {
    lbm::Tables tab;
    lbm::Units units;
    lbm::Lattice L;
    lbm::DevState S;
    int storage = LBM_F32;
    cudaStream_t stream = nullptr;  // caller's stream
    cudaStream_t cap_main = nullptr, cap_side = nullptr;  // private capture streams
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaEvent_t gfork = nullptr, gjoin = nullptr;         // events used inside graphs
    cudaGraphExec_t graph[2] = {nullptr, nullptr};        // chunk starting in buffer 0/1
    int cur = 0;
    int64_t time = 0;
    void *owned = nullptr;  // cudaMalloc'ed workspace, if the library allocated it
    void *base = nullptr;
    uint64_t bytes = 0;
    int32_t *h_probe_idx = nullptr;  // pinned host staging for probes
    float *h_probe_out = nullptr;
    uint32_t *h_status = nullptr;    // pinned copy of the status word
    cudaEvent_t status_ready = nullptr;
    bool status_pending = false;
    int64_t launches = 0;            // kernels launched by this handle
    bool deferred = false;           // created with CreateOptions::deferred
    // timing mode: events around every interior and boundary kernel
    bool timing = false;
    std::vector<lbm::StepEvents> ev_pool;
    size_t ev_used = 0;
    // temporal blocking: steps per launch (1: one-step kernels) and its tables
    int block = 1;
    lbm::WaveMaps wave;
};

