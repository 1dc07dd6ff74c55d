// Device-side interface of the spectral-element stepper (sm_103a).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "sem_plan.h"

namespace semdev {

constexpr int MAX_NP = 9;  // orders 1..8

// Per-order GLL tables passed by value to the kernels. With the loops over
// GLL points unrolled, every entry is a compile-time offset into the
// kernel-parameter constant bank and becomes an operand of the arithmetic
// instruction itself.
template <typename T>
struct Basis {
    T D[MAX_NP * MAX_NP];  // D[i*np + k] = l_k'(x_i)
    T W[MAX_NP * MAX_NP];  // W[j*np + i] = w_i w_j (quadrature weight of point (i, j))
    T w[MAX_NP];           // GLL weights
    T x[MAX_NP];           // GLL nodes
};

// Block plan on the device (layout in sem_plan.h).
struct Plan {
    const uint8_t* packet;
    const int4* hdr;           // [nblocks][3]
    const uint32_t* epos;      // [(P+1)/2][ne]
    const float4* coef;        // [2][ne] bilinear map (FP32 kernels)
    const double* G;           // [3P][ne] stored metric (FP64 kernels)
    const float* G32;          // [3P][ne] stored metric rounded to FP32 (FP32 kernels, or null: from coef)
    const double* coef64;      // [8][ne] FP64 bilinear map, 1/rho (FP64 first-order kernels)
    const int32_t* open_gid;   // open nodes, ascending
    const int32_t* open_base;
    const int32_t* open_cnt;
    const int32_t* open_rec;   // receiver index or -1
    int64_t ne, nn;
    int eb, nblocks, nopen_nodes;
    int max_packet;            // bytes, multiple of 16
    int sulen_pad, slen_pad;   // shared-memory array lengths (multiples of 16 bytes)
    int dense;
    int vec;                   // node values per 16 bytes of the storage type
};

enum Mode : int {
    MODE_THREE_LEVEL = 0,  // u^{n+1} = 2u^n - u^{n-1} + s (f e_src - K u^n)
    MODE_KAHAN = 1,        // delta += s (f e_src - K u); u += delta, Kahan-compensated
    MODE_APPLY = 2,        // out = K u
    MODE_HEUN_P = 3,       // Heun predictor on the first-order system (see StepArgs)
    MODE_HEUN_C = 4        // Heun corrector
};

// Node state of "level" m: three-level mode (u^m, u^{m-1}); Kahan mode
// (u^m, delta^{m-1/2}, c^m). Launch k of a run reads level k everywhere and
// writes level k+1 at the nodes its blocks close; when `pending` is set the
// open nodes still stand at level k-1 plus the partial sums of launch k-1,
// and every block that touches such a node finishes it to level k itself
// (bitwise the same in every block) before using it; the node's first block
// (its owner) stores that level-k state.
template <typename T>
struct StepArgs {
    const T* u_k;     // level k: u^k (MODE_APPLY: the input vector)
    const T* x_k;     //          u^{k-1} or delta^{k-1/2}
    const T* c_k;     //          compensation (Kahan)
    const T* u_km1;   // level k-1 (read at open nodes when pending)
    const T* x_km1;
    const T* c_km1;
    T* u_kp1;         // level k+1 (written at closed nodes)
    T* x_kp1;         //          (Kahan only; three-level keeps u^k in place)
    T* c_kp1;
    T* u_kw;          // level k at open nodes (owner, when pending)
    T* x_kw;
    T* c_kw;
    const T* s;       // dt^2 / M per node
    const T* part_rd; // partial sums of launch k-1
    T* part_wr;       // partial sums of this launch
    T* apply_out;     // MODE_APPLY output
    const double* src_f;  // Ricker table f(t_n)
    int64_t step;         // k
    int32_t src_gid;      // source node (new id) or -1
    double* trace;        // [nrec][trace_cap]
    int64_t trace_cap;
    int pending;
    int vec_ok;           // node arrays 16-byte aligned (vector copies allowed)
    int32_t* err;         // error word raised by a wait that gave up (may be null)
    // first-order system (Section 4.1-4.2: pressure U at global nodes,
    // velocity V at every element's local nodes, layout [2P][ne]) advanced by
    // Heun's method: the predictor reads U (u_k) and V (v_in), writes
    // U~ = U + h dU (u_kp1), V~ = V + h dV (v_out) and the rates dU (u_d1),
    // dV (v_d1); the corrector reads U~ (u_k), V~ (v_in), U (u_old), V (v_old)
    // and the rates, and writes U + h/2 (dU + dU~) (u_kp1), V + h/2 (dV + dV~)
    // (v_out). s holds 1/M; the source value is f(t_step).
    const T* v_in;
    T* v_out;
    const T* v_old;
    T* v_d1;
    const T* u_old;
    T* u_d1;
    double h;
};

// Per-shot data of a batch (device memory): the shot's plan and its level
// buffers (three-level: u[0..2]; Kahan: u, x, c [0..1]), from which the
// kernel forms the arguments of each step.
template <typename T>
struct ShotDesc {
    Plan pl;
    T* u[3];
    T* x[2];
    T* c[2];
    T* part[2];
    const T* s;
    const double* src_f;
    double* trace;
    int64_t trace_cap;
    int32_t src_gid;
    int32_t* err;     // error word of the handle or batch running the shot
};

// Per shot, advanced on the device after every launch (so that a captured
// launch sequence can be replayed): the step number of the launch's first
// step and whether the shot's open nodes are pending before it.
struct ShotClock {
    int64_t step0;
    int32_t pending0;
    int32_t pad;
};

// One batch launch: CTA i handles block cta_block[i] of shot cta_shot[i];
// step[] and pending[] hold each shot's step number and pending flag, or,
// when clock is set, the shot's step is clock[shot].step0 + offset and its
// open nodes are pending when offset > 0 or clock[shot].pending0.
struct BatchArgs {
    const void* shots;         // ShotDesc<T>[nshots]
    const int32_t* cta_shot;
    const int32_t* cta_block;
    const int64_t* step;
    const int32_t* pending;
    const ShotClock* clock;
    int32_t offset;
};

// A streamed batch launch: several steps of every shot of one order in one
// launch of nsteps * nblk CTAs, one (step, block) unit each, the units of a
// step running over the blocks of all the shots (see sem_batch_stream_kernel).
// Per block g of the order's shots, one 128-byte record: the block header,
// its shot, its block index in the shot and its padded neighbour list.
struct BatchUnit {
    int32_t hdr[12];
    int32_t shot, block, dep_stride, pad;
    int32_t dep[16];
};
struct BatchStreamArgs {
    const void* shots;          // ShotDesc<T>[nshots]
    const BatchUnit* units;     // [nblk]
    ShotClock* clock;           // [nshots]
    uint32_t* const* done;      // [nshots]: each shot's done flags
    const uint32_t* serial0;    // serial of the launch's first step (one for the whole batch)
    unsigned long long* counter;
    int32_t* err;
    int32_t nblk;               // blocks per step, all shots of the order
    int32_t nsteps;             // steps in this launch
};

// A streamed launch: several steps of one mesh (the shot's plan and level
// buffers) in one launch; see sem_stream_kernel.
// Largest padded neighbour list of a streamed block.
constexpr int kMaxStreamDeps = 64;

struct StreamArgs {
    unsigned long long* counter;  // work counter
    unsigned long long base;      // its value when this launch starts
    uint32_t* done;               // per block: serial of its last finished step
    // [nblocks][dep_stride]: the blocks sharing a node with the block, itself
    // included, padded with the block itself to dep_stride (a multiple of 4,
    // at most kMaxStreamDeps) entries
    const int32_t* dep;
    int32_t dep_stride;
    int32_t* err;                 // raised when a wait gave up
    int64_t step0;                // step number of the launch's first step
    int32_t nsteps;               // steps in this launch
    int32_t pending0;             // open nodes pending before the first step
    uint32_t serial0;             // serial of the first step (done flags)
    int64_t hold_unit;            // step * nblocks + block of the unit whose done flag is withheld (test hook), or -1
    // wavefront order: the first tiled_units tickets (whole bands of
    // band_steps steps) map through sched, one band's entries
    // (step-in-band << 24 | block), band after band; later tickets, and all
    // when sched is null, run step after step
    const uint32_t* sched;
    int32_t band_steps;
    int64_t tiled_units;
};

// Launchers; return cudaSuccess or the launch error.
cudaError_t launch_step(int np, bool fp64, int mode, const Plan& plan, const void* args, const void* basis,
                        int threads, int smem_bytes, cudaStream_t st);
// Finishes the open nodes: level k -> k+1 from part_rd (or MODE_APPLY:
// apply_out = sum of partials).
cudaError_t launch_open_finish(bool fp64, int mode, const Plan& plan, const void* args, cudaStream_t st);

// One-time FP64 precompute per element (new order) from the corner
// coordinates: bilinear coefficients (FP32, coef non-null), the stored
// metric (G64 non-null) and w_q |J_q| / (rho c^2) per slot (mloc).
cudaError_t launch_geometry(int np, int64_t ne, const double* coords, const int32_t* quads_new, const double* rho,
                            const double* vel, const Basis<double>& basis, float4* coef, double* G64, double* mloc,
                            double* coef64, float* G32, cudaStream_t st);
// The FP32 metric the step kernels form from the bilinear map (plan.coef),
// for every GLL point of every element (device element order):
// out[(e * P + q) * 3 + (0, 1, 2)] = (gxx, gxy, gyy), in FP64.
cudaError_t launch_metric_fp32(int np, const Plan& plan, const Basis<float>& basis, double* out, cudaStream_t st);
// Lumped mass through the block plan (deterministic), M[nn] in FP64; mloc
// per slot in the device element order.
cudaError_t launch_mass(const Plan& plan, int np, const double* mloc, double* partial, double* M, cudaStream_t st);
// s = num / M (num = dt^2 for the leapfrog, 1 for the first-order system;
// FP64 arithmetic, rounded once to the storage type).
cudaError_t launch_scale(const double* M, int64_t nn, double num, double* s64, float* s32, cudaStream_t st);

// Discrete adjoint of the leapfrog (FP64 or FP32 three-level storage): the
// backward update, the receiver residuals of step m, the correlation
// C += lambda^m (u^m - 2u^{m-1} + u^{m-2}) and the per-element gradient
// dJ/dc_e = -(2/c_e) sum_q mloc[e,q] C[conn[e,q]] (device element order).
cudaError_t launch_adjoint_update(bool fp64, int64_t nn, void* lam, const void* lam1, const void* lam2, const void* s,
                                  const void* klam1, cudaStream_t st);
cudaError_t launch_adjoint_receivers(bool fp64, int nrec, void* lam, const void* s, const int32_t* rec_node,
                                     const int32_t* rec_row, const double* trace, int64_t trace_cap, const double* obs,
                                     int64_t obs_cap, int64_t m, double inv_dt, cudaStream_t st);
cudaError_t launch_correlate(bool fp64, int64_t nn, double* C, const void* lam, const void* um, const void* um1,
                             const void* um2, cudaStream_t st);
// The three above in one pass over the nodes (backward update, receiver
// residuals of step m, correlation): rec_first[nn] is the first index in
// rec_order (receivers sorted by node, then index) of the node's receivers,
// or -1.
cudaError_t launch_adjoint_node(bool fp64, int64_t nn, void* lam, const void* lam1, const void* lam2, const void* s,
                                const void* klam1, const int32_t* rec_first, const int32_t* rec_order, int nrec,
                                const int32_t* rec_node, const int32_t* rec_row, const double* trace,
                                int64_t trace_cap, const double* obs, int64_t obs_cap, int64_t m, double inv_dt,
                                double* C, const void* um, const void* um1, const void* um2, cudaStream_t st);
cudaError_t launch_gradient(int64_t ne, int P, const int32_t* conn, const double* mloc, const double* C,
                            const double* vel, double* grad, cudaStream_t st);

// Threads of the step kernel for a block of eb elements (one per element,
// rounded up to whole warps).
int step_threads(int eb);
// Dynamic shared memory of the step kernel.
int smem_bytes_for(int P, int eb, int max_packet, int sulen_pad, int slen_pad, bool fp64, int mode, bool dense);

// Batch step (all shots of one order) and the step-counter advance.
// prepare_only sets the kernel's shared-memory limit (done before a graph
// capture) and launches nothing.
cudaError_t launch_batch_step(int np, bool fp64, int mode, bool prepare_only, const BatchArgs& ba, int ctas,
                              const void* basis, int threads, int smem, cudaStream_t st);
cudaError_t launch_batch_advance(int64_t* step, int32_t* pending, int nshots, cudaStream_t st);
// Streamed batch launch of sa.nsteps steps of the order-np shots
// (prepare_only: set the kernel's shared-memory limit, launch nothing), the
// advance of every shot's clock and of the batch serial by nsteps after it,
// and the CTAs of that launch shape resident at once.
cudaError_t launch_batch_stream(int np, bool fp64, int mode, bool prepare_only, const BatchStreamArgs& sa,
                                const void* basis, int threads, int smem, cudaStream_t st);
cudaError_t launch_batch_clock_advance(ShotClock* clock, int nshots, uint32_t* serial, int nsteps, cudaStream_t st);
cudaError_t batch_stream_resident_ctas(int np, bool fp64, int mode, int threads, int smem, int* out);

// Streamed steps (leapfrog modes of DENSE plans): sa.nsteps steps of the
// shot (a host ShotDesc<T> whose plan has nblocks blocks) in one launch of
// sa.nsteps * nblocks CTAs, one (step, block) unit each.
cudaError_t launch_stream(int np, bool fp64, int mode, const void* shot, const StreamArgs& sa, const void* basis,
                          int threads, int smem, int nblocks, cudaStream_t st);
// CTAs of that launch shape resident on the whole GPU at once.
// (sg: the kernel that streams the stored FP32 metric, plan.G32)
cudaError_t stream_resident_ctas(int np, bool fp64, int mode, bool sg, int threads, int smem, int* out);

}  // namespace semdev
