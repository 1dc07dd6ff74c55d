/*
 * sem.h -- C ABI of the GB300 spectral-element wave stepper.
 *
 * The library advances the 2D acoustic wave equation (Section 4.1,
 * Eqs. def_v_1 and def_u_1, eliminated to the scalar second-order form
 * (1/K) u_tt = div((1/rho) grad u) + f with K = rho c^2 and natural Neumann
 * boundaries from the weak form, Eq. def_weak_u) on an unstructured mesh of
 * quadrilaterals with a tensor-product Gauss-Lobatto-Legendre (GLL) nodal
 * basis whose nodes double as quadrature points (Section 4.2,
 * Eq. numerical_integ). One time step is:
 *   gather U_mu(q,e) per element (Section 4.2, the U_2 gather of Algorithm 1),
 *   reference gradient and per-point metric G_q = w_q |J_q| rho_e^-1 J_q^-1 J_q^-T
 *   (Eq. deriv_u with K^(e) = J^-1), transposed derivative contraction and
 *   assembly into global nodes (Eq. u_change_r_effic), the lumped inverse mass
 *   (Eq. Abar with M = 1/K) and point source (Algorithm 3), then an explicit
 *   leapfrog update, u^{n+1} = 2u^n - u^{n-1} + dt^2 M^-1 (f(t_n) e_s - K u^n).
 * Elements and nodes are stored in an order chosen by sem_reorder; the
 * Hilbert ordering is the memory reordering of Section 4.3.
 *
 * Conventions for every call:
 *  - All calls return sem_status and never throw. NULL handle or pointer
 *    arguments return SEM_ERR_INVALID_ARG. sem_last_error() gives a
 *    human-readable message for the last failing call on a handle.
 *  - Arrays passed by the caller are HOST arrays (plain C memory) unless the
 *    argument name says "dev_". They are copied; the caller keeps ownership.
 *  - User-facing arrays use the ORIGINAL numbering: vertex/element ids as
 *    passed to sem_mesh_create, and the canonical global node numbering
 *    defined below. Permutations are applied and undone inside the library.
 *  - The library owns all device memory of a handle (allocated through
 *    sem_set_allocator's callbacks when set, else cudaMalloc) and frees it
 *    in sem_destroy. A handle is not thread-safe; use one per thread.
 *  - Device work is enqueued on the stream given to sem_mesh_create
 *    (NULL = legacy default stream). Calls that return data to the host
 *    synchronise that stream.
 *
 * Canonical global node numbering (the paper adds SEM nodes to its meshes in
 * memory without fixing their labels; this library fixes one). Local point
 * (i, j), i, j in 0..p, has local index j*(p+1) + i; xi runs from corner 0 to
 * corner 1 and eta from corner 0 to corner 3 (corners counter-clockwise).
 * Global ids: first the mesh vertices in input order; then the p-1 interior
 * nodes of each edge, edges in order of first appearance when scanning
 * elements 0..E-1 over local edges (c0c1, c1c2, c2c3, c3c0), each edge's
 * nodes ordered from its lower vertex id to its higher one; then the (p-1)^2
 * interior nodes of each element, elements ascending, i fastest.
 */
#ifndef SEM_H
#define SEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SEM_OK = 0,
    SEM_ERR_INVALID_ARG = 1,  /* bad pointer, size, index, mesh or value      */
    SEM_ERR_STATE = 2,        /* call out of order (e.g. reorder after a step) */
    SEM_ERR_CUDA = 3,         /* a CUDA runtime call failed                    */
    SEM_ERR_OOM = 4,          /* device or host allocation failed              */
    SEM_ERR_TIMEOUT = 5,      /* a bounded device wait gave up                 */
    SEM_ERR_UNSUPPORTED = 6   /* order or option not built into this library   */
} sem_status;

typedef enum {
    SEM_FP64 = 0,        /* FP64 storage and arithmetic, three-level leapfrog    */
    SEM_FP32_KAHAN = 1,  /* FP32 bulk; increment-form leapfrog with a Kahan-
                            compensated accumulation of u; FP64 precompute      */
    SEM_FP32 = 2         /* FP32 bulk, plain three-level leapfrog (no Kahan)    */
} sem_precision;

typedef enum {
    SEM_ORDER_NONE = 0,     /* input order for elements and nodes ("No Strategy",
                               Section 6.1)                                      */
    SEM_ORDER_ROWMAJOR = 1, /* input element order; nodes renumbered by the
                               node procedure of Section 4.3                     */
    SEM_ORDER_RANDOM = 2,   /* Fisher-Yates shuffles of elements (splitmix64
                               stream seed+2) and of nodes (stream seed+3)       */
    SEM_ORDER_HILBERT = 3,  /* Section 4.3: elements along a generalized Hilbert
                               curve over the centroid grid, nodes renumbered by
                               first touch, ascending degree                     */
    SEM_ORDER_CONNECTIVITY = 4, /* Section 6.1 "Node Connectivity": a walk over
                               nodes (connected = sharing an element) from the
                               node with the fewest connections, always to the
                               unvisited connected node with the fewest; at a
                               dead end back along the walk; elements listed as
                               their nodes are first visited (ascending id)      */
    SEM_ORDER_DISTANCE = 5, /* Section 6.1 "Node Distance": the same walk by
                               squared distance to the lower-left corner of the
                               bounding box (ties to the lower node id)          */
    SEM_ORDER_HILBERT_WIDE = 6 /* SEM_ORDER_HILBERT with the other bounding box
                               Section 4.3 offers for changing how many elements
                               fall in a curve cell (w_b = sqrt(n_e) r, h_b =
                               sqrt(n_e)): H = ceil(sqrt(E)) cells high, W =
                               max(1, ceil(H r)) wide, r = w_m / h_m; the same
                               node renumbering. SEM_ERR_UNSUPPORTED when W x H
                               exceeds 2^30 cells                                */
} sem_ordering;

typedef enum { SEM_SRC_RICKER = 0 } sem_source_kind;

/* Where the FP32 kernels take the per-point geometric factors G_q of Eq.
 * deriv_u from (SEM_FP64 always streams its FP64 copy). Both start from the
 * FP64 precompute of Section 4.2's "precalculate" step: */
typedef enum {
    SEM_METRIC_BILINEAR = 0, /* the default: the FP64-derived bilinear map of
                                each element (b, c, d and 1/rho, 32 B per element),
                                rounded to FP32 once; G_q is formed from it in FP32
                                at every point of every step                      */
    SEM_METRIC_STORED = 1    /* G_q computed in FP64 and rounded to FP32 once,
                                stored [3P][ne] and streamed every step (12 B per
                                GLL point)                                        */
} sem_metric;

typedef enum {
    SEM_SCHEME_LEAPFROG = 0, /* second-order form M u_tt = f e_s - K u, leapfrog
                                (the default; see sem_precision)                 */
    SEM_SCHEME_HEUN = 1      /* the paper's own scheme (Section 4.2, Time
                                Integration): the first-order pressure/velocity
                                system, velocity V stored at every element's local
                                nodes (Eq. v_change), pressure U at the global nodes
                                (Eq. u_change with B = -I, F = I/rho), advanced by
                                Heun's predictor-corrector; the source y(t) enters
                                dU/dt. SEM_FP64 or SEM_FP32 only                   */
} sem_scheme;

typedef struct sem_mesh sem_mesh;

/* Optional device allocator (e.g. a framework's caching allocator). alloc
 * returns a 16-byte aligned device pointer of at least `bytes` bytes usable
 * on `stream`, or NULL on failure; free releases it. A pointer that is not
 * 16-byte aligned is released again and the call that needed it fails with
 * SEM_ERR_OOM. Applies to handles created afterwards
 * in this process. Pass NULLs to restore cudaMalloc/cudaFree. */
typedef void* (*sem_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*sem_free_fn)(void* ptr, size_t bytes, void* stream, void* ctx);
sem_status sem_set_allocator(sem_alloc_fn alloc, sem_free_fn free_fn, void* ctx);

/* Create a mesh handle (Section 4.2: unstructured mesh of non-overlapping
 * elements, each mapped from the reference element; here bilinear quads).
 *   coords [nv][2]  vertex coordinates (x, y), FP64.
 *   quads  [ne][4]  vertex ids of each quad, counter-clockwise.
 *   order           polynomial order p, 1..8 (p+1 GLL points per direction).
 *   prec            arithmetic of the time loop (see sem_precision).
 *   cuda_stream     cudaStream_t to enqueue work on (NULL = default stream).
 * Validation (SEM_ERR_INVALID_ARG): nv, ne > 0; indices in [0, nv); every
 * vertex referenced; no edge shared by more than two quads; the Jacobian
 * determinant positive at every GLL point (clockwise or degenerate quads are
 * rejected). The ordering starts as SEM_ORDER_NONE. */
sem_status sem_mesh_create(const double* coords, int64_t nv, const int32_t* quads, int64_t ne,
                           int order, sem_precision prec, void* cuda_stream, sem_mesh** out);

/* Choose the memory ordering of elements and nodes (Section 4.3 for HILBERT).
 * Must precede the first sem_step / sem_set_state / sem_apply_stiffness
 * (else SEM_ERR_STATE). `seed` is used by SEM_ORDER_RANDOM only. */
sem_status sem_reorder(sem_mesh* m, sem_ordering kind, uint64_t seed);

/* Per-element material (Section 4.1: rho and K = rho c^2, constant per
 * element as assumed before Eq. u_change). vel[ne] > 0 (wave speed c);
 * rho[ne] > 0, or NULL for rho = 1. Original element order. Called again
 * after the device data exists, it recomputes the geometric factors, the
 * lumped mass and dt^2/M on the device and keeps the plan and the state (the
 * way to re-evaluate a misfit for a new model without rebuilding). */
sem_status sem_set_model(sem_mesh* m, const double* vel, const double* rho);

/* Point source (Eq. def_u_2 source term; Algorithm 3): a Ricker wavelet
 * amp (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2) at t_n = n dt,
 * added to the global node nearest to (x, y) (Euclidean distance; ties to the
 * lowest original node id), scaled by the inverse lumped mass. f0 > 0.
 * Before the first step only. */
sem_status sem_set_source(sem_mesh* m, int kind, double f0, double t0, double amp, double x,
                          double y);

/* Receivers: xy[nrec][2] positions, each snapped like the source. Traces of
 * u at those nodes are recorded in FP64 after every step, for up to
 * max_steps steps (sem_step returns SEM_ERR_INVALID_ARG beyond that).
 * nrec = 0 removes them. Before the first step only. */
sem_status sem_set_receivers(sem_mesh* m, const double* xy, int32_t nrec, int64_t max_steps);

/* dt_cfl = min over elements of (the shortest distance between GLL points
 * adjacent along a local grid line) / c_e. The paper only says its step
 * meets the CFL condition (Section 6.2); this is the definition used here.
 * Needs the model. */
sem_status sem_cfl_dt(const sem_mesh* m, double* dt_cfl);

/* Time integration scheme (sem_scheme), before the device data is built.
 * SEM_SCHEME_HEUN with SEM_FP32_KAHAN returns SEM_ERR_UNSUPPORTED. With Heun,
 * sem_step advances Heun steps (two right-hand-side evaluations each, every
 * evaluation one step-kernel launch plus one open-node launch), traces record
 * U after each step, sem_read_wavefield / sem_get_state return U (u_prev gets
 * zeros), sem_set_state sets U and V = 0 (u_prev is ignored); the batched and
 * adjoint calls are leapfrog-only (SEM_ERR_STATE / SEM_ERR_UNSUPPORTED). */
sem_status sem_set_scheme(sem_mesh* m, int scheme);

/* Metric source of the FP32 kernels (sem_metric), before the device data is
 * built. SEM_METRIC_STORED on an SEM_FP64 handle is a no-op (FP64 always
 * stores); with SEM_SCHEME_HEUN it returns SEM_ERR_UNSUPPORTED, and so does
 * sem_set_scheme(SEM_SCHEME_HEUN) after it; handles with a stored FP32 metric
 * cannot join a batch (sem_batch_create returns SEM_ERR_UNSUPPORTED). After
 * the build: SEM_ERR_STATE. (The paper precalculates its geometric factors,
 * Section 4.2; this call chooses the FP32 copy the step streams.) */
sem_status sem_set_metric(sem_mesh* m, int metric);

/* The geometric factors G_q = w_q |J_q| / rho_e J_q^-1 J_q^-T (Eq. deriv_u,
 * with the quadrature weight of Eq. numerical_integ) exactly as the step
 * kernels use them: G[e][q][3] = (gxx, gxy, gyy) for every element e
 * (original order) and GLL point q = j (p+1) + i, in FP64. SEM_FP64 and
 * SEM_METRIC_STORED: the stored values; SEM_METRIC_BILINEAR: the FP32 values
 * the kernels form from the bilinear map, by the same device code. Builds the
 * device data if needed (needs the model); synchronises. */
sem_status sem_read_metric(sem_mesh* m, double* G);

/* Time step dt > 0 (values above sem_cfl_dt are accepted; stability is the
 * caller's business). Before the first step only. */
sem_status sem_set_dt(sem_mesh* m, double dt);

/* Advance nsteps >= 0 leapfrog steps from the current state (u^0 = u^-1 = 0
 * unless sem_set_state was called; Eq. initial_cond). Asynchronous on the
 * handle's stream. The first call builds the device data (allocation and
 * host-to-device copies). Needs the model and dt. The nodes shared between
 * element blocks are finished from per-block partial sums by the next
 * step's blocks; after a call's last step they stay partial until the next
 * sem_step call finishes them the same way, or until a call that reads or
 * replaces the state (sem_get_state, sem_read_wavefield, sem_read_traces,
 * sem_set_model, a batch step, the gradient) runs one open-node launch
 * first: what the API returns is the same, bit for bit, however the steps
 * were split into calls. */
sem_status sem_step(sem_mesh* m, int64_t nsteps);

/* Number of steps taken so far, n in t_n = n dt (the step counter of the
 * time loop, Eq. u_change's time index; no passage of its own: an accessor). */
sem_status sem_get_step(const sem_mesh* m, int64_t* step);

/* Copy traces to out[nrec][cap]: out[r*cap + k] = u at receiver r after step
 * k+1, for k < min(cap, steps taken). Synchronises the stream. Receiver
 * records are the seismograms of the multilayer model of Section 6.2 (the
 * paper records the wavefield at surface receivers; it gives no interface
 * for reading them, so this call is an accessor). */
sem_status sem_read_traces(sem_mesh* m, double* out, int64_t cap);

/* u^n at every global node, original node order, as FP64. Synchronises. */
sem_status sem_read_wavefield(sem_mesh* m, double* u);

/* Set (u^n, u^{n-1}) in original node order and the step counter n (which
 * sets t_n = n dt for the source). In FP32 modes the values are rounded to
 * FP32 once (SEM_FP32_KAHAN stores u and delta = u^n - u^{n-1}, computed in
 * FP64). Builds the device data if needed. Needs the model and dt. */
sem_status sem_set_state(sem_mesh* m, const double* u, const double* u_prev, int64_t step);

/* Read (u^n, u^{n-1}) back in original node order (either pointer may be
 * NULL). Synchronises. */
sem_status sem_get_state(sem_mesh* m, double* u, double* u_prev, int64_t* step);

/* Matrix-free stiffness application Ku = K u (Eq. u_change_r_effic in the
 * second-order form) with the handle's precision, on host arrays in original
 * node order (u[N] in, Ku[N] out). Does not change the time-stepping state.
 * Synchronises. Needs the model. On DENSE block plans every step and apply
 * launch copies each block's packet and owned node range into shared memory
 * with bulk copies whose completion barrier is waited on with the same
 * bound as the streamed waits (sem_set_stream); a wait that gave up raises
 * the device error flag, and this call (or, after a step or a device-array
 * apply, the next sem_read_wavefield, sem_get_state or sem_read_traces)
 * returns SEM_ERR_TIMEOUT. */
sem_status sem_apply_stiffness(sem_mesh* m, const double* u, double* Ku);

/* Lumped diagonal mass M_nu = sum over (e, q) with mu(q, e) = nu of
 * w_q |J_q| / (rho_e c_e^2) (Eq. Abar with M = 1/K), computed in FP64 on the
 * device, original node order. Synchronises. Needs the model. */
sem_status sem_read_mass(sem_mesh* m, double* mass);

/* Permutations chosen by sem_reorder: elem_new_of_old[ne] and
 * node_new_of_old[N] (either may be NULL). These are the element order of
 * Section 4.3 (the curve order L) and the node renumbering of the same
 * section, read back; no passage of their own: an accessor. */
sem_status sem_get_permutation(const sem_mesh* m, int64_t* elem_new_of_old,
                               int64_t* node_new_of_old);

/* Global node count N and element count E (the counts of Section 4.2's
 * global node set and element set; no passage of their own: an accessor). */
sem_status sem_get_sizes(const sem_mesh* m, int64_t* n_nodes, int64_t* n_elems);

/* Positions of the global nodes, original order, out[N][2]. */
sem_status sem_node_coordinates(const sem_mesh* m, double* xy);

/* Indices (original numbering) of the source node and receiver nodes
 * (either pointer may be NULL; rec must hold nrec entries). */
sem_status sem_get_snapped(const sem_mesh* m, int64_t* src_node, int64_t* rec_nodes);

/* Host-only ordering computation, no device needed: the element and node
 * orderings sem_reorder would choose for this mesh, as order arrays
 * (elem_order[new] = old element id, node_order[new] = old node id). Same
 * validation as sem_mesh_create. n_nodes_out receives N (may be NULL);
 * node_order must hold N entries, computable as sem_count_nodes. */
sem_status sem_compute_ordering(const double* coords, int64_t nv, const int32_t* quads, int64_t ne,
                                int order, sem_ordering kind, uint64_t seed, int64_t* elem_order,
                                int64_t* node_order);

/* Host-only self-check of the block plan that the step kernel would use for
 * this mesh, ordering, block size and storage type (fp64_storage: 8-byte
 * node values, else 4): builds the plan and replays one assembly over it on
 * the host with every index bounds-checked, on integer-valued residuals so
 * that sums are exact, and compares with the direct per-slot sum; also
 * checks that every distinct receiver node (rec_xy[nrec][2], snapped like
 * sem_set_receivers) is recorded by exactly one block; checks that no two
 * elements of one colour in a block share a node; checks that the streamed
 * loop's wavefront order (sem_set_stream_tiling; bands of 16 steps, windows
 * of 1, 4 and 16 levels) over the plan's block graph is topological. info[7] (may be NULL):
 * blocks, DENSE layout (1/0), open nodes, largest entry count, largest
 * packet bytes, partial-sum slots, most colours in a block. msg (may be
 * NULL) receives the first violation. Returns SEM_OK when consistent, SEM_ERR_STATE on a
 * violation, SEM_ERR_UNSUPPORTED when the plan cannot be built,
 * SEM_ERR_INVALID_ARG for bad input. No device is needed. */
sem_status sem_plan_check(const double* coords, int64_t nv, const int32_t* quads, int64_t ne, int order,
                          sem_ordering kind, uint64_t seed, int elems_per_block, int fp64_storage,
                          const double* rec_xy, int32_t nrec, int64_t* info, char* msg, size_t msg_cap);

/* Global node count of a mesh at polynomial order `order`, host only. */
sem_status sem_count_nodes(const int32_t* quads, int64_t nv, int64_t ne, int order,
                           int64_t* n_nodes);

/* Generalized Hilbert curve over a W x H cell grid (Section 3, after
 * Cerveny 2020; equals Listing 1's curve when W = H = 2^a): cells[k] =
 * (x, y) of the k-th visited cell, out cells[W*H][2]. Host only. */
sem_status sem_hilbert_cells(int32_t W, int32_t H, int32_t* cells);

/* Launch accounting of the time loop: steps per step-kernel launch (1, or
 * the streamed launch length of sem_set_stream when the time loop is
 * streamed; a read of the state after a sem_step call adds one open-node
 * launch, see sem_step) and the number of open nodes, i.e. nodes whose
 * elements span more than one element block (-1 before the device data is
 * built). Either pointer may be NULL. */
sem_status sem_launch_info(const sem_mesh* m, int64_t* steps_per_launch, int64_t* open_nodes);

/* Streamed time loop. With steps_per_launch = N >= 1 sem_step runs up to N
 * leapfrog steps per launch: one CTA per (step, element block) unit, each
 * CTA taking the next unit in order from a work counter once it runs; a
 * unit starts as soon as the previous step has finished at its block and at
 * every block sharing a node with it, so consecutive steps overlap and no
 * launch boundary or partly filled last wave separates them. The arithmetic
 * per unit is the per-step kernel's: the results are bitwise those of N = 0
 * (one launch per step). Used for DENSE block plans (the node numbering of
 * Section 4.3 along the element order) and the leapfrog scheme where no block
 * shares nodes with more than 64 blocks (itself included); other cases
 * launch once per step. N = -1 (the default) streams 256 steps per launch
 * where a step has at least as many element blocks as step CTAs resident on
 * the GPU at once and fewer than 8 times as many (there the partly filled
 * last wave of a launch per step costs more than the units' waits; with
 * less than one wave streaming only adds the units' waits) and launches
 * once per step otherwise.
 * Waits are bounded: a wait gives up after 1 s of the GPU's global timer
 * (checked every 64 polls of 128 ns back-off each; in any case after 2^26
 * polls); one that gives up (which no correct run does) raises
 * a device error flag, the remaining steps of the run are skipped, and the
 * next sem_read_wavefield, sem_get_state or sem_read_traces returns
 * SEM_ERR_TIMEOUT. Any time. */
sem_status sem_set_stream(sem_mesh* m, int steps_per_launch);

/* Order of the units of a streamed launch. Section 4.3 orders elements so
 * that data reused together is close in memory and in time; here the same
 * argument is carried across time steps. In step order (band_steps = 0) a
 * block's next step comes a whole step's data later (more than the L2 on the
 * workloads this library streams). In the wavefront order (band_steps = T >=
 * 1) each band of T consecutive steps of a launch runs as tiles over the
 * block graph (blocks adjacent when they share a node): blocks get levels,
 * their breadth-first distance from a pseudo-peripheral block; unit (step j
 * of the band, block b) belongs to tile floor((level(b) + j) / W), and units
 * run by tile, then step, then level, then block id. Every unit's
 * dependencies come earlier (a topological order, checked on the host before
 * upload), and a block's next step follows about W levels' worth of units
 * later, so its element data and node state are mostly still in L2. Steps of
 * a launch beyond its last whole band run in step order. window_levels = W >=
 * 1, or 0 for the automatic window (about as many blocks per step of a tile as
 * step CTAs are resident on the GPU at once). band_steps = -1 selects the
 * default, the step order: the wavefront order trades the L2 reuse for units
 * that wait on neighbours issued shortly before them, which on the meshes
 * measured cost more than it saved. The results are bitwise the same in every
 * order. Any time; takes effect at the next streamed launch. */
sem_status sem_set_stream_tiling(sem_mesh* m, int band_steps, int window_levels);

/* Band length and window of the wavefront order last uploaded for the
 * handle's streamed launches (0, 0 before any). Either pointer may be NULL. */
sem_status sem_stream_order(const sem_mesh* m, int32_t* band_steps, int32_t* window_levels);

/* Host-only construction of the wavefront order above for a block graph in
 * CSR form (dep[dep_ptr[b] .. dep_ptr[b+1]): the blocks adjacent to block b,
 * b itself included; the graph must be symmetric). sched[band_steps *
 * nblocks] receives the units as (j << 24) | b in run order; levels[nblocks]
 * (may be NULL) the breadth-first levels. SEM_ERR_INVALID_ARG for a malformed
 * graph or out-of-range sizes (band_steps 1..255, window_levels >= 1,
 * nblocks < 2^24); SEM_ERR_STATE if the built order fails the library's own
 * topological check. No device is needed. */
sem_status sem_stream_schedule(const int32_t* dep_ptr, const int32_t* dep, int32_t nblocks, int band_steps,
                               int window_levels, uint32_t* sched, int32_t* levels);

/* Test hook for the bounded waits of the streamed time loop: in the streamed
 * launch that runs step `step`, the unit of element block `block` (in the
 * plan's block order, 0 .. blocks-1) does its work but does not mark its
 * block done, so the next step's units that share a node with that block wait
 * until their wait limit (1 s of global timer), raise the error flag and stop the
 * launch; the next read-back returns SEM_ERR_TIMEOUT and clears the flag, and the
 * wavefield is not meaningful until sem_set_state. Fires once; a negative
 * step or block clears it. No effect on steps that run one launch each. */
sem_status sem_stream_withhold(sem_mesh* m, int64_t step, int32_t block);

/* Launch shape of the step kernel: elements per block (0 = default, about
 * 6400 element points per block in FP32 and 3200 in FP64, at most 256, one
 * thread per element; in FP64 on a mesh with fewer elements than that times
 * the device's SM count,
 * the elements over the SM count, at least 4, so that a step's
 * double-precision arithmetic spreads over every SM) and
 * threads per block (0 = one per element rounded up to whole warps; else a
 * multiple of 32 up to 256, raised to that minimum if smaller; the threads
 * beyond the block's elements help with staging and assembly). Before the
 * device data is built. elems_per_block * (order+1)^2 must not exceed 65535. */
sem_status sem_set_tuning(sem_mesh* m, int elems_per_block, int threads_per_block);

/* Per-kernel device timing for measurement. While enabled, sem_step records
 * CUDA events on the handle's stream around every step-kernel launch
 * ("block", one or, streamed, several steps) and every open-node launch
 * ("open"). sem_profile_read
 * synchronises the stream and returns the summed durations (milliseconds)
 * and launch counts since the last read, then resets them. Any output pointer
 * may be NULL. */
sem_status sem_profile_enable(sem_mesh* m, int enable);
sem_status sem_profile_read(sem_mesh* m, double* block_ms, int64_t* block_launches, double* open_ms,
                            int64_t* open_launches);

/* Compulsory DRAM bytes of one step-kernel launch (block_bytes; a launch
 * that finishes the previous step's open nodes) and of one open-node launch
 * (open_bytes) under the current plan and precision: every array a launch
 * touches counted once (element positions and geometry, block packets, node
 * state read and written, partial sums). Needs the device data (after the
 * first sem_step). Either pointer may be NULL. */
sem_status sem_traffic_model(const sem_mesh* m, double* block_bytes, double* open_bytes);

/* Host<->device bytes this handle's calls have copied so far. */
sem_status sem_transfer_bytes(const sem_mesh* m, int64_t* h2d, int64_t* d2h);

/* Stiffness application that allocates nothing, for callers that cannot
 * call cudaMalloc themselves or let a library do it: a real-time loop that
 * must not reach the allocator (cudaMalloc and cudaFree can synchronise the
 * device and take unbounded time), or a host process that hands all device
 * memory out from its own pool sized up front, where an extra allocation
 * fails. The paper has no counterpart; it is a deployment aid.
 *   dev_u   [N] device array, input; dev_Ku [N] device array, output. Both hold
 *           the handle's storage type (double for SEM_FP64, float otherwise)
 *           indexed by the library's storage order of the nodes
 *           (node_new_of_old from sem_get_permutation).
 * Computes dev_Ku = K dev_u like sem_apply_stiffness, enqueued on the
 * handle's stream without synchronising. The per-block partial sums go to a
 * scratch array that is a file-scope device variable of the library:
 * SEM_NOALLOC_SCRATCH_BYTES bytes, held on every GPU that loads the library
 * until the process exits. A mesh whose partial sums need more
 * (partial-sum slots x element size) gets SEM_ERR_INVALID_ARG. The handle's device
 * data must exist already (after sem_step, sem_set_state or
 * sem_apply_stiffness), else SEM_ERR_STATE. The first call on a device looks
 * up the scratch array's device address (cudaGetSymbolAddress); make that
 * first call before any stream capture. All calls share the one scratch
 * array: calls that may overlap on the GPU (different streams, handles or
 * threads) race on it. Every scratch value a call reads was written earlier
 * in the same call, so nothing needs clearing between calls. A bounded wait
 * that gave up is reported as for sem_apply_stiffness, at the next call that
 * reads back. */
#define SEM_NOALLOC_SCRATCH_BYTES (16u << 20)
sem_status sem_apply_stiffness_dev_noalloc(sem_mesh* m, const void* dev_u, void* dev_Ku);

/* Batched shots (many independent simulations advanced together). A batch
 * groups mesh handles that are configured (model and dt set; source and
 * receivers optional) with the same precision and stream; each keeps its own
 * mesh, order, ordering, model and state, and is read back with the usual
 * per-handle calls. The paper runs one simulation at a time; batching is the
 * serving-style use of the same time step.
 *   shots[nshots]   handles (distinct); the batch does not own them and must
 *                   be destroyed before any of them.
 *   autotune_steps  0: keep each handle's block size. > 0: for each order, the
 *                   not yet built handle whose element count is closest to
 *                   65,536 is timed for this many steps (20 or more give
 *                   stable choices) with each candidate elements-per-block
 *                   (48..256; the threads of a block follow: one per element,
 *                   whole warps), as one streamed launch where the handle can
 *                   stream (the way a streamed batch runs it), and every
 *                   not yet built handle of that order without its own
 *                   sem_set_tuning uses the fastest (the timed handle is then
 *                   rebuilt from its initial state).
 * Returns SEM_ERR_STATE if a handle lacks model or dt or the precisions or
 * streams differ, SEM_ERR_UNSUPPORTED for a handle with a stored FP32 metric
 * (sem_set_metric). */
typedef struct sem_batch sem_batch;
sem_status sem_batch_create(sem_mesh* const* shots, int32_t nshots, int32_t autotune_steps, sem_batch** out);

/* Advance every shot nsteps leapfrog steps. Clock-driven batch (every shot on
 * a DENSE plan with at most 16 neighbour blocks per block, as Hilbert and
 * row-major orderings give, and at least one order class streaming; see
 * sem_batch_set_stream): per polynomial order present, a streamed class runs a
 * block of 64 steps as one launch over the element blocks of all shots of
 * that order, one CTA per (step, block) unit taken from a work counter, each
 * unit waiting (bounded) for the previous step at the blocks of its own shot
 * that share a node with it (as sem_set_stream does for one mesh); a class
 * that does not stream runs 64 launches of one step each; the launches of
 * all orders and the update of the shots' clocks after them are captured
 * once as a CUDA graph and replayed, the remainder launched directly.
 * Otherwise each step is one launch per order plus a step-counter update,
 * with a 16-step graph. After
 * the last step each shot's open nodes are completed as by sem_step. The
 * first call builds the shots' device data. Results equal those of sem_step
 * on each handle with the same block size, bit for bit. A streamed wait that
 * gives up (which no correct run does) makes the call return
 * SEM_ERR_TIMEOUT. Synchronises the stream at the start (state upload) and
 * at the end of a streamed call (its error flag). */
sem_status sem_batch_step(sem_batch* b, int64_t nsteps);

/* After the first sem_batch_step: number of order classes, and per class its
 * polynomial order, elements per block (the largest in the class) and element
 * blocks per step (the CTAs of one step; any output may be NULL; arrays hold
 * nclasses entries). */
sem_status sem_batch_info(const sem_batch* b, int32_t* nclasses, int32_t* orders, int32_t* elems_per_block,
                          int32_t* ctas);

/* Which order classes stream, before the first sem_batch_step: -1 (the
 * default) streams a class where one step of it has fewer element blocks than
 * 8 times the CTAs resident at once (the upper bound of the rule
 * sem_set_stream(-1) applies to one mesh; a class with less than one wave
 * streams too, since its shots share the launch) and runs the others one
 * launch per step inside the same captured
 * block; 1 streams every class; 2 streams none but keeps the captured
 * 64-step blocks with steps taken from the shots' clocks; 0 none (one launch
 * per class and step with step counters, 16-step graphs: the scheme for
 * GATHER plans). SEM_ERR_STATE after the first step. */
sem_status sem_batch_set_stream(sem_batch* b, int mode);

/* After the first sem_batch_step: streamed = the number of order classes
 * running streamed launches (see sem_batch_step); steps_per_launch = the
 * steps of one captured block of the clock-driven path (64), 1 when the
 * batch runs one launch per class and step with step counters. Either
 * output may be NULL. */
sem_status sem_batch_mode(const sem_batch* b, int32_t* streamed, int32_t* steps_per_launch);

/* Message of the last failing batch call ("" if none). Never NULL. */
const char* sem_batch_last_error(const sem_batch* b);

/* Free the batch (not its handles). NULL is a no-op. */
void sem_batch_destroy(sem_batch* b);

/* L2 trace misfit and its gradient with respect to the per-element wave
 * speeds, by the discrete adjoint of the leapfrog time step (the paper has no
 * adjoint; the speed enters the scheme only through the lumped mass of
 * Eq. Abar with M = 1/K, K = rho c^2).
 *   d_obs[nrec][nsteps]  observed traces, receiver-major, host array;
 *   misfit               J = 1/2 sum_r sum_n (d_r^n - d_obs[r][n])^2 dt, where
 *                        d_r^n = u^{n+1} at receiver r (as sem_read_traces);
 *   grad_vel[ne]         dJ/dc_e, original element order (NULL: misfit only).
 * The run starts from rest (u^0 = u^-1 = 0) with the handle's source; the
 * adjoint lambda^m = 2 lambda^{m+1} - lambda^{m+2} - s (K lambda^{m+1} +
 * g^m / dt^2), g^m = dt (d^{m-1} - d_obs^{m-1}) at the receivers, runs backward
 * from lambda^{N+1} = lambda^{N+2} = 0 and dJ/dc_e = -(2/c_e) sum_q w_q |J_q| /
 * (rho_e c_e^2) sum_{m} lambda^m (u^m - 2 u^{m-1} + u^{m-2}) at the element's
 * nodes. Forward states are kept as checkpoints every checkpoint_every steps
 * (0 = ceil(sqrt(nsteps))) and recomputed one segment at a time on the way
 * back (sqrt(T) memory). Needs receivers with max_steps >= nsteps; SEM_FP64 or
 * SEM_FP32 handles (SEM_FP32_KAHAN returns SEM_ERR_UNSUPPORTED). Leaves the
 * handle at step nsteps of the forward run. Synchronises. */
sem_status sem_misfit_gradient(sem_mesh* m, const double* d_obs, int64_t nsteps, int64_t checkpoint_every,
                               double* misfit, double* grad_vel);

/* Message of the last failing call on this handle ("" if none). Never NULL. */
const char* sem_last_error(const sem_mesh* m);

/* Free the handle and all its device memory. NULL is a no-op. */
void sem_destroy(sem_mesh* m);

#ifdef __cplusplus
}
#endif
#endif /* SEM_H */
