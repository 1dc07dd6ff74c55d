// Host-side preprocessing of the spectral-element stepper (C++17, no CUDA).
//
// Everything here runs once per mesh: validation, the canonical numbering of
// the SEM nodes (Section 4.2, mu(p, e)), the generalized Hilbert curve and
// the element / node reorderings of Section 4.3, and the "block plan" that
// the device kernels use for deterministic, atomic-free assembly.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "sem_plan.h"

namespace semhost {

struct Mesh {
    int p = 0;                      // polynomial order
    int np = 0;                     // p + 1
    int P = 0;                      // (p + 1)^2 points per element
    int64_t nv = 0, ne = 0, nn = 0; // vertices, elements, global nodes
    std::vector<double> coords;     // [nv][2]
    std::vector<int32_t> quads;     // [ne][4]
    std::vector<int32_t> conn;      // [ne][P] canonical (original) node ids
    std::vector<int64_t> edge_lo, edge_hi, edge_first;  // canonical edges
};

// GLL nodes (ascending, exact endpoints, symmetric) and weights of order p.
void gll_rule(int p, std::vector<double>& x, std::vector<double>& w);
// D[i][j] = l_j'(x_i) (row-major, (p+1)^2 values).
void gll_derivative(const std::vector<double>& x, std::vector<double>& D);

// Checks indices, vertex use, edge multiplicity and positive Jacobians at the
// GLL points. Returns "" when valid, else the reason.
std::string validate(const double* coords, int64_t nv, const int32_t* quads, int64_t ne, int p);

// Canonical numbering (see sem.h). Fills m.conn, m.nn and the edge table.
void number_nodes(Mesh& m);
// Positions of all global nodes in original order, [nn][2].
void node_coordinates(const Mesh& m, std::vector<double>& xy);

// Generalized Hilbert curve over W x H cells: (x, y) of each visited cell.
void hilbert_cells(int64_t W, int64_t H, std::vector<int32_t>& cells);

// Orderings as order arrays (order[new] = old id).
// (Returns "" or why the curve grid cannot be built.)
std::string element_order_hilbert(const Mesh& m, std::vector<int64_t>& order, bool wide = false);
void node_degrees(const Mesh& m, std::vector<int32_t>& deg);
void renumber_nodes(const Mesh& m, const std::vector<int64_t>& elem_order,
                    const std::vector<int32_t>& deg, std::vector<int64_t>& node_order);
void random_order(int64_t n, uint64_t seed, std::vector<int64_t>& order);
// kind: 0 none, 1 rowmajor, 2 random, 3 hilbert, 4 node connectivity,
// 5 node distance (Section 6.1's strategies), 6 hilbert with the wide
// bounding box of Section 4.3. Returns "" or why the ordering cannot be built.
std::string orderings(const Mesh& m, int kind, uint64_t seed, std::vector<int64_t>& elem_order,
                      std::vector<int64_t>& node_order);

// Nearest global node (original id) to (x, y), ties to the lowest id.
int64_t snap(const std::vector<double>& node_xy, double x, double y);
// The same for nq points (qx[k * stride], qy[k * stride]) in one pass.
void snap_many(const std::vector<double>& node_xy, const double* qx, const double* qy, int64_t nq, int64_t stride,
               std::vector<int64_t>& out);

// CFL step (see sem_cfl_dt in sem.h) for per-element speeds vel[ne].
double cfl_dt(const Mesh& m, const double* vel);

// Block plan for deterministic, atomic-free assembly (layout and terms in
// sem_plan.h). conn: [ne][P] new node ids, elements in the new (memory)
// order. rec_gid: new node id of each receiver whose trace the kernels record,
// -1 for none. vec: node values per 16 bytes (4 FP32, 2 FP64). allow_dense:
// use the DENSE layout when the numbering permits it. The plan's device
// element order (dev_order[i] = index into conn of the element that thread i
// of block i / eb handles) is the memory order with each block sorted by
// colour; all element-side device data follows it.
struct BlockPlan {
    int eb = 0;
    int P = 0;
    bool dense = false;
    int64_t ne = 0, nn = 0, nblocks = 0;
    int max_entries = 0;                 // largest entry count of a block
    int max_sulen = 0;                   // largest node-value position count
    int max_slen = 0;                    // largest staged-state length
    int max_packet = 0;                  // largest packet (bytes)
    int max_colors = 0;                  // most colours in a block
    std::vector<int64_t> dev_order;      // [ne] device element order
    std::vector<uint8_t> packet;         // all packets, block after block
    std::vector<int32_t> hdr;            // [nblocks][HDR_INTS]
    std::vector<uint32_t> epos;          // [(P+1)/2][ne] packed positions, device element order
    // open nodes (touched by more than one block), ascending id, for the
    // kernels that finish them outside the step kernel
    std::vector<int32_t> open_gid, open_base, open_cnt, open_rec;
    int64_t npartial = 0;                // partial-sum slots (sum of open_cnt)
    int64_t nent_total = 0, nclosed_total = 0, nopen_entries = 0;
    // neighbours of each block: the blocks sharing a node with it, itself
    // included, ascending (CSR: dep[dep_ptr[b] .. dep_ptr[b+1]))
    std::vector<int32_t> dep_ptr, dep;
    int max_deps = 0;
};
// Returns "" on success, else why the plan cannot be built (a limit of the
// 16-bit / 8-bit fields or of the colour count exceeded).
std::string build_block_plan(const std::vector<int32_t>& conn, int64_t ne, int P, int64_t nn, int eb,
                             bool allow_dense, int vec, const std::vector<int32_t>& rec_gid, BlockPlan& plan);

// Host emulation of one step-kernel assembly plus the open-node pass over the
// plan, with every index bounds-checked, on integer-valued element residuals
// r[e][q] = u[conn[e][q]] + (e mod 7) * (q + 1) so that sums are exact:
// every slot must read its own node's value through epos, no two elements of
// one colour may share a node, and the assembled result must equal the direct
// per-slot sum. Returns "" when the plan is consistent, else the first
// violation.
std::string check_block_plan(const BlockPlan& plan, const std::vector<int32_t>& conn, int vec);

// Order of the streamed time loop's units over a band of T consecutive steps
// (unit (j, b): step j of the band at element block b). It carries Section
// 4.3's locality argument across time steps: instead of every block of step j
// before any block of step j+1 (which puts a whole step's data, more than the
// L2, between a block's two visits), units follow a wavefront over the block
// graph (blocks adjacent when they share a node). Each block gets a level, its
// breadth-first distance from a pseudo-peripheral block of its connected part
// (the far end of a first sweep), so that adjacent blocks' levels differ by at
// most one. Units are emitted by tile t = floor((level + j) / W), then step j,
// then level, then block id. A unit's dependencies, step j-1 at the block and
// at its neighbours, have level + j - 1 <= level + 1 + j - 1, hence a tile no
// later and an earlier step: the order is topological, which the streamed
// loop needs for its waits to end. A block's next step follows after about W
// levels' worth of units. Entry = (j << kSchedShift) | b.
constexpr int kSchedShift = 24;
constexpr int kSchedMaxSteps = 255;
// levels[nb] as above.
std::vector<int32_t> block_levels(const int32_t* dep_ptr, const int32_t* dep, int64_t nb);
// Window W (levels per tile) giving about target_units units per step of a
// tile: target_units over the mean number of blocks per level, at least 1.
int auto_window(const std::vector<int32_t>& levels, int64_t target_units);
// sched[T * nb]; "" on success, else why no schedule can be built.
std::string stream_schedule(const int32_t* dep_ptr, const int32_t* dep, int64_t nb, int T, int W,
                            std::vector<uint32_t>& sched, std::vector<int32_t>* levels_out);
// Checks that sched holds every unit of the band once and that every unit
// comes after step j-1 of each block in its neighbour list (itself
// included). "" when valid, else the first violation.
std::string check_stream_schedule(const int32_t* dep_ptr, const int32_t* dep, int64_t nb, int T,
                                  const std::vector<uint32_t>& sched);

}  // namespace semhost
