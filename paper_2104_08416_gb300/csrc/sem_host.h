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
void element_order_hilbert(const Mesh& m, std::vector<int64_t>& order);
void node_degrees(const Mesh& m, std::vector<int32_t>& deg);
void renumber_nodes(const Mesh& m, const std::vector<int64_t>& elem_order,
                    const std::vector<int32_t>& deg, std::vector<int64_t>& node_order);
void random_order(int64_t n, uint64_t seed, std::vector<int64_t>& order);
// kind: 0 none, 1 rowmajor, 2 random, 3 hilbert.
void orderings(const Mesh& m, int kind, uint64_t seed, std::vector<int64_t>& elem_order,
               std::vector<int64_t>& node_order);

// Nearest global node (original id) to (x, y), ties to the lowest id.
int64_t snap(const std::vector<double>& node_xy, double x, double y);

// CFL step (see sem_cfl_dt in sem.h) for per-element speeds vel[ne].
double cfl_dt(const Mesh& m, const double* vel);

// Block plan for deterministic assembly. Elements (in the new order) are cut
// into blocks of `eb` consecutive elements. Inside a block each touched
// global node is an "entry"; element slots point at their entry (lidx) and
// each entry lists its slots (a local CSR, slots ascending). An entry is
// closed when every slot of its node lies in this block: the block finishes
// that node by itself. Closed entries come first (in order of first
// appearance), then open ones; open entry k of block b writes its partial sum
// to partial[pbase_b + k], and the open-node pass adds the partials of each
// open node in ascending block order.
//
// Everything a block reads besides node values is one contiguous, 16-byte
// aligned "packet" (copied to shared memory in one go):
//   lidx  u16[nslot]      entry of each slot
//   lsl   u16[nslot]      slots of each entry (local CSR)
//   lrow  u16[nent + 1]   local CSR offsets
//   gid   i32[nent]       node id of each entry (4-byte aligned)
//   coef  f32[neb][8]     bilinear-map coefficients (16-byte aligned; filled
//                         on the device)
// with the offsets given by packet_layout().
struct PacketLayout {
    int64_t lidx, lsl, lrow, gid, coef, bytes;
};
PacketLayout packet_layout(int64_t nslot, int64_t nent, int64_t neb);

struct BlockPlan {
    int eb = 0;
    int64_t nblocks = 0;
    int max_entries = 0;                 // largest entry count of a block
    int64_t max_packet = 0;              // largest packet (bytes)
    std::vector<uint8_t> packet;         // all packets, block after block
    std::vector<int32_t> hdr;            // [nblocks][4]: packet start / 16, nent, nclosed, pbase
    std::vector<int32_t> open_gid;       // [nopen] ascending
    std::vector<int32_t> open_ptr;       // [nopen+1] into open_src
    std::vector<int32_t> open_src;       // [npartial] partial index of each contribution
    int64_t npartial = 0;
    int64_t nent_total = 0, nclosed_total = 0;
};
// conn_new: [ne][P] new node ids, elements in the new order.
void build_block_plan(const std::vector<int32_t>& conn_new, int64_t ne, int P, int64_t nn, int eb,
                      BlockPlan& plan);

}  // namespace semhost
