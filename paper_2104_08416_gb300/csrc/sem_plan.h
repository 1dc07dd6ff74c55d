// Block plan layout shared by the host builder (sem_host.cpp) and the CUDA
// kernels (sem_kernels.cu). Plain C++; compiled by g++ and nvcc.
//
// Elements, in the chosen memory order, are cut into blocks of `eb`
// consecutive elements; one CTA owns one block per step, one thread per
// element. Inside a block every distinct global node is an "entry". An entry
// is CLOSED when all element slots of its node lie in the block (the block
// finishes the node), else OPEN (the block writes a partial sum; partial sums
// of a node are added in ascending block order by whichever kernel finishes
// the node).
//
// Assembly is a colour-ordered scatter: the elements of a block are coloured
// so that two elements of one colour share no node, and sorted by colour
// inside the block (stable, so the block keeps its element set and the
// memory order keeps its locality). The threads of colour c add their
// element residuals into shared-memory accumulators in phase c; no two
// threads touch one accumulator in a phase, and every node sums its slots in
// the same fixed order on every run: no atomics, bitwise reproducible.
//
// Shared-memory positions. DENSE plans (node ids numbered by first touch
// along the element order, which the node procedure of Section 4.3
// produces): the nodes first touched by block b are the id range
// [own_start, own_start + nown); entry l < nown is node own_start + l at
// position off + l, where off = own_start % vec, so the owned range is copied
// with 16-byte vectors lined up with global memory (vec = node values per 16
// bytes); the block's other ("halo", always open) nodes follow at positions
// ulen.. with ulen = round_up(off + nown, vec). Position p < ulen holds node
// abase + p with abase = own_start - off. GATHER plans (any numbering):
// nown = ulen = 0 and position p is entry p. slen (the positions whose
// update state is staged) is ulen for DENSE and the entry count for GATHER;
// every closed entry lies below slen.
//
// Per-block packet (one 16-byte aligned run of bytes, copied to shared memory):
//   cmask  u32[(sulen + 31) / 32]  bit p set: position p is a closed entry
//   egid   i32[sulen - ulen]       node ids of positions ulen..
//   obase  i32[nopen]              first partial-sum slot of open entry o's node
//   opos   u16[nopen]              position of open entry o
//   ocnt   u8[nopen]               blocks touching that node (= its partials)
//   orank  u8[nopen]               this block's rank among them (0 = owner)
//   cstart u16[ncolors + 1]        first thread (element) of each colour
//   recs   i32[2 * nrec]           receiver records (position, receiver):
//                                  closed entries first, then open entries
//                                  this block owns
// Element-side data (global, element-fastest in the device element order so
// that a thread per element reads it coalesced): epos u32[(P+1)/2][ne], two
// u16 positions per word (slot 2h in the low half); coef float4[2][ne] (FP32
// bilinear map); G f64[3P][ne] (FP64 stored metric).
#pragma once
#include <cstdint>

#if defined(__CUDACC__)
#define SEMPLAN_HD __host__ __device__ __forceinline__
#else
#define SEMPLAN_HD inline
#endif

namespace semplan {

constexpr int MAX_BLOCKS_PER_NODE = 255;
constexpr int MAX_COLORS = 32;

// Header of block b: 12 int32 (read as three int4 on the device).
enum HeaderField : int {
    H_START = 0,      // packet start / 16
    H_NENT = 1,       // entries
    H_NOWN = 2,       // owned entries (DENSE), 0 for GATHER
    H_OWN_START = 3,  // first owned node id (DENSE), 0 for GATHER
    H_NOPEN = 4,      // open entries
    H_ULEN = 5,       // aligned owned-range length (DENSE), 0 for GATHER
    H_SLEN = 6,       // staged-state length: ulen (DENSE) or nent (GATHER)
    H_SULEN = 7,      // node-value positions: ulen + entries beyond the owned ones
    H_NCOLORS = 8,    // colours of the block's elements
    H_NREC_CLOSED = 9,
    H_NREC_OPEN = 10,
    H_RESERVED = 11
};
constexpr int HDR_INTS = 12;

struct Offsets {
    int cmask, egid, obase, opos, ocnt, orank, cstart, recs, bytes;
};

SEMPLAN_HD int align_to(int v, int a) { return (v + a - 1) / a * a; }

SEMPLAN_HD Offsets offsets(int sulen, int ulen, int nopen, int ncolors, int nrec_total) {
    Offsets L;
    L.cmask = 0;
    L.egid = L.cmask + 4 * ((sulen + 31) / 32);
    L.obase = L.egid + 4 * (sulen - ulen);
    L.opos = L.obase + 4 * nopen;
    L.ocnt = L.opos + 2 * nopen;
    L.orank = L.ocnt + nopen;
    L.cstart = align_to(L.orank + nopen, 2);
    L.recs = align_to(L.cstart + 2 * (ncolors + 1), 4);
    L.bytes = align_to(L.recs + 8 * nrec_total, 16);
    return L;
}

SEMPLAN_HD int entry_pos(int l, int nown, int off, int ulen) { return l < nown ? off + l : ulen + (l - nown); }

}  // namespace semplan
