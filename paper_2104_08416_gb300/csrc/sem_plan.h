// Block plan layout shared by the host builder (sem_host.cpp) and the CUDA
// kernels (sem_kernels.cu). Plain C++; compiled by g++ and nvcc.
//
// Elements, in the chosen memory order, are cut into blocks of `eb`
// consecutive elements; one CTA owns one block per step. Inside a block every
// distinct global node is an "entry". An entry is CLOSED when all element
// slots of its node lie in the block (the block finishes the node), else OPEN
// (the block writes a partial sum; partial sums of a node are added in
// ascending block order by whichever kernel finishes the node).
//
// Entry order and shared-memory positions. DENSE plans (node ids numbered by
// first touch along the element order, which the node procedure of Section
// 4.3 produces): the nodes first touched by block b are the id range
// [own_start, own_start + nown); entries 0..nown-1 are those nodes in id
// order, entries nown.. the block's other nodes ("halo", always open) in
// order of first appearance. GATHER plans (any numbering): nown = 0 and all
// entries in order of first appearance. Node values of entry l sit in shared
// memory at pos(l) = l < nown ? off + l : ulen + (l - nown), where
// off = own_start % vec and ulen = round_up(off + nown, vec) (both 0 for
// GATHER), so the owned range is copied with 16-byte vectors that line up with
// global memory (vec = node values per 16 bytes).
//
// Per-block packet (one 16-byte aligned run of bytes, copied to shared memory):
//   lsl   u16[nslot]    slots of each entry (slot = element * P + point),
//                       ascending, entry after entry (local CSR)
//   lrow  u16[nent + 1] CSR offsets into lsl
//   aux   u16[nent]     CLOSED, or the entry's open rank o
//   egid  i32[nent - nown] node ids of entries nown.. (4-byte aligned)
//   obase i32[nopen]    first partial-sum slot of the node of open entry o
//   oent  u16[nopen]    entry of open rank o
//   ocnt  u8[nopen]     number of blocks touching that node (= its partials)
//   orank u8[nopen]     this block's rank among them (0 = owner)
//   recs  i32[2 * (nrec_closed + nrec_open)] receiver records (4-byte
//                       aligned): (entry, receiver) for closed entries, then
//                       (open rank, receiver) for open entries this block owns
// Element-side data (global, element-fastest so a thread per element reads it
// coalesced): epos u32[(P+1)/2][ne], two u16 positions per word (slot 2h in
// the low half); coef float4[2][ne] (FP32 bilinear map); G f64[3P][ne]
// (FP64 stored metric).
#pragma once
#include <cstdint>

#if defined(__CUDACC__)
#define SEMPLAN_HD __host__ __device__ __forceinline__
#else
#define SEMPLAN_HD inline
#endif

namespace semplan {

constexpr uint16_t CLOSED = 0xFFFF;
constexpr int MAX_BLOCKS_PER_NODE = 255;

// Header of block b: 8 int32 (read as two int4 on the device).
enum HeaderField : int {
    H_START = 0,      // packet start / 16
    H_NENT = 1,       // entries
    H_NOWN = 2,       // owned entries (DENSE), 0 for GATHER
    H_OWN_START = 3,  // first owned node id (DENSE), 0 for GATHER
    H_NOPEN = 4,      // open entries
    H_ULEN = 5,       // aligned owned-range length (DENSE), 0 for GATHER
    H_SLEN = 6,       // staged-state length: ulen (DENSE) or nent (GATHER)
    H_NREC = 7        // (closed receivers << 16) | owned open receivers
};
constexpr int HDR_INTS = 8;

struct Offsets {
    int lsl, lrow, aux, egid, obase, oent, ocnt, orank, recs, bytes;
};

SEMPLAN_HD int align_to(int v, int a) { return (v + a - 1) / a * a; }

SEMPLAN_HD Offsets offsets(int nslot, int nent, int nown, int nopen, int nrec_total) {
    Offsets L;
    L.lsl = 0;
    L.lrow = L.lsl + 2 * nslot;
    L.aux = L.lrow + 2 * (nent + 1);
    L.egid = align_to(L.aux + 2 * nent, 4);
    L.obase = L.egid + 4 * (nent - nown);
    L.oent = L.obase + 4 * nopen;
    L.ocnt = L.oent + 2 * nopen;
    L.orank = L.ocnt + nopen;
    L.recs = align_to(L.orank + nopen, 4);
    L.bytes = align_to(L.recs + 8 * nrec_total, 16);
    return L;
}

SEMPLAN_HD int entry_pos(int l, int nown, int off, int ulen) { return l < nown ? off + l : ulen + (l - nown); }

}  // namespace semplan
