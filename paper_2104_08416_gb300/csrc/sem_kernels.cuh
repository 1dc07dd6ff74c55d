// Device-side interface of the spectral-element stepper (sm_103a).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace semdev {

constexpr int MAX_NP = 9;  // orders 1..8

// Per-order GLL tables passed by value to the kernels (kernel-parameter
// space is a broadcast constant bank, so every thread reads them cheaply).
template <typename T>
struct Basis {
    T D[MAX_NP * MAX_NP];  // D[i*np + k] = l_k'(x_i)
    T w[MAX_NP];           // GLL weights
    T x[MAX_NP];           // GLL nodes
};

// Block plan on the device (see semhost::BlockPlan): per-block packets and
// headers (packet start / 16, entries, closed entries, first partial slot),
// and the open-node lists.
struct Plan {
    const uint8_t* packet;
    const int4* hdr;
    const int32_t* open_gid;
    const int32_t* open_ptr;
    const int32_t* open_src;
    const int32_t* open_rec;   // receiver index of an open node, or -1 (may be null)
    int64_t ne;
    int eb;
    int nblocks;
    int nopen;
    int max_entries;
    int max_packet;
};

// Packet layout, identical to semhost::packet_layout.
struct PacketOffsets {
    int lidx, lsl, lrow, gid, coef, bytes;
};
__host__ __device__ inline PacketOffsets packet_offsets(int nslot, int nent, int neb) {
    PacketOffsets L;
    L.lidx = 0;
    L.lsl = 2 * nslot;
    L.lrow = 4 * nslot;
    L.gid = (L.lrow + 2 * (nent + 1) + 3) / 4 * 4;
    L.coef = (L.gid + 4 * nent + 15) / 16 * 16;
    L.bytes = (L.coef + 32 * neb + 15) / 16 * 16;
    return L;
}

enum Mode : int {
    MODE_THREE_LEVEL = 0,  // u^{n+1} = 2u^n - u^{n-1} + s (f e_src - K u^n)
    MODE_KAHAN = 1,        // delta += s (f e_src - K u); u += delta, Kahan-compensated
    MODE_APPLY = 2         // out = K u
};

// Geometry of the stiffness: either the per-point metric
// G_q = w_q |J_q| / rho_e * J_q^-1 J_q^-T stored as three arrays [3][ne*P]
// (Gxx, Gxy, Gyy), or the element's bilinear-map coefficients (b, c, d) and
// 1/rho from which the metric is formed at each point.
template <typename T>
struct StepArgs {
    const T* u_cur;        // u^n
    T* u_out;              // u^{n+1} (three-level: the u^{n-1} buffer, overwritten)
    const T* u_prev;       // u^{n-1} (three-level only)
    T* delta;              // Kahan mode: u^{n+1/2} increment
    T* comp;               // Kahan mode: compensation
    const T* s;            // dt^2 / M per node
    T* partial;            // partial sums of open nodes
    const T* G;            // stored metric [3][gstride] or null
    int64_t gstride;       // ne * P
    T* apply_out;          // MODE_APPLY output
    const double* src_f;   // Ricker table f(t_n)
    int64_t step;          // n
    int32_t src_gid;       // source node (new id) or -1
    const int32_t* rec_gid;  // receivers (new ids)
    const uint8_t* rec_closed;
    int32_t nrec;
    double* trace;         // [nrec][trace_cap]
    int64_t trace_cap;
};

// Launchers. Return cudaSuccess or the launch error.
cudaError_t launch_step(int np, bool fp64, int mode, bool bilinear, const Plan& plan, const void* args,
                        const void* basis, int smem_bytes, cudaStream_t st);
cudaError_t launch_open(bool fp64, int mode, const Plan& plan, const void* args, cudaStream_t st);

// One-time FP64 precompute: per element (new order) from the corner
// coordinates: the bilinear coefficients (FP32), the stored metric (FP64 or
// FP32, when G_out is non-null), and w_q |J_q| / (rho c^2) per slot.
cudaError_t launch_geometry(int np, const double* coords, const int32_t* quads_new, const double* rho,
                            const double* vel, const Plan& plan, const Basis<double>& basis, uint8_t* packet,
                            double* G64, double* mloc, cudaStream_t st);
// Lumped mass through the block plan (deterministic), M[nn] in FP64.
cudaError_t launch_mass(const Plan& plan, int P, const double* mloc, double* partial, double* M,
                        cudaStream_t st);
// s = dt^2 / M (FP64 arithmetic, rounded once to the storage type).
cudaError_t launch_scale(const double* M, int64_t nn, double dt, double* s64, float* s32, cudaStream_t st);

int smem_bytes_for(int P, int eb, int max_entries, int max_packet, bool fp64, int mode);
// Element lanes of the block kernel: elements processed side by side, one
// thread per GLL point of each (blockDim = lanes * (p+1)^2).
int lanes_for(int np);

}  // namespace semdev
