// CUDA kernels of the spectral-element time step (sm_103a).
//
// One launch of sem_step_kernel per time step; one CTA per block of
// consecutive elements (in the chosen memory order), one thread per element:
//  A. the block's packet (local assembly lists) and its owned node range
//     (values and update state) are staged in shared memory with 16-byte
//     asynchronous copies; nodes shared with other blocks ("open") are
//     gathered, or, from the second step of a run on, finished to the current
//     level from the previous launch's partial sums (deferred assembly, see
//     StepArgs);
//  B. each thread gathers its element's (p+1)^2 values (the U_2 gather of
//     Algorithm 1) into registers, forms the reference gradient with the GLL
//     derivative matrix, applies the per-point metric G_q = w_q |J_q| / rho_e
//     J_q^-1 J_q^-T (Eq. deriv_u with K^(e) = J^-1, quadrature of Eq.
//     numerical_integ) and contracts with the transposed derivative (Eq.
//     u_change_r_effic, second-order form), all in registers; the residuals go
//     to shared memory;
//  C. the block assembles its entries through the local CSR lists in a fixed
//     order. Closed nodes get the inverse lumped mass (Eq. Abar), the point
//     source (Algorithm 3) and the leapfrog update on the spot; open nodes
//     leave one partial sum per block.
// sem_open_finish_kernel completes the open nodes after the last launch of a
// run. No floating-point atomics are used, so results are bitwise reproducible.
#include "sem_kernels.cuh"

#include <map>
#include <mutex>

namespace semdev {

namespace {

using namespace semplan;

constexpr int kThreads = 256;
constexpr int kMaxStepThreads = 256;
// Resident CTAs the compiler budgets registers for: three (80 registers a
// thread, a few spilled values) for FP32 up to order 4, where the extra
// resident warps outweigh the spills; one for larger elements and FP64.
#ifndef SEM_STEP_MINB
#define SEM_STEP_MINB 3
#endif
template <int NP, typename T>
constexpr int step_min_blocks() {
    return (sizeof(T) == 4 && NP <= 5) ? SEM_STEP_MINB : 1;
}

__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// One node update from level k to k+1: assembled stiffness ku, value un,
// state xn (u^{k-1} or delta^{k-1/2}) and cn (compensation), s = dt^2/M,
// source value f. Three-level: u' = (2u - u_prev) + s (f - ku). Kahan:
// delta' = delta + s (f - ku), u' = u + delta' as a Kahan-compensated sum.
// Every operation is an explicitly rounded intrinsic, so the step kernel and
// the open-node kernel produce bitwise the same update.
template <typename T, int MODE>
struct Update {
    T u, x, c;
};
template <typename T, int MODE>
__device__ __forceinline__ Update<T, MODE> update_node(T un, T xn, T cn, T sn, T f, T ku) {
    Update<T, MODE> o;
    const T acc = sub_rn(f, ku);
    if (MODE == MODE_THREE_LEVEL) {
        o.u = fma_rn(sn, acc, sub_rn(add_rn(un, un), xn));
        o.x = un;
        o.c = T(0);
    } else {
        const T d = fma_rn(sn, acc, xn);
        const T y = sub_rn(d, cn);
        const T t = add_rn(un, y);
        o.c = sub_rn(sub_rn(t, un), y);
        o.x = d;
        o.u = t;
    }
    return o;
}

// Sum of the cnt >= 2 partial sums of an open node, in ascending block
// order (the loads of the first four are issued together). Shared by every
// kernel that finishes open nodes, so they all round the same way.
template <typename T>
__device__ __forceinline__ T sum_partials(const T* __restrict__ p, int32_t pb, int cnt) {
    T v[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) v[t] = (t < cnt) ? __ldcg(p + pb + t) : T(0);
    T s = add_rn(v[0], v[1]);
    if (cnt > 2) s = add_rn(s, v[2]);
    if (cnt > 3) s = add_rn(s, v[3]);
    for (int t = 4; t < cnt; ++t) s = add_rn(s, __ldcg(p + pb + t));
    return s;
}

// Value recorded in a trace (FP64): the compensated sum u - c in Kahan mode.
template <typename T, int MODE>
__device__ __forceinline__ double trace_value(T u, T c) {
    return MODE == MODE_KAHAN ? (double)u - (double)c : (double)u;
}

// ---------------------------------------------------------- async copies
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
template <int BYTES>
__device__ __forceinline__ void cp_async_small(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gmem), "n"(BYTES) : "memory");
}
// Moves the 128-byte line holding p into L2 (no register, no wait).
__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];\n" ::"l"(p));
}
// A wait gives up once it has lasted kWaitNs of the GPU's global timer
// (read every 64 polls; a unit normally waits microseconds at most), or,
// whatever the timer says, after kWaitPolls polls (each followed by a
// 128 ns back-off, so at least 8.6 s of nominal sleep, for a flag; a bulk
// copy's barrier is polled with the hardware's own suspend hint instead).
constexpr unsigned long long kWaitNs = 1000000000ull;
constexpr int kWaitPolls = 1 << 26;
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}

// 1-D bulk copies (the TMA engine) into shared memory, completing on an
// mbarrier of the CTA: one thread issues them, every thread waits on the
// barrier's phase. Source and destination 16-byte aligned, size a multiple
// of 16 bytes. The barrier is initialised once per unit (arrival count 1:
// the issuing thread's arrive with the expected byte count).
__device__ __forceinline__ void bulk_g2s(void* smem, const void* gmem, unsigned bytes, unsigned mb) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                 ::"r"(sa), "l"(gmem), "r"(bytes), "r"(mb) : "memory");
}
__device__ __forceinline__ void mbar_init(unsigned mb) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb) : "memory");
    // the initialisation, and this thread's earlier shared-memory accesses,
    // ordered before the copies the async proxy performs
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect(unsigned mb, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mb), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned mb, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mb), "r"(parity)
        : "memory");
    return ok != 0;
}
// Waits for phase 0 of the barrier; false if it gave up (kWaitNs of the
// global timer, or kWaitPolls polls).
__device__ __forceinline__ bool mbar_wait(unsigned mb) {
    unsigned long long t0 = 0;
    for (int n = 0; !mbar_try(mb, 0); ++n) {
        if ((n & 63) == 63) {
            const unsigned long long now = global_ns();
            if (n == 63) t0 = now;
            if (now - t0 > kWaitNs || n >= kWaitPolls) return false;
        }
    }
    return true;
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Element data, read once per step: cached in L2 only (ld.global.cg
// measured 0.6 % faster than the evict-first L1 hint on the graded mesh).
__device__ __forceinline__ uint32_t ld_stream(const uint32_t* p) { return __ldcg(p); }
__device__ __forceinline__ float4 ld_stream(const float4* p) { return __ldcg(p); }
__device__ __forceinline__ double ld_stream(const double* p) { return __ldcs(p); }
__device__ __forceinline__ float ld_stream(const float* p) { return __ldcs(p); }

// 16-byte shared-memory vector of VEC values.
template <typename T, int VEC>
__device__ __forceinline__ void load_vec(T (&v)[VEC], const T* p) {
    const float4 w = *reinterpret_cast<const float4*>(p);
    const T* t = reinterpret_cast<const T*>(&w);
#pragma unroll
    for (int k = 0; k < VEC; ++k) v[k] = t[k];
}
// 16-byte global vector of VEC values (L2 only: it is read once).
template <typename T, int VEC>
__device__ __forceinline__ void load_global_vec(T (&v)[VEC], const T* p) {
    const float4 w = __ldcg(reinterpret_cast<const float4*>(p));
    const T* t = reinterpret_cast<const T*>(&w);
#pragma unroll
    for (int k = 0; k < VEC; ++k) v[k] = t[k];
}

// Stores the values whose bit is set; one 16-byte store when all are.
template <typename T, int VEC>
__device__ __forceinline__ void store_masked(T* g, const T (&v)[VEC], uint32_t bits) {
    if (bits == (1u << VEC) - 1u) {
        float4 w;
        T* t = reinterpret_cast<T*>(&w);
#pragma unroll
        for (int k = 0; k < VEC; ++k) t[k] = v[k];
        __stcg(reinterpret_cast<float4*>(g), w);
    } else {
#pragma unroll
        for (int k = 0; k < VEC; ++k)
            if ((bits >> k) & 1u) __stcg(g + k, v[k]);
    }
}

// Copies node values [abase, abase + len) of src (len a multiple of VEC,
// abase a multiple of VEC) to dst with 16-byte copies, element by element
// where the vector would cross the end nn or the arrays are not aligned.
template <typename T>
__device__ __forceinline__ void stage_range(T* dst, const T* src, int64_t abase, int len, int64_t nn, bool vec_ok,
                                            int tid, int nt) {
    constexpr int VEC = 16 / sizeof(T);
    const int nch = len / VEC;
    for (int ch = tid; ch < nch; ch += nt) {
        const int64_t g = abase + (int64_t)ch * VEC;
        if (vec_ok && g + VEC <= nn) {
            cp_async16(dst + ch * VEC, src + g);
        } else {
#pragma unroll
            for (int t = 0; t < VEC; ++t)
                if (g + t < nn) dst[ch * VEC + t] = __ldcg(src + g + t);
        }
    }
}

// Header fields of block b (three int4).
struct BlockHdr {
    int start, nent, nown, own_start, nopen, ulen, slen, sulen, ncolors, nrc, nro;
};
__device__ __forceinline__ BlockHdr load_hdr(const int4* hdr, int b) {
    const int4 h0 = hdr[3 * b], h1 = hdr[3 * b + 1], h2 = hdr[3 * b + 2];
    BlockHdr h;
    h.start = h0.x;
    h.nent = h0.y;
    h.nown = h0.z;
    h.own_start = h0.w;
    h.nopen = h1.x;
    h.ulen = h1.y;
    h.slen = h1.z;
    h.sulen = h1.w;
    h.ncolors = h2.x;
    h.nrc = h2.y;
    h.nro = h2.z;
    return h;
}

__device__ __forceinline__ bool is_closed(const uint32_t* cmask, int p) { return (cmask[p >> 5] >> (p & 31)) & 1u; }

// First-order node update of Heun's method: dU = s (K-side sum + f) with
// s = 1/M; predictor U~ = U + h dU (and dU kept), corrector
// U + h/2 (dU_pred + dU). ui is U (predictor) or U~ (corrector).
template <typename T, int MODE>
__device__ __forceinline__ T heun_node(const StepArgs<T>& a, int64_t g, T ui, T ksum, T f) {
    const T du = __ldcg(a.s + g) * add_rn(ksum, f);
    if (MODE == MODE_HEUN_P) {
        __stcg(a.u_d1 + g, du);
        return fma_rn((T)a.h, du, ui);
    }
    const T sum = add_rn(__ldcg(a.u_d1 + g), du);
    return fma_rn((T)(0.5 * a.h), sum, __ldcg(a.u_old + g));
}

// Element part of the first-order system (Section 4.2): dV = grad u / rho at
// each local node (Eq. v_change with F = I/rho, grad = J^-T grad_ref) and the
// element's share of R (Eq. u_change_r_effic with B = -I):
// -sum_q w_q |J_q| V_q . grad phi_p(x_q) = -(D^T W) with W = w adj(J) V
// (|J| J^-1 = adj(J)). V advances in place of the element (predictor or
// corrector); r receives the negated contraction.
template <int NP, typename T, int MODE>
__device__ __forceinline__ void heun_element(const Plan& pl, const StepArgs<T>& a, const Basis<T>& bs, int64_t e,
                                             const uint32_t* pw, float4 cf0, float4 cf1, const T* su, T* r) {
    constexpr int P = NP * NP;
    T u[P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
        u[q] = su[(pw[q / 2] >> (16 * (q & 1))) & 0xFFFFu];
        r[q] = T(0);
    }
    T bx, by, cx, cy, dx, dy, rinv;
    if constexpr (sizeof(T) == 4) {
        bx = cf0.x; by = cf0.y; cx = cf0.z; cy = cf0.w; dx = cf1.x; dy = cf1.y; rinv = cf1.z;
    } else {
        bx = __ldcs(pl.coef64 + 0 * pl.ne + e);
        by = __ldcs(pl.coef64 + 1 * pl.ne + e);
        cx = __ldcs(pl.coef64 + 2 * pl.ne + e);
        cy = __ldcs(pl.coef64 + 3 * pl.ne + e);
        dx = __ldcs(pl.coef64 + 4 * pl.ne + e);
        dy = __ldcs(pl.coef64 + 5 * pl.ne + e);
        rinv = __ldcs(pl.coef64 + 6 * pl.ne + e);
    }
    const T h = (T)a.h, h2 = (T)(0.5 * a.h);
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        const T eta = bs.x[j];
        const T j00 = bx + dx * eta, j10 = by + dy * eta;
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            const int q = j * NP + i;
            const T xi = bs.x[i];
            const T j01 = cx + dx * xi, j11 = cy + dy * xi;
            T dxi = T(0), deta = T(0);
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                dxi += bs.D[i * NP + k] * u[j * NP + k];
                deta += bs.D[j * NP + k] * u[k * NP + i];
            }
            const T rdet = T(1) / (j00 * j11 - j01 * j10);
            const T vdx = (j11 * dxi - j10 * deta) * rdet * rinv;    // (J^-T grad_ref u)_x / rho
            const T vdy = (j00 * deta - j01 * dxi) * rdet * rinv;
            const int64_t ix = (int64_t)q * pl.ne + e, iy = (int64_t)(P + q) * pl.ne + e;
            const T vx = __ldcs(a.v_in + ix), vy = __ldcs(a.v_in + iy);
            const T wq = bs.W[q];
            const T wxi = wq * (j11 * vx - j01 * vy);
            const T weta = wq * (j00 * vy - j10 * vx);
#pragma unroll
            for (int m = 0; m < NP; ++m) {
                r[j * NP + m] -= bs.D[i * NP + m] * wxi;
                r[m * NP + i] -= bs.D[j * NP + m] * weta;
            }
            if (MODE == MODE_HEUN_P) {
                __stcg(a.v_d1 + ix, vdx);
                __stcg(a.v_d1 + iy, vdy);
                __stcg(a.v_out + ix, fma_rn(h, vdx, vx));
                __stcg(a.v_out + iy, fma_rn(h, vdy, vy));
            } else {
                __stcg(a.v_out + ix, fma_rn(h2, add_rn(__ldcs(a.v_d1 + ix), vdx), __ldcs(a.v_old + ix)));
                __stcg(a.v_out + iy, fma_rn(h2, add_rn(__ldcs(a.v_d1 + iy), vdy), __ldcs(a.v_old + iy)));
            }
        }
    }
}

// The FP32 metric of Eq. deriv_u, G_q = w_q |J_q| / rho_e J_q^-1 J_q^-T =
// w_q / (rho_e |J_q|) adj(J_q) adj(J_q)^T, formed at a GLL point from the
// element's bilinear map x = a + b xi + c eta + d xi eta (coefficients b, c,
// d and 1/rho in cf0 = (bx, by, cx, cy), cf1 = (dx, dy, 1/rho, -)):
// J = [j00 j01; j10 j11] with j00, j10 depending on eta only (one row of
// points) and j01, j11 on xi only (one column). Every operation is an
// explicitly rounded intrinsic, so the step kernels and sem_read_metric's
// kernel form bitwise the same values.
struct BilCol {
    float j01, j11, cB;   // cB = j11^2 + j01^2
};
struct BilRow {
    float j00, j10, cA;   // cA = j10^2 + j00^2
};
__device__ __forceinline__ BilCol bil_col(const float4& cf0, const float4& cf1, float xi) {
    BilCol c;
    c.j01 = __fmaf_rn(cf1.x, xi, cf0.z);
    c.j11 = __fmaf_rn(cf1.y, xi, cf0.w);
    c.cB = __fmaf_rn(c.j11, c.j11, __fmul_rn(c.j01, c.j01));
    return c;
}
__device__ __forceinline__ BilRow bil_row(const float4& cf0, const float4& cf1, float eta) {
    BilRow r;
    r.j00 = __fmaf_rn(cf1.x, eta, cf0.x);
    r.j10 = __fmaf_rn(cf1.y, eta, cf0.y);
    r.cA = __fmaf_rn(r.j10, r.j10, __fmul_rn(r.j00, r.j00));
    return r;
}
// wr = w_q / rho_e
__device__ __forceinline__ void bil_metric(const BilRow& r, const BilCol& c, float wr, float& gxx, float& gxy,
                                           float& gyy) {
    const float det = __fmaf_rn(r.j00, c.j11, -__fmul_rn(c.j01, r.j10));
    const float kk = __fdividef(wr, det);
    gxx = __fmul_rn(kk, c.cB);
    gyy = __fmul_rn(kk, r.cA);
    gxy = -__fmul_rn(kk, __fmaf_rn(r.j10, c.j11, __fmul_rn(r.j00, c.j01)));
}

// The loaded inputs of one open entry whose node is finished in this unit
// (position, node, partial sums, previous-level state).
template <typename T>
struct OpenIn {
    T p[4];
    T u, x, c, s;
    int64_t g;
    int pos, pb, cnt;
    bool own;
};

// One block of one mesh, one CTA (the body of the step kernels).
// Called by every thread of a block after the loads that do not depend on
// the previous step (element data, packet) are issued and before the node
// state is read; returns false (the same in every thread) to abandon the
// block. The plain step kernel has nothing to wait for.
struct NoWait {
    __device__ __forceinline__ bool operator()() const { return true; }
};

// SG: FP32 kernels stream the stored metric (pl.G32, computed in FP64 and
// rounded once) instead of forming it from the bilinear map.
template <int NP, typename T, int MODE, bool SG = false, typename Ready = NoWait>
__device__ __forceinline__ void step_block(const Plan& pl, const StepArgs<T>& a, const Basis<T>& bs, const int b,
                                           unsigned char* smem_raw, const int64_t step, const int pend,
                                           const Ready& ready = Ready(), const BlockHdr* hpre = nullptr,
                                           unsigned long long* mbar_pre = nullptr) {
    constexpr int P = NP * NP;
    constexpr int UPH = (P + 1) / 2;
    constexpr bool HEUN = MODE == MODE_HEUN_P || MODE == MODE_HEUN_C;
    constexpr bool STATE = MODE == MODE_THREE_LEVEL || MODE == MODE_KAHAN;   // leapfrog state staged
    constexpr bool KAHAN = MODE == MODE_KAHAN;
    // FP32: metric from the bilinear map (or stored, SG); FP64: stored metric
    constexpr bool BIL = sizeof(T) == 4 && !SG;
    constexpr int VEC = 16 / sizeof(T);
    uint8_t* spk = smem_raw;
    T* su = reinterpret_cast<T*>(smem_raw + pl.max_packet);   // node values at the positions
    // DENSE plans read s, u^{k-1} or delta and the compensation straight
    // from global memory in phase C (contiguous, 16-byte loads one chunk
    // ahead) instead of staging them: less shared memory per block and
    // fewer copies in the staging round trip (reading delta there too
    // measured 3.5 % faster on the graded 512 x 512 mesh)
    const bool direct = pl.dense;
    T* ss = su + pl.sulen_pad;                                        // staged s
    T* sx = ss + (STATE && !direct ? pl.slen_pad : 0);                // staged u^{k-1} or delta (GATHER)
    T* sc = sx + (STATE && !direct ? pl.slen_pad : 0);                // staged compensation
    T* acc = sc + (KAHAN && !direct ? pl.slen_pad : 0);               // assembled K u at the positions

    const int tid = threadIdx.x, nt = blockDim.x;
    const BlockHdr h = hpre ? *hpre : load_hdr(pl.hdr, b);
    const int64_t e0 = (int64_t)b * pl.eb;
    const int neb = (int)min((int64_t)pl.eb, pl.ne - e0);
    const Offsets L = offsets(h.sulen, h.ulen, h.nopen, h.ncolors, h.nrc + h.nro);
    const int off = pl.dense ? h.own_start % VEC : 0;
    const int64_t abase = (int64_t)h.own_start - off;
    const bool has_el = tid < neb;
    // source values of this launch (the point source is one node)
    T f_now = T(0), f_prev = T(0);
    if ((STATE || HEUN) && a.src_gid >= 0) {
        f_now = (T)a.src_f[step];
        if (STATE && pend) f_prev = (T)a.src_f[step - 1];
    }
    const int64_t e = e0 + tid;
    // the element-array stride, opaque to the compiler: a kernel that runs
    // several blocks in a loop would otherwise compute the per-slot addresses
    // once, ahead of the loop, and hold them in registers throughout
    int64_t nes = pl.ne;
    asm volatile("" : "+l"(nes));

    // element-side data straight into registers (coalesced across threads)
    uint32_t pw[UPH];
    float4 cf0 = make_float4(0.f, 0.f, 0.f, 0.f), cf1 = cf0;
    if (has_el) {
#pragma unroll
        for (int k = 0; k < UPH; ++k) pw[k] = ld_stream(pl.epos + (int64_t)k * nes + e);
        if constexpr (BIL) {
            cf0 = ld_stream(pl.coef + e);
            cf1 = ld_stream(pl.coef + nes + e);
        }
    }

    // A1. packet, owned node range, zeroed accumulators. DENSE plans with
    // 16-byte aligned node arrays copy the packet and the owned range of u
    // with 1-D bulk copies issued by thread 0 (one instruction per range),
    // completing on two mbarriers (packet, u), so that the open entries'
    // loads can go out as soon as the packet is in, while u is still landing;
    // a caller may have issued the packet copy already (mbar_pre: the
    // streamed kernel does it while its neighbour wait is under way). Other
    // plans copy with 16-byte cp.async per thread.
    const bool bulk = pl.dense && a.vec_ok != 0;
    __shared__ __align__(8) unsigned long long s_mbar_own[2];
    unsigned long long* mbp = mbar_pre ? mbar_pre : s_mbar_own;
    const unsigned mbk = (unsigned)__cvta_generic_to_shared(mbp);
    const unsigned mbu = (unsigned)__cvta_generic_to_shared(mbp + 1);
    {
        const uint8_t* gpk = pl.packet + (int64_t)h.start * 16;
        if (bulk) {
            if (!mbar_pre && tid == 0) {
                mbar_init(mbk);
                mbar_init(mbu);
                mbar_arrive_expect(mbk, (unsigned)L.bytes);
                bulk_g2s(spk, gpk, (unsigned)L.bytes, mbk);
            }
        } else {
            for (int o = tid * 16; o < L.bytes; o += nt * 16) cp_async16(spk + o, gpk + o);
        }
        float4* az = reinterpret_cast<float4*>(acc);
        const int nz = (h.sulen * (int)sizeof(T) + 15) / 16;
        for (int k = tid; k < nz; k += nt) az[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (!ready()) {
            // the packet copy in flight completes before the CTA leaves
            if (bulk) {
                __syncthreads();
                mbar_wait(mbk);
            }
            cp_async_commit();
            cp_async_wait_all();
            return;
        }
        if (pl.dense) {
            if (bulk) {
                // the chunks wholly inside the array by one copy; the last
                // block's tail, if the array ends inside a chunk, by loads
                const int nchunk = h.ulen / VEC;
                const int64_t room = (pl.nn - abase) / VEC;
                const int nfull = (int)max((int64_t)0, min((int64_t)nchunk, room));
                if (tid == 0) {
                    const unsigned ub = (unsigned)nfull * 16u;
                    // u as other blocks' stores left it (made visible to this
                    // CTA by the neighbour wait or the launch boundary), ordered
                    // before the copy engine's reads
                    asm volatile("fence.proxy.async.global;\n" ::: "memory");
                    mbar_arrive_expect(mbu, ub);
                    if (ub) bulk_g2s(su, a.u_k + abase, ub, mbu);
                }
                for (int ch = nfull + tid; ch < nchunk; ch += nt) {
                    const int64_t g = abase + (int64_t)ch * VEC;
#pragma unroll
                    for (int t = 0; t < VEC; ++t)
                        if (g + t < pl.nn) su[ch * VEC + t] = __ldcg(a.u_k + g + t);
                }
            } else {
                stage_range(su, a.u_k, abase, h.ulen, pl.nn, false, tid, nt);
            }
            if (STATE) {
                // s, u^{k-1} or delta and the compensation, read in phase C
                // chunk by chunk: into L2 now, so that phase C's first loads
                // do not wait on DRAM (32 values per 128-byte line)
                const int nline = (h.slen * (int)sizeof(T) + 127) / 128;
                for (int l = tid; l < nline; l += nt) {
                    prefetch_l2(a.s + abase + (int64_t)l * (128 / sizeof(T)));
                    prefetch_l2(a.x_k + abase + (int64_t)l * (128 / sizeof(T)));
                    if (KAHAN) prefetch_l2(a.c_k + abase + (int64_t)l * (128 / sizeof(T)));
                }
            }
        }
        if (bulk) {
            // the barriers' initialisation seen by every thread (when this
            // block did it), then the packet; a copy that never completes
            // (the wait is bounded) abandons the unit and raises the error word
            if (!mbar_pre) __syncthreads();
            if (__syncthreads_or(!mbar_wait(mbk))) {
                if (tid == 0 && a.err) atomicExch(a.err, 1);
                if (pl.dense) mbar_wait(mbu);   // the copy of u in flight, bounded too
                return;
            }
        } else {
            cp_async_commit();
            cp_async_wait_all();
            __syncthreads();
        }
    }
    const uint32_t* cmask = reinterpret_cast<const uint32_t*>(spk + L.cmask);
    const int32_t* egid = reinterpret_cast<const int32_t*>(spk + L.egid);
    const int32_t* obase = reinterpret_cast<const int32_t*>(spk + L.obase);
    const uint16_t* opos = reinterpret_cast<const uint16_t*>(spk + L.opos);
    const uint8_t* ocnt = spk + L.ocnt;
    const uint8_t* orank = spk + L.orank;
    const uint16_t* cstart = reinterpret_cast<const uint16_t*>(spk + L.cstart);
    const int32_t* recs = reinterpret_cast<const int32_t*>(spk + L.recs);

    // A2. closed positions of GATHER plans; open entries
    if (!pl.dense) {
        for (int p = tid; p < h.slen; p += nt)
            if (is_closed(cmask, p)) {
                const int32_t g = egid[p];
                cp_async_small<sizeof(T)>(su + p, a.u_k + g);
                if (STATE) {
                    cp_async_small<sizeof(T)>(ss + p, a.s + g);
                    cp_async_small<sizeof(T)>(sx + p, a.x_k + g);
                    if (KAHAN) cp_async_small<sizeof(T)>(sc + p, a.c_k + g);
                }
            }
    }
    const bool pending = STATE && pend;
    bool staged_ok = true;
    if (!pending) {
        // level k stored whole: u^k at the open entries outside the staged
        // range (those inside it are staged)
        for (int o = tid; o < h.nopen; o += nt) {
            const int pos = opos[o];
            if (pos < h.ulen) continue;
            su[pos] = __ldcg(a.u_k + egid[pos - h.ulen]);
        }
        if (bulk) staged_ok = mbar_wait(mbu);
    } else {
        // two open entries per pass, every load of both issued before either
        // is used: one round trip per pass; the first pass's loads go out
        // before the wait for the staged u, which the finished values
        // overwrite
        auto fetch = [&](int o, OpenIn<T>& in) {
            in.pos = opos[o];
            in.g = in.pos < h.ulen ? abase + in.pos : (int64_t)egid[in.pos - h.ulen];
            in.pb = obase[o];
            in.cnt = ocnt[o];
            in.own = orank[o] == 0;
#pragma unroll
            for (int t = 0; t < 4; ++t) in.p[t] = (t < in.cnt) ? __ldcg(a.part_rd + in.pb + t) : T(0);
            in.u = __ldcg(a.u_km1 + in.g);
            in.x = __ldcg(a.x_km1 + in.g);
            in.c = KAHAN ? __ldcg(a.c_km1 + in.g) : T(0);
            in.s = __ldcg(a.s + in.g);
        };
        auto finish = [&](const OpenIn<T>& in) {
            // partial sums in ascending block order, as sum_partials adds them
            T ku = add_rn(in.p[0], in.p[1]);
            if (in.cnt > 2) ku = add_rn(ku, in.p[2]);
            if (in.cnt > 3) ku = add_rn(ku, in.p[3]);
            for (int t = 4; t < in.cnt; ++t) ku = add_rn(ku, __ldcg(a.part_rd + in.pb + t));
            const T f = (in.g == a.src_gid) ? f_prev : T(0);
            const Update<T, MODE> up = update_node<T, MODE>(in.u, in.x, in.c, in.s, f, ku);
            su[in.pos] = up.u;
            if (in.own) {
                __stcg(a.u_kw + in.g, up.u);
                if (KAHAN) {
                    __stcg(a.x_kw + in.g, up.x);
                    __stcg(a.c_kw + in.g, up.c);
                    if (!direct) sc[in.pos] = up.c;  // for a receiver record (the owner's entries are staged)
                }
            }
        };
        const int o0 = tid, o1 = tid + nt;
        OpenIn<T> in0, in1;
        if (o0 < h.nopen) fetch(o0, in0);
        if (o1 < h.nopen) fetch(o1, in1);
        if (bulk) staged_ok = mbar_wait(mbu);
        if (staged_ok) {
            if (o0 < h.nopen) finish(in0);
            if (o1 < h.nopen) finish(in1);
            for (int q0 = tid + 2 * nt; q0 < h.nopen; q0 += 2 * nt) {
                const int q1 = q0 + nt;
                fetch(q0, in0);
                if (q1 < h.nopen) fetch(q1, in1);
                finish(in0);
                if (q1 < h.nopen) finish(in1);
            }
        }
    }
    cp_async_commit();
    cp_async_wait_all();
    if (__syncthreads_or(!staged_ok)) {
        if (tid == 0 && a.err) atomicExch(a.err, 1);
        if (bulk) mbar_wait(mbu);   // once more (bounded) for the copy of u in flight
        return;
    }
    if (pending && h.nro > 0) {
        for (int k = tid; k < h.nro; k += nt) {
            const int pos = recs[2 * (h.nrc + k)], r = recs[2 * (h.nrc + k) + 1];
            // the owner's entries lie in the owned range (DENSE) or the staged one
            const T cw = KAHAN ? (direct ? __ldcg(a.c_kw + abase + pos) : sc[pos]) : T(0);
            a.trace[(int64_t)r * a.trace_cap + step - 1] = trace_value<T, MODE>(su[pos], cw);
        }
    }

    // B. element contraction in registers
    T r[P];
    if (HEUN && has_el) {
        heun_element<NP, T, MODE>(pl, a, bs, e, pw, cf0, cf1, su, r);
    } else if (has_el) {
        T u[P];
#pragma unroll
        for (int q = 0; q < P; ++q) {
            u[q] = su[(pw[q / 2] >> (16 * (q & 1))) & 0xFFFFu];
            r[q] = T(0);
        }
        // per-column (xi = x_i) parts of the Jacobian, hoisted out of the rows
        BilCol col[NP];
        if constexpr (BIL) {
#pragma unroll
            for (int i = 0; i < NP; ++i) col[i] = bil_col(cf0, cf1, (float)bs.x[i]);
        }
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            BilRow row{};
            if constexpr (BIL) row = bil_row(cf0, cf1, (float)bs.x[j]);
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                const int q = j * NP + i;
                T dxi = T(0), deta = T(0);
#pragma unroll
                for (int k = 0; k < NP; ++k) {
                    dxi += bs.D[i * NP + k] * u[j * NP + k];
                    deta += bs.D[j * NP + k] * u[k * NP + i];
                }
                T gxx, gxy, gyy;
                if constexpr (BIL) {
                    float fx, fxy, fy;
                    bil_metric(row, col[i], __fmul_rn((float)bs.W[q], cf1.z), fx, fxy, fy);
                    gxx = fx;
                    gxy = fxy;
                    gyy = fy;
                } else if constexpr (SG) {
                    gxx = ld_stream(pl.G32 + (int64_t)q * nes + e);
                    gxy = ld_stream(pl.G32 + (int64_t)(P + q) * nes + e);
                    gyy = ld_stream(pl.G32 + (int64_t)(2 * P + q) * nes + e);
                } else {
                    gxx = ld_stream(pl.G + (int64_t)q * nes + e);
                    gxy = ld_stream(pl.G + (int64_t)(P + q) * nes + e);
                    gyy = ld_stream(pl.G + (int64_t)(2 * P + q) * nes + e);
                }
                const T F1 = gxx * dxi + gxy * deta;
                const T F2 = gxy * dxi + gyy * deta;
#pragma unroll
                for (int m = 0; m < NP; ++m) {
                    r[j * NP + m] += bs.D[i * NP + m] * F1;
                    r[m * NP + i] += bs.D[j * NP + m] * F2;
                }
            }
        }
    }
    // colour-ordered scatter: in phase c only the threads of colour c add,
    // and they share no node
    // (an element's slots are distinct nodes, so all reads go first, then
    // all writes, without read-after-write waits between slots)
    for (int c = 0; c < h.ncolors; ++c) {
        if (tid >= cstart[c] && tid < cstart[c + 1]) {
            T v[P];
#pragma unroll
            for (int q = 0; q < P; ++q) v[q] = acc[(pw[q / 2] >> (16 * (q & 1))) & 0xFFFFu];
#pragma unroll
            for (int q = 0; q < P; ++q) acc[(pw[q / 2] >> (16 * (q & 1))) & 0xFFFFu] = v[q] + r[q];
        }
        __syncthreads();
    }

    // C. closed positions finish their node; open entries leave a partial sum
    if (pl.dense) {
        // VEC consecutive positions per thread: 16-byte shared-memory reads,
        // and 16-byte stores where all VEC positions are closed
        const int nch = h.slen / VEC;
        T s_nx[VEC], c_nx[VEC], x_nx[VEC];
        if (STATE && direct && tid < nch) {
            load_global_vec<T, VEC>(s_nx, a.s + abase + (int64_t)tid * VEC);
            load_global_vec<T, VEC>(x_nx, a.x_k + abase + (int64_t)tid * VEC);
            if (KAHAN) load_global_vec<T, VEC>(c_nx, a.c_k + abase + (int64_t)tid * VEC);
        }
        for (int ch = tid; ch < nch; ch += nt) {
            const int p0 = ch * VEC;
            T vu[VEC], vr[VEC], vx[VEC], vc[VEC], vs[VEC];
            if (STATE && direct) {
#pragma unroll
                for (int t = 0; t < VEC; ++t) {
                    vs[t] = s_nx[t];
                    vx[t] = x_nx[t];
                    vc[t] = KAHAN ? c_nx[t] : T(0);
                }
                const int chn = ch + nt;
                if (chn < nch) {
                    load_global_vec<T, VEC>(s_nx, a.s + abase + (int64_t)chn * VEC);
                    load_global_vec<T, VEC>(x_nx, a.x_k + abase + (int64_t)chn * VEC);
                    if (KAHAN) load_global_vec<T, VEC>(c_nx, a.c_k + abase + (int64_t)chn * VEC);
                }
            }
            const uint32_t bits = (cmask[p0 >> 5] >> (p0 & 31)) & ((1u << VEC) - 1u);
            if (bits == 0) continue;
            const int64_t g0 = abase + p0;
            if constexpr (HEUN) {
                T ui[VEC], ku[VEC], out[VEC];
                load_vec<T, VEC>(ui, su + p0);
                load_vec<T, VEC>(ku, acc + p0);
                // closed positions only: the predictor also stores the rate
                // dU at the node, and the chunk's other positions are open
                // nodes (finished by the open-node kernel) or, at the ends of
                // the owned range, nodes of the neighbouring blocks
#pragma unroll
                for (int t = 0; t < VEC; ++t) {
                    const T f = (g0 + t == a.src_gid) ? f_now : T(0);
                    out[t] = ((bits >> t) & 1u) ? heun_node<T, MODE>(a, g0 + t, ui[t], ku[t], f) : T(0);
                }
                store_masked<T, VEC>(a.u_kp1 + g0, out, bits);
                if (MODE == MODE_HEUN_C && h.nrc > 0) {
#pragma unroll
                    for (int t = 0; t < VEC; ++t)
                        if ((bits >> t) & 1u) su[p0 + t] = out[t];
                }
                continue;
            }
            load_vec<T, VEC>(vr, acc + p0);
            if (MODE == MODE_APPLY) {
                store_masked<T, VEC>(a.apply_out + g0, vr, a.vec_ok ? bits : (bits | (1u << VEC)));
                continue;
            }
            load_vec<T, VEC>(vu, su + p0);
            if (!direct) {
                load_vec<T, VEC>(vx, sx + p0);
                load_vec<T, VEC>(vs, ss + p0);
                if (KAHAN) load_vec<T, VEC>(vc, sc + p0);
            }
#pragma unroll
            for (int t = 0; t < VEC; ++t) {
                const T f = (g0 + t == a.src_gid) ? f_now : T(0);
                const Update<T, MODE> up = update_node<T, MODE>(vu[t], vx[t], KAHAN ? vc[t] : T(0), vs[t], f, vr[t]);
                vu[t] = up.u;
                vx[t] = up.x;
                vc[t] = up.c;
            }
            store_masked<T, VEC>(a.u_kp1 + g0, vu, bits);
            if (KAHAN) {
                store_masked<T, VEC>(a.x_kp1 + g0, vx, bits);
                store_masked<T, VEC>(a.c_kp1 + g0, vc, bits);
            }
            if (h.nrc > 0) {
#pragma unroll
                for (int t = 0; t < VEC; ++t)
                    if ((bits >> t) & 1u) {
                        su[p0 + t] = vu[t];
                        if (KAHAN) (direct ? acc : sc)[p0 + t] = vc[t];   // acc[p] is no longer needed
                    }
            }
        }
    } else {
        for (int p = tid; p < h.slen; p += nt) {
            if (!is_closed(cmask, p)) continue;
            const int64_t g = egid[p];
            if (MODE == MODE_APPLY) {
                __stcg(a.apply_out + g, acc[p]);
            } else if constexpr (HEUN) {
                const T f = (g == a.src_gid) ? f_now : T(0);
                const T out = heun_node<T, MODE>(a, g, su[p], acc[p], f);
                __stcg(a.u_kp1 + g, out);
                if (MODE == MODE_HEUN_C && h.nrc > 0) su[p] = out;
            } else {
                const T f = (g == a.src_gid) ? f_now : T(0);
                const Update<T, MODE> up = update_node<T, MODE>(su[p], sx[p], KAHAN ? sc[p] : T(0), ss[p], f, acc[p]);
                __stcg(a.u_kp1 + g, up.u);
                if (KAHAN) {
                    __stcg(a.x_kp1 + g, up.x);
                    __stcg(a.c_kp1 + g, up.c);
                }
                if (h.nrc > 0) {
                    su[p] = up.u;
                    if (KAHAN) sc[p] = up.c;
                }
            }
        }
    }
    for (int o = tid; o < h.nopen; o += nt) __stcg(a.part_wr + obase[o] + orank[o], acc[opos[o]]);
    if ((STATE || MODE == MODE_HEUN_C) && h.nrc > 0) {
        __syncthreads();
        // the corrector of step n runs with step = n + 1 (source at t_{n+1})
        const int64_t tix = HEUN ? step - 1 : step;
        for (int k = tid; k < h.nrc; k += nt) {
            const int pos = recs[2 * k], r2 = recs[2 * k + 1];
            a.trace[(int64_t)r2 * a.trace_cap + tix] =
                trace_value<T, MODE>(su[pos], KAHAN ? (direct ? acc : sc)[pos] : T(0));
        }
    }
}

// One step of one mesh: CTA b handles block b.
template <int NP, typename T, int MODE, bool SG = false>
__global__ void __launch_bounds__(kMaxStepThreads, (step_min_blocks<NP, T>()))
    sem_step_kernel(const Plan pl, const StepArgs<T> a, const Basis<T> bs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    step_block<NP, T, MODE, SG>(pl, a, bs, blockIdx.x, smem_raw, a.step, a.pending);
}

// Arguments of launch k of a shot, from its level buffers (the same
// assignment as the host's for a single mesh).
template <typename T, int MODE>
__device__ __forceinline__ StepArgs<T> shot_step_args(const ShotDesc<T>& d, int64_t k, int pending) {
    StepArgs<T> a;
    auto m3 = [](int64_t v) { return (int)(((v % 3) + 3) % 3); };
    if (MODE == MODE_KAHAN) {
        a.u_k = d.u[k & 1];
        a.x_k = d.x[k & 1];
        a.c_k = d.c[k & 1];
        a.u_km1 = d.u[(k + 1) & 1];
        a.x_km1 = d.x[(k + 1) & 1];
        a.c_km1 = d.c[(k + 1) & 1];
        a.u_kp1 = d.u[(k + 1) & 1];
        a.x_kp1 = d.x[(k + 1) & 1];
        a.c_kp1 = d.c[(k + 1) & 1];
        a.u_kw = d.u[k & 1];
        a.x_kw = d.x[k & 1];
        a.c_kw = d.c[k & 1];
    } else {
        a.u_k = d.u[m3(k)];
        a.x_k = d.u[m3(k - 1)];
        a.c_k = nullptr;
        a.u_km1 = d.u[m3(k - 1)];
        a.x_km1 = d.u[m3(k - 2)];
        a.c_km1 = nullptr;
        a.u_kp1 = d.u[m3(k + 1)];
        a.x_kp1 = nullptr;
        a.c_kp1 = nullptr;
        a.u_kw = d.u[m3(k)];
        a.x_kw = nullptr;
        a.c_kw = nullptr;
    }
    a.s = d.s;
    a.part_rd = d.part[(k + 1) & 1];
    a.part_wr = d.part[k & 1];
    a.apply_out = nullptr;
    a.src_f = d.src_f;
    a.step = k;
    a.src_gid = d.src_gid;
    a.trace = d.trace;
    a.trace_cap = d.trace_cap;
    a.pending = pending;
    a.vec_ok = 1;
    a.err = d.err;
    return a;
}

// One step of every shot of a batch whose elements have this order: CTA i
// handles block cta_block[i] of shot cta_shot[i]; the shot's step number and
// whether its open nodes are pending come from device memory, so a captured
// sequence of launches can be replayed.
template <int NP, typename T, int MODE>
__global__ void __launch_bounds__(kMaxStepThreads, (step_min_blocks<NP, T>()))
    sem_batch_step_kernel(const BatchArgs ba, const Basis<T> bs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Plan s_pl;
    __shared__ StepArgs<T> s_a;
    const int shot = ba.cta_shot[blockIdx.x];
    if (threadIdx.x == 0) {
        const ShotDesc<T>& d = static_cast<const ShotDesc<T>*>(ba.shots)[shot];
        s_pl = d.pl;
        if (ba.clock) {
            const ShotClock c = ba.clock[shot];
            s_a = shot_step_args<T, MODE>(d, c.step0 + ba.offset, (ba.offset > 0 || c.pending0) ? 1 : 0);
        } else {
            s_a = shot_step_args<T, MODE>(d, ba.step[shot], ba.pending[shot]);
        }
    }
    __syncthreads();
    step_block<NP, T, MODE>(s_pl, s_a, bs, ba.cta_block[blockIdx.x], smem_raw, s_a.step, s_a.pending);
}

#ifndef SEM_KERNEL_NP
// After a batch step: every shot's step number advances and its open nodes
// are pending from now on.
__global__ void batch_advance_kernel(int64_t* step, int32_t* pending, int nshots) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nshots) {
        step[i] += 1;
        pending[i] = 1;
    }
}
#endif

// ------------------------------------------------------- streamed time loop

__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(uint32_t* p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed_gpu(const int32_t* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}


// Unit (i, b) of a launch from its ticket offset u (0 <= u < total): step
// order, or the band's wavefront order for the first tiled_units tickets.
__device__ __forceinline__ void unit_of(const StreamArgs& sa, int nb, long long u, int& ui, int& ub) {
    if (u < sa.tiled_units) {
        const long long band_units = (long long)sa.band_steps * nb;
        const long long band = u / band_units;
        const uint32_t en = __ldg(sa.sched + (u - band * band_units));
        ui = (int)(band * sa.band_steps) + (int)(en >> 24);
        ub = (int)(en & 0xFFFFFFu);
    } else {
        ui = (int)(u / nb);
        ub = (int)(u - (long long)ui * nb);
    }
}

// Bounded wait for one done flag: true once it reaches `need` (acquire,
// GPU scope), false when the wait gave up or another unit raised the error
// flag.
__device__ __forceinline__ bool wait_flag(const uint32_t* f, uint32_t need, const int32_t* err) {
    unsigned long long t0 = 0;
    for (int n = 0; (int32_t)(ld_acquire_gpu(f) - need) < 0; ++n) {
        if ((n & 63) == 63) {
            const unsigned long long now = global_ns();
            if (n == 63) t0 = now;
            if (now - t0 > kWaitNs || n >= kWaitPolls || ld_relaxed_gpu(err) != 0) return false;
        }
        __nanosleep(128);
    }
    return true;
}

// step_block's "ready" hook of a streamed unit: the neighbours were awaited
// in the unit's prologue; a unit whose wait gave up stops here.
struct PrologueWaited {
    const int* fail;
    __device__ __forceinline__ bool operator()() const { return *fail == 0; }
};

// Several steps of one mesh in one launch of nsteps * nblocks CTAs. Each
// CTA, once running, takes the next ticket from a work counter and runs its
// unit (step i of the launch, block b): i * nblocks + b in step order, or the
// band's wavefront order (StreamArgs::sched, a topological order of the
// dependencies below built on the host), so units start in ticket order
// whatever order the hardware runs CTAs in. Unit (i, b) first waits until
// step i-1 has finished at b and at every block sharing a node with b: those
// are exactly the blocks whose partial sums, open-node states and closed-node
// values it reads, and whose reads of the buffers it overwrites (the level
// buffers and the partial-sum buffers rotate with the step) precede its
// writes. A unit waits only on units taken earlier, by CTAs that are running
// or finished, so the waits end; each is still bounded, and a wait that
// gives up raises the error flag, after which every unit still to start
// returns at once. The arithmetic per unit is step_block's, so the result is
// bitwise that of one launch per step. DENSE plans only: the gathers of
// GATHER plans stage through L1, which is not coherent with the other CTAs'
// writes within a launch.
template <int NP, typename T, int MODE, bool SG = false>
__global__ void __launch_bounds__(kMaxStepThreads, (step_min_blocks<NP, T>()))
    sem_stream_kernel(const ShotDesc<T> d, const StreamArgs sa, const Basis<T> bs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ StepArgs<T> s_a;
    __shared__ BlockHdr s_h;
    __shared__ int s_i, s_b;
    __shared__ __align__(16) int32_t s_dep[kMaxStreamDeps];
    __shared__ int s_fail;
    __shared__ __align__(8) unsigned long long s_mb[2];
    const int nb = d.pl.nblocks;
    const long long total = (long long)sa.nsteps * nb;
    if (threadIdx.x == 0) {
        // the ticket and the error flag are fetched together (one round trip)
        const unsigned long long t = atomicAdd(sa.counter, 1ull);
        const int raised = ld_relaxed_gpu(sa.err);
        const long long u = raised != 0 ? total : (long long)(t - sa.base);
        int ui = -1, ub = 0;
        if (u >= 0 && u < total) unit_of(sa, nb, u, ui, ub);
        s_i = ui;
        s_b = ub;
        s_fail = 0;
        if (ui >= 0) {
            // the unit's step arguments and block header, for every thread
            s_a = shot_step_args<T, MODE>(d, sa.step0 + ui, (ui > 0 || sa.pending0) ? 1 : 0);
            const BlockHdr hh = load_hdr(d.pl.hdr, ub);
            s_h = hh;
            const int4* dr = reinterpret_cast<const int4*>(sa.dep + (int64_t)ub * sa.dep_stride);
            for (int q = 0; q < sa.dep_stride / 4; ++q) reinterpret_cast<int4*>(s_dep)[q] = dr[q];
            if (d.pl.dense) {
                // the block's packet (static) is copied while the neighbour
                // wait below is under way; step_block waits for it
                const unsigned m0 = (unsigned)__cvta_generic_to_shared(&s_mb[0]);
                mbar_init(m0);
                mbar_init((unsigned)__cvta_generic_to_shared(&s_mb[1]));
                const Offsets L = offsets(hh.sulen, hh.ulen, hh.nopen, hh.ncolors, hh.nrc + hh.nro);
                mbar_arrive_expect(m0, (unsigned)L.bytes);
                bulk_g2s(smem_raw, d.pl.packet + (int64_t)hh.start * 16, (unsigned)L.bytes, m0);
            }
        }
    }
    // the neighbours' previous step, awaited by warp 0 (one flag per lane)
    // before the unit issues any other load of its own (only the packet's
    // bulk copy, which the copy engine carries, is under way). Measured on
    // the graded 512 x 512 mesh: polling with the element data and packet
    // loads of the threads already in flight took 5.6k cycles per unit
    // against 1.1k here, so the early poll shortens the unit although the
    // element loads now start one round trip later.
    __syncwarp();
    if (threadIdx.x < 32 && s_i > 0) {
        const uint32_t need = sa.serial0 + (uint32_t)(s_i - 1);
        bool ok = true;
        for (int t = (int)threadIdx.x; t < sa.dep_stride; t += 32) ok = ok && wait_flag(sa.done + s_dep[t], need, sa.err);
        if (!ok) s_fail = 1;
    }
    __syncthreads();
    const int i = s_i;
    const int b = s_b;
    if (i < 0) return;
    const int64_t k = sa.step0 + i;
    const int pend = (i > 0 || sa.pending0) ? 1 : 0;
    const PrologueWaited w{&s_fail};
    step_block<NP, T, MODE, SG>(d.pl, s_a, bs, b, smem_raw, k, pend, w, &s_h, d.pl.dense ? s_mb : nullptr);
    // every thread's stores of the unit precede the flag: the barrier orders
    // them before thread 0's release store (release at GPU scope covers what
    // the barrier made it observe)
    __syncthreads();
    if (s_fail) {
        if (threadIdx.x == 0) atomicExch(sa.err, 1);
        return;
    }
    if (threadIdx.x == 0 && (long long)i * nb + b != sa.hold_unit) st_release_gpu(sa.done + b, sa.serial0 + (uint32_t)i);
}

// Several steps of every shot of one order in one launch of
// nsteps * nblk CTAs (batched shots streamed like sem_stream_kernel): each
// CTA takes the next ticket from the launch's work counter; ticket u is
// unit (i = u / nblk, g = u % nblk): step i of the launch at block g of the
// order's blocks, i.e. block units[g].block of shot units[g].shot. The unit
// waits until step i-1 has finished at that block and at every block of the
// same shot sharing a node with it (the record's neighbour list, the shot's
// done flags, one serial sequence for the whole batch), runs step_block on
// the shot's plan and level buffers at the shot's own step number, and
// releases its block's done flag. As in sem_stream_kernel a unit waits only
// on units taken earlier, every wait is bounded, and the arithmetic is
// step_block's: bitwise the result of one launch per shot and step.
template <int NP, typename T, int MODE>
__global__ void __launch_bounds__(kMaxStepThreads, (step_min_blocks<NP, T>()))
    sem_batch_stream_kernel(const BatchStreamArgs ba, const Basis<T> bs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Plan s_pl;
    __shared__ StepArgs<T> s_a;
    __shared__ BlockHdr s_h;
    __shared__ __align__(16) int32_t s_dep[16];
    __shared__ int s_i, s_b, s_shot, s_stride, s_fail;
    __shared__ uint32_t s_serial0;
    const long long total = (long long)ba.nsteps * ba.nblk;
    if (threadIdx.x == 0) {
        const unsigned long long t = atomicAdd(ba.counter, 1ull);
        const int raised = ld_relaxed_gpu(ba.err);
        const uint32_t serial0 = __ldcg(ba.serial0);
        const long long u = raised != 0 ? total : (long long)t;
        int ui = -1;
        s_fail = 0;
        if (u < total) {
            ui = (int)(u / ba.nblk);
            const BatchUnit* rec = ba.units + (u - (long long)ui * ba.nblk);
            const int4* r4 = reinterpret_cast<const int4*>(rec);
            const int4 h0 = r4[0], h1 = r4[1], h2 = r4[2], meta = r4[3];
            BlockHdr h;
            h.start = h0.x; h.nent = h0.y; h.nown = h0.z; h.own_start = h0.w;
            h.nopen = h1.x; h.ulen = h1.y; h.slen = h1.z; h.sulen = h1.w;
            h.ncolors = h2.x; h.nrc = h2.y; h.nro = h2.z;
            s_h = h;
            s_shot = meta.x;
            s_b = meta.y;
            s_stride = meta.z;
            for (int q = 0; q < meta.z / 4; ++q) reinterpret_cast<int4*>(s_dep)[q] = r4[4 + q];
        }
        s_i = ui;
        s_serial0 = serial0;
    }
    // warp 0 only (its lanes see thread 0's writes after __syncwarp): lanes
    // 0..15 await the neighbours' previous step (at most 16, one flag each)
    // before any other load, as in sem_stream_kernel; lane 16 meanwhile
    // fetches the shot's descriptor and clock
    __syncwarp();
    if (threadIdx.x < 32) {
        const int lane = (int)threadIdx.x, ui = s_i;
        if (lane < 16) {
            if (ui > 0 && lane < s_stride &&
                !wait_flag(ba.done[s_shot] + s_dep[lane], s_serial0 + (uint32_t)(ui - 1), ba.err))
                s_fail = 1;
        } else if (lane == 16 && ui >= 0) {
            const ShotDesc<T>& d = static_cast<const ShotDesc<T>*>(ba.shots)[s_shot];
            const ShotClock c = ba.clock[s_shot];
            s_pl = d.pl;
            s_a = shot_step_args<T, MODE>(d, c.step0 + ui, (ui > 0 || c.pending0) ? 1 : 0);
        }
    }
    __syncthreads();
    if (s_i < 0) return;
    const PrologueWaited w{&s_fail};
    step_block<NP, T, MODE>(s_pl, s_a, bs, s_b, smem_raw, s_a.step, s_a.pending, w, &s_h);
    __syncthreads();
    if (s_fail) {
        if (threadIdx.x == 0) atomicExch(ba.err, 1);
        return;
    }
    if (threadIdx.x == 0) st_release_gpu(ba.done[s_shot] + s_b, s_serial0 + (uint32_t)s_i);
}

// After a streamed batch launch of n steps: every shot's clock and the
// batch serial advance by n, and the open nodes are pending from now on.
#ifndef SEM_KERNEL_NP
__global__ void batch_clock_advance_kernel(ShotClock* clock, int nshots, uint32_t* serial, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nshots) {
        clock[i].step0 += n;
        clock[i].pending0 = 1;
    }
    if (i == 0) *serial += (uint32_t)n;
}
#endif

template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads) sem_open_finish_kernel(const Plan pl, const StepArgs<T> a) {
    for (int k = blockIdx.x * kThreads + threadIdx.x; k < pl.nopen_nodes; k += gridDim.x * kThreads) {
        const int32_t pb = pl.open_base[k];
        const int cnt = pl.open_cnt[k];
        const T acc = sum_partials(a.part_rd, pb, cnt);
        const int32_t g = pl.open_gid[k];
        if (MODE == MODE_APPLY) {
            a.apply_out[g] = acc;
            continue;
        }
        if constexpr (MODE == MODE_HEUN_P || MODE == MODE_HEUN_C) {
            const T f = (g == a.src_gid) ? (T)a.src_f[a.step] : T(0);
            const T out = heun_node<T, MODE>(a, g, a.u_k[g], acc, f);
            a.u_kp1[g] = out;
            const int r = pl.open_rec[k];
            if (MODE == MODE_HEUN_C && r >= 0) a.trace[(int64_t)r * a.trace_cap + a.step - 1] = (double)out;
            continue;
        } else {
        const T f = (g == a.src_gid) ? (T)a.src_f[a.step] : T(0);
        const Update<T, MODE> up =
            update_node<T, MODE>(a.u_k[g], a.x_k[g], MODE == MODE_KAHAN ? a.c_k[g] : T(0), a.s[g], f, acc);
        a.u_kp1[g] = up.u;
        if (MODE == MODE_KAHAN) {
            a.x_kp1[g] = up.x;
            a.c_kp1[g] = up.c;
        }
        const int r = pl.open_rec[k];
        if (r >= 0) a.trace[(int64_t)r * a.trace_cap + a.step] = trace_value<T, MODE>(up.u, up.c);
        }
    }
}

#ifndef SEM_KERNEL_NP
// ------------------------------------------------------------ precompute
__global__ void geometry_kernel(int np, int64_t ne, const double* __restrict__ coords,
                                const int32_t* __restrict__ quads, const double* __restrict__ rho,
                                const double* __restrict__ vel, const Basis<double> bs, float4* coef, double* G64,
                                double* mloc, double* coef64, float* G32) {
    const int P = np * np;
    const int64_t total = ne * P;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = t / P;
        const int q = (int)(t - e * P);
        const int j = q / np, i = q - j * np;
        double X[4], Y[4];
        for (int c = 0; c < 4; ++c) {
            const int32_t v = quads[e * 4 + c];
            X[c] = coords[(int64_t)v * 2];
            Y[c] = coords[(int64_t)v * 2 + 1];
        }
        // bilinear map X = a + b xi + c eta + d xi eta
        const double bx = 0.25 * ((X[1] - X[0]) + (X[2] - X[3]));
        const double by = 0.25 * ((Y[1] - Y[0]) + (Y[2] - Y[3]));
        const double cx = 0.25 * ((X[3] - X[0]) + (X[2] - X[1]));
        const double cy = 0.25 * ((Y[3] - Y[0]) + (Y[2] - Y[1]));
        const double dx = 0.25 * ((X[0] - X[1]) + (X[2] - X[3]));
        const double dy = 0.25 * ((Y[0] - Y[1]) + (Y[2] - Y[3]));
        const double rinv = 1.0 / rho[e];
        if (q == 0 && coef != nullptr) {
            coef[e] = make_float4((float)bx, (float)by, (float)cx, (float)cy);
            coef[ne + e] = make_float4((float)dx, (float)dy, (float)rinv, 0.0f);
        }
        if (q == 0 && coef64 != nullptr) {
            const double c8[8] = {bx, by, cx, cy, dx, dy, rinv, 0.0};
            for (int k = 0; k < 8; ++k) coef64[(int64_t)k * ne + e] = c8[k];
        }
        const double xi = bs.x[i], eta = bs.x[j];
        const double j00 = bx + dx * eta, j10 = by + dy * eta;
        const double j01 = cx + dx * xi, j11 = cy + dy * xi;
        const double det = j00 * j11 - j01 * j10;
        const double wq = bs.w[i] * bs.w[j];
        const double k = wq * rinv / det;
        const double gxx = k * (j11 * j11 + j01 * j01);
        const double gxy = -k * (j10 * j11 + j00 * j01);
        const double gyy = k * (j10 * j10 + j00 * j00);
        if (G64 != nullptr) {
            G64[(int64_t)q * ne + e] = gxx;
            G64[(int64_t)(P + q) * ne + e] = gxy;
            G64[(int64_t)(2 * P + q) * ne + e] = gyy;
        }
        if (G32 != nullptr) {   // the same FP64 values, rounded once
            G32[(int64_t)q * ne + e] = (float)gxx;
            G32[(int64_t)(P + q) * ne + e] = (float)gxy;
            G32[(int64_t)(2 * P + q) * ne + e] = (float)gyy;
        }
        if (mloc != nullptr) mloc[t] = wq * det * rinv / (vel[e] * vel[e]);
    }
}
#endif

// Lumped mass through the block plan: the same colour-ordered scatter as the
// step kernel, in FP64, of w_q |J_q| / (rho c^2) per slot (mloc, device
// element order); one thread per element.
template <int NP>
__global__ void __launch_bounds__(kMaxStepThreads) mass_block_kernel(const Plan pl, const double* __restrict__ mloc,
                                                                    double* partial, double* M) {
    constexpr int P = NP * NP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* acc = reinterpret_cast<double*>(smem_raw);
    const int b = blockIdx.x;
    const int tid = threadIdx.x, nt = blockDim.x;
    const BlockHdr h = load_hdr(pl.hdr, b);
    const int64_t e0 = (int64_t)b * pl.eb;
    const int neb = (int)min((int64_t)pl.eb, pl.ne - e0);
    const Offsets L = offsets(h.sulen, h.ulen, h.nopen, h.ncolors, h.nrc + h.nro);
    const uint8_t* pk = pl.packet + (int64_t)h.start * 16;
    const uint32_t* cmask = reinterpret_cast<const uint32_t*>(pk + L.cmask);
    const int32_t* egid = reinterpret_cast<const int32_t*>(pk + L.egid);
    const int32_t* obase = reinterpret_cast<const int32_t*>(pk + L.obase);
    const uint16_t* opos = reinterpret_cast<const uint16_t*>(pk + L.opos);
    const uint8_t* orank = pk + L.orank;
    const uint16_t* cstart = reinterpret_cast<const uint16_t*>(pk + L.cstart);
    const int off = pl.dense ? h.own_start % pl.vec : 0;
    const int64_t abase = (int64_t)h.own_start - off;
    for (int p = tid; p < h.sulen; p += nt) acc[p] = 0.0;
    __syncthreads();
    for (int c = 0; c < h.ncolors; ++c) {
        if (tid < neb && tid >= cstart[c] && tid < cstart[c + 1]) {
            const int64_t e = e0 + tid;
            for (int q = 0; q < P; ++q) {
                const uint32_t w = pl.epos[(int64_t)(q / 2) * pl.ne + e];
                acc[(w >> (16 * (q & 1))) & 0xFFFFu] += mloc[e * P + q];
            }
        }
        __syncthreads();
    }
    for (int p = tid; p < h.slen; p += nt)
        if (is_closed(cmask, p)) M[p < h.ulen ? abase + p : (int64_t)egid[p - h.ulen]] = acc[p];
    for (int o = tid; o < h.nopen; o += nt) partial[obase[o] + orank[o]] = acc[opos[o]];
}

// The FP32 metric as the step kernels form it, written out in FP64 (one
// thread per element, device element order): sem_read_metric's kernel.
template <int NP>
__global__ void __launch_bounds__(kThreads) metric_fp32_kernel(const Plan pl, const Basis<float> bs, double* out) {
    constexpr int P = NP * NP;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < pl.ne; e += (int64_t)gridDim.x * blockDim.x) {
        const float4 cf0 = pl.coef[e], cf1 = pl.coef[pl.ne + e];
        for (int j = 0; j < NP; ++j) {
            const BilRow row = bil_row(cf0, cf1, bs.x[j]);
            for (int i = 0; i < NP; ++i) {
                const int q = j * NP + i;
                float gxx, gxy, gyy;
                bil_metric(row, bil_col(cf0, cf1, bs.x[i]), __fmul_rn(bs.W[q], cf1.z), gxx, gxy, gyy);
                out[(e * P + q) * 3 + 0] = gxx;
                out[(e * P + q) * 3 + 1] = gxy;
                out[(e * P + q) * 3 + 2] = gyy;
            }
        }
    }
}

#ifndef SEM_KERNEL_NP
__global__ void mass_open_kernel(const Plan pl, const double* __restrict__ partial, double* M) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < pl.nopen_nodes; k += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int t = 0; t < pl.open_cnt[k]; ++t) acc += partial[pl.open_base[k] + t];
        M[pl.open_gid[k]] = acc;
    }
}

__global__ void scale_kernel(const double* __restrict__ M, int64_t nn, double num, double* s64, float* s32) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nn; g += (int64_t)gridDim.x * blockDim.x) {
        const double v = num / M[g];
        if (s64) s64[g] = v;
        if (s32) s32[g] = (float)v;
    }
}

// ------------------------------------------------------------ adjoint
// lambda^m = 2 lambda^{m+1} - lambda^{m+2} - s (K lambda^{m+1}) (the
// leapfrog recurrence run backward; receiver residuals are added after).
template <typename T>
__global__ void adjoint_update_kernel(int64_t nn, T* lam, const T* __restrict__ lam1, const T* __restrict__ lam2,
                                      const T* __restrict__ s, const T* __restrict__ klam1) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nn; g += (int64_t)gridDim.x * blockDim.x)
        lam[g] = fma_rn(-s[g], klam1[g], sub_rn(add_rn(lam1[g], lam1[g]), lam2[g]));
}

// Receiver residuals of step m: lambda^m[node_r] -= s (trace_r^{m-1} - obs_r^{m-1}) / dt,
// receivers in ascending order by one thread (two receivers may share a node).
template <typename T>
__global__ void adjoint_receivers_kernel(int nrec, T* lam, const T* __restrict__ s, const int32_t* rec_node,
                                         const int32_t* rec_row, const double* trace, int64_t trace_cap,
                                         const double* obs, int64_t obs_cap, int64_t m, double inv_dt) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    for (int r = 0; r < nrec; ++r) {
        const int32_t g = rec_node[r];
        const double res = trace[(int64_t)rec_row[r] * trace_cap + m - 1] - obs[(int64_t)r * obs_cap + m - 1];
        lam[g] = (T)((double)lam[g] - (double)s[g] * res * inv_dt);
    }
}

// One backward step at every node, fused: lambda^m = 2 lambda^{m+1} -
// lambda^{m+2} - s (K lambda^{m+1}); then the receiver residuals of step m
// at receiver nodes, lambda^m -= s (trace_r^{m-1} - obs_r^{m-1}) / dt for the
// node's receivers in ascending order (rec_first[g]: the first of them in
// rec_order, the receivers sorted by (node, index), or -1); then
// C += lambda^m (u^m - 2 u^{m-1} + u^{m-2}) in FP64. The same operations in
// the same order as the three separate kernels below, so bitwise the same.
template <typename T>
__global__ void adjoint_node_kernel(int64_t nn, T* lam, const T* __restrict__ lam1, const T* __restrict__ lam2,
                                    const T* __restrict__ s, const T* __restrict__ klam1,
                                    const int32_t* __restrict__ rec_first, const int32_t* __restrict__ rec_order,
                                    int nrec, const int32_t* __restrict__ rec_node, const int32_t* __restrict__ rec_row,
                                    const double* __restrict__ trace, int64_t trace_cap, const double* __restrict__ obs,
                                    int64_t obs_cap, int64_t m, double inv_dt, double* C, const T* __restrict__ um,
                                    const T* __restrict__ um1, const T* __restrict__ um2) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nn; g += (int64_t)gridDim.x * blockDim.x) {
        const T sg = s[g];
        T l = fma_rn(-sg, klam1[g], sub_rn(add_rn(lam1[g], lam1[g]), lam2[g]));
        const int k0 = rec_first[g];
        if (k0 >= 0) {
            for (int k = k0; k < nrec && rec_node[rec_order[k]] == (int32_t)g; ++k) {
                const int r = rec_order[k];
                const double res = trace[(int64_t)rec_row[r] * trace_cap + m - 1] - obs[(int64_t)r * obs_cap + m - 1];
                l = (T)((double)l - (double)sg * res * inv_dt);
            }
        }
        lam[g] = l;
        const double a = ((double)um[g] - 2.0 * (double)um1[g]) + (double)um2[g];
        C[g] = fma((double)l, a, C[g]);
    }
}

// C += lambda^m (u^m - 2 u^{m-1} + u^{m-2}), accumulated in FP64.
template <typename T>
__global__ void correlate_kernel(int64_t nn, double* C, const T* __restrict__ lam, const T* __restrict__ um,
                                 const T* __restrict__ um1, const T* __restrict__ um2) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nn; g += (int64_t)gridDim.x * blockDim.x) {
        const double a = ((double)um[g] - 2.0 * (double)um1[g]) + (double)um2[g];
        C[g] = fma((double)lam[g], a, C[g]);
    }
}

// dJ/dc_e = sum_q dM/dc_e C = -(2 / c_e) sum_q mloc[e, q] C[node(e, q)],
// mloc = w_q |J_q| / (rho_e c_e^2); one thread per element, points in order.
__global__ void gradient_kernel(int64_t ne, int P, const int32_t* __restrict__ conn, const double* __restrict__ mloc,
                                const double* __restrict__ C, const double* __restrict__ vel, double* grad) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int q = 0; q < P; ++q) acc = fma(mloc[e * P + q], C[conn[e * P + q]], acc);
        grad[e] = -2.0 * acc / vel[e];
    }
}

int grid_for(int64_t n, int threads) {
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 152 * 64) g = 152 * 64;
    return (int)g;
}
#endif

}  // namespace

// ------------------------------------------------------ per-order launchers
// The kernels templated on the order are instantiated one order per
// translation unit: this file is compiled once per order with
// SEM_KERNEL_NP = p + 1 (those units define the launchers below for their
// order only) and once without it (the dispatchers and the order-independent
// kernels), so that the orders compile in parallel.
template <int NP>
cudaError_t step_np(bool fp64, int mode, const Plan& pl, const void* args, const void* basis, int threads, int smem,
                    cudaStream_t st);
template <int NP>
cudaError_t metric_np(const Plan& pl, const Basis<float>& basis, double* out, cudaStream_t st);
template <int NP>
cudaError_t batch_np(bool fp64, int mode, bool prepare_only, const BatchArgs& ba, int ctas, const void* basis,
                     int threads, int smem, cudaStream_t st);
template <int NP>
cudaError_t stream_np(bool fp64, int mode, const void* shot, const StreamArgs& sa, const void* basis, int threads,
                      int smem, int64_t ctas, cudaStream_t st);
template <int NP>
cudaError_t resident_np(bool fp64, int mode, bool sg, int threads, int smem, int* out);
template <int NP>
cudaError_t bstream_np(bool fp64, int mode, bool prepare_only, const BatchStreamArgs& ba, const void* basis,
                       int threads, int smem, cudaStream_t st);
template <int NP>
cudaError_t bresident_np(bool fp64, int mode, int threads, int smem, int* out);
template <int NP>
cudaError_t mass_np(const Plan& pl, const double* mloc, double* partial, double* M, int threads, int smem,
                    cudaStream_t st);

#ifdef SEM_KERNEL_NP
namespace {

// Raises the dynamic shared-memory limit of a kernel to at least `smem` and
// never lowers it: handles with different block sizes share one kernel, and
// a limit set for a smaller block would make a later launch of a larger one
// fail. One table per translation unit (each kernel lives in one unit).
std::mutex g_smem_mu;
std::map<const void*, int> g_smem_limit;
template <typename K>
cudaError_t raise_smem(K kern, int smem) {
    const void* f = reinterpret_cast<const void*>(kern);
    std::lock_guard<std::mutex> lk(g_smem_mu);
    int& lim = g_smem_limit[f];
    if (smem <= lim) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) lim = smem;
    return e;
}

template <int NP, typename T, int MODE, bool SG = false>
cudaError_t launch_step_t(const Plan& pl, const void* args, const void* basis, int threads, int smem, cudaStream_t st) {
    auto kern = sem_step_kernel<NP, T, MODE, SG>;
    const cudaError_t e = raise_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<pl.nblocks, threads, smem, st>>>(pl, *static_cast<const StepArgs<T>*>(args),
                                            *static_cast<const Basis<T>*>(basis));
    return cudaGetLastError();
}

template <int NP, typename T, int MODE>
cudaError_t launch_batch_t(bool prepare_only, const BatchArgs& ba, int ctas, const void* basis, int threads, int smem,
                           cudaStream_t st) {
    auto kern = sem_batch_step_kernel<NP, T, MODE>;
    if (prepare_only) return raise_smem(kern, smem);
    kern<<<ctas, threads, smem, st>>>(ba, *static_cast<const Basis<T>*>(basis));
    return cudaGetLastError();
}

template <int NP, typename T, int MODE, bool SG = false>
cudaError_t stream_t(const void* shot, const StreamArgs& sa, const void* basis, int threads, int smem, int64_t ctas,
                     cudaStream_t st) {
    auto kern = sem_stream_kernel<NP, T, MODE, SG>;
    {
        const cudaError_t e = raise_smem(kern, smem);
        if (e != cudaSuccess) return e;
    }
    if (ctas < 1 || ctas > 2147483647LL) return cudaErrorInvalidValue;
    kern<<<(unsigned)ctas, threads, smem, st>>>(*static_cast<const ShotDesc<T>*>(shot), sa,
                                                *static_cast<const Basis<T>*>(basis));
    return cudaGetLastError();
}

template <int NP, typename T, int MODE, bool SG = false>
cudaError_t stream_resident_t(int threads, int smem, int* out) {
    auto kern = sem_stream_kernel<NP, T, MODE, SG>;
    cudaError_t e = raise_smem(kern, smem);
    int per_sm = 0, dev = 0, sms = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) *out = per_sm * sms;
    return e;
}

template <int NP, typename T, int MODE>
cudaError_t bstream_t(bool prepare_only, const BatchStreamArgs& ba, const void* basis, int threads, int smem,
                      cudaStream_t st) {
    auto kern = sem_batch_stream_kernel<NP, T, MODE>;
    if (prepare_only) return raise_smem(kern, smem);
    const long long ctas = (long long)ba.nsteps * ba.nblk;
    if (ctas < 1 || ctas > 2147483647LL) return cudaErrorInvalidValue;
    kern<<<(unsigned)ctas, threads, smem, st>>>(ba, *static_cast<const Basis<T>*>(basis));
    return cudaGetLastError();
}

template <int NP, typename T, int MODE>
cudaError_t bresident_t(int threads, int smem, int* out) {
    auto kern = sem_batch_stream_kernel<NP, T, MODE>;
    cudaError_t e = raise_smem(kern, smem);
    int per_sm = 0, dev = 0, sms = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) *out = per_sm * sms;
    return e;
}

}  // namespace

template <int NP>
cudaError_t bstream_np(bool fp64, int mode, bool prepare_only, const BatchStreamArgs& ba, const void* basis,
                       int threads, int smem, cudaStream_t st) {
    if (fp64) {
        if (mode == MODE_THREE_LEVEL)
            return bstream_t<NP, double, MODE_THREE_LEVEL>(prepare_only, ba, basis, threads, smem, st);
        return cudaErrorInvalidValue;
    }
    if (mode == MODE_THREE_LEVEL) return bstream_t<NP, float, MODE_THREE_LEVEL>(prepare_only, ba, basis, threads, smem, st);
    if (mode == MODE_KAHAN) return bstream_t<NP, float, MODE_KAHAN>(prepare_only, ba, basis, threads, smem, st);
    return cudaErrorInvalidValue;
}

template <int NP>
cudaError_t bresident_np(bool fp64, int mode, int threads, int smem, int* out) {
    if (fp64) {
        if (mode == MODE_THREE_LEVEL) return bresident_t<NP, double, MODE_THREE_LEVEL>(threads, smem, out);
        return cudaErrorInvalidValue;
    }
    if (mode == MODE_THREE_LEVEL) return bresident_t<NP, float, MODE_THREE_LEVEL>(threads, smem, out);
    if (mode == MODE_KAHAN) return bresident_t<NP, float, MODE_KAHAN>(threads, smem, out);
    return cudaErrorInvalidValue;
}

template <int NP>
cudaError_t step_np(bool fp64, int mode, const Plan& pl, const void* args, const void* basis, int threads, int smem,
                    cudaStream_t st) {
    if (fp64) {
        switch (mode) {
            case MODE_THREE_LEVEL: return launch_step_t<NP, double, MODE_THREE_LEVEL>(pl, args, basis, threads, smem, st);
            case MODE_APPLY: return launch_step_t<NP, double, MODE_APPLY>(pl, args, basis, threads, smem, st);
            case MODE_HEUN_P: return launch_step_t<NP, double, MODE_HEUN_P>(pl, args, basis, threads, smem, st);
            case MODE_HEUN_C: return launch_step_t<NP, double, MODE_HEUN_C>(pl, args, basis, threads, smem, st);
            default: return cudaErrorInvalidValue;
        }
    }
    if (pl.G32) {
        switch (mode) {
            case MODE_THREE_LEVEL:
                return launch_step_t<NP, float, MODE_THREE_LEVEL, true>(pl, args, basis, threads, smem, st);
            case MODE_KAHAN: return launch_step_t<NP, float, MODE_KAHAN, true>(pl, args, basis, threads, smem, st);
            case MODE_APPLY: return launch_step_t<NP, float, MODE_APPLY, true>(pl, args, basis, threads, smem, st);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (mode) {
        case MODE_THREE_LEVEL: return launch_step_t<NP, float, MODE_THREE_LEVEL>(pl, args, basis, threads, smem, st);
        case MODE_KAHAN: return launch_step_t<NP, float, MODE_KAHAN>(pl, args, basis, threads, smem, st);
        case MODE_APPLY: return launch_step_t<NP, float, MODE_APPLY>(pl, args, basis, threads, smem, st);
        case MODE_HEUN_P: return launch_step_t<NP, float, MODE_HEUN_P>(pl, args, basis, threads, smem, st);
        case MODE_HEUN_C: return launch_step_t<NP, float, MODE_HEUN_C>(pl, args, basis, threads, smem, st);
        default: return cudaErrorInvalidValue;
    }
}

template <int NP>
cudaError_t batch_np(bool fp64, int mode, bool prepare_only, const BatchArgs& ba, int ctas, const void* basis,
                     int threads, int smem, cudaStream_t st) {
    if (fp64) {
        if (mode == MODE_THREE_LEVEL)
            return launch_batch_t<NP, double, MODE_THREE_LEVEL>(prepare_only, ba, ctas, basis, threads, smem, st);
        return cudaErrorInvalidValue;
    }
    if (mode == MODE_THREE_LEVEL)
        return launch_batch_t<NP, float, MODE_THREE_LEVEL>(prepare_only, ba, ctas, basis, threads, smem, st);
    if (mode == MODE_KAHAN) return launch_batch_t<NP, float, MODE_KAHAN>(prepare_only, ba, ctas, basis, threads, smem, st);
    return cudaErrorInvalidValue;
}

template <int NP>
cudaError_t stream_np(bool fp64, int mode, const void* shot, const StreamArgs& sa, const void* basis, int threads,
                      int smem, int64_t ctas, cudaStream_t st) {
    if (fp64) {
        if (mode == MODE_THREE_LEVEL) return stream_t<NP, double, MODE_THREE_LEVEL>(shot, sa, basis, threads, smem, ctas, st);
        return cudaErrorInvalidValue;
    }
    if (static_cast<const ShotDesc<float>*>(shot)->pl.G32) {
        if (mode == MODE_THREE_LEVEL)
            return stream_t<NP, float, MODE_THREE_LEVEL, true>(shot, sa, basis, threads, smem, ctas, st);
        if (mode == MODE_KAHAN) return stream_t<NP, float, MODE_KAHAN, true>(shot, sa, basis, threads, smem, ctas, st);
        return cudaErrorInvalidValue;
    }
    if (mode == MODE_THREE_LEVEL) return stream_t<NP, float, MODE_THREE_LEVEL>(shot, sa, basis, threads, smem, ctas, st);
    if (mode == MODE_KAHAN) return stream_t<NP, float, MODE_KAHAN>(shot, sa, basis, threads, smem, ctas, st);
    return cudaErrorInvalidValue;
}

template <int NP>
cudaError_t resident_np(bool fp64, int mode, bool sg, int threads, int smem, int* out) {
    if (fp64) {
        if (mode == MODE_THREE_LEVEL) return stream_resident_t<NP, double, MODE_THREE_LEVEL>(threads, smem, out);
        return cudaErrorInvalidValue;
    }
    if (sg) {
        if (mode == MODE_THREE_LEVEL) return stream_resident_t<NP, float, MODE_THREE_LEVEL, true>(threads, smem, out);
        if (mode == MODE_KAHAN) return stream_resident_t<NP, float, MODE_KAHAN, true>(threads, smem, out);
        return cudaErrorInvalidValue;
    }
    if (mode == MODE_THREE_LEVEL) return stream_resident_t<NP, float, MODE_THREE_LEVEL>(threads, smem, out);
    if (mode == MODE_KAHAN) return stream_resident_t<NP, float, MODE_KAHAN>(threads, smem, out);
    return cudaErrorInvalidValue;
}

template <int NP>
cudaError_t mass_np(const Plan& pl, const double* mloc, double* partial, double* M, int threads, int smem,
                    cudaStream_t st) {
    cudaError_t e = raise_smem(mass_block_kernel<NP>, smem);
    if (e != cudaSuccess) return e;
    mass_block_kernel<NP><<<pl.nblocks, threads, smem, st>>>(pl, mloc, partial, M);
    return cudaGetLastError();
}

template <int NP>
cudaError_t metric_np(const Plan& pl, const Basis<float>& basis, double* out, cudaStream_t st) {
    int64_t g = (pl.ne + kThreads - 1) / kThreads;
    if (g < 1) g = 1;
    if (g > 152 * 64) g = 152 * 64;
    metric_fp32_kernel<NP><<<(int)g, kThreads, 0, st>>>(pl, basis, out);
    return cudaGetLastError();
}

template cudaError_t step_np<SEM_KERNEL_NP>(bool, int, const Plan&, const void*, const void*, int, int, cudaStream_t);
template cudaError_t metric_np<SEM_KERNEL_NP>(const Plan&, const Basis<float>&, double*, cudaStream_t);
template cudaError_t batch_np<SEM_KERNEL_NP>(bool, int, bool, const BatchArgs&, int, const void*, int, int,
                                            cudaStream_t);
template cudaError_t stream_np<SEM_KERNEL_NP>(bool, int, const void*, const StreamArgs&, const void*, int, int,
                                             int64_t, cudaStream_t);
template cudaError_t resident_np<SEM_KERNEL_NP>(bool, int, bool, int, int, int*);
template cudaError_t bstream_np<SEM_KERNEL_NP>(bool, int, bool, const BatchStreamArgs&, const void*, int, int,
                                              cudaStream_t);
template cudaError_t bresident_np<SEM_KERNEL_NP>(bool, int, int, int, int*);
template cudaError_t mass_np<SEM_KERNEL_NP>(const Plan&, const double*, double*, double*, int, int, cudaStream_t);

#else  // the dispatchers and the order-independent kernels

#define SEM_NP_SWITCH(np, CALL)        \
    switch (np) {                      \
        case 2: return CALL(2);        \
        case 3: return CALL(3);        \
        case 4: return CALL(4);        \
        case 5: return CALL(5);        \
        case 6: return CALL(6);        \
        case 7: return CALL(7);        \
        case 8: return CALL(8);        \
        case 9: return CALL(9);        \
        default: return cudaErrorInvalidValue; \
    }

cudaError_t launch_batch_step(int np, bool fp64, int mode, bool prepare_only, const BatchArgs& ba, int ctas,
                              const void* basis, int threads, int smem, cudaStream_t st) {
    if (threads < 1 || threads > kMaxStepThreads) return cudaErrorInvalidValue;
#define SEM_CALL(N) batch_np<N>(fp64, mode, prepare_only, ba, ctas, basis, threads, smem, st)
    SEM_NP_SWITCH(np, SEM_CALL)
#undef SEM_CALL
}

cudaError_t launch_batch_advance(int64_t* step, int32_t* pending, int nshots, cudaStream_t st) {
    batch_advance_kernel<<<(nshots + 255) / 256, 256, 0, st>>>(step, pending, nshots);
    return cudaGetLastError();
}

cudaError_t launch_batch_stream(int np, bool fp64, int mode, bool prepare_only, const BatchStreamArgs& sa,
                                const void* basis, int threads, int smem, cudaStream_t st) {
    if (threads < 1 || threads > kMaxStepThreads) return cudaErrorInvalidValue;
#define SEM_CALL(N) bstream_np<N>(fp64, mode, prepare_only, sa, basis, threads, smem, st)
    SEM_NP_SWITCH(np, SEM_CALL)
#undef SEM_CALL
}

cudaError_t launch_batch_clock_advance(ShotClock* clock, int nshots, uint32_t* serial, int nsteps, cudaStream_t st) {
    batch_clock_advance_kernel<<<(nshots + 255) / 256, 256, 0, st>>>(clock, nshots, serial, nsteps);
    return cudaGetLastError();
}

cudaError_t batch_stream_resident_ctas(int np, bool fp64, int mode, int threads, int smem, int* out) {
    *out = 0;
#define SEM_CALL(N) bresident_np<N>(fp64, mode, threads, smem, out)
    SEM_NP_SWITCH(np, SEM_CALL)
#undef SEM_CALL
}

cudaError_t stream_resident_ctas(int np, bool fp64, int mode, bool sg, int threads, int smem, int* out) {
    *out = 0;
#define SEM_CALL(N) resident_np<N>(fp64, mode, sg, threads, smem, out)
    SEM_NP_SWITCH(np, SEM_CALL)
#undef SEM_CALL
}

cudaError_t launch_stream(int np, bool fp64, int mode, const void* shot, const StreamArgs& sa, const void* basis,
                          int threads, int smem, int nblocks, cudaStream_t st) {
    if (threads < 1 || threads > kMaxStepThreads) return cudaErrorInvalidValue;
    const int64_t ctas = (int64_t)sa.nsteps * (int64_t)nblocks;
#define SEM_CALL(N) stream_np<N>(fp64, mode, shot, sa, basis, threads, smem, ctas, st)
    SEM_NP_SWITCH(np, SEM_CALL)
#undef SEM_CALL
}

cudaError_t launch_metric_fp32(int np, const Plan& pl, const Basis<float>& basis, double* out, cudaStream_t st) {
    if (!pl.coef) return cudaErrorInvalidValue;
#define SEM_CALL(N) metric_np<N>(pl, basis, out, st)
    SEM_NP_SWITCH(np, SEM_CALL)
#undef SEM_CALL
}

int step_threads(int eb) {
    int t = (eb + 31) / 32 * 32;
    return t < 32 ? 32 : t;
}

int smem_bytes_for(int P, int eb, int max_packet, int sulen_pad, int slen_pad, bool fp64, int mode, bool dense) {
    (void)P;
    (void)eb;
    const int sz = fp64 ? 8 : 4;
    const bool direct = dense;
    const bool leap = mode == MODE_THREE_LEVEL || mode == MODE_KAHAN;
    const int staged = !leap ? 0 : (direct ? 0 : (mode == MODE_KAHAN ? 3 : 2));
    return max_packet + (2 * sulen_pad + staged * slen_pad) * sz;
}

cudaError_t launch_step(int np, bool fp64, int mode, const Plan& pl, const void* args, const void* basis,
                        int threads, int smem, cudaStream_t st) {
    if (threads < 1 || threads > kMaxStepThreads || threads < pl.eb) return cudaErrorInvalidValue;
#define SEM_CALL(N) step_np<N>(fp64, mode, pl, args, basis, threads, smem, st)
    SEM_NP_SWITCH(np, SEM_CALL)
#undef SEM_CALL
}

cudaError_t launch_open_finish(bool fp64, int mode, const Plan& pl, const void* args, cudaStream_t st) {
    if (pl.nopen_nodes == 0) return cudaSuccess;
    const int grid = grid_for(pl.nopen_nodes, kThreads);
    if (fp64) {
        const auto& a = *static_cast<const StepArgs<double>*>(args);
        if (mode == MODE_THREE_LEVEL) sem_open_finish_kernel<double, MODE_THREE_LEVEL><<<grid, kThreads, 0, st>>>(pl, a);
        else if (mode == MODE_APPLY) sem_open_finish_kernel<double, MODE_APPLY><<<grid, kThreads, 0, st>>>(pl, a);
        else if (mode == MODE_HEUN_P) sem_open_finish_kernel<double, MODE_HEUN_P><<<grid, kThreads, 0, st>>>(pl, a);
        else if (mode == MODE_HEUN_C) sem_open_finish_kernel<double, MODE_HEUN_C><<<grid, kThreads, 0, st>>>(pl, a);
        else return cudaErrorInvalidValue;
    } else {
        const auto& a = *static_cast<const StepArgs<float>*>(args);
        if (mode == MODE_THREE_LEVEL) sem_open_finish_kernel<float, MODE_THREE_LEVEL><<<grid, kThreads, 0, st>>>(pl, a);
        else if (mode == MODE_KAHAN) sem_open_finish_kernel<float, MODE_KAHAN><<<grid, kThreads, 0, st>>>(pl, a);
        else if (mode == MODE_APPLY) sem_open_finish_kernel<float, MODE_APPLY><<<grid, kThreads, 0, st>>>(pl, a);
        else if (mode == MODE_HEUN_P) sem_open_finish_kernel<float, MODE_HEUN_P><<<grid, kThreads, 0, st>>>(pl, a);
        else if (mode == MODE_HEUN_C) sem_open_finish_kernel<float, MODE_HEUN_C><<<grid, kThreads, 0, st>>>(pl, a);
        else return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_adjoint_update(bool fp64, int64_t nn, void* lam, const void* lam1, const void* lam2, const void* s,
                                  const void* klam1, cudaStream_t st) {
    const int grid = grid_for(nn, kThreads);
    if (fp64)
        adjoint_update_kernel<double><<<grid, kThreads, 0, st>>>(nn, (double*)lam, (const double*)lam1,
                                                                (const double*)lam2, (const double*)s,
                                                                (const double*)klam1);
    else
        adjoint_update_kernel<float><<<grid, kThreads, 0, st>>>(nn, (float*)lam, (const float*)lam1,
                                                               (const float*)lam2, (const float*)s,
                                                               (const float*)klam1);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_receivers(bool fp64, int nrec, void* lam, const void* s, const int32_t* rec_node,
                                     const int32_t* rec_row, const double* trace, int64_t trace_cap, const double* obs,
                                     int64_t obs_cap, int64_t m, double inv_dt, cudaStream_t st) {
    if (fp64)
        adjoint_receivers_kernel<double><<<1, 32, 0, st>>>(nrec, (double*)lam, (const double*)s, rec_node, rec_row,
                                                           trace, trace_cap, obs, obs_cap, m, inv_dt);
    else
        adjoint_receivers_kernel<float><<<1, 32, 0, st>>>(nrec, (float*)lam, (const float*)s, rec_node, rec_row,
                                                          trace, trace_cap, obs, obs_cap, m, inv_dt);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_node(bool fp64, int64_t nn, void* lam, const void* lam1, const void* lam2, const void* s,
                                const void* klam1, const int32_t* rec_first, const int32_t* rec_order, int nrec,
                                const int32_t* rec_node, const int32_t* rec_row, const double* trace,
                                int64_t trace_cap, const double* obs, int64_t obs_cap, int64_t m, double inv_dt,
                                double* C, const void* um, const void* um1, const void* um2, cudaStream_t st) {
    const int grid = grid_for(nn, kThreads);
    if (fp64)
        adjoint_node_kernel<double><<<grid, kThreads, 0, st>>>(
            nn, (double*)lam, (const double*)lam1, (const double*)lam2, (const double*)s, (const double*)klam1,
            rec_first, rec_order, nrec, rec_node, rec_row, trace, trace_cap, obs, obs_cap, m, inv_dt, C,
            (const double*)um, (const double*)um1, (const double*)um2);
    else
        adjoint_node_kernel<float><<<grid, kThreads, 0, st>>>(
            nn, (float*)lam, (const float*)lam1, (const float*)lam2, (const float*)s, (const float*)klam1, rec_first,
            rec_order, nrec, rec_node, rec_row, trace, trace_cap, obs, obs_cap, m, inv_dt, C, (const float*)um,
            (const float*)um1, (const float*)um2);
    return cudaGetLastError();
}

cudaError_t launch_correlate(bool fp64, int64_t nn, double* C, const void* lam, const void* um, const void* um1,
                             const void* um2, cudaStream_t st) {
    const int grid = grid_for(nn, kThreads);
    if (fp64)
        correlate_kernel<double><<<grid, kThreads, 0, st>>>(nn, C, (const double*)lam, (const double*)um,
                                                           (const double*)um1, (const double*)um2);
    else
        correlate_kernel<float><<<grid, kThreads, 0, st>>>(nn, C, (const float*)lam, (const float*)um,
                                                          (const float*)um1, (const float*)um2);
    return cudaGetLastError();
}

cudaError_t launch_gradient(int64_t ne, int P, const int32_t* conn, const double* mloc, const double* C,
                            const double* vel, double* grad, cudaStream_t st) {
    gradient_kernel<<<grid_for(ne, kThreads), kThreads, 0, st>>>(ne, P, conn, mloc, C, vel, grad);
    return cudaGetLastError();
}

cudaError_t launch_geometry(int np, int64_t ne, const double* coords, const int32_t* quads_new, const double* rho,
                            const double* vel, const Basis<double>& basis, float4* coef, double* G64, double* mloc,
                            double* coef64, float* G32, cudaStream_t st) {
    geometry_kernel<<<grid_for(ne * np * np, kThreads), kThreads, 0, st>>>(np, ne, coords, quads_new, rho, vel, basis,
                                                                          coef, G64, mloc, coef64, G32);
    return cudaGetLastError();
}

cudaError_t launch_mass(const Plan& pl, int np, const double* mloc, double* partial, double* M, cudaStream_t st) {
    const int threads = step_threads(pl.eb);
    const int smem = pl.sulen_pad * 8;
    cudaError_t e = cudaSuccess;
    switch (np) {
#define SEM_MASS_CASE(N) \
    case N: e = mass_np<N>(pl, mloc, partial, M, threads, smem, st); break;
        SEM_MASS_CASE(2)
        SEM_MASS_CASE(3)
        SEM_MASS_CASE(4)
        SEM_MASS_CASE(5)
        SEM_MASS_CASE(6)
        SEM_MASS_CASE(7)
        SEM_MASS_CASE(8)
        SEM_MASS_CASE(9)
#undef SEM_MASS_CASE
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    if (pl.nopen_nodes > 0) mass_open_kernel<<<grid_for(pl.nopen_nodes, kThreads), kThreads, 0, st>>>(pl, partial, M);
    return cudaGetLastError();
}

cudaError_t launch_scale(const double* M, int64_t nn, double num, double* s64, float* s32, cudaStream_t st) {
    scale_kernel<<<grid_for(nn, kThreads), kThreads, 0, st>>>(M, nn, num, s64, s32);
    return cudaGetLastError();
}

#endif  // SEM_KERNEL_NP

}  // namespace semdev
