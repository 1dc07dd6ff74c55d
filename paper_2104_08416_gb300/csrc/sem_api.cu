// C ABI of the spectral-element stepper (declarations and contracts in
// include/sem.h). Host orchestration: validation, orderings and the block
// plan come from sem_host.cpp; all per-step arithmetic runs in the kernels of
// sem_kernels.cu on the handle's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <atomic>
#include <map>
#include <thread>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/sem.h"
#include "sem_host.h"
#include "sem_kernels.cuh"

namespace {

std::mutex g_alloc_mu;
sem_alloc_fn g_alloc = nullptr;
sem_free_fn g_free = nullptr;
void* g_alloc_ctx = nullptr;

struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct sem_mesh {
    semhost::Mesh mesh;
    sem_precision prec = SEM_FP64;
    cudaStream_t stream = nullptr;
    std::string err;
    // allocator captured at creation
    sem_alloc_fn alloc = nullptr;
    sem_free_fn free_fn = nullptr;
    void* alloc_ctx = nullptr;
    std::vector<DevBuf> bufs;

    int ordering = SEM_ORDER_NONE;
    uint64_t seed = 0;
    std::vector<int64_t> elem_order, node_order;  // order[new] = old
    std::vector<int64_t> elem_new, node_new;      // new id of each old id
    std::vector<double> node_xy;                  // original order

    bool have_model = false;
    std::vector<double> vel, rho;
    bool have_src = false;
    double f0 = 0, t0 = 0, amp = 0, sx = 0, sy = 0;
    int64_t src_node = -1;  // original id
    int32_t nrec = 0;
    int64_t trace_cap = 0;
    std::vector<int64_t> rec_nodes;  // original ids
    std::vector<int32_t> rec_row;    // -1, or the earlier receiver on the same node
    bool have_dt = false;
    double dt = 0;
    int eb_request = 0;
    int sm_count = 0;           // SMs of the handle's device (0: unknown), for the default block size
    int scheme = 0;             // SEM_SCHEME_LEAPFROG or SEM_SCHEME_HEUN
    int threads_request = 0;

    // device state (host_* hold the host part of the build until the device part)
    bool built = false;
    bool host_ready = false;
    std::vector<int32_t> host_quads;
    std::vector<double> host_rho, host_vel;
    int64_t step = 0;
    int64_t stepped_calls = 0;
    // the open nodes of the last leapfrog step still stand as partial sums:
    // the next step finishes them as any step does, and a call that reads or
    // replaces the state first runs the open-node kernel (flush_pending)
    bool open_pending = false;
    semhost::BlockPlan plan;
    semdev::Plan dplan{};
    int smem = 0;
    int threads = 0;
    // streamed time loop (sem_set_stream): up to stream_steps steps per
    // launch (0: one launch per step) where the plan allows it (stream_ok),
    // per-block neighbour lists and done flags
    int stream_steps = -1;            // -1: automatic (see streamed())
    bool stream_ok = false;
    int resident_ctas = 0;            // step CTAs resident on the GPU at once
    int32_t* d_dep = nullptr;         // [nblocks][dep_stride] padded neighbour lists
    int32_t dep_stride = 0;
    uint32_t* d_done = nullptr;
    unsigned long long* d_counter = nullptr;
    // the counter's value when the next streamed launch starts: every CTA of
    // a launch takes exactly one ticket, so it grows by the launch's units
    // and needs no reset between launches
    unsigned long long ticket_base = 0;
    int32_t* d_err = nullptr;
    uint32_t serial = 1;              // serial of the next streamed step
    int64_t hold_step = -1;           // test hook: (step, block) whose done flag is withheld
    int32_t hold_block = -1;
    // wavefront order of the streamed units (sem_set_stream_tiling):
    // band_req steps per band (-1: default, 0: step order), window_req
    // levels per tile (0: automatic); d_sched holds one band's order, built
    // for (sched_T, sched_W)
    int band_req = -1;
    int window_req = 0;
    uint32_t* d_sched = nullptr;
    size_t sched_cap = 0;
    int sched_T = 0, sched_W = 0;
    int auto_window = 0;              // window of window_req = 0 (resident CTAs per step of a tile)
    semdev::Basis<double> basis64{};
    semdev::Basis<float> basis32{};
    double* d_coords = nullptr;
    int32_t* d_quads = nullptr;
    double* d_rho = nullptr;
    double* d_vel = nullptr;
    uint8_t* d_packet = nullptr;
    double* d_G64 = nullptr;
    float* d_G32 = nullptr;       // stored FP32 metric (SEM_METRIC_STORED)
    double* d_metric_out = nullptr;   // sem_read_metric's output buffer
    int metric = SEM_METRIC_BILINEAR;
    double* d_coef64 = nullptr;   // FP64 bilinear map (first-order system, FP64)
    void* d_v[2] = {nullptr, nullptr};   // first-order system: V, V~ ([2P][ne])
    void* d_vd1 = nullptr;               // predictor rate of V
    void* d_ud1 = nullptr;               // predictor rate of U
    double* d_mloc = nullptr;
    double* d_M = nullptr;
    void* d_s = nullptr;
    // node state by level (see semdev::StepArgs): three-level mode keeps
    // u^m in d_u[m % 3]; Kahan mode keeps (u^m, delta^{m-1/2}, c^m) in
    // (d_u, d_x, d_c)[m % 2]
    void* d_u[3] = {nullptr, nullptr, nullptr};
    void* d_x[2] = {nullptr, nullptr};
    void* d_c[2] = {nullptr, nullptr};
    void* d_part[2] = {nullptr, nullptr};
    void* d_apply_in = nullptr;
    void* d_apply_out = nullptr;
    double* d_src = nullptr;
    int64_t src_cap = 0;
    double* d_trace = nullptr;
    // adjoint (allocated by the first sem_misfit_gradient)
    int64_t adj_steps = 0, adj_kc = 0;
    void* d_lam[3] = {nullptr, nullptr, nullptr};
    void* d_klam = nullptr;
    double* d_C = nullptr;
    double* d_obs = nullptr;
    double* d_grad = nullptr;
    int32_t* d_conn_dev = nullptr;
    int32_t* d_rec_node = nullptr;
    int32_t* d_rec_row = nullptr;
    int32_t* d_rec_order = nullptr;   // receivers sorted by (node, index)
    int32_t* d_rec_first = nullptr;   // [nn]: first of a node's receivers in d_rec_order, or -1
    std::vector<void*> d_chk;   // per checkpoint: u^{n0}, u^{n0-1}
    std::vector<void*> d_seg;   // recomputed states of one segment
    // measurement
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_block, ev_open;
    int64_t h2d = 0, d2h = 0;
};

namespace {

sem_status fail(sem_mesh* m, sem_status st, const std::string& msg) {
    if (m) m->err = msg;
    return st;
}

sem_status cuda_fail(sem_mesh* m, cudaError_t e, const char* where) {
    return fail(m, SEM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define SEM_CUDA(call)                                          \
    do {                                                        \
        cudaError_t _e = (call);                                \
        if (_e != cudaSuccess) return cuda_fail(m, _e, #call);  \
    } while (0)

void* dev_alloc(sem_mesh* m, size_t bytes) {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~size_t(255);
    void* p = nullptr;
    if (m->alloc) {
        p = m->alloc(bytes, (void*)m->stream, m->alloc_ctx);
        // the kernels copy node arrays with 16-byte vectors: a pointer off
        // that boundary is handed back and reported as a failed allocation
        if (p && ((uintptr_t)p % 16) != 0) {
            if (m->free_fn) m->free_fn(p, bytes, (void*)m->stream, m->alloc_ctx);
            p = nullptr;
        }
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) m->bufs.push_back({p, bytes});
    return p;
}

void dev_free_all(sem_mesh* m) {
    if (!m->bufs.empty()) cudaStreamSynchronize(m->stream);
    for (auto& b : m->bufs) {
        if (m->free_fn) m->free_fn(b.ptr, b.bytes, (void*)m->stream, m->alloc_ctx);
        else cudaFree(b.ptr);
    }
    m->bufs.clear();
}

template <typename T>
sem_status upload(sem_mesh* m, T** dst, const T* src, size_t n) {
    *dst = static_cast<T*>(dev_alloc(m, n * sizeof(T)));
    if (!*dst) return fail(m, SEM_ERR_OOM, "device allocation failed");
    if (n) {
        cudaError_t e = cudaMemcpyAsync(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice, m->stream);
        m->h2d += (int64_t)(n * sizeof(T));
        if (e != cudaSuccess) return cuda_fail(m, e, "cudaMemcpyAsync H2D");
        // host vectors may die right after this call returns
        e = cudaStreamSynchronize(m->stream);
        if (e != cudaSuccess) return cuda_fail(m, e, "cudaStreamSynchronize");
    }
    return SEM_OK;
}

sem_status zeros(sem_mesh* m, void** dst, size_t bytes) {
    *dst = dev_alloc(m, bytes);
    if (!*dst) return fail(m, SEM_ERR_OOM, "device allocation failed");
    cudaError_t e = cudaMemsetAsync(*dst, 0, bytes, m->stream);
    if (e != cudaSuccess) return cuda_fail(m, e, "cudaMemsetAsync");
    return SEM_OK;
}

bool fp64(const sem_mesh* m) { return m->prec == SEM_FP64; }
size_t tsize(const sem_mesh* m) { return fp64(m) ? 8 : 4; }
// s = dt^2 / M for the leapfrog, 1 / M for the first-order system.
double scale_numerator(const sem_mesh* m) { return m->scheme == SEM_SCHEME_HEUN ? 1.0 : m->dt * m->dt; }

int mode_of(const sem_mesh* m) {
    return m->prec == SEM_FP32_KAHAN ? semdev::MODE_KAHAN : semdev::MODE_THREE_LEVEL;
}

template <typename T>
void fill_basis(semdev::Basis<T>& b, int p) {
    std::vector<double> x, w, D;
    semhost::gll_rule(p, x, w);
    semhost::gll_derivative(x, D);
    std::memset(&b, 0, sizeof(b));
    const int n = p + 1;
    for (int i = 0; i < n; ++i) {
        b.x[i] = (T)x[i];
        b.w[i] = (T)w[i];
        for (int k = 0; k < n; ++k) b.D[i * n + k] = (T)D[(size_t)i * n + k];
    }
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) b.W[j * n + i] = (T)(w[(size_t)i] * w[(size_t)j]);
}

sem_status compute_orderings(sem_mesh* m) {
    std::vector<int64_t> eo, no;
    const std::string why = semhost::orderings(m->mesh, m->ordering, m->seed, eo, no);
    if (!why.empty()) return fail(m, SEM_ERR_UNSUPPORTED, why);
    m->elem_order.swap(eo);
    m->node_order.swap(no);
    m->elem_new.assign(m->elem_order.size(), 0);
    m->node_new.assign(m->node_order.size(), 0);
    for (size_t k = 0; k < m->elem_order.size(); ++k) m->elem_new[(size_t)m->elem_order[k]] = (int64_t)k;
    for (size_t k = 0; k < m->node_order.size(); ++k) m->node_new[(size_t)m->node_order[k]] = (int64_t)k;
    return SEM_OK;
}

sem_status fill_source(sem_mesh* m, int64_t upto) {
    // Ricker values f(t_n), t_n = n dt, tabulated in FP64 on the host.
    if (upto <= m->src_cap) return SEM_OK;
    int64_t cap = std::max<int64_t>(upto, std::max<int64_t>(1024, m->src_cap * 2));
    std::vector<double> f((size_t)cap, 0.0);
    if (m->have_src) {
        for (int64_t n = 0; n < cap; ++n) {
            double a = M_PI * m->f0 * ((double)n * m->dt - m->t0);
            a = a * a;
            f[(size_t)n] = m->amp * (1.0 - 2.0 * a) * std::exp(-a);
        }
    }
    double* d = nullptr;
    sem_status st = upload(m, &d, f.data(), f.size());
    if (st != SEM_OK) return st;
    m->d_src = d;  // the old table stays allocated until sem_destroy
    m->src_cap = cap;
    return SEM_OK;
}

// Smallest default block of a small mesh (elements).
constexpr int kMinSmallMeshEb = 4;

// SMs of the current device, or 0 when it cannot be queried.
int device_sm_count() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return sms;
}

int default_eb(int np, bool f64) {
    // about 6400 element points per block (FP32), at most 256 elements
    // (threads). FP64 blocks hold half as many (128 elements at order 4):
    // the FP64 kernels use about 254 registers per thread, so a 256-thread
    // block is alone on its SM and its memory phases leave the FP64 units
    // idle; two half-size blocks per SM overlap one's memory phases with the
    // other's arithmetic (graded 512 x 512, order 4: 10.6 against 9.8 G
    // node-updates/s; layered 4096 x 1024: 11.1 against 10.2 G)
    const int P = np * np;
    int eb = ((f64 ? 3200 : 6400) + P / 2) / P;
    if (eb > 256) eb = 256;
    if (eb < 1) eb = 1;
    return eb;
}

int vec_of(const sem_mesh* m) { return fp64(m) ? 2 : 4; }

constexpr int kSmemLimit = 227 * 1024;

// Shared memory the step kernel needs for the handle's plan (the larger of
// the time-stepping and the stiffness-only mode).
int plan_smem_bytes(const sem_mesh* m, int P) {
    const auto& pl = m->plan;
    const int v = vec_of(m);
    const int sulen_pad = (pl.max_sulen + v - 1) / v * v;
    const int slen_pad = (pl.max_slen + v - 1) / v * v;
    const int a = semdev::smem_bytes_for(P, pl.eb, pl.max_packet, sulen_pad, slen_pad, fp64(m), mode_of(m), pl.dense);
    const int b =
        semdev::smem_bytes_for(P, pl.eb, pl.max_packet, sulen_pad, slen_pad, fp64(m), semdev::MODE_APPLY, pl.dense);
    return std::max(std::max(a, b), sulen_pad * 8);
}

// Node arrays are allocated to a multiple of 16 bytes plus one vector so
// the kernels' aligned 16-byte copies of owned ranges never leave them.
size_t node_bytes(const sem_mesh* m) {
    const int64_t v = vec_of(m);
    return (size_t)(((m->mesh.nn + v - 1) / v + 1) * v) * tsize(m);
}

// Host part of the device data: orderings, receivers, block plan, and the
// element data in the plan's device order (kept until the device part). No
// CUDA calls, so several handles can run it in parallel threads.
sem_status build_host(sem_mesh* m) {
    if (m->built || m->host_ready) return SEM_OK;
    if (!m->have_model) return fail(m, SEM_ERR_STATE, "sem_set_model must come first");
    const auto& M = m->mesh;
    const int P = M.P;
    if (m->elem_order.empty()) {
        sem_status so = compute_orderings(m);
        if (so != SEM_OK) return so;
    }
    // permuted connectivity and element data
    std::vector<int32_t> conn_new((size_t)(M.ne * P));
    std::vector<int32_t> quads_new((size_t)M.ne * 4);
    std::vector<double> rho_new((size_t)M.ne), vel_new((size_t)M.ne);
    {
        // independent per element: split over host threads
        const int64_t T = std::max<int64_t>(
            1, std::min<int64_t>(std::min(16u, std::max(1u, std::thread::hardware_concurrency())), M.ne / 16384));
        auto part = [&](int64_t t) {
            for (int64_t en = M.ne * t / T; en < M.ne * (t + 1) / T; ++en) {
                const int64_t eo = m->elem_order[(size_t)en];
                for (int q = 0; q < P; ++q)
                    conn_new[(size_t)(en * P + q)] = (int32_t)m->node_new[(size_t)M.conn[(size_t)(eo * P + q)]];
                for (int c = 0; c < 4; ++c) quads_new[(size_t)en * 4 + c] = M.quads[(size_t)eo * 4 + c];
                rho_new[(size_t)en] = m->rho[(size_t)eo];
                vel_new[(size_t)en] = m->vel[(size_t)eo];
            }
        };
        std::vector<std::thread> pool;
        for (int64_t t = 1; t < T; ++t) pool.emplace_back(part, t);
        part(0);
        for (auto& th : pool) th.join();
    }
    // receivers: new node ids; a second receiver on the same node copies the
    // first one's trace on the host
    std::vector<int32_t> rec_gid((size_t)m->nrec, -1);
    m->rec_row.assign((size_t)m->nrec, -1);
    for (int32_t r = 0; r < m->nrec; ++r) {
        const int32_t g = (int32_t)m->node_new[(size_t)m->rec_nodes[(size_t)r]];
        for (int32_t q = 0; q < r; ++q)
            if (rec_gid[(size_t)q] == g) {
                m->rec_row[(size_t)r] = q;
                break;
            }
        if (m->rec_row[(size_t)r] < 0) rec_gid[(size_t)r] = g;
    }
    int eb = m->eb_request > 0 ? m->eb_request : default_eb(M.np, fp64(m));
    // small FP64 meshes (default size only): at least one block per SM, so
    // that a step's double-precision arithmetic, slow per SM on this GPU,
    // spreads over all of them (FP32 small meshes keep the larger blocks:
    // there a step is bound by one unit's chain of round trips, and fewer
    // blocks share fewer nodes)
    if (m->eb_request <= 0 && fp64(m) && m->sm_count > 0 && M.ne < (int64_t)eb * m->sm_count)
        eb = (int)std::max<int64_t>(kMinSmallMeshEb, (M.ne + m->sm_count - 1) / m->sm_count);
    if ((int64_t)eb * P > 65535) eb = 65535 / P;
    if (eb > 256) eb = 256;
    // the default block size shrinks until the step kernel's shared memory
    // fits (scattered orderings touch more distinct nodes per block)
    for (;;) {
        std::string why = semhost::build_block_plan(conn_new, M.ne, P, M.nn, eb, true, vec_of(m), rec_gid, m->plan);
        if (!why.empty()) return fail(m, SEM_ERR_UNSUPPORTED, "block plan: " + why);
        const int need = plan_smem_bytes(m, P);
        if (need <= kSmemLimit || m->eb_request > 0 || eb <= 4) break;
        eb = std::max(4, (int)((double)eb * 0.9 * kSmemLimit / need));
    }
    conn_new.clear();
    conn_new.shrink_to_fit();
    const auto& pl = m->plan;
    // element data in the plan's device order (blocks sorted by colour)
    {
        std::vector<int32_t> qd((size_t)M.ne * 4);
        std::vector<double> rd((size_t)M.ne), vd((size_t)M.ne);
        for (int64_t i = 0; i < M.ne; ++i) {
            const int64_t en = pl.dev_order[(size_t)i];
            for (int c = 0; c < 4; ++c) qd[(size_t)i * 4 + c] = quads_new[(size_t)en * 4 + c];
            rd[(size_t)i] = rho_new[(size_t)en];
            vd[(size_t)i] = vel_new[(size_t)en];
        }
        m->host_quads.swap(qd);
        m->host_rho.swap(rd);
        m->host_vel.swap(vd);
    }
    m->host_ready = true;
    return SEM_OK;
}

sem_status build(sem_mesh* m) {
    if (m->built) return SEM_OK;
    if (!m->host_ready && m->sm_count == 0) m->sm_count = device_sm_count();
    sem_status st = build_host(m);
    if (st != SEM_OK) return st;
    const auto& M = m->mesh;
    const int P = M.P;
    const auto& pl = m->plan;
    const std::vector<int32_t>& quads_new = m->host_quads;
    const std::vector<double>& rho_new = m->host_rho;
    const std::vector<double>& vel_new = m->host_vel;
    const int v = vec_of(m);
    const int sulen_pad = (pl.max_sulen + v - 1) / v * v;
    const int slen_pad = (pl.max_slen + v - 1) / v * v;
    m->threads = std::max(semdev::step_threads(pl.eb), m->threads_request);
    m->smem = semdev::smem_bytes_for(P, pl.eb, pl.max_packet, sulen_pad, slen_pad, fp64(m), mode_of(m), pl.dense);
    const int smem_apply = semdev::smem_bytes_for(P, pl.eb, pl.max_packet, sulen_pad, slen_pad, fp64(m),
                                                  semdev::MODE_APPLY, pl.dense);
    if (std::max(m->smem, smem_apply) > kSmemLimit)
        return fail(m, SEM_ERR_UNSUPPORTED, "block plan does not fit in shared memory; lower sem_set_tuning");

    uint8_t* packet;
    int32_t *hdr, *open_gid, *open_base, *open_cnt, *open_rec;
    uint32_t* epos;
    if ((st = upload(m, &packet, pl.packet.data(), pl.packet.size())) != SEM_OK) return st;
    if ((st = upload(m, &hdr, pl.hdr.data(), pl.hdr.size())) != SEM_OK) return st;
    if ((st = upload(m, &epos, pl.epos.data(), pl.epos.size())) != SEM_OK) return st;
    if ((st = upload(m, &open_gid, pl.open_gid.data(), pl.open_gid.size())) != SEM_OK) return st;
    if ((st = upload(m, &open_base, pl.open_base.data(), pl.open_base.size())) != SEM_OK) return st;
    if ((st = upload(m, &open_cnt, pl.open_cnt.data(), pl.open_cnt.size())) != SEM_OK) return st;
    if ((st = upload(m, &open_rec, pl.open_rec.data(), pl.open_rec.size())) != SEM_OK) return st;
    m->d_packet = packet;
    semdev::Plan& dp = m->dplan;
    dp.packet = packet;
    dp.hdr = reinterpret_cast<const int4*>(hdr);
    dp.epos = epos;
    dp.coef = nullptr;
    dp.G = nullptr;
    dp.G32 = nullptr;
    dp.open_gid = open_gid;
    dp.open_base = open_base;
    dp.open_cnt = open_cnt;
    dp.open_rec = open_rec;
    dp.ne = M.ne;
    dp.nn = M.nn;
    dp.eb = pl.eb;
    dp.nblocks = (int)pl.nblocks;
    dp.nopen_nodes = (int)pl.open_gid.size();
    dp.max_packet = pl.max_packet;
    dp.sulen_pad = sulen_pad;
    dp.slen_pad = slen_pad;
    dp.dense = pl.dense ? 1 : 0;
    dp.vec = vec_of(m);

    fill_basis(m->basis64, M.p);
    fill_basis(m->basis32, M.p);

    // FP64 geometry and mass on the device
    if ((st = upload(m, &m->d_coords, M.coords.data(), M.coords.size())) != SEM_OK) return st;
    if ((st = upload(m, &m->d_quads, quads_new.data(), quads_new.size())) != SEM_OK) return st;
    if ((st = upload(m, &m->d_rho, rho_new.data(), rho_new.size())) != SEM_OK) return st;
    if ((st = upload(m, &m->d_vel, vel_new.data(), vel_new.size())) != SEM_OK) return st;
    const size_t nslot = (size_t)(M.ne * P);
    m->d_mloc = (double*)dev_alloc(m, nslot * 8);
    m->d_M = (double*)dev_alloc(m, (size_t)M.nn * 8);
    const size_t pbytes = (size_t)std::max<int64_t>(pl.npartial, 1) * 8;
    m->d_part[0] = dev_alloc(m, pbytes);
    m->d_part[1] = dev_alloc(m, pbytes);
    if (!m->d_mloc || !m->d_M || !m->d_part[0] || !m->d_part[1])
        return fail(m, SEM_ERR_OOM, "device allocation failed");
    float4* coef = nullptr;
    if (fp64(m)) {
        m->d_G64 = (double*)dev_alloc(m, nslot * 3 * 8);
        if (!m->d_G64) return fail(m, SEM_ERR_OOM, "device allocation failed");
        dp.G = m->d_G64;
    } else {
        coef = (float4*)dev_alloc(m, (size_t)M.ne * 2 * sizeof(float4));
        if (!coef) return fail(m, SEM_ERR_OOM, "device allocation failed");
        dp.coef = coef;
        if (m->metric == SEM_METRIC_STORED) {
            m->d_G32 = (float*)dev_alloc(m, nslot * 3 * 4);
            if (!m->d_G32) return fail(m, SEM_ERR_OOM, "device allocation failed");
            dp.G32 = m->d_G32;
        }
    }
    if (m->scheme == SEM_SCHEME_HEUN && fp64(m)) {
        m->d_coef64 = (double*)dev_alloc(m, (size_t)M.ne * 8 * 8);
        if (!m->d_coef64) return fail(m, SEM_ERR_OOM, "device allocation failed");
        dp.coef64 = m->d_coef64;
    }
    SEM_CUDA(semdev::launch_geometry(M.np, M.ne, m->d_coords, m->d_quads, m->d_rho, m->d_vel, m->basis64, coef,
                                     m->d_G64, m->d_mloc, m->d_coef64, m->d_G32, m->stream));
    SEM_CUDA(semdev::launch_mass(dp, M.np, m->d_mloc, (double*)m->d_part[0], m->d_M, m->stream));

    // time-stepping state
    const size_t nb = node_bytes(m);
    const int nu = m->prec == SEM_FP32_KAHAN ? 2 : 3;
    for (int k = 0; k < nu; ++k)
        if ((st = zeros(m, &m->d_u[k], nb)) != SEM_OK) return st;
    if ((st = zeros(m, &m->d_s, nb)) != SEM_OK) return st;
    if (m->prec == SEM_FP32_KAHAN) {
        for (int k = 0; k < 2; ++k) {
            if ((st = zeros(m, &m->d_x[k], nb)) != SEM_OK) return st;
            if ((st = zeros(m, &m->d_c[k], nb)) != SEM_OK) return st;
        }
    }
    if (m->scheme == SEM_SCHEME_HEUN) {
        const size_t vb = (size_t)M.ne * (size_t)P * 2 * tsize(m);
        for (auto& v : m->d_v)
            if ((st = zeros(m, &v, vb)) != SEM_OK) return st;
        if ((st = zeros(m, &m->d_vd1, vb)) != SEM_OK) return st;
        if ((st = zeros(m, &m->d_ud1, nb)) != SEM_OK) return st;
    }
    if (m->have_dt) {
        SEM_CUDA(semdev::launch_scale(m->d_M, M.nn, scale_numerator(m), fp64(m) ? (double*)m->d_s : nullptr,
                                      fp64(m) ? nullptr : (float*)m->d_s, m->stream));
    }
    if (m->nrec > 0) {
        void* tr = nullptr;
        if ((st = zeros(m, &tr, (size_t)m->nrec * (size_t)m->trace_cap * 8)) != SEM_OK) return st;
        m->d_trace = (double*)tr;
    }
    // error word: raised on the device by a bounded wait that gave up (a
    // streamed unit's neighbour flags, a bulk copy's barrier)
    {
        void* er = nullptr;
        if ((st = zeros(m, &er, 4)) != SEM_OK) return st;
        m->d_err = (int32_t*)er;
    }
    // streamed time loop: leapfrog on a DENSE plan
    m->stream_ok = false;
    const int md = mode_of(m);
    if (pl.dense && m->scheme == SEM_SCHEME_LEAPFROG && (md == semdev::MODE_KAHAN || md == semdev::MODE_THREE_LEVEL) &&
        pl.max_deps <= semdev::kMaxStreamDeps) {
        // neighbour lists padded with the block itself to a common multiple
        // of 4 entries (one 16-byte row load per unit)
        const int stride = (pl.max_deps + 3) / 4 * 4;
        std::vector<int32_t> pad((size_t)pl.nblocks * (size_t)stride);
        for (int64_t b = 0; b < pl.nblocks; ++b)
            for (int t = 0; t < stride; ++t) {
                const int32_t k = pl.dep_ptr[(size_t)b] + t;
                pad[(size_t)b * stride + t] = k < pl.dep_ptr[(size_t)b + 1] ? pl.dep[(size_t)k] : (int32_t)b;
            }
        m->dep_stride = stride;
        if ((st = upload(m, &m->d_dep, pad.data(), pad.size())) != SEM_OK) return st;
        void *done = nullptr, *ctr = nullptr;
        if ((st = zeros(m, &done, (size_t)pl.nblocks * 4)) != SEM_OK) return st;
        if ((st = zeros(m, &ctr, 8)) != SEM_OK) return st;
        m->d_done = (uint32_t*)done;
        m->d_counter = (unsigned long long*)ctr;
        m->ticket_base = 0;
        m->serial = 1;
        int res = 0;
        SEM_CUDA(semdev::stream_resident_ctas(M.np, fp64(m), md, m->d_G32 != nullptr, m->threads, m->smem, &res));
        m->resident_ctas = res;
        m->stream_ok = res > 0;
    }
    cudaError_t e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return cuda_fail(m, e, "build");
    std::vector<int32_t>().swap(m->host_quads);
    std::vector<double>().swap(m->host_rho);
    std::vector<double>().swap(m->host_vel);
    m->host_ready = false;
    m->built = true;
    return SEM_OK;
}

// Element data of the current model in the plan's device order.
void device_order_model(const sem_mesh* m, std::vector<double>& rho_d, std::vector<double>& vel_d) {
    const int64_t ne = m->mesh.ne;
    rho_d.resize((size_t)ne);
    vel_d.resize((size_t)ne);
    for (int64_t i = 0; i < ne; ++i) {
        const int64_t eo = m->elem_order[(size_t)m->plan.dev_order[(size_t)i]];
        rho_d[(size_t)i] = m->rho[(size_t)eo];
        vel_d[(size_t)i] = m->vel[(size_t)eo];
    }
}

// New model on a built handle: geometry factors, lumped mass and dt^2/M are
// recomputed on the device; the plan and the state stay.
sem_status refresh_model(sem_mesh* m) {
    std::vector<double> rd, vd;
    device_order_model(m, rd, vd);
    SEM_CUDA(cudaMemcpyAsync(m->d_rho, rd.data(), rd.size() * 8, cudaMemcpyHostToDevice, m->stream));
    SEM_CUDA(cudaMemcpyAsync(m->d_vel, vd.data(), vd.size() * 8, cudaMemcpyHostToDevice, m->stream));
    m->h2d += (int64_t)(rd.size() + vd.size()) * 8;
    SEM_CUDA(semdev::launch_geometry(m->mesh.np, m->mesh.ne, m->d_coords, m->d_quads, m->d_rho, m->d_vel, m->basis64,
                                     const_cast<float4*>(m->dplan.coef), m->d_G64, m->d_mloc, m->d_coef64, m->d_G32,
                                     m->stream));
    SEM_CUDA(semdev::launch_mass(m->dplan, m->mesh.np, m->d_mloc, (double*)m->d_part[0], m->d_M, m->stream));
    if (m->have_dt)
        SEM_CUDA(semdev::launch_scale(m->d_M, m->mesh.nn, scale_numerator(m), fp64(m) ? (double*)m->d_s : nullptr,
                                      fp64(m) ? nullptr : (float*)m->d_s, m->stream));
    SEM_CUDA(cudaStreamSynchronize(m->stream));
    return SEM_OK;
}

// Buffers of level m.
void* level_u(const sem_mesh* m, int64_t lv) {
    return m->prec == SEM_FP32_KAHAN ? m->d_u[lv & 1] : m->d_u[((lv % 3) + 3) % 3];
}
void* level_x(const sem_mesh* m, int64_t lv) {
    return m->prec == SEM_FP32_KAHAN ? m->d_x[lv & 1] : m->d_u[(((lv - 1) % 3) + 3) % 3];
}
void* level_c(const sem_mesh* m, int64_t lv) { return m->prec == SEM_FP32_KAHAN ? m->d_c[lv & 1] : nullptr; }

// Arguments of launch k (reads level k, writes level k+1 at closed nodes).
template <typename T>
semdev::StepArgs<T> step_args(sem_mesh* m, int64_t k, bool pending) {
    semdev::StepArgs<T> a{};
    a.u_k = (const T*)level_u(m, k);
    a.x_k = (const T*)level_x(m, k);
    a.c_k = (const T*)level_c(m, k);
    a.u_km1 = (const T*)level_u(m, k - 1);
    a.x_km1 = (const T*)level_x(m, k - 1);
    a.c_km1 = (const T*)level_c(m, k - 1);
    a.u_kp1 = (T*)level_u(m, k + 1);
    a.x_kp1 = m->prec == SEM_FP32_KAHAN ? (T*)level_x(m, k + 1) : nullptr;
    a.c_kp1 = (T*)level_c(m, k + 1);
    a.u_kw = (T*)level_u(m, k);
    a.x_kw = m->prec == SEM_FP32_KAHAN ? (T*)level_x(m, k) : nullptr;
    a.c_kw = (T*)level_c(m, k);
    a.s = (const T*)m->d_s;
    a.part_rd = (const T*)m->d_part[(k + 1) & 1];
    a.part_wr = (T*)m->d_part[k & 1];
    a.apply_out = nullptr;
    a.src_f = m->d_src;
    a.step = k;
    a.src_gid = m->have_src ? (int32_t)m->node_new[(size_t)m->src_node] : -1;
    a.trace = m->d_trace;
    a.trace_cap = m->trace_cap;
    a.pending = pending ? 1 : 0;
    a.vec_ok = 1;
    a.err = m->d_err;
    return a;
}

cudaEvent_t take_event(sem_mesh* m) {
    if (!m->ev_pool.empty()) {
        cudaEvent_t e = m->ev_pool.back();
        m->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

const void* basis_of(const sem_mesh* m) {
    return fp64(m) ? (const void*)&m->basis64 : (const void*)&m->basis32;
}

// Device descriptor of the mesh's plan and level buffers (streamed
// launches and batches form each step's arguments from it).
template <typename T>
semdev::ShotDesc<T> shot_desc(const sem_mesh* m) {
    semdev::ShotDesc<T> d{};
    d.pl = m->dplan;
    for (int k = 0; k < 3; ++k) d.u[k] = (T*)m->d_u[k];
    for (int k = 0; k < 2; ++k) {
        d.x[k] = (T*)m->d_x[k];
        d.c[k] = (T*)m->d_c[k];
        d.part[k] = (T*)m->d_part[k];
    }
    d.s = (const T*)m->d_s;
    d.src_f = m->d_src;
    d.trace = m->d_trace;
    d.trace_cap = m->trace_cap;
    d.src_gid = m->have_src ? (int32_t)m->node_new[(size_t)m->src_node] : -1;
    d.err = m->d_err;
    return d;
}

// Streamed where the plan allows it and either asked for, or (automatic)
// where one launch per step would leave much of the GPU idle: at least one
// and fewer than 8 waves of resident CTAs per step, so that the partly
// filled last wave and the launch boundary cost more than the streamed
// units' own waits. With less than one wave every unit of a step runs at
// once either way, and streamed units only add their ticket, neighbour wait
// and release to each step (measured: homogeneous 128 x 128, FP64, 152
// blocks: 7.1 G node-updates/s one launch per step against 4.6 G streamed;
// FP32+Kahan 64 x 64, 16 blocks: 5.3 against 4.3 G).
constexpr int kAutoStreamSteps = 256;
constexpr int kAutoStreamWaves = 8;
bool streamed(const sem_mesh* m) {
    if (!m->stream_ok || m->stream_steps == 0) return false;
    if (m->stream_steps > 0) return true;
    return m->plan.nblocks >= (int64_t)m->resident_ctas &&
           m->plan.nblocks < (int64_t)kAutoStreamWaves * m->resident_ctas;
}
int64_t stream_len(const sem_mesh* m) { return m->stream_steps > 0 ? m->stream_steps : kAutoStreamSteps; }

// Band length and window of the wavefront order (0 steps: step order, the
// default: on the graded and layered meshes the wavefront order ran slower,
// its units waiting on neighbours issued shortly before them).
constexpr int kDefaultBandSteps = 0;
int band_steps_of(const sem_mesh* m) {
    const int T = m->band_req < 0 ? kDefaultBandSteps : m->band_req;
    return m->plan.nblocks >= ((int64_t)1 << semhost::kSchedShift) ? 0 : T;
}

// One band's wavefront order on the device for the current band length and
// window (built on the host, checked, uploaded once per setting).
sem_status ensure_schedule(sem_mesh* m, int T) {
    const auto& pl = m->plan;
    if (m->auto_window <= 0)
        m->auto_window = semhost::auto_window(semhost::block_levels(pl.dep_ptr.data(), pl.dep.data(), pl.nblocks),
                                              std::max(1, m->resident_ctas));
    const int W = m->window_req > 0 ? m->window_req : m->auto_window;
    if (m->d_sched && m->sched_T == T && m->sched_W == W) return SEM_OK;
    std::vector<uint32_t> sched;
    std::string why = semhost::stream_schedule(pl.dep_ptr.data(), pl.dep.data(), pl.nblocks, T, W, sched, nullptr);
    if (why.empty()) why = semhost::check_stream_schedule(pl.dep_ptr.data(), pl.dep.data(), pl.nblocks, T, sched);
    if (!why.empty()) return fail(m, SEM_ERR_STATE, "wavefront order: " + why);
    if (!m->d_sched || m->sched_cap < sched.size()) {
        void* p = nullptr;
        sem_status st = zeros(m, &p, sched.size() * 4);
        if (st != SEM_OK) return st;
        m->d_sched = (uint32_t*)p;
        m->sched_cap = sched.size();
    }
    SEM_CUDA(cudaMemcpyAsync(m->d_sched, sched.data(), sched.size() * 4, cudaMemcpyHostToDevice, m->stream));
    m->h2d += (int64_t)(sched.size() * 4);
    SEM_CUDA(cudaStreamSynchronize(m->stream));
    m->sched_T = T;
    m->sched_W = W;
    return SEM_OK;
}

// Steps k = m->step .. m->step + n - 1 as one streamed launch (pending: the
// open nodes of step m->step - 1 are not finished yet), recorded with events
// when profiling. Whole bands of the launch run in the wavefront order, the
// rest step after step.
sem_status launch_stream_steps(sem_mesh* m, int64_t n, bool pending) {
    const int T = band_steps_of(m);
    semdev::StreamArgs sa{};
    if (T > 0 && n >= T) {
        sem_status st = ensure_schedule(m, T);
        if (st != SEM_OK) return st;
        sa.sched = m->d_sched;
        sa.band_steps = T;
        sa.tiled_units = (n / T) * T * m->plan.nblocks;
    }
    sa.counter = m->d_counter;
    sa.base = m->ticket_base;
    sa.done = m->d_done;
    sa.dep = m->d_dep;
    sa.dep_stride = m->dep_stride;
    sa.err = m->d_err;
    sa.step0 = m->step;
    sa.nsteps = (int32_t)n;
    sa.pending0 = pending ? 1 : 0;
    sa.serial0 = m->serial;
    sa.hold_unit = -1;
    if (m->hold_step >= m->step && m->hold_step < m->step + n) {
        sa.hold_unit = (m->hold_step - m->step) * m->plan.nblocks + m->hold_block;
        m->hold_step = -1;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (m->profiling) {
        e0 = take_event(m);
        e1 = take_event(m);
        if (!e0 || !e1) return fail(m, SEM_ERR_CUDA, "cudaEventCreate failed");
    }
    cudaError_t e = e0 ? cudaEventRecord(e0, m->stream) : cudaSuccess;
    if (e == cudaSuccess) {
        if (fp64(m)) {
            auto d = shot_desc<double>(m);
            e = semdev::launch_stream(m->mesh.np, true, mode_of(m), &d, sa, basis_of(m), m->threads, m->smem,
                                      (int)m->plan.nblocks, m->stream);
        } else {
            auto d = shot_desc<float>(m);
            e = semdev::launch_stream(m->mesh.np, false, mode_of(m), &d, sa, basis_of(m), m->threads, m->smem,
                                      (int)m->plan.nblocks, m->stream);
        }
    }
    if (e == cudaSuccess && e1) e = cudaEventRecord(e1, m->stream);
    if (e != cudaSuccess) return cuda_fail(m, e, "streamed step launch");
    if (m->profiling) m->ev_block.push_back({e0, e1});
    m->serial += (uint32_t)n;
    m->ticket_base += (unsigned long long)n * (unsigned long long)m->plan.nblocks;
    m->step += n;
    return SEM_OK;
}

sem_status launch_one_step(sem_mesh* m, bool pending);

// Steps of one sem_step call: streamed launches of up to stream_steps steps,
// else one launch per step.
sem_status launch_steps(sem_mesh* m, int64_t nsteps) {
    sem_status st;
    const bool p0 = m->open_pending;
    for (int64_t k = 0; k < nsteps;) {
        if (streamed(m)) {
            // at most 2^31 - 1 CTAs per launch
            const int64_t cap = std::max<int64_t>(1, 2147483647LL / std::max<int64_t>(1, m->plan.nblocks));
            const int64_t n = std::min<int64_t>(std::min<int64_t>(nsteps - k, stream_len(m)), cap);
            if ((st = launch_stream_steps(m, n, k > 0 || p0)) != SEM_OK) return st;
            k += n;
        } else {
            if ((st = launch_one_step(m, k > 0 || p0)) != SEM_OK) return st;
            k += 1;
        }
        m->open_pending = true;
    }
    return SEM_OK;
}

// A wait of a streamed launch that gave up leaves the error flag raised; it
// is reported once and cleared (the state is then the caller's to reset).
sem_status check_stream_error(sem_mesh* m) {
    if (!m->d_err) return SEM_OK;
    int32_t h = 0;
    SEM_CUDA(cudaMemcpyAsync(&h, m->d_err, 4, cudaMemcpyDeviceToHost, m->stream));
    SEM_CUDA(cudaStreamSynchronize(m->stream));
    if (h != 0) {
        SEM_CUDA(cudaMemsetAsync(m->d_err, 0, 4, m->stream));
        SEM_CUDA(cudaStreamSynchronize(m->stream));
        return fail(m, SEM_ERR_TIMEOUT,
                    "a step gave up waiting (a streamed unit for a neighbouring block, or a block for its bulk copy); "
                    "steps were skipped");
    }
    return SEM_OK;
}

// Launch k of a run: the step kernel (pending = not the first launch of the
// run), recorded with events when profiling.
sem_status launch_one_step(sem_mesh* m, bool pending) {
    const bool f64 = fp64(m);
    const int mode = mode_of(m);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (m->profiling) {
        e0 = take_event(m);
        e1 = take_event(m);
        if (!e0 || !e1) return fail(m, SEM_ERR_CUDA, "cudaEventCreate failed");
    }
    cudaError_t e = e0 ? cudaEventRecord(e0, m->stream) : cudaSuccess;
    if (e == cudaSuccess) {
        if (f64) {
            auto a = step_args<double>(m, m->step, pending);
            e = semdev::launch_step(m->mesh.np, true, mode, m->dplan, &a, basis_of(m), m->threads, m->smem, m->stream);
        } else {
            auto a = step_args<float>(m, m->step, pending);
            e = semdev::launch_step(m->mesh.np, false, mode, m->dplan, &a, basis_of(m), m->threads, m->smem, m->stream);
        }
    }
    if (e == cudaSuccess && e1) e = cudaEventRecord(e1, m->stream);
    if (e != cudaSuccess) return cuda_fail(m, e, "step launch");
    if (m->profiling) m->ev_block.push_back({e0, e1});
    m->step++;
    return SEM_OK;
}

sem_status launch_flush(sem_mesh* m);
// The open nodes of the last step finished (the open-node kernel), if they
// are still partial sums.
sem_status flush_pending(sem_mesh* m) {
    if (!m->open_pending) return SEM_OK;
    m->open_pending = false;
    return launch_flush(m);
}

// After the last launch k of a run: finish the open nodes to level k+1.
sem_status launch_flush(sem_mesh* m) {
    const bool f64 = fp64(m);
    const int mode = mode_of(m);
    const int64_t k = m->step - 1;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (m->profiling) {
        e0 = take_event(m);
        e1 = take_event(m);
        if (!e0 || !e1) return fail(m, SEM_ERR_CUDA, "cudaEventCreate failed");
    }
    cudaError_t e = e0 ? cudaEventRecord(e0, m->stream) : cudaSuccess;
    if (e == cudaSuccess) {
        if (f64) {
            auto a = step_args<double>(m, k, false);
            a.part_rd = (const double*)m->d_part[k & 1];
            e = semdev::launch_open_finish(true, mode, m->dplan, &a, m->stream);
        } else {
            auto a = step_args<float>(m, k, false);
            a.part_rd = (const float*)m->d_part[k & 1];
            e = semdev::launch_open_finish(false, mode, m->dplan, &a, m->stream);
        }
    }
    if (e == cudaSuccess && e1) e = cudaEventRecord(e1, m->stream);
    if (e != cudaSuccess) return cuda_fail(m, e, "open-node launch");
    if (m->profiling) m->ev_open.push_back({e0, e1});
    return SEM_OK;
}

// One step of Heun's method on the first-order system: predictor and
// corrector, each a step-kernel launch plus the open-node launch.
template <typename T>
sem_status heun_launches(sem_mesh* m) {
    const bool f64 = fp64(m);
    semdev::StepArgs<T> a{};
    a.s = (const T*)m->d_s;
    a.src_f = m->d_src;
    a.src_gid = m->have_src ? (int32_t)m->node_new[(size_t)m->src_node] : -1;
    a.trace = m->d_trace;
    a.trace_cap = m->trace_cap;
    a.vec_ok = 1;
    a.err = m->d_err;
    a.h = m->dt;
    a.u_d1 = (T*)m->d_ud1;
    a.v_d1 = (T*)m->d_vd1;
    a.part_wr = (T*)m->d_part[0];
    a.part_rd = (const T*)m->d_part[0];
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (m->profiling) {
        e0 = take_event(m);
        e1 = take_event(m);
        if (!e0 || !e1) return fail(m, SEM_ERR_CUDA, "cudaEventCreate failed");
        SEM_CUDA(cudaEventRecord(e0, m->stream));
    }
    for (int phase = 0; phase < 2; ++phase) {
        const int mode = phase == 0 ? semdev::MODE_HEUN_P : semdev::MODE_HEUN_C;
        a.step = m->step + phase;                       // source at t_n, then t_{n+1}
        a.u_k = (const T*)m->d_u[phase];                // U, then U~
        a.u_kp1 = (T*)m->d_u[phase == 0 ? 1 : 0];       // U~, then U (in place)
        a.u_old = (const T*)m->d_u[0];
        a.v_in = (const T*)m->d_v[phase];               // V, then V~
        a.v_out = (T*)m->d_v[phase == 0 ? 1 : 0];       // V~, then V (in place)
        a.v_old = (const T*)m->d_v[0];
        SEM_CUDA(semdev::launch_step(m->mesh.np, f64, mode, m->dplan, &a, basis_of(m), m->threads, m->smem,
                                     m->stream));
        SEM_CUDA(semdev::launch_open_finish(f64, mode, m->dplan, &a, m->stream));
    }
    if (m->profiling) {
        SEM_CUDA(cudaEventRecord(e1, m->stream));
        m->ev_block.push_back({e0, e1});
    }
    m->step++;
    return SEM_OK;
}

sem_status launch_heun_step(sem_mesh* m) { return fp64(m) ? heun_launches<double>(m) : heun_launches<float>(m); }

// K u for u in the library's storage type and order (dev_in), into dev_out,
// with `partial` as scratch for the open entries' partial sums.
sem_status launch_apply(sem_mesh* m, const void* dev_in, void* dev_out, void* partial) {
    const bool f64 = fp64(m);
    // 16-byte vector copies and stores need both vectors 16-byte aligned
    const bool vok = ((uintptr_t)dev_in % 16) == 0 && ((uintptr_t)dev_out % 16) == 0;
    cudaError_t e;
    if (f64) {
        semdev::StepArgs<double> a{};
        a.u_k = (const double*)dev_in;
        a.apply_out = (double*)dev_out;
        a.part_wr = (double*)partial;
        a.part_rd = (const double*)partial;
        a.vec_ok = vok;
        a.src_gid = -1;
        a.err = m->d_err;
        e = semdev::launch_step(m->mesh.np, true, semdev::MODE_APPLY, m->dplan, &a, basis_of(m), m->threads, m->smem,
                                m->stream);
        if (e == cudaSuccess) e = semdev::launch_open_finish(true, semdev::MODE_APPLY, m->dplan, &a, m->stream);
    } else {
        semdev::StepArgs<float> a{};
        a.u_k = (const float*)dev_in;
        a.apply_out = (float*)dev_out;
        a.part_wr = (float*)partial;
        a.part_rd = (const float*)partial;
        a.vec_ok = vok;
        a.src_gid = -1;
        a.err = m->d_err;
        e = semdev::launch_step(m->mesh.np, false, semdev::MODE_APPLY, m->dplan, &a, basis_of(m), m->threads,
                                m->smem, m->stream);
        if (e == cudaSuccess) e = semdev::launch_open_finish(false, semdev::MODE_APPLY, m->dplan, &a, m->stream);
    }
    if (e != cudaSuccess) return cuda_fail(m, e, "apply launch");
    return SEM_OK;
}

template <typename T>
void to_new_order(const sem_mesh* m, const double* src, std::vector<T>& dst) {
    dst.resize(m->node_order.size());
    for (size_t k = 0; k < dst.size(); ++k) dst[k] = (T)src[(size_t)m->node_order[k]];
}

sem_status read_nodes(sem_mesh* m, const void* dptr, bool as_f64, std::vector<double>& out_new) {
    const size_t nn = (size_t)m->mesh.nn;
    out_new.assign(nn, 0.0);
    if (as_f64) {
        SEM_CUDA(cudaMemcpyAsync(out_new.data(), dptr, nn * 8, cudaMemcpyDeviceToHost, m->stream));
        m->d2h += (int64_t)(nn * 8);
        SEM_CUDA(cudaStreamSynchronize(m->stream));
    } else {
        std::vector<float> tmp(nn);
        SEM_CUDA(cudaMemcpyAsync(tmp.data(), dptr, nn * 4, cudaMemcpyDeviceToHost, m->stream));
        m->d2h += (int64_t)(nn * 4);
        SEM_CUDA(cudaStreamSynchronize(m->stream));
        for (size_t k = 0; k < nn; ++k) out_new[k] = (double)tmp[k];
    }
    return SEM_OK;
}

void to_original(const sem_mesh* m, const std::vector<double>& v_new, double* out) {
    for (size_t k = 0; k < v_new.size(); ++k) out[(size_t)m->node_order[k]] = v_new[k];
}

sem_status write_nodes(sem_mesh* m, void* dptr, const double* src_orig) {
    if (fp64(m)) {
        std::vector<double> v;
        to_new_order(m, src_orig, v);
        SEM_CUDA(cudaMemcpyAsync(dptr, v.data(), v.size() * 8, cudaMemcpyHostToDevice, m->stream));
        m->h2d += (int64_t)(v.size() * 8);
        SEM_CUDA(cudaStreamSynchronize(m->stream));
    } else {
        std::vector<float> v;
        to_new_order(m, src_orig, v);
        SEM_CUDA(cudaMemcpyAsync(dptr, v.data(), v.size() * 4, cudaMemcpyHostToDevice, m->stream));
        m->h2d += (int64_t)(v.size() * 4);
        SEM_CUDA(cudaStreamSynchronize(m->stream));
    }
    return SEM_OK;
}

bool before_first_step(sem_mesh* m) { return !m->built; }

}  // namespace

extern "C" {

sem_status sem_set_allocator(sem_alloc_fn alloc, sem_free_fn free_fn, void* ctx) {
    if ((alloc == nullptr) != (free_fn == nullptr)) return SEM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc = alloc;
    g_free = free_fn;
    g_alloc_ctx = ctx;
    return SEM_OK;
}

sem_status sem_mesh_create(const double* coords, int64_t nv, const int32_t* quads, int64_t ne, int order,
                           sem_precision prec, void* cuda_stream, sem_mesh** out) {
    if (!out) return SEM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!coords || !quads) return SEM_ERR_INVALID_ARG;
    if (prec != SEM_FP64 && prec != SEM_FP32_KAHAN && prec != SEM_FP32) return SEM_ERR_INVALID_ARG;
    if (ne > 0 && (ne * (int64_t)(order + 1) * (order + 1) >= (int64_t)1 << 31)) return SEM_ERR_UNSUPPORTED;
    std::string why = semhost::validate(coords, nv, quads, ne, order);
    if (!why.empty()) return SEM_ERR_INVALID_ARG;
    sem_mesh* m = new (std::nothrow) sem_mesh();
    if (!m) return SEM_ERR_OOM;
    try {
        m->mesh.p = order;
        m->mesh.nv = nv;
        m->mesh.ne = ne;
        m->mesh.coords.assign(coords, coords + nv * 2);
        m->mesh.quads.assign(quads, quads + ne * 4);
        semhost::number_nodes(m->mesh);
    } catch (const std::bad_alloc&) {
        delete m;
        return SEM_ERR_OOM;
    }
    if (m->mesh.nn >= ((int64_t)1 << 31)) {
        delete m;
        return SEM_ERR_UNSUPPORTED;
    }
    m->prec = prec;
    m->stream = (cudaStream_t)cuda_stream;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        m->alloc = g_alloc;
        m->free_fn = g_free;
        m->alloc_ctx = g_alloc_ctx;
    }
    *out = m;
    return SEM_OK;
}

sem_status sem_reorder(sem_mesh* m, sem_ordering kind, uint64_t seed) {
    if (!m) return SEM_ERR_INVALID_ARG;
    if ((int)kind < 0 || (int)kind > 6) return fail(m, SEM_ERR_INVALID_ARG, "unknown ordering");
    if (!before_first_step(m)) return fail(m, SEM_ERR_STATE, "sem_reorder after the device data was built");
    const int old_kind = m->ordering;
    const uint64_t old_seed = m->seed;
    m->ordering = (int)kind;
    m->seed = seed;
    sem_status st;
    try {
        st = compute_orderings(m);
    } catch (const std::bad_alloc&) {
        st = fail(m, SEM_ERR_OOM, "host allocation failed");
    }
    if (st != SEM_OK) {
        m->ordering = old_kind;
        m->seed = old_seed;
    }
    return st;
}

sem_status sem_set_model(sem_mesh* m, const double* vel, const double* rho) {
    if (!m || !vel) return m ? fail(m, SEM_ERR_INVALID_ARG, "vel is NULL") : SEM_ERR_INVALID_ARG;
    const int64_t ne = m->mesh.ne;
    for (int64_t e = 0; e < ne; ++e) {
        if (!(vel[e] > 0.0) || !std::isfinite(vel[e])) return fail(m, SEM_ERR_INVALID_ARG, "vel must be > 0");
        if (rho && (!(rho[e] > 0.0) || !std::isfinite(rho[e]))) return fail(m, SEM_ERR_INVALID_ARG, "rho must be > 0");
    }
    m->vel.assign(vel, vel + ne);
    if (rho) m->rho.assign(rho, rho + ne);
    else m->rho.assign((size_t)ne, 1.0);
    m->have_model = true;
    if (m->built) {
        // the pending open nodes belong to the old model's step
        if (sem_status sf = flush_pending(m)) return sf;
        return refresh_model(m);
    }
    return SEM_OK;
}

static void ensure_node_xy(sem_mesh* m) {
    if (m->node_xy.empty()) semhost::node_coordinates(m->mesh, m->node_xy);
}

sem_status sem_set_source(sem_mesh* m, int kind, double f0, double t0, double amp, double x, double y) {
    if (!m) return SEM_ERR_INVALID_ARG;
    if (kind != SEM_SRC_RICKER) return fail(m, SEM_ERR_INVALID_ARG, "unknown source kind");
    if (!(f0 > 0.0) || !std::isfinite(t0) || !std::isfinite(amp) || !std::isfinite(x) || !std::isfinite(y))
        return fail(m, SEM_ERR_INVALID_ARG, "bad source parameters");
    if (!before_first_step(m)) return fail(m, SEM_ERR_STATE, "sem_set_source after the first step");
    ensure_node_xy(m);
    m->f0 = f0;
    m->t0 = t0;
    m->amp = amp;
    m->sx = x;
    m->sy = y;
    m->src_node = semhost::snap(m->node_xy, x, y);
    m->have_src = true;
    return SEM_OK;
}

sem_status sem_set_receivers(sem_mesh* m, const double* xy, int32_t nrec, int64_t max_steps) {
    if (!m) return SEM_ERR_INVALID_ARG;
    if (nrec < 0 || (nrec > 0 && (!xy || max_steps < 1))) return fail(m, SEM_ERR_INVALID_ARG, "bad receivers");
    if (!before_first_step(m)) return fail(m, SEM_ERR_STATE, "sem_set_receivers after the first step");
    ensure_node_xy(m);
    m->rec_nodes.assign((size_t)nrec, 0);
    {
        std::vector<int64_t> got;
        semhost::snap_many(m->node_xy, xy, xy + 1, nrec, 2, got);
        for (int32_t r = 0; r < nrec; ++r) m->rec_nodes[(size_t)r] = got[(size_t)r];
    }
    m->nrec = nrec;
    m->trace_cap = nrec > 0 ? max_steps : 0;
    return SEM_OK;
}

sem_status sem_cfl_dt(const sem_mesh* m, double* dt_cfl) {
    if (!m || !dt_cfl) return SEM_ERR_INVALID_ARG;
    if (!m->have_model) return SEM_ERR_STATE;
    *dt_cfl = semhost::cfl_dt(m->mesh, m->vel.data());
    return SEM_OK;
}

sem_status sem_set_scheme(sem_mesh* m, int scheme) {
    if (!m) return SEM_ERR_INVALID_ARG;
    if (scheme != SEM_SCHEME_LEAPFROG && scheme != SEM_SCHEME_HEUN) return fail(m, SEM_ERR_INVALID_ARG, "unknown scheme");
    if (!before_first_step(m)) return fail(m, SEM_ERR_STATE, "sem_set_scheme after the device data was built");
    if (scheme == SEM_SCHEME_HEUN && m->prec == SEM_FP32_KAHAN)
        return fail(m, SEM_ERR_UNSUPPORTED, "the first-order scheme runs on SEM_FP64 or SEM_FP32");
    if (scheme == SEM_SCHEME_HEUN && m->metric == SEM_METRIC_STORED && !fp64(m))
        return fail(m, SEM_ERR_UNSUPPORTED, "the first-order scheme forms its FP32 metric from the bilinear map");
    m->scheme = scheme;
    return SEM_OK;
}

sem_status sem_set_metric(sem_mesh* m, int metric) {
    if (!m) return SEM_ERR_INVALID_ARG;
    if (metric != SEM_METRIC_BILINEAR && metric != SEM_METRIC_STORED)
        return fail(m, SEM_ERR_INVALID_ARG, "unknown metric source");
    if (!before_first_step(m)) return fail(m, SEM_ERR_STATE, "sem_set_metric after the device data was built");
    if (fp64(m)) return SEM_OK;
    if (metric == SEM_METRIC_STORED && m->scheme == SEM_SCHEME_HEUN)
        return fail(m, SEM_ERR_UNSUPPORTED, "the first-order scheme forms its FP32 metric from the bilinear map");
    m->metric = metric;
    return SEM_OK;
}

sem_status sem_read_metric(sem_mesh* m, double* G) {
    if (!m || !G) return SEM_ERR_INVALID_ARG;
    if (!m->have_model) return fail(m, SEM_ERR_STATE, "sem_set_model must come first");
    sem_status st = build(m);
    if (st != SEM_OK) return st;
    const int64_t ne = m->mesh.ne;
    const int P = m->mesh.P;
    const size_t nslot = (size_t)ne * (size_t)P;
    std::vector<double> g(nslot * 3);   // [dev element][q][3]
    if (fp64(m) || m->d_G32) {
        // stored [3P][ne], element-fastest
        std::vector<double> raw(nslot * 3);
        if (fp64(m)) {
            SEM_CUDA(cudaMemcpyAsync(raw.data(), m->d_G64, raw.size() * 8, cudaMemcpyDeviceToHost, m->stream));
            m->d2h += (int64_t)(raw.size() * 8);
        } else {
            std::vector<float> r32(nslot * 3);
            SEM_CUDA(cudaMemcpyAsync(r32.data(), m->d_G32, r32.size() * 4, cudaMemcpyDeviceToHost, m->stream));
            m->d2h += (int64_t)(r32.size() * 4);
            SEM_CUDA(cudaStreamSynchronize(m->stream));
            for (size_t k = 0; k < raw.size(); ++k) raw[k] = (double)r32[k];
        }
        SEM_CUDA(cudaStreamSynchronize(m->stream));
        for (int64_t e = 0; e < ne; ++e)
            for (int q = 0; q < P; ++q)
                for (int c = 0; c < 3; ++c)
                    g[((size_t)e * P + q) * 3 + c] = raw[((size_t)c * P + q) * (size_t)ne + (size_t)e];
    } else {
        if (!m->d_metric_out) {
            m->d_metric_out = (double*)dev_alloc(m, nslot * 3 * 8);
            if (!m->d_metric_out) return fail(m, SEM_ERR_OOM, "device allocation failed");
        }
        SEM_CUDA(semdev::launch_metric_fp32(m->mesh.np, m->dplan, m->basis32, m->d_metric_out, m->stream));
        SEM_CUDA(cudaMemcpyAsync(g.data(), m->d_metric_out, g.size() * 8, cudaMemcpyDeviceToHost, m->stream));
        m->d2h += (int64_t)(g.size() * 8);
        SEM_CUDA(cudaStreamSynchronize(m->stream));
    }
    // device element i is original element elem_order[dev_order[i]]
    for (int64_t i = 0; i < ne; ++i) {
        const int64_t eo = m->elem_order[(size_t)m->plan.dev_order[(size_t)i]];
        std::copy(g.begin() + (size_t)i * P * 3, g.begin() + (size_t)(i + 1) * P * 3, G + (size_t)eo * P * 3);
    }
    return SEM_OK;
}

sem_status sem_set_dt(sem_mesh* m, double dt) {
    if (!m) return SEM_ERR_INVALID_ARG;
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(m, SEM_ERR_INVALID_ARG, "dt must be > 0");
    if (!before_first_step(m)) return fail(m, SEM_ERR_STATE, "sem_set_dt after the device data was built");
    m->dt = dt;
    m->have_dt = true;
    return SEM_OK;
}

sem_status sem_set_tuning(sem_mesh* m, int elems_per_block, int threads_per_block) {
    if (!m) return SEM_ERR_INVALID_ARG;
    if (elems_per_block < 0 || elems_per_block > 256 || (int64_t)elems_per_block * m->mesh.P > 65535)
        return fail(m, SEM_ERR_INVALID_ARG, "elems_per_block out of range");
    if (threads_per_block < 0 || threads_per_block > 256 || threads_per_block % 32 != 0)
        return fail(m, SEM_ERR_INVALID_ARG, "threads_per_block must be 0 or a multiple of 32 up to 256");
    if (!before_first_step(m)) return fail(m, SEM_ERR_STATE, "sem_set_tuning after the device data was built");
    m->eb_request = elems_per_block;
    m->threads_request = threads_per_block;
    return SEM_OK;
}

sem_status sem_set_stream(sem_mesh* m, int steps_per_launch) {
    if (!m) return SEM_ERR_INVALID_ARG;
    if (steps_per_launch < -1 || steps_per_launch > 65536)
        return fail(m, SEM_ERR_INVALID_ARG, "steps_per_launch must be in -1..65536");
    m->stream_steps = steps_per_launch;
    return SEM_OK;
}

sem_status sem_set_stream_tiling(sem_mesh* m, int band_steps, int window_levels) {
    if (!m) return SEM_ERR_INVALID_ARG;
    if (band_steps < -1 || band_steps > semhost::kSchedMaxSteps)
        return fail(m, SEM_ERR_INVALID_ARG, "band_steps must be in -1..255");
    if (window_levels < 0) return fail(m, SEM_ERR_INVALID_ARG, "window_levels must be >= 0");
    m->band_req = band_steps;
    m->window_req = window_levels;
    return SEM_OK;
}

sem_status sem_stream_order(const sem_mesh* m, int32_t* band_steps, int32_t* window_levels) {
    if (!m) return SEM_ERR_INVALID_ARG;
    if (band_steps) *band_steps = m->sched_T;
    if (window_levels) *window_levels = m->sched_W;
    return SEM_OK;
}

sem_status sem_stream_schedule(const int32_t* dep_ptr, const int32_t* dep, int32_t nblocks, int band_steps,
                               int window_levels, uint32_t* sched, int32_t* levels) {
    if (!dep_ptr || !dep || !sched || nblocks < 1 || band_steps < 1 || window_levels < 1) return SEM_ERR_INVALID_ARG;
    if (dep_ptr[0] != 0) return SEM_ERR_INVALID_ARG;
    for (int32_t b = 0; b < nblocks; ++b) {
        if (dep_ptr[b + 1] < dep_ptr[b]) return SEM_ERR_INVALID_ARG;
        bool self = false;
        for (int32_t t = dep_ptr[b]; t < dep_ptr[b + 1]; ++t) {
            if (dep[t] < 0 || dep[t] >= nblocks) return SEM_ERR_INVALID_ARG;
            self = self || dep[t] == b;
        }
        if (!self) return SEM_ERR_INVALID_ARG;
    }
    // the graph must be symmetric (sharing a node is)
    for (int32_t b = 0; b < nblocks; ++b)
        for (int32_t t = dep_ptr[b]; t < dep_ptr[b + 1]; ++t) {
            const int32_t c = dep[t];
            if (std::find(dep + dep_ptr[c], dep + dep_ptr[c + 1], b) == dep + dep_ptr[c + 1]) return SEM_ERR_INVALID_ARG;
        }
    std::vector<uint32_t> sc;
    std::vector<int32_t> lev;
    std::string why = semhost::stream_schedule(dep_ptr, dep, nblocks, band_steps, window_levels, sc, &lev);
    if (!why.empty()) return SEM_ERR_INVALID_ARG;
    why = semhost::check_stream_schedule(dep_ptr, dep, nblocks, band_steps, sc);
    if (!why.empty()) return SEM_ERR_STATE;
    std::memcpy(sched, sc.data(), sc.size() * 4);
    if (levels) std::memcpy(levels, lev.data(), lev.size() * 4);
    return SEM_OK;
}

sem_status sem_stream_withhold(sem_mesh* m, int64_t step, int32_t block) {
    if (!m) return SEM_ERR_INVALID_ARG;
    if (step < 0 || block < 0) {
        m->hold_step = -1;
        m->hold_block = -1;
        return SEM_OK;
    }
    m->hold_step = step;
    m->hold_block = block;
    return SEM_OK;
}

sem_status sem_step(sem_mesh* m, int64_t nsteps) {
    if (!m) return SEM_ERR_INVALID_ARG;
    if (nsteps < 0) return fail(m, SEM_ERR_INVALID_ARG, "nsteps < 0");
    if (!m->have_model || !m->have_dt) return fail(m, SEM_ERR_STATE, "model and dt must be set before sem_step");
    sem_status st = build(m);
    if (st != SEM_OK) return st;
    if (m->nrec > 0 && m->step + nsteps > m->trace_cap)
        return fail(m, SEM_ERR_INVALID_ARG, "steps beyond the receivers' max_steps");
    if (nsteps == 0) return SEM_OK;
    if ((st = fill_source(m, m->step + nsteps + 1)) != SEM_OK) return st;
    if (m->scheme == SEM_SCHEME_HEUN) {
        for (int64_t k = 0; k < nsteps; ++k)
            if ((st = launch_heun_step(m)) != SEM_OK) return st;
        m->stepped_calls++;
        return SEM_OK;
    }
    // every launch but the first of a stored level finishes the open nodes
    // of the previous step itself; those of the last step stay pending until
    // the next sem_step finishes them the same way, or a read of the state
    // runs the open-node kernel
    if ((st = launch_steps(m, nsteps)) != SEM_OK) return st;
    m->stepped_calls++;
    return SEM_OK;
}

sem_status sem_get_step(const sem_mesh* m, int64_t* step) {
    if (!m || !step) return SEM_ERR_INVALID_ARG;
    *step = m->step;
    return SEM_OK;
}

sem_status sem_read_traces(sem_mesh* m, double* out, int64_t cap) {
    if (!m || !out || cap < 0) return SEM_ERR_INVALID_ARG;
    if (m->nrec == 0 || cap == 0) return SEM_OK;
    if (!m->built) {
        std::fill(out, out + (size_t)m->nrec * (size_t)cap, 0.0);
        return SEM_OK;
    }
    sem_status st = flush_pending(m);
    if (st != SEM_OK) return st;
    if ((st = check_stream_error(m)) != SEM_OK) return st;
    const int64_t n = std::min(cap, m->step);
    std::fill(out, out + (size_t)m->nrec * (size_t)cap, 0.0);
    if (n > 0) {
        SEM_CUDA(cudaMemcpy2DAsync(out, (size_t)cap * 8, m->d_trace, (size_t)m->trace_cap * 8, (size_t)n * 8,
                                   (size_t)m->nrec, cudaMemcpyDeviceToHost, m->stream));
        m->d2h += (int64_t)n * 8 * m->nrec;
    }
    SEM_CUDA(cudaStreamSynchronize(m->stream));
    for (int32_t r = 0; r < m->nrec; ++r) {
        const int32_t q = m->rec_row[(size_t)r];
        if (q >= 0) std::copy(out + (size_t)q * cap, out + (size_t)(q + 1) * cap, out + (size_t)r * cap);
    }
    return SEM_OK;
}

sem_status sem_read_wavefield(sem_mesh* m, double* u) { return sem_get_state(m, u, nullptr, nullptr); }

sem_status sem_set_state(sem_mesh* m, const double* u, const double* u_prev, int64_t step) {
    if (!m || !u || !u_prev || step < 0) return SEM_ERR_INVALID_ARG;
    if (!m->have_model || !m->have_dt) return fail(m, SEM_ERR_STATE, "model and dt must be set first");
    sem_status st = build(m);
    if (st != SEM_OK) return st;
    if (m->nrec > 0 && step > m->trace_cap) return fail(m, SEM_ERR_INVALID_ARG, "step beyond max_steps");
    m->step = step;
    m->open_pending = false;   // the state is replaced whole
    if (m->scheme == SEM_SCHEME_HEUN) {
        if ((st = write_nodes(m, m->d_u[0], u)) != SEM_OK) return st;
        const size_t vb = (size_t)m->mesh.ne * (size_t)m->mesh.P * 2 * tsize(m);
        SEM_CUDA(cudaMemsetAsync(m->d_v[0], 0, vb, m->stream));
        SEM_CUDA(cudaStreamSynchronize(m->stream));
        return SEM_OK;
    }
    if ((st = write_nodes(m, level_u(m, step), u)) != SEM_OK) return st;
    if (m->prec == SEM_FP32_KAHAN) {
        std::vector<double> d((size_t)m->mesh.nn);
        for (size_t k = 0; k < d.size(); ++k) d[k] = u[k] - u_prev[k];
        if ((st = write_nodes(m, level_x(m, step), d.data())) != SEM_OK) return st;
        SEM_CUDA(cudaMemsetAsync(level_c(m, step), 0, (size_t)m->mesh.nn * 4, m->stream));
        SEM_CUDA(cudaStreamSynchronize(m->stream));
    } else {
        if ((st = write_nodes(m, level_x(m, step), u_prev)) != SEM_OK) return st;
    }
    return SEM_OK;
}

sem_status sem_get_state(sem_mesh* m, double* u, double* u_prev, int64_t* step) {
    if (!m) return SEM_ERR_INVALID_ARG;
    if (step) *step = m->step;
    const size_t nn = (size_t)m->mesh.nn;
    if (!m->built) {
        if (u) std::fill(u, u + nn, 0.0);
        if (u_prev) std::fill(u_prev, u_prev + nn, 0.0);
        return SEM_OK;
    }
    if (sem_status sf = flush_pending(m)) return sf;
    if (sem_status se = check_stream_error(m)) return se;
    std::vector<double> un, tmp;
    if (m->scheme == SEM_SCHEME_HEUN) {
        sem_status st = read_nodes(m, m->d_u[0], fp64(m), un);
        if (st != SEM_OK) return st;
        if (u) to_original(m, un, u);
        if (u_prev) std::fill(u_prev, u_prev + nn, 0.0);
        return SEM_OK;
    }
    sem_status st = read_nodes(m, level_u(m, m->step), fp64(m), un);
    if (st != SEM_OK) return st;
    if (m->prec == SEM_FP32_KAHAN) {
        // compensated value u - c; u^{n-1} = u^n - delta^{n-1/2}
        if ((st = read_nodes(m, level_c(m, m->step), false, tmp)) != SEM_OK) return st;
        for (size_t k = 0; k < nn; ++k) un[k] -= tmp[k];
        if (u_prev) {
            if ((st = read_nodes(m, level_x(m, m->step), false, tmp)) != SEM_OK) return st;
            for (size_t k = 0; k < nn; ++k) tmp[k] = un[k] - tmp[k];
            to_original(m, tmp, u_prev);
        }
    } else if (u_prev) {
        if ((st = read_nodes(m, level_x(m, m->step), fp64(m), tmp)) != SEM_OK) return st;
        to_original(m, tmp, u_prev);
    }
    if (u) to_original(m, un, u);
    return SEM_OK;
}

sem_status sem_apply_stiffness(sem_mesh* m, const double* u, double* Ku) {
    if (!m || !u || !Ku) return SEM_ERR_INVALID_ARG;
    if (!m->have_model) return fail(m, SEM_ERR_STATE, "sem_set_model must come first");
    sem_status st = build(m);
    if (st != SEM_OK) return st;
    const size_t nb = node_bytes(m);
    if (!m->d_apply_in) {
        m->d_apply_in = dev_alloc(m, nb);
        m->d_apply_out = dev_alloc(m, nb);
        if (!m->d_apply_in || !m->d_apply_out) return fail(m, SEM_ERR_OOM, "device allocation failed");
    }
    if ((st = write_nodes(m, m->d_apply_in, u)) != SEM_OK) return st;
    // the partial-sum buffer of the step that comes next is free: every
    // launch that reads partials first has them written by its predecessor
    if ((st = launch_apply(m, m->d_apply_in, m->d_apply_out, m->d_part[m->step & 1])) != SEM_OK) return st;
    std::vector<double> out;
    if ((st = read_nodes(m, m->d_apply_out, fp64(m), out)) != SEM_OK) return st;
    if ((st = check_stream_error(m)) != SEM_OK) return st;
    to_original(m, out, Ku);
    return SEM_OK;
}

sem_status sem_read_mass(sem_mesh* m, double* mass) {
    if (!m || !mass) return SEM_ERR_INVALID_ARG;
    if (!m->have_model) return fail(m, SEM_ERR_STATE, "sem_set_model must come first");
    sem_status st = build(m);
    if (st != SEM_OK) return st;
    std::vector<double> v;
    if ((st = read_nodes(m, m->d_M, true, v)) != SEM_OK) return st;
    to_original(m, v, mass);
    return SEM_OK;
}

sem_status sem_get_permutation(const sem_mesh* mc, int64_t* elem_new_of_old, int64_t* node_new_of_old) {
    sem_mesh* m = const_cast<sem_mesh*>(mc);
    if (!m) return SEM_ERR_INVALID_ARG;
    if (m->elem_order.empty()) {
        sem_status so = compute_orderings(m);
        if (so != SEM_OK) return so;
    }
    if (elem_new_of_old) std::copy(m->elem_new.begin(), m->elem_new.end(), elem_new_of_old);
    if (node_new_of_old) std::copy(m->node_new.begin(), m->node_new.end(), node_new_of_old);
    return SEM_OK;
}

sem_status sem_get_sizes(const sem_mesh* m, int64_t* n_nodes, int64_t* n_elems) {
    if (!m) return SEM_ERR_INVALID_ARG;
    if (n_nodes) *n_nodes = m->mesh.nn;
    if (n_elems) *n_elems = m->mesh.ne;
    return SEM_OK;
}

sem_status sem_node_coordinates(const sem_mesh* mc, double* xy) {
    sem_mesh* m = const_cast<sem_mesh*>(mc);
    if (!m || !xy) return SEM_ERR_INVALID_ARG;
    ensure_node_xy(m);
    std::copy(m->node_xy.begin(), m->node_xy.end(), xy);
    return SEM_OK;
}

sem_status sem_get_snapped(const sem_mesh* m, int64_t* src_node, int64_t* rec_nodes) {
    if (!m) return SEM_ERR_INVALID_ARG;
    if (src_node) *src_node = m->have_src ? m->src_node : -1;
    if (rec_nodes) std::copy(m->rec_nodes.begin(), m->rec_nodes.end(), rec_nodes);
    return SEM_OK;
}

sem_status sem_plan_check(const double* coords, int64_t nv, const int32_t* quads, int64_t ne, int order,
                          sem_ordering kind, uint64_t seed, int elems_per_block, int fp64_storage,
                          const double* rec_xy, int32_t nrec, int64_t* info, char* msg, size_t msg_cap) {
    auto say = [&](const std::string& t) {
        if (msg && msg_cap > 0) {
            const size_t n = std::min(msg_cap - 1, t.size());
            std::memcpy(msg, t.data(), n);
            msg[n] = 0;
        }
    };
    say("");
    if (!coords || !quads || (nrec > 0 && !rec_xy) || nrec < 0) return SEM_ERR_INVALID_ARG;
    if ((int)kind < 0 || (int)kind > 6 || elems_per_block < 1 || elems_per_block > 256) return SEM_ERR_INVALID_ARG;
    const std::string bad = semhost::validate(coords, nv, quads, ne, order);
    if (!bad.empty()) {
        say(bad);
        return SEM_ERR_INVALID_ARG;
    }
    semhost::Mesh mm;
    mm.p = order;
    mm.nv = nv;
    mm.ne = ne;
    mm.coords.assign(coords, coords + nv * 2);
    mm.quads.assign(quads, quads + ne * 4);
    semhost::number_nodes(mm);
    std::vector<int64_t> eo, no;
    {
        const std::string why = semhost::orderings(mm, (int)kind, seed, eo, no);
        if (!why.empty()) {
            say(why);
            return SEM_ERR_UNSUPPORTED;
        }
    }
    std::vector<int64_t> nnew(no.size());
    for (size_t k = 0; k < no.size(); ++k) nnew[(size_t)no[k]] = (int64_t)k;
    const int P = mm.P;
    std::vector<int32_t> conn_new((size_t)(ne * P));
    for (int64_t en = 0; en < ne; ++en)
        for (int q = 0; q < P; ++q)
            conn_new[(size_t)(en * P + q)] = (int32_t)nnew[(size_t)mm.conn[(size_t)(eo[(size_t)en] * P + q)]];
    std::vector<double> xy;
    semhost::node_coordinates(mm, xy);
    std::vector<int32_t> rec_gid((size_t)nrec, -1);
    for (int32_t r = 0; r < nrec; ++r) {
        const int32_t g = (int32_t)nnew[(size_t)semhost::snap(xy, rec_xy[2 * r], rec_xy[2 * r + 1])];
        bool dup = false;
        for (int32_t q = 0; q < r; ++q) dup = dup || rec_gid[(size_t)q] == g;
        if (!dup) rec_gid[(size_t)r] = g;
    }
    const int vec = fp64_storage ? 2 : 4;
    semhost::BlockPlan pl;
    std::string why = semhost::build_block_plan(conn_new, ne, P, mm.nn, elems_per_block, true, vec, rec_gid, pl);
    if (!why.empty()) {
        say(why);
        return SEM_ERR_UNSUPPORTED;
    }
    if (info) {
        info[0] = pl.nblocks;
        info[1] = pl.dense ? 1 : 0;
        info[2] = (int64_t)pl.open_gid.size();
        info[3] = pl.max_entries;
        info[4] = pl.max_packet;
        info[5] = pl.npartial;
        info[6] = pl.max_colors;
    }
    why = semhost::check_block_plan(pl, conn_new, vec);
    if (!why.empty()) {
        say(why);
        return SEM_ERR_STATE;
    }
    // the streamed loop's wavefront order over this plan's block graph
    for (int W : {1, 4, 16}) {
        std::vector<uint32_t> sched;
        why = semhost::stream_schedule(pl.dep_ptr.data(), pl.dep.data(), pl.nblocks, 16, W, sched, nullptr);
        if (why.empty()) why = semhost::check_stream_schedule(pl.dep_ptr.data(), pl.dep.data(), pl.nblocks, 16, sched);
        if (!why.empty()) {
            say("wavefront order: " + why);
            return SEM_ERR_STATE;
        }
    }
    // receivers: every distinct receiver node is recorded exactly once
    std::vector<int> seen((size_t)nrec, 0);
    for (int64_t b = 0; b < pl.nblocks; ++b) {
        const int32_t* h = &pl.hdr[(size_t)b * semplan::HDR_INTS];
        const int nrc = h[semplan::H_NREC_CLOSED], nro = h[semplan::H_NREC_OPEN];
        const semplan::Offsets L = semplan::offsets(h[semplan::H_SULEN], h[semplan::H_ULEN], h[semplan::H_NOPEN],
                                                    h[semplan::H_NCOLORS], nrc + nro);
        const int32_t* recs = reinterpret_cast<const int32_t*>(pl.packet.data() + (size_t)h[0] * 16 + L.recs);
        for (int k = 0; k < nrc + nro; ++k) {
            const int r = recs[2 * k + 1];
            if (r < 0 || r >= nrec) {
                say("receiver record out of range");
                return SEM_ERR_STATE;
            }
            seen[(size_t)r]++;
        }
    }
    for (size_t k = 0; k < pl.open_rec.size(); ++k)
        if (pl.open_rec[k] >= 0) seen[(size_t)pl.open_rec[k]] += 1000;  // finished again by the open-node pass
    for (int32_t r = 0; r < nrec; ++r) {
        const int want = rec_gid[(size_t)r] < 0 ? 0 : 1;
        const int got = seen[(size_t)r] % 1000;
        const bool open_node = seen[(size_t)r] >= 1000;
        if ((want == 0 && seen[(size_t)r] != 0) || (want == 1 && !(got == 1))) {
            say("receiver " + std::to_string(r) + " recorded " + std::to_string(got) + " times in blocks");
            return SEM_ERR_STATE;
        }
        (void)open_node;
    }
    return SEM_OK;
}

sem_status sem_count_nodes(const int32_t* quads, int64_t nv, int64_t ne, int order, int64_t* n_nodes) {
    if (!quads || !n_nodes || nv <= 0 || ne <= 0 || order < 1 || order > 8) return SEM_ERR_INVALID_ARG;
    for (int64_t i = 0; i < ne * 4; ++i)
        if (quads[i] < 0 || quads[i] >= nv) return SEM_ERR_INVALID_ARG;
    semhost::Mesh mm;
    mm.p = order;
    mm.nv = nv;
    mm.ne = ne;
    mm.quads.assign(quads, quads + ne * 4);
    semhost::number_nodes(mm);
    *n_nodes = mm.nn;
    return SEM_OK;
}

sem_status sem_compute_ordering(const double* coords, int64_t nv, const int32_t* quads, int64_t ne, int order,
                                sem_ordering kind, uint64_t seed, int64_t* elem_order, int64_t* node_order) {
    if (!coords || !quads || !elem_order || !node_order) return SEM_ERR_INVALID_ARG;
    if ((int)kind < 0 || (int)kind > 6) return SEM_ERR_INVALID_ARG;
    if (!semhost::validate(coords, nv, quads, ne, order).empty()) return SEM_ERR_INVALID_ARG;
    semhost::Mesh mm;
    mm.p = order;
    mm.nv = nv;
    mm.ne = ne;
    mm.coords.assign(coords, coords + nv * 2);
    mm.quads.assign(quads, quads + ne * 4);
    semhost::number_nodes(mm);
    std::vector<int64_t> eo, no;
    if (!semhost::orderings(mm, (int)kind, seed, eo, no).empty()) return SEM_ERR_UNSUPPORTED;
    std::copy(eo.begin(), eo.end(), elem_order);
    std::copy(no.begin(), no.end(), node_order);
    return SEM_OK;
}

sem_status sem_hilbert_cells(int32_t W, int32_t H, int32_t* cells) {
    if (!cells || W < 1 || H < 1) return SEM_ERR_INVALID_ARG;
    std::vector<int32_t> c;
    semhost::hilbert_cells(W, H, c);
    std::copy(c.begin(), c.end(), cells);
    return SEM_OK;
}

sem_status sem_launch_info(const sem_mesh* m, int64_t* steps_per_launch, int64_t* open_nodes) {
    if (!m) return SEM_ERR_INVALID_ARG;
    if (steps_per_launch) *steps_per_launch = m->built && streamed(m) ? stream_len(m) : 1;
    if (open_nodes) *open_nodes = m->built ? (int64_t)m->plan.open_gid.size() : -1;
    return SEM_OK;
}

sem_status sem_profile_enable(sem_mesh* m, int enable) {
    if (!m) return SEM_ERR_INVALID_ARG;
    m->profiling = enable != 0;
    return SEM_OK;
}

sem_status sem_profile_read(sem_mesh* m, double* block_ms, int64_t* block_launches, double* open_ms,
                            int64_t* open_launches) {
    if (!m) return SEM_ERR_INVALID_ARG;
    SEM_CUDA(cudaStreamSynchronize(m->stream));
    double tb = 0.0, to = 0.0;
    for (auto& pr : m->ev_block) {
        float ms = 0.f;
        SEM_CUDA(cudaEventElapsedTime(&ms, pr.first, pr.second));
        tb += ms;
    }
    for (auto& pr : m->ev_open) {
        float ms = 0.f;
        SEM_CUDA(cudaEventElapsedTime(&ms, pr.first, pr.second));
        to += ms;
    }
    if (block_ms) *block_ms = tb;
    if (open_ms) *open_ms = to;
    if (block_launches) *block_launches = (int64_t)m->ev_block.size();
    if (open_launches) *open_launches = (int64_t)m->ev_open.size();
    for (auto& pr : m->ev_block) m->ev_pool.push_back(pr.first), m->ev_pool.push_back(pr.second);
    for (auto& pr : m->ev_open) m->ev_pool.push_back(pr.first), m->ev_pool.push_back(pr.second);
    m->ev_block.clear();
    m->ev_open.clear();
    return SEM_OK;
}

sem_status sem_traffic_model(const sem_mesh* m, double* block_bytes, double* open_bytes) {
    if (!m) return SEM_ERR_INVALID_ARG;
    if (!m->built) return SEM_ERR_STATE;
    const auto& pl = m->plan;
    const double ts = (double)tsize(m);
    const double ne = (double)m->mesh.ne, nn = (double)m->mesh.nn;
    const double slots = ne * m->mesh.P;
    const bool kahan = m->prec == SEM_FP32_KAHAN;
    const double nopen_nodes = (double)pl.open_gid.size();
    const double nclosed = (double)pl.nclosed_total;
    const double nopen_entries = (double)pl.nopen_entries;
    // element side: packed positions, geometry (FP32 bilinear map or FP64 metric)
    const double elem = (double)pl.epos.size() * 4.0 + (fp64(m) ? slots * 3.0 * ts : ne * 32.0);
    const double plan = (double)pl.packet.size() + (double)pl.nblocks * 32.0;
    // closed nodes: read u, s and the update state, write u and the state
    const double state_words = kahan ? 3.0 : 2.0;          // u, delta, c  |  u, u_prev
    const double closed_rw = nclosed * ts * ((1.0 + state_words) + (kahan ? 3.0 : 1.0));
    // open entries of a pending launch: partials of the node, level k-1
    // state and s; the owner stores level k; every open entry writes a partial
    double part_per_node = 0.0;
    for (int32_t c : pl.open_cnt) part_per_node += c;
    const double avg_cnt = nopen_nodes > 0 ? part_per_node / nopen_nodes : 0.0;
    const double open_rw = nopen_entries * ts * (avg_cnt + 1.0 + state_words + 1.0) + nopen_nodes * ts * state_words;
    (void)nn;
    if (block_bytes) *block_bytes = elem + plan + closed_rw + open_rw;
    // open-node pass after the last launch: lists, partials, state in and out
    if (open_bytes)
        *open_bytes = nopen_nodes * (16.0 + ts * (avg_cnt + 1.0 + 2.0 * state_words + (kahan ? 1.0 : 0.0)));
    return SEM_OK;
}

sem_status sem_transfer_bytes(const sem_mesh* m, int64_t* h2d, int64_t* d2h) {
    if (!m) return SEM_ERR_INVALID_ARG;
    if (h2d) *h2d = m->h2d;
    if (d2h) *d2h = m->d2h;
    return SEM_OK;
}

const char* sem_last_error(const sem_mesh* m) {
    if (!m) return "NULL handle";
    return m->err.c_str();
}

void sem_destroy(sem_mesh* m) {
    if (!m) return;
    dev_free_all(m);
    for (auto& pr : m->ev_block) m->ev_pool.push_back(pr.first), m->ev_pool.push_back(pr.second);
    for (auto& pr : m->ev_open) m->ev_pool.push_back(pr.first), m->ev_pool.push_back(pr.second);
    for (cudaEvent_t e : m->ev_pool) cudaEventDestroy(e);
    delete m;
}

// ------------------------------------------------ misfit gradient (adjoint)
}  // extern "C"

namespace {

sem_status adjoint_alloc(sem_mesh* m, int64_t nsteps, int64_t kc) {
    const size_t nb = node_bytes(m);
    if (!m->d_C) {
        for (auto& l : m->d_lam)
            if (!(l = dev_alloc(m, nb))) return fail(m, SEM_ERR_OOM, "device allocation failed");
        m->d_klam = dev_alloc(m, nb);
        m->d_C = (double*)dev_alloc(m, (size_t)m->mesh.nn * 8);
        m->d_grad = (double*)dev_alloc(m, (size_t)m->mesh.ne * 8);
        m->d_rec_node = (int32_t*)dev_alloc(m, (size_t)std::max(m->nrec, 1) * 4);
        m->d_rec_row = (int32_t*)dev_alloc(m, (size_t)std::max(m->nrec, 1) * 4);
        if (!m->d_klam || !m->d_C || !m->d_grad || !m->d_rec_node || !m->d_rec_row)
            return fail(m, SEM_ERR_OOM, "device allocation failed");
        // connectivity in the device element order (new node ids)
        const auto& M = m->mesh;
        std::vector<int32_t> cd((size_t)(M.ne * M.P));
        for (int64_t i = 0; i < M.ne; ++i) {
            const int64_t eo = m->elem_order[(size_t)m->plan.dev_order[(size_t)i]];
            for (int q = 0; q < M.P; ++q)
                cd[(size_t)(i * M.P + q)] = (int32_t)m->node_new[(size_t)M.conn[(size_t)(eo * M.P + q)]];
        }
        sem_status st = upload(m, &m->d_conn_dev, cd.data(), cd.size());
        if (st != SEM_OK) return st;
        std::vector<int32_t> rn((size_t)m->nrec), rr((size_t)m->nrec);
        for (int32_t r = 0; r < m->nrec; ++r) {
            rn[(size_t)r] = (int32_t)m->node_new[(size_t)m->rec_nodes[(size_t)r]];
            rr[(size_t)r] = m->rec_row[(size_t)r] >= 0 ? m->rec_row[(size_t)r] : r;
        }
        SEM_CUDA(cudaMemcpyAsync(m->d_rec_node, rn.data(), rn.size() * 4, cudaMemcpyHostToDevice, m->stream));
        SEM_CUDA(cudaMemcpyAsync(m->d_rec_row, rr.data(), rr.size() * 4, cudaMemcpyHostToDevice, m->stream));
        // receivers sorted by (node, index), and per node the first of them
        std::vector<int32_t> order((size_t)m->nrec), first((size_t)m->mesh.nn, -1);
        for (int32_t r = 0; r < m->nrec; ++r) order[(size_t)r] = r;
        std::stable_sort(order.begin(), order.end(),
                         [&](int32_t a, int32_t b) { return rn[(size_t)a] < rn[(size_t)b]; });
        for (int32_t k = m->nrec - 1; k >= 0; --k) first[(size_t)rn[(size_t)order[(size_t)k]]] = k;
        if (order.empty()) order.push_back(0);   // never read (no receivers), keeps the upload non-empty
        if ((st = upload(m, &m->d_rec_order, order.data(), order.size())) != SEM_OK) return st;
        if ((st = upload(m, &m->d_rec_first, first.data(), first.size())) != SEM_OK) return st;
        SEM_CUDA(cudaStreamSynchronize(m->stream));
    }
    if (nsteps > m->adj_steps || kc != m->adj_kc) {
        // checkpoints and segment buffers (the old ones stay until sem_destroy)
        const int64_t nchk = (nsteps + kc - 1) / kc + 1;
        m->d_chk.assign((size_t)(2 * nchk), nullptr);
        for (auto& c : m->d_chk)
            if (!(c = dev_alloc(m, nb))) return fail(m, SEM_ERR_OOM, "device allocation failed (checkpoints)");
        m->d_seg.assign((size_t)(kc + 1), nullptr);
        for (auto& c : m->d_seg)
            if (!(c = dev_alloc(m, nb))) return fail(m, SEM_ERR_OOM, "device allocation failed (segment)");
        m->d_obs = (double*)dev_alloc(m, (size_t)std::max(m->nrec, 1) * (size_t)nsteps * 8);
        if (!m->d_obs) return fail(m, SEM_ERR_OOM, "device allocation failed");
        m->adj_steps = nsteps;
        m->adj_kc = kc;
    }
    return SEM_OK;
}

sem_status copy_dev(sem_mesh* m, void* dst, const void* src) {
    SEM_CUDA(cudaMemcpyAsync(dst, src, (size_t)m->mesh.nn * tsize(m), cudaMemcpyDeviceToDevice, m->stream));
    return SEM_OK;
}

// n steps from a stored level (open nodes completed).
sem_status run_steps(sem_mesh* m, int64_t n) {
    sem_status st;
    if ((st = launch_steps(m, n)) != SEM_OK) return st;
    return flush_pending(m);
}

}  // namespace

extern "C" {

sem_status sem_misfit_gradient(sem_mesh* m, const double* d_obs, int64_t nsteps, int64_t checkpoint_every,
                               double* misfit, double* grad_vel) {
    if (!m || !d_obs || nsteps < 1 || checkpoint_every < 0) return SEM_ERR_INVALID_ARG;
    if (m->prec == SEM_FP32_KAHAN || m->scheme != SEM_SCHEME_LEAPFROG)
        return fail(m, SEM_ERR_UNSUPPORTED, "the adjoint runs on leapfrog SEM_FP64 or SEM_FP32 (three-level) handles");
    if (!m->have_model || !m->have_dt) return fail(m, SEM_ERR_STATE, "model and dt must be set first");
    if (m->nrec < 1 || m->trace_cap < nsteps)
        return fail(m, SEM_ERR_STATE, "receivers with max_steps >= nsteps must be set first");
    sem_status st = build(m);
    if (st != SEM_OK) return st;
    if ((st = fill_source(m, nsteps)) != SEM_OK) return st;
    int64_t kc = checkpoint_every;
    if (kc == 0) kc = std::max<int64_t>(1, (int64_t)std::ceil(std::sqrt((double)nsteps)));
    kc = std::min(kc, nsteps);
    if ((st = adjoint_alloc(m, nsteps, kc)) != SEM_OK) return st;
    const bool f64 = fp64(m);
    const size_t nb = (size_t)m->mesh.nn * tsize(m);
    const int64_t nchk = (nsteps + kc - 1) / kc;
    // forward from rest, a checkpoint (u^{n0}, u^{n0-1}) every kc steps
    for (auto* u : m->d_u) SEM_CUDA(cudaMemsetAsync(u, 0, nb, m->stream));
    SEM_CUDA(cudaMemsetAsync(m->d_trace, 0, (size_t)m->nrec * (size_t)m->trace_cap * 8, m->stream));
    m->step = 0;
    m->open_pending = false;   // the state restarts from rest
    for (int64_t c = 0; c < nchk; ++c) {
        const int64_t n0 = c * kc;
        if ((st = copy_dev(m, m->d_chk[(size_t)(2 * c)], level_u(m, n0))) != SEM_OK) return st;
        if ((st = copy_dev(m, m->d_chk[(size_t)(2 * c + 1)], level_x(m, n0))) != SEM_OK) return st;
        if ((st = run_steps(m, std::min(kc, nsteps - n0))) != SEM_OK) return st;
    }
    // the final state, restored at the end
    void* fin_u = m->d_chk[(size_t)(2 * nchk)];
    void* fin_x = m->d_chk[(size_t)(2 * nchk + 1)];
    if ((st = copy_dev(m, fin_u, level_u(m, nsteps))) != SEM_OK) return st;
    if ((st = copy_dev(m, fin_x, level_x(m, nsteps))) != SEM_OK) return st;
    // misfit from the traces
    std::vector<double> tr((size_t)m->nrec * (size_t)nsteps);
    if ((st = sem_read_traces(m, tr.data(), nsteps)) != SEM_OK) return st;
    double J = 0.0;
    for (size_t k = 0; k < tr.size(); ++k) {
        const double d = tr[k] - d_obs[k];
        J += d * d;
    }
    J *= 0.5 * m->dt;
    if (misfit) *misfit = J;
    if (!grad_vel) {
        m->step = nsteps;
        return SEM_OK;
    }
    SEM_CUDA(cudaMemcpyAsync(m->d_obs, d_obs, tr.size() * 8, cudaMemcpyHostToDevice, m->stream));
    m->h2d += (int64_t)(tr.size() * 8);
    // backward: lambda^{N+1} = lambda^{N+2} = 0, segments last to first
    for (auto* l : m->d_lam) SEM_CUDA(cudaMemsetAsync(l, 0, nb, m->stream));
    SEM_CUDA(cudaMemsetAsync(m->d_C, 0, (size_t)m->mesh.nn * 8, m->stream));
    auto lam = [&](int64_t k) { return m->d_lam[(size_t)(((k % 3) + 3) % 3)]; };
    const double inv_dt = 1.0 / m->dt;
    for (int64_t c = nchk - 1; c >= 0; --c) {
        const int64_t n0 = c * kc, n1 = std::min(n0 + kc, nsteps);
        // recompute u^{n0..n1} from the checkpoint
        if ((st = copy_dev(m, level_u(m, n0), m->d_chk[(size_t)(2 * c)])) != SEM_OK) return st;
        if ((st = copy_dev(m, level_x(m, n0), m->d_chk[(size_t)(2 * c + 1)])) != SEM_OK) return st;
        m->step = n0;
        if ((st = copy_dev(m, m->d_seg[0], m->d_chk[(size_t)(2 * c)])) != SEM_OK) return st;
        for (int64_t j = 1; j <= n1 - n0; ++j) {
            if ((st = run_steps(m, 1)) != SEM_OK) return st;
            if ((st = copy_dev(m, m->d_seg[(size_t)j], level_u(m, n0 + j))) != SEM_OK) return st;
        }
        auto u_at = [&](int64_t k) -> const void* {
            return k >= n0 ? m->d_seg[(size_t)(k - n0)] : m->d_chk[(size_t)(2 * c + 1)];
        };
        // per backward step: K lambda (step kernel in apply mode and the
        // open-node kernel), then one fused node pass
        for (int64_t mm = n1; mm > n0; --mm) {
            if ((st = launch_apply(m, lam(mm + 1), m->d_klam, m->d_part[0])) != SEM_OK) return st;
            SEM_CUDA(semdev::launch_adjoint_node(f64, m->mesh.nn, lam(mm), lam(mm + 1), lam(mm + 2), m->d_s, m->d_klam,
                                                 m->d_rec_first, m->d_rec_order, m->nrec, m->d_rec_node, m->d_rec_row,
                                                 m->d_trace, m->trace_cap, m->d_obs, nsteps, mm, inv_dt, m->d_C,
                                                 u_at(mm), u_at(mm - 1), u_at(mm - 2), m->stream));
        }
    }
    SEM_CUDA(semdev::launch_gradient(m->mesh.ne, m->mesh.P, m->d_conn_dev, m->d_mloc, m->d_C, m->d_vel, m->d_grad,
                                     m->stream));
    std::vector<double> g((size_t)m->mesh.ne);
    SEM_CUDA(cudaMemcpyAsync(g.data(), m->d_grad, g.size() * 8, cudaMemcpyDeviceToHost, m->stream));
    m->d2h += (int64_t)(g.size() * 8);
    // restore the state after the forward run
    if ((st = copy_dev(m, level_u(m, nsteps), fin_u)) != SEM_OK) return st;
    if ((st = copy_dev(m, level_x(m, nsteps), fin_x)) != SEM_OK) return st;
    SEM_CUDA(cudaStreamSynchronize(m->stream));
    m->step = nsteps;
    if ((st = check_stream_error(m)) != SEM_OK) return st;
    for (int64_t i = 0; i < m->mesh.ne; ++i) grad_vel[(size_t)m->elem_order[(size_t)m->plan.dev_order[(size_t)i]]] = g[(size_t)i];
    return SEM_OK;
}

// ------------------------------------------------ allocation-free variant
}  // extern "C"

namespace {
// Scratch of sem_apply_stiffness_dev_noalloc: partial sums of open entries.
// A file-scope device array, so the call needs no allocation. In host code
// the name is only a host-side stand-in; its device address comes from
// cudaGetSymbolAddress, looked up once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SEM_NOALLOC_SCRATCH_BYTES];
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[256] = {};

cudaError_t noalloc_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}
}  // namespace

extern "C" {

sem_status sem_apply_stiffness_dev_noalloc(sem_mesh* m, const void* dev_u, void* dev_Ku) {
    if (!m || !dev_u || !dev_Ku) return SEM_ERR_INVALID_ARG;
    if (!m->built)
        return fail(m, SEM_ERR_STATE, "device data not built: call sem_step, sem_set_state or sem_apply_stiffness once");
    const int64_t need = m->plan.npartial * (int64_t)tsize(m);
    if ((double)need > (double)SEM_NOALLOC_SCRATCH_BYTES)
        return fail(m, SEM_ERR_INVALID_ARG,
                    "mesh needs " + std::to_string(need) + " bytes of partial sums, above the allocation-free limit of " +
                        std::to_string((unsigned)SEM_NOALLOC_SCRATCH_BYTES) + " bytes");
    void* scratch = nullptr;
    cudaError_t e = noalloc_scratch(&scratch);
    if (e != cudaSuccess) return cuda_fail(m, e, "cudaGetSymbolAddress");
    return launch_apply(m, dev_u, dev_Ku, scratch);
}

}  // extern "C"

// ------------------------------------------------------------ batched shots
struct sem_batch {
    std::vector<sem_mesh*> shots;
    cudaStream_t stream = nullptr;     // the shots' stream; NULL = legacy default
    cudaStream_t own = nullptr;        // created when the shots use the legacy default stream
    cudaStream_t run = nullptr;        // where the batch enqueues (graphs cannot capture the legacy stream)
    sem_precision prec = SEM_FP64;
    std::string err;
    struct Class {
        int np = 0;
        int threads = 0, smem = 0, ctas = 0;
        int eb = 0;
        int32_t* d_cta_shot = nullptr;
        int32_t* d_cta_block = nullptr;
        // streamed batch: one record per block of the class's shots, and
        // the class launch's work counter
        semdev::BatchUnit* d_units = nullptr;
        unsigned long long* d_counter = nullptr;
        bool streamed = false;   // streamed launches; else one launch per step (clock path)
    };
    std::vector<Class> classes;
    // streamed batch (every shot streamable): each order class runs a block
    // of steps as one launch over the blocks of all its shots
    bool streamed = false;                 // the clock-driven path (some class streams)
    int stream_mode = -1;                  // sem_batch_set_stream: -1 automatic, 0 never, 1 every class, 2 clock path, no class
    int stream_steps = 64;                 // steps per streamed launch (one graph replay)
    semdev::ShotClock* d_clock = nullptr;  // [nshots]
    uint32_t** d_done = nullptr;           // [nshots]: each shot's done flags
    uint32_t* d_serial = nullptr;          // serial of the next launch's first step
    int32_t* d_err = nullptr;
    uint32_t serial = 1;
    void* d_desc = nullptr;
    size_t desc_bytes = 0;
    int64_t* d_step = nullptr;
    int32_t* d_pending = nullptr;
    std::vector<void*> allocs;
    bool ready = false;
    int graph_steps = 0;
    cudaGraphExec_t graph = nullptr;
    cudaGraphExec_t sgraph = nullptr;      // one streamed block of stream_steps steps
};

namespace {

sem_status bfail(sem_batch* b, sem_status st, const std::string& msg) {
    if (b) b->err = msg;
    return st;
}

void* balloc(sem_batch* b, size_t bytes) {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    b->allocs.push_back(p);
    return p;
}

// Frees a handle's device data so that it can be built again (used by the
// autotuner); the handle's settings stay.
void unbuild(sem_mesh* m) {
    dev_free_all(m);
    m->d_G32 = nullptr;
    m->d_metric_out = nullptr;
    // adjoint buffers went with the rest: the next sem_misfit_gradient
    // allocates them again
    m->adj_steps = m->adj_kc = 0;
    for (auto& l : m->d_lam) l = nullptr;
    m->d_klam = nullptr;
    m->d_C = nullptr;
    m->d_obs = nullptr;
    m->d_grad = nullptr;
    m->d_conn_dev = nullptr;
    m->d_rec_node = m->d_rec_row = m->d_rec_order = m->d_rec_first = nullptr;
    m->d_err = nullptr;
    m->d_done = nullptr;
    m->d_counter = nullptr;
    m->d_dep = nullptr;
    m->stream_ok = false;
    m->d_chk.clear();
    m->d_seg.clear();
    m->built = false;
    m->open_pending = false;
    m->step = 0;
    m->d_src = nullptr;
    m->src_cap = 0;
    m->d_trace = nullptr;
    m->d_apply_in = m->d_apply_out = nullptr;
    for (auto& u : m->d_u) u = nullptr;
    for (auto& x : m->d_x) x = nullptr;
    for (auto& c : m->d_c) c = nullptr;
    for (auto& p : m->d_part) p = nullptr;
    m->plan = semhost::BlockPlan();
    m->host_ready = false;
}


// Per-shot descriptors (re-uploaded before every batch step: source tables
// may have grown).
sem_status upload_desc(sem_batch* b) {
    const size_t n = b->shots.size();
    std::vector<uint8_t> host;
    if (b->prec == SEM_FP64) {
        std::vector<semdev::ShotDesc<double>> v(n);
        for (size_t i = 0; i < n; ++i) {
            v[i] = shot_desc<double>(b->shots[i]);
            if (b->d_err) v[i].err = b->d_err;
        }
        host.assign(reinterpret_cast<uint8_t*>(v.data()), reinterpret_cast<uint8_t*>(v.data() + n));
    } else {
        std::vector<semdev::ShotDesc<float>> v(n);
        for (size_t i = 0; i < n; ++i) {
            v[i] = shot_desc<float>(b->shots[i]);
            if (b->d_err) v[i].err = b->d_err;
        }
        host.assign(reinterpret_cast<uint8_t*>(v.data()), reinterpret_cast<uint8_t*>(v.data() + n));
    }
    if (!b->d_desc) {
        b->desc_bytes = host.size();
        b->d_desc = balloc(b, b->desc_bytes);
        if (!b->d_desc) return bfail(b, SEM_ERR_OOM, "device allocation failed");
    }
    if (cudaMemcpyAsync(b->d_desc, host.data(), host.size(), cudaMemcpyHostToDevice, b->run) != cudaSuccess ||
        cudaStreamSynchronize(b->run) != cudaSuccess)
        return bfail(b, SEM_ERR_CUDA, "descriptor upload failed");
    return SEM_OK;
}

// Time per step of one handle (after two warm-up steps), in ms: one
// streamed launch of `steps` steps where the handle can stream (the way a
// streamed batch runs it), else one launch per step.
sem_status time_handle(sem_mesh* m, int steps, double* ms) {
    sem_status st;
    if ((st = build(m)) != SEM_OK) return st;
    if ((st = fill_source(m, steps + 2)) != SEM_OK) return st;
    const bool stream = m->stream_ok && m->dep_stride <= 16;
    if (stream) {
        if ((st = launch_stream_steps(m, 2, false)) != SEM_OK) return st;
    } else {
        for (int k = 0; k < 2; ++k)
            if ((st = launch_one_step(m, k > 0)) != SEM_OK) return st;
    }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return fail(m, SEM_ERR_CUDA, "event");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(m, SEM_ERR_CUDA, "event");
    }
    cudaEventRecord(e0, m->stream);
    if (stream) {
        st = launch_stream_steps(m, steps, true);
    } else {
        for (int k = 0; k < steps; ++k)
            if ((st = launch_one_step(m, true)) != SEM_OK) break;
    }
    cudaEventRecord(e1, m->stream);
    float t = 0.f;
    if (st == SEM_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
        st = fail(m, SEM_ERR_CUDA, "event timing");
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = t / steps;
    return st;
}

// Launches of one batch step: every order class, then the counter advance.
sem_status batch_launch_step(sem_batch* b) {
    const bool f64 = b->prec == SEM_FP64;
    const int mode = b->prec == SEM_FP32_KAHAN ? semdev::MODE_KAHAN : semdev::MODE_THREE_LEVEL;
    for (auto& c : b->classes) {
        // step counters, no clocks (clock = nullptr, offset = 0)
        semdev::BatchArgs ba{b->d_desc, c.d_cta_shot, c.d_cta_block, b->d_step, b->d_pending, nullptr, 0};
        const sem_mesh* m0 = nullptr;
        for (auto* m : b->shots)
            if (m->mesh.np == c.np) {
                m0 = m;
                break;
            }
        const void* basis = f64 ? (const void*)&m0->basis64 : (const void*)&m0->basis32;
        cudaError_t e = semdev::launch_batch_step(c.np, f64, mode, false, ba, c.ctas, basis, c.threads, c.smem, b->run);
        if (e != cudaSuccess) return bfail(b, SEM_ERR_CUDA, std::string("batch step launch: ") + cudaGetErrorString(e));
    }
    cudaError_t e = semdev::launch_batch_advance(b->d_step, b->d_pending, (int)b->shots.size(), b->run);
    if (e != cudaSuccess) return bfail(b, SEM_ERR_CUDA, std::string("batch advance: ") + cudaGetErrorString(e));
    return SEM_OK;
}

// Streamed launches of n steps: every order class as one launch over the
// blocks of its shots, then the shots' clocks and the batch serial advance.
sem_status batch_launch_stream(sem_batch* b, int n) {
    const bool f64 = b->prec == SEM_FP64;
    const int mode = b->prec == SEM_FP32_KAHAN ? semdev::MODE_KAHAN : semdev::MODE_THREE_LEVEL;
    for (auto& c : b->classes) {
        const sem_mesh* m0 = nullptr;
        for (auto* m : b->shots)
            if (m->mesh.np == c.np) {
                m0 = m;
                break;
            }
        const void* basis = f64 ? (const void*)&m0->basis64 : (const void*)&m0->basis32;
        if (!c.streamed) {
            // one launch per step over the class's blocks, steps from the clocks
            for (int o = 0; o < n; ++o) {
                semdev::BatchArgs ba{b->d_desc, c.d_cta_shot, c.d_cta_block, nullptr, nullptr, b->d_clock, o};
                cudaError_t e = semdev::launch_batch_step(c.np, f64, mode, false, ba, c.ctas, basis, c.threads, c.smem,
                                                          b->run);
                if (e != cudaSuccess)
                    return bfail(b, SEM_ERR_CUDA, std::string("batch step launch: ") + cudaGetErrorString(e));
            }
            continue;
        }
        semdev::BatchStreamArgs sa{};
        sa.shots = b->d_desc;
        sa.units = c.d_units;
        sa.clock = b->d_clock;
        sa.done = b->d_done;
        sa.serial0 = b->d_serial;
        sa.counter = c.d_counter;
        sa.err = b->d_err;
        sa.nblk = c.ctas;
        sa.nsteps = n;
        if (cudaMemsetAsync(c.d_counter, 0, 8, b->run) != cudaSuccess)
            return bfail(b, SEM_ERR_CUDA, "work counter reset failed");
        cudaError_t e = semdev::launch_batch_stream(c.np, f64, mode, false, sa, basis, c.threads, c.smem, b->run);
        if (e != cudaSuccess)
            return bfail(b, SEM_ERR_CUDA, std::string("streamed batch launch: ") + cudaGetErrorString(e));
    }
    cudaError_t e = semdev::launch_batch_clock_advance(b->d_clock, (int)b->shots.size(), b->d_serial, n, b->run);
    if (e != cudaSuccess) return bfail(b, SEM_ERR_CUDA, std::string("batch clock advance: ") + cudaGetErrorString(e));
    return SEM_OK;
}

// Device records of a streamed batch (after the shots are built): per class
// one BatchUnit per block of its shots, the clocks, done-flag table, serial
// and error flag. A class streams where a step of it has fewer than
// kAutoStreamWaves waves of resident CTAs (the upper bound of the rule
// sem_step applies to one mesh: with more, the per-unit ticket, waits and
// release cost more than a launch per step loses at its last wave; a class
// with less than one wave still streams, since a batch of small shots would
// otherwise pay a launch per class and step); the other classes run one launch
// per step inside the same captured block, their steps taken from the
// shots' clocks. Returns false (the batch keeps one launch per class and
// step, with step counters) when a shot cannot stream or no class would.
bool batch_prepare_stream(sem_batch* b) {
    if (b->stream_mode == 0) return false;
    for (auto* m : b->shots)
        if (!m->stream_ok || m->dep_stride > 16) return false;
    const bool f64 = b->prec == SEM_FP64;
    const int mode = b->prec == SEM_FP32_KAHAN ? semdev::MODE_KAHAN : semdev::MODE_THREE_LEVEL;
    int nstream = 0;
    for (auto& c : b->classes) {
        int res = 0;
        if (semdev::batch_stream_resident_ctas(c.np, f64, mode, c.threads, c.smem, &res) != cudaSuccess) return false;
        c.streamed = b->stream_mode == 1 || (b->stream_mode == -1 && (int64_t)c.ctas < (int64_t)kAutoStreamWaves * res);
        nstream += c.streamed ? 1 : 0;
    }
    if (nstream == 0 && b->stream_mode != 2) return false;
    for (auto& c : b->classes) {
        if (!c.streamed) continue;
        std::vector<semdev::BatchUnit> units;
        for (size_t i = 0; i < b->shots.size(); ++i) {
            const sem_mesh* m = b->shots[i];
            if (m->mesh.np != c.np) continue;
            const auto& pl = m->plan;
            for (int64_t k = 0; k < pl.nblocks; ++k) {
                semdev::BatchUnit u{};
                for (int f = 0; f < 12; ++f) u.hdr[f] = pl.hdr[(size_t)k * 12 + f];
                u.shot = (int32_t)i;
                u.block = (int32_t)k;
                u.dep_stride = m->dep_stride;
                for (int t = 0; t < 16; ++t) {
                    const int32_t q = pl.dep_ptr[(size_t)k] + t;
                    u.dep[t] = (t < m->dep_stride && q < pl.dep_ptr[(size_t)k + 1]) ? pl.dep[(size_t)q] : (int32_t)k;
                }
                units.push_back(u);
            }
        }
        c.d_units = (semdev::BatchUnit*)balloc(b, units.size() * sizeof(semdev::BatchUnit));
        c.d_counter = (unsigned long long*)balloc(b, 8);
        if (!c.d_units || !c.d_counter) return false;
        if (cudaMemcpy(c.d_units, units.data(), units.size() * sizeof(semdev::BatchUnit), cudaMemcpyHostToDevice) !=
            cudaSuccess)
            return false;
        semdev::BatchStreamArgs none{};
        if (semdev::launch_batch_stream(c.np, f64, mode, true, none, nullptr, c.threads, c.smem, b->run) != cudaSuccess)
            return false;
    }
    const size_t n = b->shots.size();
    b->d_clock = (semdev::ShotClock*)balloc(b, n * sizeof(semdev::ShotClock));
    b->d_done = (uint32_t**)balloc(b, n * sizeof(uint32_t*));
    b->d_serial = (uint32_t*)balloc(b, 4);
    b->d_err = (int32_t*)balloc(b, 4);
    if (!b->d_clock || !b->d_done || !b->d_serial || !b->d_err) return false;
    std::vector<uint32_t*> done(n);
    for (size_t i = 0; i < n; ++i) done[i] = b->shots[i]->d_done;
    if (cudaMemcpy(b->d_done, done.data(), n * sizeof(uint32_t*), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(b->d_err, 0, 4) != cudaSuccess)
        return false;
    return true;
}

sem_status batch_prepare(sem_batch* b) {
    if (b->ready) return SEM_OK;
    if (!b->run) {
        if (b->stream) {
            b->run = b->stream;
        } else {
            if (cudaStreamCreate(&b->own) != cudaSuccess) return bfail(b, SEM_ERR_CUDA, "stream creation failed");
            b->run = b->own;
        }
    }
    const bool f64 = b->prec == SEM_FP64;
    const int mode = b->prec == SEM_FP32_KAHAN ? semdev::MODE_KAHAN : semdev::MODE_THREE_LEVEL;
    {
        // host parts of all shots in parallel, then the device parts in order
        std::atomic<size_t> next(0);
        const unsigned hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
        std::vector<std::thread> workers;
        for (unsigned w = 0; w < hw; ++w)
            workers.emplace_back([&]() {
                for (size_t i = next++; i < b->shots.size(); i = next++) build_host(b->shots[i]);
            });
        for (auto& t : workers) t.join();
    }
    for (auto* m : b->shots) {
        sem_status st = build(m);
        if (st != SEM_OK) return bfail(b, st, std::string("shot build: ") + m->err);
    }
    std::map<int, std::vector<int>> by_order;
    for (size_t i = 0; i < b->shots.size(); ++i) by_order[b->shots[i]->mesh.np].push_back((int)i);
    for (auto& kv : by_order) {
        sem_batch::Class c;
        c.np = kv.first;
        std::vector<int32_t> cs, cb;
        for (int i : kv.second) {
            const sem_mesh* m = b->shots[(size_t)i];
            c.threads = std::max(c.threads, m->threads);
            c.smem = std::max(c.smem, m->smem);
            c.eb = std::max(c.eb, m->plan.eb);
            for (int64_t k = 0; k < m->plan.nblocks; ++k) {
                cs.push_back(i);
                cb.push_back((int32_t)k);
            }
        }
        c.ctas = (int)cs.size();
        c.d_cta_shot = (int32_t*)balloc(b, cs.size() * 4);
        c.d_cta_block = (int32_t*)balloc(b, cb.size() * 4);
        if (!c.d_cta_shot || !c.d_cta_block) return bfail(b, SEM_ERR_OOM, "device allocation failed");
        if (cudaMemcpy(c.d_cta_shot, cs.data(), cs.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(c.d_cta_block, cb.data(), cb.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
            return bfail(b, SEM_ERR_CUDA, "cta map upload failed");
        semdev::BatchArgs none{};
        cudaError_t e = semdev::launch_batch_step(c.np, f64, mode, true, none, 0, nullptr, c.threads, c.smem, b->run);
        if (e != cudaSuccess) return bfail(b, SEM_ERR_CUDA, std::string("batch kernel set-up: ") + cudaGetErrorString(e));
        b->classes.push_back(c);
    }
    b->d_step = (int64_t*)balloc(b, b->shots.size() * 8);
    b->d_pending = (int32_t*)balloc(b, b->shots.size() * 4);
    if (!b->d_step || !b->d_pending) return bfail(b, SEM_ERR_OOM, "device allocation failed");
    b->streamed = batch_prepare_stream(b);
    cudaGetLastError();
    b->ready = true;
    return SEM_OK;
}

}  // namespace

// sem_batch_step of a streamed batch: each shot's done flags restart from
// zero and the batch serial from 1, the clocks start at the shots' steps;
// blocks of stream_steps steps replay one captured graph (per class: reset
// of the work counter, one streamed launch; then the clock advance), the
// remainder is launched directly; then the open nodes of every shot.
sem_status batch_step_streamed(sem_batch* b, int64_t nsteps) {
    sem_status st;
    const size_t n = b->shots.size();
    std::vector<semdev::ShotClock> clk(n);
    for (size_t i = 0; i < n; ++i) {
        sem_mesh* m = b->shots[i];
        clk[i].step0 = m->step;
        clk[i].pending0 = 0;
        if (cudaMemsetAsync(m->d_done, 0, (size_t)m->plan.nblocks * 4, b->run) != cudaSuccess)
            return bfail(b, SEM_ERR_CUDA, "done flags reset failed");
    }
    b->serial = 1;
    if (cudaMemcpyAsync(b->d_clock, clk.data(), n * sizeof(semdev::ShotClock), cudaMemcpyHostToDevice, b->run) !=
            cudaSuccess ||
        cudaMemcpyAsync(b->d_serial, &b->serial, 4, cudaMemcpyHostToDevice, b->run) != cudaSuccess ||
        cudaStreamSynchronize(b->run) != cudaSuccess)
        return bfail(b, SEM_ERR_CUDA, "batch clock upload failed");
    const int G = b->stream_steps;
    int64_t done = 0;
    if (nsteps >= G) {
        if (!b->sgraph) {
            cudaGraph_t g = nullptr;
            if (cudaStreamBeginCapture(b->run, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
                return bfail(b, SEM_ERR_CUDA, "graph capture begin failed");
            const sem_status cst = batch_launch_stream(b, G);
            const cudaError_t ce = cudaStreamEndCapture(b->run, &g);
            if (cst != SEM_OK) {
                if (g) cudaGraphDestroy(g);
                return cst;
            }
            if (ce != cudaSuccess) return bfail(b, SEM_ERR_CUDA, "graph capture failed");
            const cudaError_t ie = cudaGraphInstantiate(&b->sgraph, g, 0);
            cudaGraphDestroy(g);
            if (ie != cudaSuccess) {
                b->sgraph = nullptr;
                return bfail(b, SEM_ERR_CUDA, "graph instantiation failed");
            }
        }
        for (; done + G <= nsteps; done += G)
            if (cudaGraphLaunch(b->sgraph, b->run) != cudaSuccess) return bfail(b, SEM_ERR_CUDA, "graph launch failed");
    }
    if (done < nsteps && (st = batch_launch_stream(b, (int)(nsteps - done))) != SEM_OK) return st;
    // a bounded wait that gave up: reported once, flag cleared
    int32_t raised = 0;
    if (cudaMemcpyAsync(&raised, b->d_err, 4, cudaMemcpyDeviceToHost, b->run) != cudaSuccess ||
        cudaStreamSynchronize(b->run) != cudaSuccess)
        return bfail(b, SEM_ERR_CUDA, "batch error flag read failed");
    b->serial = (uint32_t)(1 + nsteps);
    for (auto* m : b->shots) {
        m->step += nsteps;
        m->serial = b->serial;
        if ((st = launch_flush(m)) != SEM_OK) return bfail(b, st, m->err);
        m->stepped_calls++;
    }
    if (raised) {
        cudaMemsetAsync(b->d_err, 0, 4, b->run);
        cudaStreamSynchronize(b->run);
        return bfail(b, SEM_ERR_TIMEOUT, "a streamed batch step gave up waiting for a neighbouring block");
    }
    return SEM_OK;
}

extern "C" {

sem_status sem_batch_create(sem_mesh* const* shots, int32_t nshots, int32_t autotune_steps, sem_batch** out) {
    if (!shots || nshots < 1 || !out || autotune_steps < 0) return SEM_ERR_INVALID_ARG;
    *out = nullptr;
    sem_batch* b = new (std::nothrow) sem_batch();
    if (!b) return SEM_ERR_OOM;
    for (int32_t i = 0; i < nshots; ++i) {
        sem_mesh* m = shots[i];
        if (!m) {
            delete b;
            return SEM_ERR_INVALID_ARG;
        }
        for (auto* o : b->shots)
            if (o == m) {
                delete b;
                return SEM_ERR_INVALID_ARG;
            }
        b->shots.push_back(m);
    }
    sem_mesh* m0 = b->shots[0];
    b->stream = m0->stream;
    b->prec = m0->prec;
    for (auto* m : b->shots) {
        if (m->prec != b->prec || m->stream != b->stream || !m->have_model || !m->have_dt ||
            m->scheme != SEM_SCHEME_LEAPFROG) {
            delete b;
            return SEM_ERR_STATE;
        }
        if (m->metric == SEM_METRIC_STORED) {
            delete b;
            return SEM_ERR_UNSUPPORTED;
        }
    }
    // autotuner: per order, the not yet built shot whose element count is
    // closest to 65,536 (large enough to fill the GPU, small enough to plan
    // quickly) is timed with each candidate block size; every unbuilt shot of
    // that order then uses the fastest
    if (autotune_steps > 0) {
        std::map<int, std::vector<sem_mesh*>> by_order;
        for (auto* m : b->shots)
            if (!m->built && m->eb_request == 0) by_order[m->mesh.np].push_back(m);
        for (auto& kv : by_order) {
            sem_mesh* big = kv.second[0];
            auto dist = [](const sem_mesh* m) { return std::llabs((long long)m->mesh.ne - 65536LL); };
            for (auto* m : kv.second)
                if (dist(m) < dist(big)) big = m;
            const int P = kv.first * kv.first;
            int best = 0;
            double best_ms = 1e300;
            for (int eb : {48, 64, 96, 128, 160, 192, 224, 256}) {
                if ((int64_t)eb * P > 65535 || eb > std::max<int64_t>(big->mesh.ne, 48)) continue;
                big->eb_request = eb;
                double ms = 0.0;
                const sem_status st = time_handle(big, autotune_steps, &ms);
                unbuild(big);
                if (st == SEM_OK && ms < best_ms) {
                    best_ms = ms;
                    best = eb;
                }
            }
            for (auto* m : kv.second) m->eb_request = best;
        }
    }
    *out = b;
    return SEM_OK;
}

sem_status sem_batch_step(sem_batch* b, int64_t nsteps) {
    if (!b || nsteps < 0) return SEM_ERR_INVALID_ARG;
    sem_status st = batch_prepare(b);
    if (st != SEM_OK) return st;
    if (nsteps == 0) return SEM_OK;
    // a shot stepped on its own since the last batch step: its open nodes
    // finished first (the batch starts from stored levels)
    bool flushed = false;
    for (auto* m : b->shots) {
        if (!m->open_pending) continue;
        flushed = true;
        if ((st = flush_pending(m)) != SEM_OK) return bfail(b, st, m->err);
    }
    if (flushed && cudaStreamSynchronize(b->shots[0]->stream) != cudaSuccess)
        return bfail(b, SEM_ERR_CUDA, "open-node launch failed");
    for (auto* m : b->shots) {
        if (m->nrec > 0 && m->step + nsteps > m->trace_cap)
            return bfail(b, SEM_ERR_INVALID_ARG, "steps beyond a shot's receiver max_steps");
        if ((st = fill_source(m, m->step + nsteps)) != SEM_OK) return bfail(b, st, m->err);
    }
    if ((st = upload_desc(b)) != SEM_OK) return st;
    const size_t n = b->shots.size();
    if (b->streamed) return batch_step_streamed(b, nsteps);
    std::vector<int64_t> steps(n);
    for (size_t i = 0; i < n; ++i) steps[i] = b->shots[i]->step;
    if (cudaMemcpyAsync(b->d_step, steps.data(), n * 8, cudaMemcpyHostToDevice, b->run) != cudaSuccess ||
        cudaMemsetAsync(b->d_pending, 0, n * 4, b->run) != cudaSuccess ||
        cudaStreamSynchronize(b->run) != cudaSuccess)
        return bfail(b, SEM_ERR_CUDA, "step counters upload failed");
    // a block of steps captured once as a CUDA graph and replayed; the
    // remainder is launched directly
    const int G = 16;
    int64_t done = 0;
    if (nsteps >= G) {
        if (!b->graph) {
            cudaGraph_t g = nullptr;
            if (cudaStreamBeginCapture(b->run, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
                return bfail(b, SEM_ERR_CUDA, "graph capture begin failed");
            sem_status cst = SEM_OK;
            for (int k = 0; k < G && cst == SEM_OK; ++k) cst = batch_launch_step(b);
            const cudaError_t ce = cudaStreamEndCapture(b->run, &g);
            if (cst != SEM_OK) {
                if (g) cudaGraphDestroy(g);
                return cst;
            }
            if (ce != cudaSuccess) return bfail(b, SEM_ERR_CUDA, "graph capture failed");
            const cudaError_t ie = cudaGraphInstantiate(&b->graph, g, 0);
            cudaGraphDestroy(g);
            if (ie != cudaSuccess) {
                b->graph = nullptr;
                return bfail(b, SEM_ERR_CUDA, "graph instantiation failed");
            }
            b->graph_steps = G;
        }
        for (; done + G <= nsteps; done += G)
            if (cudaGraphLaunch(b->graph, b->run) != cudaSuccess) return bfail(b, SEM_ERR_CUDA, "graph launch failed");
    }
    for (; done < nsteps; ++done)
        if ((st = batch_launch_step(b)) != SEM_OK) return st;
    // host step counters, then the open nodes of every shot
    for (auto* m : b->shots) {
        m->step += nsteps;
        if ((st = launch_flush(m)) != SEM_OK) return bfail(b, st, m->err);
        m->stepped_calls++;
    }
    return SEM_OK;
}

sem_status sem_batch_info(const sem_batch* b, int32_t* nclasses, int32_t* orders, int32_t* elems_per_block,
                          int32_t* ctas) {
    if (!b) return SEM_ERR_INVALID_ARG;
    if (!b->ready) return SEM_ERR_STATE;
    if (nclasses) *nclasses = (int32_t)b->classes.size();
    for (size_t i = 0; i < b->classes.size(); ++i) {
        if (orders) orders[i] = b->classes[i].np - 1;
        if (elems_per_block) elems_per_block[i] = b->classes[i].eb;
        if (ctas) ctas[i] = b->classes[i].ctas;
    }
    return SEM_OK;
}

sem_status sem_batch_set_stream(sem_batch* b, int mode) {
    if (!b || mode < -1 || mode > 2) return SEM_ERR_INVALID_ARG;
    if (b->ready) return bfail(b, SEM_ERR_STATE, "sem_batch_set_stream after the first sem_batch_step");
    b->stream_mode = mode;
    return SEM_OK;
}

sem_status sem_batch_mode(const sem_batch* b, int32_t* streamed, int32_t* steps_per_launch) {
    if (!b) return SEM_ERR_INVALID_ARG;
    if (!b->ready) return SEM_ERR_STATE;
    int32_t n = 0;
    if (b->streamed)
        for (const auto& c : b->classes) n += c.streamed ? 1 : 0;
    if (streamed) *streamed = n;
    if (steps_per_launch) *steps_per_launch = b->streamed ? b->stream_steps : 1;
    return SEM_OK;
}

const char* sem_batch_last_error(const sem_batch* b) {
    if (!b) return "NULL batch";
    return b->err.c_str();
}

void sem_batch_destroy(sem_batch* b) {
    if (!b) return;
    cudaStreamSynchronize(b->run);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->sgraph) cudaGraphExecDestroy(b->sgraph);
    for (void* p : b->allocs) cudaFree(p);
    delete b;
}

}  // extern "C"
