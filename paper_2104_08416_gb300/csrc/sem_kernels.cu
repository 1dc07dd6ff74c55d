// CUDA kernels of the spectral-element time step (sm_103a).
//
// One step = two launches:
//  * sem_block_kernel: one CTA per block of consecutive elements (in the
//    chosen memory order). It gathers u at the block's nodes (the U_2 gather
//    of Algorithm 1), forms the reference gradient with the GLL derivative
//    matrix, applies the per-point metric (Eq. deriv_u with K^(e) = J^-1 and
//    the quadrature weights of Eq. numerical_integ), contracts with the
//    transposed derivative (Eq. u_change_r_effic, second-order form) and
//    assembles the element residuals of the block in shared memory through
//    the block's local node lists, in a fixed order. Nodes whose elements all
//    lie in the block are finished on the spot: inverse lumped mass (Eq.
//    Abar), point source (Algorithm 3) and leapfrog update. Nodes shared with
//    other blocks write one partial sum per block.
//  * sem_open_kernel: one thread per shared ("open") node adds its partial
//    sums in ascending block order and finishes the node.
// No floating-point atomics are used, so results are bitwise reproducible.
#include "sem_kernels.cuh"

namespace semdev {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }

// Finish node g whose assembled stiffness is ku and whose current value is
// un; st0/st1/st2 are its staged state (s, then u^{n-1} or delta, comp).
// Returns the new value in FP64 (for a receiver trace); in Kahan mode that is
// the compensated sum u - c.
template <typename T, int MODE>
__device__ __forceinline__ double finish_node(const StepArgs<T>& a, int32_t g, T ku, T un, T st0, T st1, T st2) {
    if (MODE == MODE_APPLY) {
        a.apply_out[g] = ku;
        return (double)ku;
    }
    T f = T(0);
    if (g == a.src_gid) f = (T)a.src_f[a.step];
    const T acc = f - ku;
    if (MODE == MODE_THREE_LEVEL) {
        const T un1 = (T(2) * un - st1) + st0 * acc;
        a.u_out[g] = un1;
        return (double)un1;
    } else {
        // increment form: delta^{n+1/2} = delta^{n-1/2} + s (f - K u^n),
        // u^{n+1} = u^n + delta^{n+1/2} with a Kahan-compensated sum.
        const T d = st1 + st0 * acc;
        const T y = sub_rn(d, st2);
        const T t = un + y;
        const T c = sub_rn(sub_rn(t, un), y);
        a.delta[g] = d;
        a.comp[g] = c;
        a.u_out[g] = t;
        return (double)t - (double)c;
    }
}

// Same, loading the node state from global memory.
template <typename T, int MODE>
__device__ __forceinline__ double finish_node_global(const StepArgs<T>& a, int32_t g, T ku, T un) {
    if (MODE == MODE_APPLY) return finish_node<T, MODE>(a, g, ku, un, T(0), T(0), T(0));
    if (MODE == MODE_THREE_LEVEL) return finish_node<T, MODE>(a, g, ku, un, a.s[g], a.u_prev[g], T(0));
    return finish_node<T, MODE>(a, g, ku, un, a.s[g], a.delta[g], a.comp[g]);
}

// Keeps a value in a register: the compiler cannot re-derive it from memory.
__device__ __forceinline__ float pin(float v) {
    asm volatile("" : "+f"(v));
    return v;
}
__device__ __forceinline__ double pin(double v) {
    asm volatile("" : "+d"(v));
    return v;
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
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Metric G = w |J| / rho * J^-1 J^-T at a point (xi, eta) of weight wq,
// from the element's bilinear-map coefficients (b, c, d, 1/rho):
// X(xi, eta) = a0 + b xi + c eta + d xi eta, so J = [b + d eta | c + d xi], and
// w |J| / rho * J^-1 J^-T = w / (rho |J|) * adj(J) adj(J)^T.
template <typename T>
__device__ __forceinline__ void metric_bilinear(const float4 c0, const float4 c1, float xi, float eta, float wq,
                                                T& gxx, T& gxy, T& gyy) {
    const float j00 = c0.x + c1.x * eta, j10 = c0.y + c1.y * eta;
    const float j01 = c0.z + c1.x * xi, j11 = c0.w + c1.y * xi;
    const float det = j00 * j11 - j01 * j10;
    const float k = wq * c1.z / det;
    gxx = (T)(k * (j11 * j11 + j01 * j01));
    gxy = (T)(-k * (j10 * j11 + j00 * j01));
    gyy = (T)(k * (j10 * j10 + j00 * j00));
}

// Elements processed side by side by one CTA: each thread keeps one GLL point
// (i, j) of one element lane for the whole kernel, so its rows and columns of
// the derivative matrix live in registers.
template <int NP>
struct Lanes {
    static constexpr int P = NP * NP;
    static constexpr int EBW = (kThreads / P) > 0 ? (kThreads / P) : 1;
    static constexpr int THREADS = EBW * P;
};

template <int NP, typename T, int MODE, bool BIL>
__global__ void __launch_bounds__(Lanes<NP>::THREADS) sem_block_kernel(const Plan pl, const StepArgs<T> a,
                                                                       const Basis<T> bs) {
    constexpr int P = NP * NP;
    constexpr int EBW = Lanes<NP>::EBW;
    constexpr int NT = Lanes<NP>::THREADS;
    constexpr bool STAGE = MODE != MODE_APPLY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint8_t* spk = smem_raw;                                          // packet
    T* su = reinterpret_cast<T*>(smem_raw + pl.max_packet);           // [max_entries] u at the entries
    T* st0 = su + pl.max_entries;                                     // staged node state
    T* st1 = st0 + (STAGE ? pl.max_entries : 0);
    T* st2 = st1 + (STAGE ? pl.max_entries : 0);
    T* sue = st2 + (MODE == MODE_KAHAN ? pl.max_entries : 0);         // [eb*P] element values, then residuals
    T* sf1 = sue + pl.eb * P;                                         // [eb*P] flux, xi component
    T* sf2 = sf1 + pl.eb * P;                                         // [eb*P] flux, eta component

    const int b = blockIdx.x;
    const int4 hd = pl.hdr[b];
    const int nent = hd.y, nclosed = hd.z, pbase = hd.w;
    const int64_t e0 = (int64_t)b * pl.eb;
    const int neb = (int)min((int64_t)pl.eb, pl.ne - e0);
    const int nslot = neb * P;
    const PacketOffsets L = packet_offsets(nslot, nent, neb);
    const int tid = threadIdx.x;
    const int q = tid % P, lane_el = tid / P;
    const int j = q / NP, i = q - j * NP;

    // 0. stage the block's packet (indices, local lists, geometry) with
    //    16-byte asynchronous copies
    {
        const uint8_t* gpk = pl.packet + (int64_t)hd.x * 16;
        for (int off = tid * 16; off < L.bytes; off += NT * 16) cp_async16(spk + off, gpk + off);
        cp_async_commit();
    }
    // GLL tables to shared memory (kernel parameters indexed per thread would
    // serialise in the constant cache), then this thread's derivative rows and
    // columns into registers, pinned there
    __shared__ T sD[P];
    __shared__ float sxw[2 * NP];
    for (int t = tid; t < P; t += NT) sD[t] = bs.D[t];
    for (int t = tid; t < NP; t += NT) {
        sxw[t] = (float)bs.x[t];
        sxw[NP + t] = (float)bs.w[t];
    }
    __syncthreads();
    T Di[NP], Dj[NP], DTi[NP], DTj[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        Di[k] = pin(sD[i * NP + k]);
        Dj[k] = pin(sD[j * NP + k]);
        DTi[k] = pin(sD[k * NP + i]);
        DTj[k] = pin(sD[k * NP + j]);
    }
    const float xi = pin(sxw[i]), eta = pin(sxw[j]);
    const float wq = pin(sxw[NP + i] * sxw[NP + j]);
    cp_async_wait<0>();
    __syncthreads();
    const uint16_t* lidx = reinterpret_cast<const uint16_t*>(spk + L.lidx);
    const uint16_t* lsl = reinterpret_cast<const uint16_t*>(spk + L.lsl);
    const uint16_t* lrow = reinterpret_cast<const uint16_t*>(spk + L.lrow);
    const int32_t* gid = reinterpret_cast<const int32_t*>(spk + L.gid);
    const float4* coef = reinterpret_cast<const float4*>(spk + L.coef);

    // 1. gather u at the entries (group 1), then the closed nodes' state (group 2)
    for (int l = tid; l < nent; l += NT) cp_async_small<sizeof(T)>(su + l, a.u_cur + gid[l]);
    cp_async_commit();
    if (STAGE) {
        for (int l = tid; l < nclosed; l += NT) {
            const int32_t g = gid[l];
            cp_async_small<sizeof(T)>(st0 + l, a.s + g);
            if (MODE == MODE_THREE_LEVEL) {
                cp_async_small<sizeof(T)>(st1 + l, a.u_prev + g);
            } else {
                cp_async_small<sizeof(T)>(st1 + l, a.delta + g);
                cp_async_small<sizeof(T)>(st2 + l, a.comp + g);
            }
        }
    }
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    // 2. element-local copies U_mu(q,e)
    for (int el = lane_el; el < neb; el += EBW) sue[el * P + q] = su[lidx[el * P + q]];
    __syncthreads();
    // 3. reference gradient, metric, fluxes
    for (int el = lane_el; el < neb; el += EBW) {
        const T* ue = sue + el * P;
        T dxi = T(0), deta = T(0);
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            dxi += Di[k] * ue[j * NP + k];
            deta += Dj[k] * ue[k * NP + i];
        }
        T gxx, gxy, gyy;
        if constexpr (BIL) {
            metric_bilinear<T>(coef[el * 2], coef[el * 2 + 1], xi, eta, wq, gxx, gxy, gyy);
        } else {
            const int64_t sl = (e0 + el) * P + q;
            gxx = a.G[sl];
            gxy = a.G[sl + a.gstride];
            gyy = a.G[sl + 2 * a.gstride];
        }
        sf1[el * P + q] = gxx * dxi + gxy * deta;
        sf2[el * P + q] = gxy * dxi + gyy * deta;
    }
    __syncthreads();
    // 4. transposed derivative: element residuals (stored over sue)
    for (int el = lane_el; el < neb; el += EBW) {
        const T* f1 = sf1 + el * P;
        const T* f2 = sf2 + el * P;
        T r = T(0);
#pragma unroll
        for (int k = 0; k < NP; ++k) r += DTi[k] * f1[j * NP + k] + DTj[k] * f2[k * NP + i];
        sue[el * P + q] = r;
    }
    cp_async_wait<0>();
    __syncthreads();
    // 5. assembly in fixed (slot-ascending) order; closed nodes are finished
    //    here, open ones leave a partial sum
    for (int l = tid; l < nent; l += NT) {
        const int r0 = lrow[l], r1 = lrow[l + 1];
        T acc = T(0);
        for (int t = r0; t < r1; ++t) acc += sue[lsl[t]];
        if (l >= nclosed) {
            a.partial[pbase + (l - nclosed)] = acc;
        } else if (STAGE) {
            finish_node<T, MODE>(a, gid[l], acc, su[l], st0[l], st1[l], MODE == MODE_KAHAN ? st2[l] : T(0));
        } else {
            finish_node<T, MODE>(a, gid[l], acc, su[l], T(0), T(0), T(0));
        }
    }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads) sem_open_kernel(const Plan pl, const StepArgs<T> a) {
    // receivers at closed nodes: their value is final once the block kernel ended
    if (MODE != MODE_APPLY && blockIdx.x == 0 && a.nrec > 0) {
        for (int r = threadIdx.x; r < a.nrec; r += kThreads)
            if (a.rec_closed[r]) {
                const int32_t g = a.rec_gid[r];
                double v = (double)a.u_out[g];
                if (MODE == MODE_KAHAN) v -= (double)a.comp[g];
                a.trace[(int64_t)r * a.trace_cap + a.step] = v;
            }
    }
    for (int k = blockIdx.x * kThreads + threadIdx.x; k < pl.nopen; k += gridDim.x * kThreads) {
        const int p0 = pl.open_ptr[k], p1 = pl.open_ptr[k + 1];
        T acc = T(0);
        for (int t = p0; t < p1; ++t) acc += a.partial[pl.open_src[t]];
        const int32_t g = pl.open_gid[k];
        const T un = (MODE == MODE_APPLY) ? T(0) : a.u_cur[g];
        const double v = finish_node_global<T, MODE>(a, g, acc, un);
        if (MODE != MODE_APPLY && pl.open_rec != nullptr) {
            const int r = pl.open_rec[k];
            if (r >= 0) a.trace[(int64_t)r * a.trace_cap + a.step] = v;
        }
    }
}

// ------------------------------------------------------------ precompute
__global__ void geometry_kernel(int np, const double* __restrict__ coords, const int32_t* __restrict__ quads,
                                const double* __restrict__ rho, const double* __restrict__ vel, const Plan pl,
                                const Basis<double> bs, uint8_t* packet, double* G64, double* mloc) {
    const int P = np * np;
    const int64_t ne = pl.ne;
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
        // bilinear coefficients: X = a + b xi + c eta + d xi eta
        const double bx = 0.25 * ((X[1] - X[0]) + (X[2] - X[3]));
        const double by = 0.25 * ((Y[1] - Y[0]) + (Y[2] - Y[3]));
        const double cx = 0.25 * ((X[3] - X[0]) + (X[2] - X[1]));
        const double cy = 0.25 * ((Y[3] - Y[0]) + (Y[2] - Y[1]));
        const double dx = 0.25 * ((X[0] - X[1]) + (X[2] - X[3]));
        const double dy = 0.25 * ((Y[0] - Y[1]) + (Y[2] - Y[3]));
        const double rinv = 1.0 / rho[e];
        if (q == 0 && packet != nullptr) {
            const int b = (int)(e / pl.eb);
            const int el = (int)(e - (int64_t)b * pl.eb);
            const int neb = (int)min((int64_t)pl.eb, ne - (int64_t)b * pl.eb);
            const int4 hd = pl.hdr[b];
            const PacketOffsets L = packet_offsets(neb * P, hd.y, neb);
            float4* cf = reinterpret_cast<float4*>(packet + (int64_t)hd.x * 16 + L.coef) + el * 2;
            cf[0] = make_float4((float)bx, (float)by, (float)cx, (float)cy);
            cf[1] = make_float4((float)dx, (float)dy, (float)rinv, 0.0f);
        }
        const double xi = bs.x[i], eta = bs.x[j];
        const double j00 = bx + dx * eta, j10 = by + dy * eta;
        const double j01 = cx + dx * xi, j11 = cy + dy * xi;
        const double det = j00 * j11 - j01 * j10;
        const double wq = bs.w[i] * bs.w[j];
        const double k = wq * rinv / det;
        if (G64 != nullptr) {
            G64[t] = k * (j11 * j11 + j01 * j01);
            G64[t + total] = -k * (j10 * j11 + j00 * j01);
            G64[t + 2 * total] = k * (j10 * j10 + j00 * j00);
        }
        if (mloc != nullptr) mloc[t] = wq * det * rinv / (vel[e] * vel[e]);
    }
}

__global__ void __launch_bounds__(kThreads) mass_block_kernel(const Plan pl, int P, const double* __restrict__ mloc,
                                                             double* partial, double* M) {
    const int b = blockIdx.x;
    const int4 hd = pl.hdr[b];
    const int64_t e0 = (int64_t)b * pl.eb;
    const int neb = (int)min((int64_t)pl.eb, pl.ne - e0);
    const PacketOffsets L = packet_offsets(neb * P, hd.y, neb);
    const uint8_t* pk = pl.packet + (int64_t)hd.x * 16;
    const uint16_t* lsl = reinterpret_cast<const uint16_t*>(pk + L.lsl);
    const uint16_t* lrow = reinterpret_cast<const uint16_t*>(pk + L.lrow);
    const int32_t* gid = reinterpret_cast<const int32_t*>(pk + L.gid);
    const int64_t s0 = e0 * P;
    for (int l = threadIdx.x; l < hd.y; l += kThreads) {
        double acc = 0.0;
        for (int t = lrow[l]; t < lrow[l + 1]; ++t) acc += mloc[s0 + lsl[t]];
        if (l >= hd.z) partial[hd.w + (l - hd.z)] = acc;
        else M[gid[l]] = acc;
    }
}

__global__ void mass_open_kernel(const Plan pl, const double* __restrict__ partial, double* M) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < pl.nopen; k += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int t = pl.open_ptr[k]; t < pl.open_ptr[k + 1]; ++t) acc += partial[pl.open_src[t]];
        M[pl.open_gid[k]] = acc;
    }
}

__global__ void scale_kernel(const double* __restrict__ M, int64_t nn, double dt, double* s64, float* s32) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nn; g += (int64_t)gridDim.x * blockDim.x) {
        const double v = (dt * dt) / M[g];
        if (s64) s64[g] = v;
        if (s32) s32[g] = (float)v;
    }
}

int grid_for(int64_t n, int threads) {
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 152 * 64) g = 152 * 64;
    return (int)g;
}

template <int NP, typename T, int MODE, bool BIL>
cudaError_t launch_block_t(const Plan& pl, const void* args, const void* basis, int smem, cudaStream_t st) {
    auto kern = sem_block_kernel<NP, T, MODE, BIL>;
    static int configured = 0;
    if (smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    kern<<<pl.nblocks, Lanes<NP>::THREADS, smem, st>>>(pl, *static_cast<const StepArgs<T>*>(args),
                                             *static_cast<const Basis<T>*>(basis));
    return cudaGetLastError();
}

template <typename T, int MODE, bool BIL>
cudaError_t dispatch_np(int np, const Plan& pl, const void* args, const void* basis, int smem, cudaStream_t st) {
    switch (np) {
        case 2: return launch_block_t<2, T, MODE, BIL>(pl, args, basis, smem, st);
        case 3: return launch_block_t<3, T, MODE, BIL>(pl, args, basis, smem, st);
        case 4: return launch_block_t<4, T, MODE, BIL>(pl, args, basis, smem, st);
        case 5: return launch_block_t<5, T, MODE, BIL>(pl, args, basis, smem, st);
        case 6: return launch_block_t<6, T, MODE, BIL>(pl, args, basis, smem, st);
        case 7: return launch_block_t<7, T, MODE, BIL>(pl, args, basis, smem, st);
        case 8: return launch_block_t<8, T, MODE, BIL>(pl, args, basis, smem, st);
        case 9: return launch_block_t<9, T, MODE, BIL>(pl, args, basis, smem, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

int lanes_for(int np) {
    switch (np) {
        case 2: return Lanes<2>::EBW;
        case 3: return Lanes<3>::EBW;
        case 4: return Lanes<4>::EBW;
        case 5: return Lanes<5>::EBW;
        case 6: return Lanes<6>::EBW;
        case 7: return Lanes<7>::EBW;
        case 8: return Lanes<8>::EBW;
        case 9: return Lanes<9>::EBW;
        default: return 1;
    }
}

int smem_bytes_for(int P, int eb, int max_entries, int max_packet, bool fp64, int mode) {
    const int sz = fp64 ? 8 : 4;
    const int staged = mode == MODE_KAHAN ? 3 : (mode == MODE_THREE_LEVEL ? 2 : 0);
    return max_packet + (max_entries * (1 + staged) + 3 * eb * P) * sz;
}

cudaError_t launch_step(int np, bool fp64, int mode, bool bilinear, const Plan& pl, const void* args,
                        const void* basis, int smem, cudaStream_t st) {
    if (fp64) {
        if (bilinear) return cudaErrorInvalidValue;
        switch (mode) {
            case MODE_THREE_LEVEL: return dispatch_np<double, MODE_THREE_LEVEL, false>(np, pl, args, basis, smem, st);
            case MODE_APPLY: return dispatch_np<double, MODE_APPLY, false>(np, pl, args, basis, smem, st);
            default: return cudaErrorInvalidValue;
        }
    }
    if (bilinear) {
        switch (mode) {
            case MODE_THREE_LEVEL: return dispatch_np<float, MODE_THREE_LEVEL, true>(np, pl, args, basis, smem, st);
            case MODE_KAHAN: return dispatch_np<float, MODE_KAHAN, true>(np, pl, args, basis, smem, st);
            case MODE_APPLY: return dispatch_np<float, MODE_APPLY, true>(np, pl, args, basis, smem, st);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (mode) {
        case MODE_KAHAN: return dispatch_np<float, MODE_KAHAN, false>(np, pl, args, basis, smem, st);
        case MODE_APPLY: return dispatch_np<float, MODE_APPLY, false>(np, pl, args, basis, smem, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_open(bool fp64, int mode, const Plan& pl, const void* args, cudaStream_t st) {
    const int grid = grid_for(pl.nopen, kThreads);
    if (fp64) {
        const auto& a = *static_cast<const StepArgs<double>*>(args);
        if (mode == MODE_THREE_LEVEL) sem_open_kernel<double, MODE_THREE_LEVEL><<<grid, kThreads, 0, st>>>(pl, a);
        else if (mode == MODE_APPLY) sem_open_kernel<double, MODE_APPLY><<<grid, kThreads, 0, st>>>(pl, a);
        else return cudaErrorInvalidValue;
    } else {
        const auto& a = *static_cast<const StepArgs<float>*>(args);
        if (mode == MODE_THREE_LEVEL) sem_open_kernel<float, MODE_THREE_LEVEL><<<grid, kThreads, 0, st>>>(pl, a);
        else if (mode == MODE_KAHAN) sem_open_kernel<float, MODE_KAHAN><<<grid, kThreads, 0, st>>>(pl, a);
        else sem_open_kernel<float, MODE_APPLY><<<grid, kThreads, 0, st>>>(pl, a);
    }
    return cudaGetLastError();
}

cudaError_t launch_geometry(int np, const double* coords, const int32_t* quads_new, const double* rho,
                            const double* vel, const Plan& plan, const Basis<double>& basis, uint8_t* packet,
                            double* G64, double* mloc, cudaStream_t st) {
    geometry_kernel<<<grid_for(plan.ne * np * np, kThreads), kThreads, 0, st>>>(np, coords, quads_new, rho, vel, plan,
                                                                               basis, packet, G64, mloc);
    return cudaGetLastError();
}

cudaError_t launch_mass(const Plan& pl, int P, const double* mloc, double* partial, double* M, cudaStream_t st) {
    mass_block_kernel<<<pl.nblocks, kThreads, 0, st>>>(pl, P, mloc, partial, M);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    mass_open_kernel<<<grid_for(pl.nopen, kThreads), kThreads, 0, st>>>(pl, partial, M);
    return cudaGetLastError();
}

cudaError_t launch_scale(const double* M, int64_t nn, double dt, double* s64, float* s32, cudaStream_t st) {
    scale_kernel<<<grid_for(nn, kThreads), kThreads, 0, st>>>(M, nn, dt, s64, s32);
    return cudaGetLastError();
}

}  // namespace semdev
