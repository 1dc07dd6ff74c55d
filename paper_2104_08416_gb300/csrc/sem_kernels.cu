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
// un. Returns the new value in FP64 (for a receiver trace); in Kahan mode that
// is the compensated sum u - c.
template <typename T, int MODE>
__device__ __forceinline__ double finish_node(const StepArgs<T>& a, int32_t g, T ku, T un) {
    if (MODE == MODE_APPLY) {
        a.apply_out[g] = ku;
        return (double)ku;
    }
    T f = T(0);
    if (g == a.src_gid) f = (T)a.src_f[a.step];
    const T acc = f - ku;
    if (MODE == MODE_THREE_LEVEL) {
        const T up = a.u_prev[g];
        const T un1 = (T(2) * un - up) + a.s[g] * acc;
        a.u_out[g] = un1;
        return (double)un1;
    } else {
        // increment form: delta^{n+1/2} = delta^{n-1/2} + s (f - K u^n),
        // u^{n+1} = u^n + delta^{n+1/2} with a Kahan-compensated sum.
        const T d = a.delta[g] + a.s[g] * acc;
        const T y = sub_rn(d, a.comp[g]);
        const T t = un + y;
        const T c = sub_rn(sub_rn(t, un), y);
        a.delta[g] = d;
        a.comp[g] = c;
        a.u_out[g] = t;
        return (double)t - (double)c;
    }
}

// Metric G = w |J| / rho * J^-1 J^-T at local point (i, j) of element e.
template <typename T, bool BIL>
__device__ __forceinline__ void metric(const StepArgs<T>& a, const Basis<T>& bs, int64_t e, int64_t slot, int i,
                                       int j, T& gxx, T& gxy, T& gyy) {
    if constexpr (BIL) {
        // X(xi, eta) = a0 + b xi + c eta + d xi eta, so J = [b + d eta | c + d xi];
        // w |J| / rho * J^-1 J^-T = w / (rho |J|) * adj(J) adj(J)^T.
        const float4 c0 = __ldg(&a.coef[e * 2 + 0]);  // bx, by, cx, cy
        const float4 c1 = __ldg(&a.coef[e * 2 + 1]);  // dx, dy, 1/rho, unused
        const float xi = (float)bs.x[i], eta = (float)bs.x[j];
        const float j00 = c0.x + c1.x * eta, j10 = c0.y + c1.y * eta;
        const float j01 = c0.z + c1.x * xi, j11 = c0.w + c1.y * xi;
        const float det = j00 * j11 - j01 * j10;
        const float k = ((float)bs.w[i] * (float)bs.w[j]) * c1.z / det;
        gxx = (T)(k * (j11 * j11 + j01 * j01));
        gxy = (T)(-k * (j10 * j11 + j00 * j01));
        gyy = (T)(k * (j10 * j10 + j00 * j00));
    } else {
        gxx = a.G[slot];
        gxy = a.G[slot + a.gstride];
        gyy = a.G[slot + 2 * a.gstride];
    }
}

template <int NP, typename T, int MODE, bool BIL>
__global__ void __launch_bounds__(kThreads) sem_block_kernel(const Plan pl, const StepArgs<T> a,
                                                              const Basis<T> bs) {
    constexpr int P = NP * NP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* su = reinterpret_cast<T*>(smem_raw);        // [max_entries] u at the block's nodes
    T* sue = su + pl.max_entries;                  // [eb*P] element values, then residuals
    T* sf1 = sue + (int64_t)pl.eb * P;             // [eb*P] flux, xi component
    T* sf2 = sf1 + (int64_t)pl.eb * P;             // [eb*P] flux, eta component

    const int b = blockIdx.x;
    const int64_t e0 = (int64_t)b * pl.eb;
    const int neb = (int)min((int64_t)pl.eb, pl.ne - e0);
    const int nslot = neb * P;
    const int64_t s0 = e0 * P;
    const int ent0 = pl.ent_ptr[b];
    const int nent = pl.ent_ptr[b + 1] - ent0;
    const int tid = threadIdx.x;

    // 1. gather u at the block's nodes
    for (int l = tid; l < nent; l += kThreads) su[l] = a.u_cur[pl.ent_gid[ent0 + l]];
    __syncthreads();
    // 2. element-local copies U_mu(q,e)
    for (int s = tid; s < nslot; s += kThreads) sue[s] = su[pl.lidx[s0 + s]];
    __syncthreads();
    // 3. reference gradient, metric, fluxes
    for (int s = tid; s < nslot; s += kThreads) {
        const int el = s / P, q = s - el * P;
        const int j = q / NP, i = q - j * NP;
        const T* ue = sue + el * P;
        T dxi = T(0), deta = T(0);
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            dxi += bs.D[i * NP + k] * ue[j * NP + k];
            deta += bs.D[j * NP + k] * ue[k * NP + i];
        }
        T gxx, gxy, gyy;
        metric<T, BIL>(a, bs, e0 + el, s0 + s, i, j, gxx, gxy, gyy);
        sf1[s] = gxx * dxi + gxy * deta;
        sf2[s] = gxy * dxi + gyy * deta;
    }
    __syncthreads();
    // 4. transposed derivative: element residuals (stored over sue)
    for (int s = tid; s < nslot; s += kThreads) {
        const int el = s / P, q = s - el * P;
        const int j = q / NP, i = q - j * NP;
        const T* f1 = sf1 + el * P;
        const T* f2 = sf2 + el * P;
        T r = T(0);
#pragma unroll
        for (int k = 0; k < NP; ++k) r += bs.D[k * NP + i] * f1[j * NP + k] + bs.D[k * NP + j] * f2[k * NP + i];
        sue[s] = r;
    }
    __syncthreads();
    // 5. assembly in fixed (slot-ascending) order; finish closed nodes
    const uint16_t* lrow = pl.lrow + ent0 + b;
    for (int l = tid; l < nent; l += kThreads) {
        const int r0 = lrow[l], r1 = lrow[l + 1];
        T acc = T(0);
        for (int t = r0; t < r1; ++t) acc += sue[pl.lsl[s0 + t]];
        const int32_t ps = pl.ent_pslot[ent0 + l];
        if (ps >= 0) {
            a.partial[ps] = acc;
        } else {
            finish_node<T, MODE>(a, pl.ent_gid[ent0 + l], acc, su[l]);
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
        for (int t = p0; t < p1; ++t) acc += a.partial[t];
        const int32_t g = pl.open_gid[k];
        const T un = (MODE == MODE_APPLY) ? T(0) : a.u_cur[g];
        const double v = finish_node<T, MODE>(a, g, acc, un);
        if (MODE != MODE_APPLY && pl.open_rec != nullptr) {
            const int r = pl.open_rec[k];
            if (r >= 0) a.trace[(int64_t)r * a.trace_cap + a.step] = v;
        }
    }
}

// ------------------------------------------------------------ precompute
__global__ void geometry_kernel(int np, const double* __restrict__ coords, const int32_t* __restrict__ quads,
                                const double* __restrict__ rho, const double* __restrict__ vel, int64_t ne,
                                const Basis<double> bs, float4* coef, double* G64, float* G32,
                                double* mloc) {
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
        // bilinear coefficients: X = a + b xi + c eta + d xi eta
        const double bx = 0.25 * ((X[1] - X[0]) + (X[2] - X[3]));
        const double by = 0.25 * ((Y[1] - Y[0]) + (Y[2] - Y[3]));
        const double cx = 0.25 * ((X[3] - X[0]) + (X[2] - X[1]));
        const double cy = 0.25 * ((Y[3] - Y[0]) + (Y[2] - Y[1]));
        const double dx = 0.25 * ((X[0] - X[1]) + (X[2] - X[3]));
        const double dy = 0.25 * ((Y[0] - Y[1]) + (Y[2] - Y[3]));
        const double rinv = 1.0 / rho[e];
        if (q == 0 && coef != nullptr) {
            coef[e * 2 + 0] = make_float4((float)bx, (float)by, (float)cx, (float)cy);
            coef[e * 2 + 1] = make_float4((float)dx, (float)dy, (float)rinv, 0.0f);
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
            G64[t] = gxx;
            G64[t + total] = gxy;
            G64[t + 2 * total] = gyy;
        }
        if (G32 != nullptr) {
            G32[t] = (float)gxx;
            G32[t + total] = (float)gxy;
            G32[t + 2 * total] = (float)gyy;
        }
        if (mloc != nullptr) mloc[t] = wq * det * rinv / (vel[e] * vel[e]);
    }
}

__global__ void __launch_bounds__(kThreads) mass_block_kernel(const Plan pl, int P, const double* __restrict__ mloc,
                                                             double* partial, double* M) {
    const int b = blockIdx.x;
    const int64_t s0 = (int64_t)b * pl.eb * P;
    const int ent0 = pl.ent_ptr[b];
    const int nent = pl.ent_ptr[b + 1] - ent0;
    const uint16_t* lrow = pl.lrow + ent0 + b;
    for (int l = threadIdx.x; l < nent; l += kThreads) {
        double acc = 0.0;
        for (int t = lrow[l]; t < lrow[l + 1]; ++t) acc += mloc[s0 + pl.lsl[s0 + t]];
        const int32_t ps = pl.ent_pslot[ent0 + l];
        if (ps >= 0) partial[ps] = acc;
        else M[pl.ent_gid[ent0 + l]] = acc;
    }
}

__global__ void mass_open_kernel(const Plan pl, const double* __restrict__ partial, double* M) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < pl.nopen; k += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int t = pl.open_ptr[k]; t < pl.open_ptr[k + 1]; ++t) acc += partial[t];
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
    kern<<<pl.nblocks, kThreads, smem, st>>>(pl, *static_cast<const StepArgs<T>*>(args),
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

int smem_bytes_for(int P, int eb, int max_entries, bool fp64) {
    const int sz = fp64 ? 8 : 4;
    return (max_entries + 3 * eb * P) * sz;
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
                            const double* vel, int64_t ne, const Basis<double>& basis, float4* coef, double* G64,
                            float* G32, double* mloc, cudaStream_t st) {
    geometry_kernel<<<grid_for(ne * np * np, kThreads), kThreads, 0, st>>>(np, coords, quads_new, rho, vel, ne, basis,
                                                                          coef, G64, G32, mloc);
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
