// Non-hot kernels of libplbm: initial equilibrium, moments of the stored state,
// deterministic FP64 reductions and population import/export.  All arithmetic
// here is FP64 regardless of the storage precision.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "plbm.h"
#include "plbm_device.cuh"

namespace plbm {

cudaError_t launch_step_f64(const LatticeParams&, const void*, void*, bool, cudaStream_t);
cudaError_t launch_step_f32(const LatticeParams&, const void*, void*, bool, cudaStream_t);
cudaError_t launch_step_f16(const LatticeParams&, const void*, void*, bool, cudaStream_t);
cudaError_t launch_step_bf16(const LatticeParams&, const void*, void*, bool, cudaStream_t);

cudaError_t launch_batch_f32(const PairParams*, int, int, int, int, int, const unsigned short*, cudaStream_t);
cudaError_t launch_batch_f16(const PairParams*, int, int, int, int, int, const unsigned short*, cudaStream_t);
cudaError_t launch_batch_bf16(const PairParams*, int, int, int, int, int, const unsigned short*, cudaStream_t);
cudaError_t batch_occupancy_f32(int, int*);
cudaError_t batch_occupancy_f16(int, int*);
cudaError_t batch_occupancy_bf16(int, int*);

cudaError_t launch_batch_node_f64(int, const LatticeParams*, const NodeSpan*, int, int, int, const unsigned short*,
                                  cudaStream_t);
cudaError_t launch_batch_node_f32(int, const LatticeParams*, const NodeSpan*, int, int, int, const unsigned short*,
                                  cudaStream_t);
cudaError_t launch_batch_node_f16(int, const LatticeParams*, const NodeSpan*, int, int, int, const unsigned short*,
                                  cudaStream_t);
cudaError_t launch_batch_node_bf16(int, const LatticeParams*, const NodeSpan*, int, int, int, const unsigned short*,
                                   cudaStream_t);
cudaError_t batch_node_occupancy_f64(int, int*);
cudaError_t batch_node_occupancy_f32(int, int*);
cudaError_t batch_node_occupancy_f16(int, int*);
cudaError_t batch_node_occupancy_bf16(int, int*);

cudaError_t launch_batch_node(int prec, int q1, const LatticeParams* inst, const NodeSpan* span, int total_tiles,
                              int ctas, int parity, const unsigned short* tile_inst, cudaStream_t stream) {
    switch (prec) {
        case kF64: return launch_batch_node_f64(q1, inst, span, total_tiles, ctas, parity, tile_inst, stream);
        case kF32: return launch_batch_node_f32(q1, inst, span, total_tiles, ctas, parity, tile_inst, stream);
        case kF16Dev: return launch_batch_node_f16(q1, inst, span, total_tiles, ctas, parity, tile_inst, stream);
        case kBF16Dev: return launch_batch_node_bf16(q1, inst, span, total_tiles, ctas, parity, tile_inst, stream);
    }
    return cudaErrorInvalidValue;
}

cudaError_t batch_node_occupancy(int prec, int q1, int* blocks_per_sm) {
    switch (prec) {
        case kF64: return batch_node_occupancy_f64(q1, blocks_per_sm);
        case kF32: return batch_node_occupancy_f32(q1, blocks_per_sm);
        case kF16Dev: return batch_node_occupancy_f16(q1, blocks_per_sm);
        case kBF16Dev: return batch_node_occupancy_bf16(q1, blocks_per_sm);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_batch(int prec, const PairParams* inst, int ninst, int total_tiles, int block_x,
                         int ctas, int parity, const unsigned short* tile_inst, cudaStream_t stream) {
    switch (prec) {
        case kF32: return launch_batch_f32(inst, ninst, total_tiles, block_x, ctas, parity, tile_inst, stream);
        case kF16Dev: return launch_batch_f16(inst, ninst, total_tiles, block_x, ctas, parity, tile_inst, stream);
        case kBF16Dev: return launch_batch_bf16(inst, ninst, total_tiles, block_x, ctas, parity, tile_inst, stream);
    }
    return cudaErrorInvalidValue;
}

cudaError_t batch_occupancy(int prec, int block_x, int* blocks_per_sm) {
    switch (prec) {
        case kF32: return batch_occupancy_f32(block_x, blocks_per_sm);
        case kF16Dev: return batch_occupancy_f16(block_x, blocks_per_sm);
        case kBF16Dev: return batch_occupancy_bf16(block_x, blocks_per_sm);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_step(int prec, const LatticeParams& P, const void* src, void* dst, bool reduce,
                        cudaStream_t stream) {
    switch (prec) {
        case kF64: return launch_step_f64(P, src, dst, reduce, stream);
        case kF32: return launch_step_f32(P, src, dst, reduce, stream);
        case kF16Dev: return launch_step_f16(P, src, dst, reduce, stream);
        case kBF16Dev: return launch_step_bf16(P, src, dst, reduce, stream);
    }
    return cudaErrorInvalidValue;
}

// FP64 equilibrium of one node, Eq. (eq:eqdist) with Eq. (eq:rdr) per axis and
// the tensor product of Sec. 2.1.  out[p], p = ix*q1 + iy.
__device__ void node_feq_f64(const LatticeParams& P, double rho, double ux, double uy, double th,
                             double* out) {
    double rx[kMaxQ1], ry[kMaxQ1], mu[kMaxQ1];
    const int q1 = P.q1;
    for (int a = 0; a < P.dim; ++a) {
        const double u = (a == 0) ? ux : uy;
        mu[0] = 1.0;
        mu[1] = u;
        for (int n = 1; n + 1 < q1; ++n) mu[n + 1] = u * mu[n] + (double)n * th * mu[n - 1];
        for (int i = 0; i < q1; ++i) {
            double r = 0.0;
            for (int n = 0; n < q1; ++n) r += P.C[i * q1 + n] * mu[n];
            if (a == 0) rx[i] = r; else ry[i] = r;
        }
    }
    if (P.dim == 1) {
        for (int i = 0; i < q1; ++i) out[i] = rho * rx[i];
    } else {
        for (int i = 0; i < q1; ++i)
            for (int j = 0; j < q1; ++j) out[i * q1 + j] = rho * rx[i] * ry[j];
    }
}

// Moments of one node from FP64 populations.
__device__ void node_moments_f64(const LatticeParams& P, const double* f, double& rho, double& ux,
                                 double& uy, double& th, double& e, double& jx_o, double& jy_o) {
    double r = 0.0, jx = 0.0, jy = 0.0, en = 0.0;
    for (int p = 0; p < P.q; ++p) {
        const int ix = (P.dim == 1) ? p : p / P.q1;
        const int iy = (P.dim == 1) ? 0 : p % P.q1;
        const double vx = (double)P.v[ix];
        const double vy = (P.dim == 1) ? 0.0 : (double)P.v[iy];
        r += f[p];
        jx += vx * f[p];
        jy += vy * f[p];
        en += (vx * vx + vy * vy) * f[p];
    }
    rho = r;
    ux = jx / r;
    uy = jy / r;
    th = (en / r - (ux * ux + uy * uy)) / (double)P.dim;
    e = en;
    jx_o = jx;
    jy_o = jy;
}

// Check of one node's initial fields, made by the initialisation kernels that read
// them anyway: a non-finite value sets PLBM_STATUS_NONFINITE, otherwise rho <= 0
// PLBM_STATUS_RHO_NONPOS and theta <= 0 PLBM_STATUS_THETA_NONPOS.
__device__ __forceinline__ void check_init_node(const LatticeParams& P, const double* rho, const double* ux,
                                                const double* uy, const double* theta, long long n) {
    const double r = rho[n], a = ux[n];
    const double b = (P.dim == 2 && uy) ? uy[n] : 0.0;
    const bool has_t = !(P.isothermal || theta == nullptr);
    const double t = has_t ? theta[n] : 1.0;
    if (isfinite(r) && isfinite(a) && isfinite(b) && isfinite(t) && r > 0.0 && t > 0.0) return;
    unsigned bits = 0u;
    if (!isfinite(r) || !isfinite(a) || !isfinite(b) || !isfinite(t)) bits |= PLBM_STATUS_NONFINITE;
    if (isfinite(r) && !(r > 0.0)) bits |= PLBM_STATUS_RHO_NONPOS;
    if (isfinite(t) && !(t > 0.0)) bits |= PLBM_STATUS_THETA_NONPOS;
    atomicOr(P.status, bits);
}

template <typename S>
__global__ void k_init(const __grid_constant__ LatticeParams P, const double* __restrict__ rho,
                       const double* __restrict__ ux, const double* __restrict__ uy,
                       const double* __restrict__ theta, S* __restrict__ f, int y0) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = y0 + blockIdx.y;
    if (x >= P.nx) return;
    const long long n = (long long)y * P.nx + x;
    check_init_node(P, rho, ux, uy, theta, n);
    const double th = (P.isothermal || theta == nullptr) ? P.theta0 : theta[n];
    double feq[kMaxQ];
    node_feq_f64(P, rho[n], ux[n], (P.dim == 2 && uy) ? uy[n] : 0.0, th, feq);
    for (int p = 0; p < P.q; ++p) f[elem_index(P, p, x, y)] = Storage<S>::from_f64(feq[p], P.W0[p]);
}

// Compile-time q1 versions of the two kernels above (arrays in registers, no
// integer division per population); the same FP64 formulas, the moments from
// the row and column sums S_i = sum_j f_ij, T_j = sum_i f_ij.
template <typename S, int Q1, int DIM>
__global__ void k_init_q(const __grid_constant__ LatticeParams P, const double* __restrict__ rho,
                         const double* __restrict__ ux, const double* __restrict__ uy,
                         const double* __restrict__ theta, S* __restrict__ f, int y0) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = y0 + blockIdx.y;
    if (x >= P.nx) return;
    const long long n = (long long)y * P.nx + x;
    check_init_node(P, rho, ux, uy, theta, n);
    const double th = (P.isothermal || theta == nullptr) ? P.theta0 : theta[n];
    double r[DIM][Q1];
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const double u = a == 0 ? ux[n] : (uy ? uy[n] : 0.0);
        double mu[Q1];
        mu[0] = 1.0;
        if (Q1 > 1) mu[1] = u;
#pragma unroll
        for (int k = 1; k + 1 < Q1; ++k) mu[k + 1] = u * mu[k] + (double)k * th * mu[k - 1];
#pragma unroll
        for (int i = 0; i < Q1; ++i) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < Q1; ++k) s += P.C[i * Q1 + k] * mu[k];
            r[a][i] = s;
        }
    }
    const double rh = rho[n];
#pragma unroll
    for (int i = 0; i < Q1; ++i) {
        const double ri = rh * r[0][i];
#pragma unroll
        for (int j = 0; j < (DIM == 2 ? Q1 : 1); ++j) {
            const int p = DIM == 2 ? i * Q1 + j : i;
            const double fe = DIM == 2 ? ri * r[DIM - 1][j] : ri;
            f[elem_index(P, p, x, y)] = Storage<S>::from_f64(fe, P.W0[p]);
        }
    }
}

template <typename S, int Q1, int DIM>
__global__ void k_moments_q(const __grid_constant__ LatticeParams P, const S* __restrict__ f, double* rho,
                            double* ux, double* uy, double* theta, int y0) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = y0 + blockIdx.y;
    if (x >= P.nx) return;
    double Sx[Q1], Ty[Q1];
#pragma unroll
    for (int i = 0; i < Q1; ++i) Sx[i] = Ty[i] = 0.0;
#pragma unroll
    for (int i = 0; i < Q1; ++i)
#pragma unroll
        for (int j = 0; j < (DIM == 2 ? Q1 : 1); ++j) {
            const int p = DIM == 2 ? i * Q1 + j : i;
            const double v = Storage<S>::to_f64(f[elem_index(P, p, x, y)], P.W0[p]);
            Sx[i] += v;
            Ty[j] += v;
        }
    double m0 = 0.0, jx = 0.0, jy = 0.0, en = 0.0;
#pragma unroll
    for (int i = 0; i < Q1; ++i) {
        const double vi = (double)P.v[i];
        m0 += Sx[i];
        jx += vi * Sx[i];
        en += vi * vi * Sx[i];
        if (DIM == 2) {
            jy += vi * Ty[i];
            en += vi * vi * Ty[i];
        }
    }
    const double a = jx / m0, b = jy / m0;
    const long long n = (long long)y * P.nx + x;
    if (rho) rho[n] = m0;
    if (ux) ux[n] = a;
    if (uy) uy[n] = b;
    if (theta) theta[n] = (en / m0 - (a * a + b * b)) / (double)DIM;
}

// Initial state of a 16/32-bit handle with a symmetric five-velocity set, in the
// FP32 deviation arithmetic of its own collision: per axis the constraint form
// of the rule (dmu_n = mu_n(u, theta) - mu_n(0, theta0), n = 1..4;
// O_b = (dmu3 - a^2 dmu1) / (2b(b^2 - a^2)), O_a = (dmu1 - 2b O_b) / (2a),
// E_b = (dmu4 - a^2 dmu2) / (2b^2(b^2 - a^2)), E_a = (dmu2 - 2b^2 E_b) / (2a^2),
// dr = (-2(E_a + E_b), E_a +- O_a, E_b +- O_b)), then
// f^eq - w0 = X_i (w_j + dr^y_j) + w_i dr^y_j with X_i = (rho - 1) w_i + rho dr^x_i
// (in 1D: X_i).  The inputs enter as the small quantities rho - 1, u and
// theta - theta0, formed in FP64.
__device__ __forceinline__ void sym5_dev(const LatticeParams& P, float u, float dth, float (&dr)[5]) {
    const float u2 = u * u;
    const float th = P.theta0f + dth;
    const float dm1 = u;
    const float dm2 = u2 + dth;
    const float dm3 = u * (u2 + 3.0f * th);
    const float dm4 = u2 * (u2 + 6.0f * th) + 3.0f * dth * (th + P.theta0f);
    const float Ob = (dm3 - P.sa2 * dm1) * P.kOb;
    const float Oa = (dm1 - 2.0f * P.sb * Ob) * P.kOa;
    const float Eb = (dm4 - P.sa2 * dm2) * P.kEb;
    const float Ea = (dm2 - 2.0f * P.sb2 * Eb) * P.kEa;
    dr[0] = -2.0f * (Ea + Eb);
    dr[1] = Ea + Oa;
    dr[2] = Ea - Oa;
    dr[3] = Eb + Ob;
    dr[4] = Eb - Ob;
}

template <typename S, int DIM>
__global__ void k_init_sym5_dev(const __grid_constant__ LatticeParams P, const double* __restrict__ rho,
                                const double* __restrict__ ux, const double* __restrict__ uy,
                                const double* __restrict__ theta, S* __restrict__ f, int y0) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = y0 + blockIdx.y;
    if (x >= P.nx) return;
    const long long n = (long long)y * P.nx + x;
    check_init_node(P, rho, ux, uy, theta, n);
    const float dth = (P.isothermal || theta == nullptr) ? 0.0f : (float)(theta[n] - P.theta0);
    const float drho = (float)(rho[n] - 1.0);
    const float rh = 1.0f + drho;
    float drx[5], dry[5];
    sym5_dev(P, (float)ux[n], dth, drx);
    if (DIM == 2) sym5_dev(P, uy ? (float)uy[n] : 0.0f, dth, dry);
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const float X = fmaf(drho, P.w1f[i], rh * drx[i]);
        if (DIM == 1) {
            Storage<S>::store(f + elem_index(P, i, x, y), X);
        } else {
#pragma unroll
            for (int j = 0; j < 5; ++j)
                Storage<S>::store(f + elem_index(P, i * 5 + j, x, y),
                                  fmaf(X, P.w1f[j] + dry[j], P.w1f[i] * dry[j]));
        }
    }
}

// Moments of a 16/32-bit (deviation) state: the row and column sums of the
// stored deviations g in float-float arithmetic (an FP32 pair hi + lo carried
// through error-free sums and products, ~2^-48 relative), then
// rho = 1 + sum g, j = sum v g, E = d theta0 + sum |v|^2 g (the rest identities of
// the 1D rule) and theta = (E / rho - |u|^2) / d in FP64.
// (FF, ff_add, ff_scale, ff_f64: plbm_device.cuh)

template <typename S, int Q1, int DIM>
__global__ void k_moments_dev(const __grid_constant__ LatticeParams P, const S* __restrict__ f, double* rho,
                              double* ux, double* uy, double* theta, int y0) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = y0 + blockIdx.y;
    if (x >= P.nx) return;
    FF Sx[Q1], Ty[Q1];
#pragma unroll
    for (int i = 0; i < Q1; ++i) Sx[i] = Ty[i] = FF{0.0f, 0.0f};
#pragma unroll
    for (int i = 0; i < Q1; ++i)
#pragma unroll
        for (int j = 0; j < (DIM == 2 ? Q1 : 1); ++j) {
            const int p = DIM == 2 ? i * Q1 + j : i;
            const float g = Storage<S>::load(f + elem_index(P, p, x, y));
            Sx[i] = ff_add(Sx[i], g);
            if (DIM == 2) Ty[j] = ff_add(Ty[j], g);
        }
    FF dm{0.0f, 0.0f}, jx = dm, jy = dm, de = dm;
#pragma unroll
    for (int i = 0; i < Q1; ++i) {
        const float vi = (float)P.v[i];
        dm = ff_add(dm, Sx[i]);
        jx = ff_add(jx, ff_scale(Sx[i], vi));
        de = ff_add(de, ff_scale(ff_scale(Sx[i], vi), vi));
        if (DIM == 2) {
            jy = ff_add(jy, ff_scale(Ty[i], vi));
            de = ff_add(de, ff_scale(ff_scale(Ty[i], vi), vi));
        }
    }
    const double r = 1.0 + ff_f64(dm);
    const double ir = 1.0 / r;
    const double a = ff_f64(jx) * ir, b = DIM == 2 ? ff_f64(jy) * ir : 0.0;
    const long long n = (long long)y * P.nx + x;
    if (rho) rho[n] = r;
    if (ux) ux[n] = a;
    if (uy) uy[n] = b;
    if (theta) theta[n] = (((double)DIM * P.theta0 + ff_f64(de)) * ir - (a * a + b * b)) / (double)DIM;
}

template <typename S>
__global__ void k_moments(const __grid_constant__ LatticeParams P, const S* __restrict__ f,
                          double* rho, double* ux, double* uy, double* theta, int y0) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = y0 + blockIdx.y;
    if (x >= P.nx) return;
    double fn[kMaxQ];
    for (int p = 0; p < P.q; ++p) fn[p] = Storage<S>::to_f64(f[elem_index(P, p, x, y)], P.W0[p]);
    double r, a, b, t, e, jx, jy;
    node_moments_f64(P, fn, r, a, b, t, e, jx, jy);
    const long long n = (long long)y * P.nx + x;
    if (rho) rho[n] = r;
    if (ux) ux[n] = a;
    if (uy) uy[n] = b;
    if (theta) theta[n] = t;
}

// Moments of the stored state packed for the surrogate: F[n] = (rho, u_x, u_y,
// theta) in FP32 and the network input x[n] = bf16((F - mean_in) * istd_in).
// FP32 arithmetic on the deviations g = f - w0 (the network's input is bf16 and
// its fields FP32): rho = 1 + sum g, j = sum v g, E = 2 theta0 + sum |v|^2 g
// (the rest sums the 1D rule reproduces), with the row and column sums of g
// factorising the velocity weights.
template <typename S>
__device__ __forceinline__ float dev_f32(const S* f, long long i, double w0) {
    return Storage<S>::load(f + i);
}
template <>
__device__ __forceinline__ float dev_f32<double>(const double* f, long long i, double w0) {
    return (float)(__ldg(f + i) - w0);
}

// refs (batched launch, grid.z = lattice): lattice blockIdx.z reads refs[z].f and
// writes its fields at refs[z].index * nx * ny of the stacks F and x.
template <typename S, int Q1>
__global__ void k_moments_pack(const __grid_constant__ LatticeParams P, const S* __restrict__ f,
                               float4* __restrict__ F, __nv_bfloat16* __restrict__ x, float4 mean_in,
                               float4 istd_in, const LatticeRef* __restrict__ refs) {
    const int xx = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (xx >= P.nx) return;
    if (refs) {
        const LatticeRef r = refs[blockIdx.z];
        f = static_cast<const S*>(r.f);
        const long long off = r.index * P.nx * P.ny;
        F += off;
        x += off * 4;
    }
    constexpr int kQ1 = Q1 ? Q1 : kMaxQ1;
    const int q1 = Q1 ? Q1 : P.q1;
    float sx[kQ1], ty[kQ1];
#pragma unroll
    for (int i = 0; i < kQ1; ++i) sx[i] = ty[i] = 0.0f;
#pragma unroll
    for (int i = 0; i < kQ1; ++i) {
        if (i >= q1) break;
#pragma unroll
        for (int j = 0; j < kQ1; ++j) {
            if (j >= q1) break;
            const int p = i * q1 + j;
            const float g = dev_f32<S>(f, elem_index(P, p, xx, y), P.W0[p]);
            sx[i] += g;
            ty[j] += g;
        }
    }
    // rest sums: sum w0 = 1, sum v w0 = 0, sum |v|^2 w0 = 2 theta0
    float dr = 0.0f, jx = 0.0f, jy = 0.0f, de = 0.0f;
#pragma unroll
    for (int i = 0; i < kQ1; ++i) {
        if (i >= q1) break;
        const float v = (float)P.v[i];
        dr += sx[i];
        jx += v * sx[i];
        jy += v * ty[i];
        de += v * v * (sx[i] + ty[i]);
    }
    const float rho = 1.0f + dr;
    const float ir = 1.0f / rho;
    const float ux = jx * ir, uy = jy * ir;
    const float th = P.theta0f + 0.5f * ((de - 2.0f * P.theta0f * dr) * ir - (ux * ux + uy * uy));
    const long long n = (long long)y * P.nx + xx;
    const float4 v = make_float4(rho, ux, uy, th);
    F[n] = v;
    __nv_bfloat162 lo = __floats2bfloat162_rn((v.x - mean_in.x) * istd_in.x, (v.y - mean_in.y) * istd_in.y);
    __nv_bfloat162 hi = __floats2bfloat162_rn((v.z - mean_in.z) * istd_in.z, (v.w - mean_in.w) * istd_in.w);
    uint2 o;
    o.x = *reinterpret_cast<uint32_t*>(&lo);
    o.y = *reinterpret_cast<uint32_t*>(&hi);
    reinterpret_cast<uint2*>(x)[n] = o;
}

template <typename S>
__global__ void __launch_bounds__(kBlockX) k_reduce_state(const __grid_constant__ LatticeParams P,
                                                          const S* __restrict__ f) {
    const int x = blockIdx.x * kBlockX + threadIdx.x;
    const int y = blockIdx.y;
    NodeDiag d;
    diag_zero(d);
    if (x < P.nx) {
        double fn[kMaxQ];
        for (int p = 0; p < P.q; ++p) fn[p] = Storage<S>::to_f64(f[elem_index(P, p, x, y)], P.W0[p]);
        double r, a, b, t, e, jx, jy;
        node_moments_f64(P, fn, r, a, b, t, e, jx, jy);
        d.mass = r;
        d.jx = jx;
        d.jy = jy;
        d.energy = e;
        d.rho_min = r;
        d.theta_min = t;
        flag_status<double>(P, r, t);
    }
    const int blk = blockIdx.y * gridDim.x + blockIdx.x;
    block_reduce_diag<kBlockX>(d, P.partials + (long long)blk * kPartialStride);
}

// The same record for 16/32-bit storage with compile-time q1, on the FP32 pipe:
// per node the row and column sums of the stored deviations in float-float,
// mass - 1 = sum g, j = sum v g, E - d theta0 = sum |v|^2 g, then the block sums
// in float-float (block_reduce_diagf); the minima from FP32 rho and theta.
template <typename S, int Q1, int DIM>
__global__ void __launch_bounds__(kBlockX) k_reduce_state_dev(const __grid_constant__ LatticeParams P,
                                                              const S* __restrict__ f) {
    const int x = blockIdx.x * kBlockX + threadIdx.x;
    const int y = blockIdx.y;
    NodeDiagF d;
    diagf_zero(d);
    double rmin = 1e300, tmin = 1e300;
    if (x < P.nx) {
        FF Sx[Q1], Ty[Q1];
#pragma unroll
        for (int i = 0; i < Q1; ++i) Sx[i] = Ty[i] = FF{0.0f, 0.0f};
#pragma unroll
        for (int i = 0; i < Q1; ++i)
#pragma unroll
            for (int j = 0; j < (DIM == 2 ? Q1 : 1); ++j) {
                const int p = DIM == 2 ? i * Q1 + j : i;
                const float g = Storage<S>::load(f + elem_index(P, p, x, y));
                Sx[i] = ff_add(Sx[i], g);
                if (DIM == 2) Ty[j] = ff_add(Ty[j], g);
            }
        FF dm{0.0f, 0.0f}, jx = dm, jy = dm, de = dm;
#pragma unroll
        for (int i = 0; i < Q1; ++i) {
            const float vi = (float)P.v[i];
            dm = ff_add(dm, Sx[i]);
            jx = ff_add(jx, ff_scale(Sx[i], vi));
            de = ff_add(de, ff_scale(ff_scale(Sx[i], vi), vi));
            if (DIM == 2) {
                jy = ff_add(jy, ff_scale(Ty[i], vi));
                de = ff_add(de, ff_scale(ff_scale(Ty[i], vi), vi));
            }
        }
        // rho and theta of the node in FP64 (the minima are reported in FP64)
        const double rho = 1.0 + ff_f64(dm);
        const double ir = 1.0 / rho;
        const double ux = ff_f64(jx) * ir, uy = DIM == 2 ? ff_f64(jy) * ir : 0.0;
        const double th = (((double)DIM * P.theta0 + ff_f64(de)) * ir - (ux * ux + uy * uy)) / (double)DIM;
        flag_status<double>(P, rho, th);
        d.dmass = dm;
        d.jx = jx;
        d.jy = jy;
        d.denergy = de;
        d.n = 1.0f;
        rmin = rho;
        tmin = th;
    }
    const int blk = blockIdx.y * gridDim.x + blockIdx.x;
    block_reduce_diagf<kBlockX, true>(d, (double)DIM * P.theta0, P.partials + (long long)blk * kPartialStride, rmin,
                                      tmin);
}

// One block of kFinalThreads threads sums the per-block partials in a fixed
// order, so the result is bit-reproducible for a given lattice.
constexpr int kFinalThreads = 512;
__global__ void __launch_bounds__(kFinalThreads) k_finalize(const double* __restrict__ partials,
                                                            int nblocks, double* __restrict__ out) {
    __shared__ double sh[6][kFinalThreads];
    double r[6] = {0, 0, 0, 0, 1e300, 1e300};
    for (int b = threadIdx.x; b < nblocks; b += kFinalThreads) {
        const double* q = partials + (long long)b * kPartialStride;
        r[0] += q[0];
        r[1] += q[1];
        r[2] += q[2];
        r[3] += q[3];
        r[4] = fmin(r[4], q[4]);
        r[5] = fmin(r[5], q[5]);
    }
    for (int k = 0; k < 6; ++k) sh[k][threadIdx.x] = r[k];
    __syncthreads();
    for (int s = kFinalThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + s];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + s];
            sh[2][threadIdx.x] += sh[2][threadIdx.x + s];
            sh[3][threadIdx.x] += sh[3][threadIdx.x + s];
            sh[4][threadIdx.x] = fmin(sh[4][threadIdx.x], sh[4][threadIdx.x + s]);
            sh[5][threadIdx.x] = fmin(sh[5][threadIdx.x], sh[5][threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x < 6) out[threadIdx.x] = sh[threadIdx.x][0];
}

template <typename S>
__global__ void k_get_pop(const __grid_constant__ LatticeParams P, const S* __restrict__ f,
                          double* __restrict__ out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    const int p = blockIdx.z;
    if (x >= P.nx) return;
    const double v = Storage<S>::to_f64(f[elem_index(P, p, x, y)], P.W0[p]);
    out[((long long)p * P.ny + y) * P.nx + x] = v;
}

template <typename S>
__global__ void k_set_pop(const __grid_constant__ LatticeParams P, const double* __restrict__ in,
                          S* __restrict__ f) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    const int p = blockIdx.z;
    if (x >= P.nx) return;
    f[elem_index(P, p, x, y)] = Storage<S>::from_f64(in[((long long)p * P.ny + y) * P.nx + x], P.W0[p]);
}

#define PLBM_DISPATCH(prec, CALL)                                        \
    switch (prec) {                                                      \
        case kF64: { using S = double; CALL; break; }                    \
        case kF32: { using S = float; CALL; break; }                     \
        case kF16Dev: { using S = __half; CALL; break; }                 \
        case kBF16Dev: { using S = __nv_bfloat16; CALL; break; }         \
        default: return cudaErrorInvalidValue;                           \
    }

// The deviation-storage precisions only.
#define PLBM_DISPATCH_DEV(prec, CALL)                                    \
    switch (prec) {                                                      \
        case kF32: { using S = float; CALL; break; }                     \
        case kF16Dev: { using S = __half; CALL; break; }                 \
        case kBF16Dev: { using S = __nv_bfloat16; CALL; break; }         \
        default: return cudaErrorInvalidValue;                           \
    }

// Initial fields are checked on the device before the state is built from them:
// a non-finite value sets PLBM_STATUS_NONFINITE, rho <= 0 PLBM_STATUS_RHO_NONPOS,
// theta <= 0 PLBM_STATUS_THETA_NONPOS.  One atomic per warp that found any.
__global__ void k_check_fields(FieldSet F, long long n, unsigned* __restrict__ status) {
    unsigned bits = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        for (int k = 0; k < F.count; ++k) {
            const double v = F.field[k][i];
            if (!isfinite(v)) bits |= PLBM_STATUS_NONFINITE;
            else if (k == F.rho && !(v > 0.0)) bits |= PLBM_STATUS_RHO_NONPOS;
            else if (k == F.theta && !(v > 0.0)) bits |= PLBM_STATUS_THETA_NONPOS;
        }
    }
    bits = __reduce_or_sync(0xffffffffu, bits);
    if ((threadIdx.x & 31) == 0 && bits) atomicOr(status, bits);
}

cudaError_t launch_check_fields(const FieldSet& F, long long n, unsigned* status, cudaStream_t stream) {
    if (n <= 0 || F.count <= 0) return cudaSuccess;
    const long long blocks = (n + 255) / 256;
    k_check_fields<<<(int)(blocks < 4096 ? blocks : 4096), 256, 0, stream>>>(F, n, status);
    return cudaGetLastError();
}

cudaError_t launch_init(int prec, const LatticeParams& P, const double* rho, const double* ux,
                        const double* uy, const double* theta, void* f, cudaStream_t stream, int y0, int y1) {
    if (y1 < 0) y1 = P.ny;
    if (y1 <= y0) return cudaSuccess;
    dim3 grid((P.nx + 127) / 128, y1 - y0);
#define PLBM_INIT_DEV(DIMv)                                                                            \
    if (P.dim == DIMv) {                                                                               \
        PLBM_DISPATCH_DEV(prec, (k_init_sym5_dev<S, DIMv><<<grid, 128, 0, stream>>>(P, rho, ux, uy, theta, \
                                                                                 static_cast<S*>(f), y0))); \
        return cudaGetLastError();                                                                     \
    }
    if (prec != kF64 && P.sym5) {
        PLBM_INIT_DEV(2)
        PLBM_INIT_DEV(1)
    }
#undef PLBM_INIT_DEV
#define PLBM_INIT_Q(Q1v, DIMv)                                                                          \
    if (P.q1 == Q1v && P.dim == DIMv) {                                                                 \
        PLBM_DISPATCH(prec, (k_init_q<S, Q1v, DIMv><<<grid, 128, 0, stream>>>(P, rho, ux, uy, theta,     \
                                                                              static_cast<S*>(f), y0)));  \
        return cudaGetLastError();                                                                      \
    }
    PLBM_INIT_Q(3, 2)
    PLBM_INIT_Q(4, 2)
    PLBM_INIT_Q(5, 2)
    PLBM_INIT_Q(5, 1)
#undef PLBM_INIT_Q
    PLBM_DISPATCH(prec, (k_init<S><<<grid, 128, 0, stream>>>(P, rho, ux, uy, theta,
                                                             static_cast<S*>(f), y0)));
    return cudaGetLastError();
}

cudaError_t launch_moments(int prec, const LatticeParams& P, const void* f, double* rho,
                           double* ux, double* uy, double* theta, cudaStream_t stream, int y0, int y1) {
    if (y1 < 0) y1 = P.ny;
    if (y1 <= y0) return cudaSuccess;
    dim3 grid((P.nx + 127) / 128, y1 - y0);
#define PLBM_MOM_Q(Q1v, DIMv)                                                                           \
    if (P.q1 == Q1v && P.dim == DIMv) {                                                                 \
        if (prec == kF64)                                                                               \
            k_moments_q<double, Q1v, DIMv><<<grid, 128, 0, stream>>>(                                   \
                P, static_cast<const double*>(f), rho, ux, uy, theta, y0);                                  \
        else                                                                                            \
            PLBM_DISPATCH_DEV(prec, (k_moments_dev<S, Q1v, DIMv><<<grid, 128, 0, stream>>>(             \
                                    P, static_cast<const S*>(f), rho, ux, uy, theta, y0)));                 \
        return cudaGetLastError();                                                                      \
    }
    PLBM_MOM_Q(3, 2)
    PLBM_MOM_Q(4, 2)
    PLBM_MOM_Q(5, 2)
    PLBM_MOM_Q(5, 1)
#undef PLBM_MOM_Q
    PLBM_DISPATCH(prec, (k_moments<S><<<grid, 128, 0, stream>>>(P, static_cast<const S*>(f), rho,
                                                                ux, uy, theta, y0)));
    return cudaGetLastError();
}

cudaError_t launch_moments_pack(int prec, const LatticeParams& P, const void* f, float* F, void* x,
                                const float* mean_in, const float* std_in, cudaStream_t stream) {
    if (P.dim != 2) return cudaErrorInvalidValue;
    const float4 mi = make_float4(mean_in[0], mean_in[1], mean_in[2], mean_in[3]);
    const float4 si = make_float4(1.f / std_in[0], 1.f / std_in[1], 1.f / std_in[2], 1.f / std_in[3]);
    dim3 grid((P.nx + 127) / 128, P.ny);
    const LatticeRef* none = nullptr;
    if (P.q1 == 5) {
        PLBM_DISPATCH(prec, (k_moments_pack<S, 5><<<grid, 128, 0, stream>>>(
                                P, static_cast<const S*>(f), reinterpret_cast<float4*>(F),
                                static_cast<__nv_bfloat16*>(x), mi, si, none)));
    } else {
        PLBM_DISPATCH(prec, (k_moments_pack<S, 0><<<grid, 128, 0, stream>>>(
                                P, static_cast<const S*>(f), reinterpret_cast<float4*>(F),
                                static_cast<__nv_bfloat16*>(x), mi, si, none)));
    }
    return cudaGetLastError();
}

cudaError_t launch_moments_pack_batch(int prec, const LatticeParams& P, const LatticeRef* refs, int n, float* F,
                                      void* x, const float* mean_in, const float* std_in, cudaStream_t stream) {
    if (P.dim != 2 || n < 1 || n > 65535) return cudaErrorInvalidValue;
    const float4 mi = make_float4(mean_in[0], mean_in[1], mean_in[2], mean_in[3]);
    const float4 si = make_float4(1.f / std_in[0], 1.f / std_in[1], 1.f / std_in[2], 1.f / std_in[3]);
    dim3 grid((P.nx + 127) / 128, P.ny, n);
    if (P.q1 == 5) {
        PLBM_DISPATCH(prec, (k_moments_pack<S, 5><<<grid, 128, 0, stream>>>(
                                P, nullptr, reinterpret_cast<float4*>(F), static_cast<__nv_bfloat16*>(x), mi, si,
                                refs)));
    } else {
        PLBM_DISPATCH(prec, (k_moments_pack<S, 0><<<grid, 128, 0, stream>>>(
                                P, nullptr, reinterpret_cast<float4*>(F), static_cast<__nv_bfloat16*>(x), mi, si,
                                refs)));
    }
    return cudaGetLastError();
}

cudaError_t launch_finalize(const LatticeParams& P, int nblocks, double* out, cudaStream_t stream) {
    k_finalize<<<1, kFinalThreads, 0, stream>>>(P.partials, nblocks, out);
    return cudaGetLastError();
}

cudaError_t launch_reduce_state(int prec, const LatticeParams& P, const void* f, double* out,
                                cudaStream_t stream) {
    dim3 grid((P.nx + kBlockX - 1) / kBlockX, P.ny);
    bool done = false;
#define PLBM_RED_Q(Q1v, DIMv)                                                                           \
    if (!done && prec != kF64 && P.q1 == Q1v && P.dim == DIMv) {                                        \
        PLBM_DISPATCH_DEV(prec, (k_reduce_state_dev<S, Q1v, DIMv><<<grid, kBlockX, 0, stream>>>(         \
                                    P, static_cast<const S*>(f))));                                     \
        done = true;                                                                                    \
    }
    PLBM_RED_Q(3, 2)
    PLBM_RED_Q(4, 2)
    PLBM_RED_Q(5, 2)
    PLBM_RED_Q(5, 1)
#undef PLBM_RED_Q
    if (!done)
        PLBM_DISPATCH(prec, (k_reduce_state<S><<<grid, kBlockX, 0, stream>>>(P, static_cast<const S*>(f))));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_finalize(P, reduce_blocks(P), out, stream);
}

cudaError_t launch_get_populations(int prec, const LatticeParams& P, const void* f, double* out,
                                   cudaStream_t stream) {
    dim3 grid((P.nx + 127) / 128, P.ny, P.q);
    PLBM_DISPATCH(prec, (k_get_pop<S><<<grid, 128, 0, stream>>>(P, static_cast<const S*>(f), out)));
    return cudaGetLastError();
}

cudaError_t launch_set_populations(int prec, const LatticeParams& P, const double* in, void* f,
                                   cudaStream_t stream) {
    dim3 grid((P.nx + 127) / 128, P.ny, P.q);
    PLBM_DISPATCH(prec, (k_set_pop<S><<<grid, 128, 0, stream>>>(P, in, static_cast<S*>(f))));
    return cudaGetLastError();
}

}  // namespace plbm
