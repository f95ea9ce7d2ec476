// Three-dimensional lattices (Sec. 2.1: D3 models are the tensor product of
// three 1D rules with one scalar theta), periodic in x, y and z.
//
// Population p = (a * q1 + b) * q1 + c has velocity (v[a], v[b], v[c]); storage
// [q][nz][ny][pitch] (row index z * ny + y of elem_index).  The rest equilibrium
// is the product w0_p = w_a w_b w_c of the 1D rest weights.
//
// k_stream_collide3<S> (FP32 arithmetic; FP32, FP16 or BF16 storage of the
// deviation g = f - w0; symmetric five-velocity sets (0, +-a, +-b), D3Q125):
//   * pull of the 125 populations (Eq. eq:srt read as pull + collide), one node
//     per thread, coalesced along x;
//   * moments from the row sums S_a = sum_{b,c} g, T_b, U_c of the deviations,
//     with the rest sums sum w0 = 1, sum v w0 = 0, sum |v|^2 w0 = 3 theta0 (the
//     1D rule reproduces mu_0, mu_1, mu_2): rho - 1 = sum S, j = sum v S (per
//     axis), E - 3 theta0 = sum v^2 (S + T + U), and
//     theta - theta0 = ((E - 3 theta0 rho) / rho - |u|^2) / 3 from these small
//     quantities (no cancellation against the rest values);
//   * per axis the rule of Eq. eq:rdr in constraint form: with
//     dmu_n = mu_n(u, theta) - mu_n(0, theta0), n = 1..4,
//     O_b = (dmu3 - a^2 dmu1) / (2 b (b^2 - a^2)), O_a = (dmu1 - 2 b O_b) / (2 a),
//     E_b = (dmu4 - a^2 dmu2) / (2 b^2 (b^2 - a^2)), E_a = (dmu2 - 2 b^2 E_b) / (2 a^2),
//     r_{+-a} = w_a + E_a +- O_a, r_{+-b} = w_b + E_b +- O_b, r_0 = w_0 - 2 (E_a + E_b),
//     so the moments the rule must reproduce hold to the rounding of these few
//     operations (FP32-rounded Lagrange coefficients would break them);
//   * f^eq - w0 = rho r^x r^y r^z - w^x w^y w^z
//               = d_a (r^y_b r^z_c) + w_a (dr^y_b r^z_c + w_b dr^z_c),  d_a = rho r^x_a - w_a;
//   * BGK: g' = g + omega (f^eq - w0 - g).
// k_stream_collide3_f64: FP64 storage of f, any q1 <= 5, thermal or isothermal,
// the plain formulas (an ALU-bound path).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "plbm_device.cuh"

namespace plbm {

namespace {

constexpr int kB3 = 128;       // threads per block along x
constexpr int kQ1 = 5;         // D3Q125
constexpr int kQ3 = kQ1 * kQ1 * kQ1;

__device__ __forceinline__ int wrap_add(int i, int d, int n) {
    const int s = i + d;
    return s >= n ? s - n : s;
}

// Per-axis rule deviations dr_i = r_i(u, theta) - w_i for (0, a, -a, b, -b),
// given dth = theta - theta0.
__device__ __forceinline__ void axis_dev(const LatticeParams& P, float u, float dth, float (&dr)[kQ1]) {
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

template <typename S>
__global__ void __launch_bounds__(kB3, 2) k_stream_collide3(const __grid_constant__ LatticeParams P,
                                                           const S* __restrict__ src, S* __restrict__ dst) {
    const int x = blockIdx.x * kB3 + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= P.nx) return;
    int xs[kQ1], ys[kQ1], zs[kQ1];
#pragma unroll
    for (int i = 0; i < kQ1; ++i) {
        xs[i] = wrap_add(x, P.vxm[i], P.nx);
        ys[i] = wrap_add(y, P.vym[i], P.ny);
        zs[i] = wrap_add(z, P.vzm[i], P.nz);
    }
    float g[kQ3];
    float Sa[kQ1], Tb[kQ1], Uc[kQ1];
#pragma unroll
    for (int i = 0; i < kQ1; ++i) Sa[i] = Tb[i] = Uc[i] = 0.0f;
#pragma unroll
    for (int b = 0; b < kQ1; ++b)
#pragma unroll
        for (int c = 0; c < kQ1; ++c) {
            const long long row = ((long long)zs[c] * P.ny + ys[b]) * P.pitch;
#pragma unroll
            for (int a = 0; a < kQ1; ++a) {
                const int p = (a * kQ1 + b) * kQ1 + c;
                g[p] = Storage<S>::load(src + (long long)p * P.plane + row + xs[a]);
            }
        }
#pragma unroll
    for (int a = 0; a < kQ1; ++a)
#pragma unroll
        for (int b = 0; b < kQ1; ++b)
#pragma unroll
            for (int c = 0; c < kQ1; ++c) {
                const float v = g[(a * kQ1 + b) * kQ1 + c];
                Sa[a] += v;
                Tb[b] += v;
                Uc[c] += v;
            }
    float drho = 0.0f, jx = 0.0f, jy = 0.0f, jz = 0.0f, de = 0.0f;
#pragma unroll
    for (int i = 0; i < kQ1; ++i) {
        const float vi = (float)P.v[i];
        drho += Sa[i];
        jx += vi * Sa[i];
        jy += vi * Tb[i];
        jz += vi * Uc[i];
        de += vi * vi * (Sa[i] + Tb[i] + Uc[i]);
    }
    const float rho = 1.0f + drho;
    const float ir = 1.0f / rho;
    const float ux = jx * ir, uy = jy * ir, uz = jz * ir;
    const float dth = ((de - 3.0f * P.theta0f * drho) * ir - (ux * ux + uy * uy + uz * uz)) * (1.0f / 3.0f);
    flag_status<float>(P, rho, P.theta0f + dth);
    float drx[kQ1], dry[kQ1], drz[kQ1];
    axis_dev(P, ux, dth, drx);
    axis_dev(P, uy, dth, dry);
    axis_dev(P, uz, dth, drz);
    float da[kQ1];  // rho r^x_a - w_a = (rho - 1) w_a + rho dr^x_a
#pragma unroll
    for (int a = 0; a < kQ1; ++a) da[a] = fmaf(drho, P.w1f[a], rho * drx[a]);
    const float om = P.omegaf;
    const long long here = ((long long)z * P.ny + y) * P.pitch + x;
#pragma unroll
    for (int b = 0; b < kQ1; ++b)
#pragma unroll
        for (int c = 0; c < kQ1; ++c) {
            const float rzc = P.w1f[c] + drz[c];
            const float Pbc = (P.w1f[b] + dry[b]) * rzc;
            const float Qbc = dry[b] * rzc + P.w1f[b] * drz[c];
#pragma unroll
            for (int a = 0; a < kQ1; ++a) {
                const int p = (a * kQ1 + b) * kQ1 + c;
                const float d = fmaf(da[a], Pbc, P.w1f[a] * Qbc);
                Storage<S>::store(dst + (long long)p * P.plane + here, fmaf(om, d - g[p], g[p]));
            }
        }
}

// FP64: any q1 <= 5; fin[p] pulled, moments, f^eq from C and the Gaussian moments.
__device__ void rule_f64(const LatticeParams& P, double u, double th, double* r) {
    double mu[kMaxQ1];
    const int q1 = P.q1;
    mu[0] = 1.0;
    mu[1] = u;
    for (int n = 1; n + 1 < q1; ++n) mu[n + 1] = u * mu[n] + (double)n * th * mu[n - 1];
    for (int i = 0; i < q1; ++i) {
        double s = 0.0;
        for (int n = 0; n < q1; ++n) s += P.C[i * q1 + n] * mu[n];
        r[i] = s;
    }
}

__device__ void moments3_f64(const LatticeParams& P, const double* f, double* m) {
    const int q1 = P.q1;
    double m0 = 0.0, mx = 0.0, my = 0.0, mz = 0.0, en = 0.0;
    for (int a = 0; a < q1; ++a)
        for (int b = 0; b < q1; ++b)
            for (int c = 0; c < q1; ++c) {
                const double fv = f[(a * q1 + b) * q1 + c];
                const double cx = P.v[a], cy = P.v[b], cz = P.v[c];
                m0 += fv;
                mx += cx * fv;
                my += cy * fv;
                mz += cz * fv;
                en += (cx * cx + cy * cy + cz * cz) * fv;
            }
    m[0] = m0;
    m[1] = mx / m0;
    m[2] = my / m0;
    m[3] = mz / m0;
    m[4] = (en / m0 - (m[1] * m[1] + m[2] * m[2] + m[3] * m[3])) / 3.0;
    m[5] = mx;
    m[6] = my;
    m[7] = mz;
    m[8] = en;
}

__device__ void feq3_f64(const LatticeParams& P, double rho, double ux, double uy, double uz, double th,
                         double* out) {
    double ra[kMaxQ1], rb[kMaxQ1], rc[kMaxQ1];
    rule_f64(P, ux, th, ra);
    rule_f64(P, uy, th, rb);
    rule_f64(P, uz, th, rc);
    const int q1 = P.q1;
    for (int a = 0; a < q1; ++a)
        for (int b = 0; b < q1; ++b)
            for (int c = 0; c < q1; ++c) out[(a * q1 + b) * q1 + c] = rho * ra[a] * rb[b] * rc[c];
}

__device__ __forceinline__ double w0_3(const LatticeParams& P, int p) {
    const int q1 = P.q1;
    const int a = p / (q1 * q1), b = (p / q1) % q1, c = p % q1;
    return P.w1[a] * P.w1[b] * P.w1[c];
}

__global__ void __launch_bounds__(kB3) k_stream_collide3_f64(const __grid_constant__ LatticeParams P,
                                                             const double* __restrict__ src,
                                                             double* __restrict__ dst) {
    const int x = blockIdx.x * kB3 + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= P.nx) return;
    const int q1 = P.q1;
    double fin[kQ3], fe[kQ3], m[9];
    for (int a = 0; a < q1; ++a)
        for (int b = 0; b < q1; ++b)
            for (int c = 0; c < q1; ++c) {
                const int p = (a * q1 + b) * q1 + c;
                const long long row = ((long long)wrap_add(z, P.vzm[c], P.nz) * P.ny + wrap_add(y, P.vym[b], P.ny)) *
                                      P.pitch;
                fin[p] = src[(long long)p * P.plane + row + wrap_add(x, P.vxm[a], P.nx)];
            }
    moments3_f64(P, fin, m);
    flag_status<double>(P, m[0], m[4]);
    feq3_f64(P, m[0], m[1], m[2], m[3], P.isothermal ? P.theta0 : m[4], fe);
    const long long here = ((long long)z * P.ny + y) * P.pitch + x;
    const double om = P.omega;
    for (int p = 0; p < q1 * q1 * q1; ++p) dst[(long long)p * P.plane + here] = (1.0 - om) * fin[p] + om * fe[p];
}

template <typename S>
__global__ void k_init3(const __grid_constant__ LatticeParams P, const double* __restrict__ rho,
                        const double* __restrict__ ux, const double* __restrict__ uy, const double* __restrict__ uz,
                        const double* __restrict__ theta, S* __restrict__ f) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= P.nx) return;
    const long long n = ((long long)z * P.ny + y) * P.nx + x;
    const double th = (P.isothermal || theta == nullptr) ? P.theta0 : theta[n];
    double fe[kQ3];
    feq3_f64(P, rho[n], ux ? ux[n] : 0.0, uy ? uy[n] : 0.0, uz ? uz[n] : 0.0, th, fe);
    const long long here = ((long long)z * P.ny + y) * P.pitch + x;
    for (int p = 0; p < P.q; ++p) f[(long long)p * P.plane + here] = Storage<S>::from_f64(fe[p], w0_3(P, p));
}

template <typename S>
__global__ void k_moments3(const __grid_constant__ LatticeParams P, const S* __restrict__ f, double* rho,
                           double* ux, double* uy, double* uz, double* theta) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= P.nx) return;
    const long long here = ((long long)z * P.ny + y) * P.pitch + x;
    double fn[kQ3], m[9];
    for (int p = 0; p < P.q; ++p) fn[p] = Storage<S>::to_f64(f[(long long)p * P.plane + here], w0_3(P, p));
    moments3_f64(P, fn, m);
    const long long n = ((long long)z * P.ny + y) * P.nx + x;
    if (rho) rho[n] = m[0];
    if (ux) ux[n] = m[1];
    if (uy) uy[n] = m[2];
    if (uz) uz[n] = m[3];
    if (theta) theta[n] = m[4];
}

// Per-block FP64 record: mass, j_x, j_y, energy, min rho, min theta, j_z.
template <typename S>
__global__ void __launch_bounds__(kB3) k_reduce3(const __grid_constant__ LatticeParams P, const S* __restrict__ f) {
    __shared__ double sh[7][kB3];
    const int x = blockIdx.x * kB3 + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    double r[7] = {0, 0, 0, 0, 1e300, 1e300, 0};
    if (x < P.nx) {
        const long long here = ((long long)z * P.ny + y) * P.pitch + x;
        double fn[kQ3], m[9];
        for (int p = 0; p < P.q; ++p) fn[p] = Storage<S>::to_f64(f[(long long)p * P.plane + here], w0_3(P, p));
        moments3_f64(P, fn, m);
        r[0] = m[0];
        r[1] = m[5];
        r[2] = m[6];
        r[3] = m[8];
        r[4] = m[0];
        r[5] = m[4];
        r[6] = m[7];
        flag_status<double>(P, m[0], m[4]);
    }
    for (int k = 0; k < 7; ++k) sh[k][threadIdx.x] = r[k];
    __syncthreads();
    for (int s = kB3 / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            for (int k = 0; k < 7; ++k) {
                const double o = sh[k][threadIdx.x + s];
                sh[k][threadIdx.x] = (k == 4 || k == 5) ? fmin(sh[k][threadIdx.x], o) : sh[k][threadIdx.x] + o;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x < 7) {
        const long long blk = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        P.partials[blk * kPartialStride + threadIdx.x] = sh[threadIdx.x][0];
    }
}

__global__ void k_finalize3(const double* __restrict__ partials, long long nblocks, double* __restrict__ out) {
    __shared__ double sh[7][256];
    double r[7] = {0, 0, 0, 0, 1e300, 1e300, 0};
    for (long long b = threadIdx.x; b < nblocks; b += 256) {
        const double* q = partials + b * kPartialStride;
        for (int k = 0; k < 7; ++k) r[k] = (k == 4 || k == 5) ? fmin(r[k], q[k]) : r[k] + q[k];
    }
    for (int k = 0; k < 7; ++k) sh[k][threadIdx.x] = r[k];
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int k = 0; k < 7; ++k) {
                const double o = sh[k][threadIdx.x + s];
                sh[k][threadIdx.x] = (k == 4 || k == 5) ? fmin(sh[k][threadIdx.x], o) : sh[k][threadIdx.x] + o;
            }
        __syncthreads();
    }
    if (threadIdx.x < 7) out[threadIdx.x] = sh[threadIdx.x][0];
}

template <typename S>
__global__ void k_get_pop3(const __grid_constant__ LatticeParams P, const S* __restrict__ f, double* __restrict__ out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= P.nx) return;
    const long long here = ((long long)z * P.ny + y) * P.pitch + x;
    const long long vol = (long long)P.nx * P.ny * P.nz;
    const long long n = ((long long)z * P.ny + y) * P.nx + x;
    for (int p = 0; p < P.q; ++p) out[p * vol + n] = Storage<S>::to_f64(f[(long long)p * P.plane + here], w0_3(P, p));
}

template <typename S>
__global__ void k_set_pop3(const __grid_constant__ LatticeParams P, const double* __restrict__ in, S* __restrict__ f) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= P.nx) return;
    const long long here = ((long long)z * P.ny + y) * P.pitch + x;
    const long long vol = (long long)P.nx * P.ny * P.nz;
    const long long n = ((long long)z * P.ny + y) * P.nx + x;
    for (int p = 0; p < P.q; ++p) f[(long long)p * P.plane + here] = Storage<S>::from_f64(in[p * vol + n], w0_3(P, p));
}

dim3 grid3(const LatticeParams& P) { return dim3((P.nx + kB3 - 1) / kB3, P.ny, P.nz); }

#define PLBM_DISPATCH3(prec, CALL)                                       \
    switch (prec) {                                                      \
        case kF64: { using S = double; CALL; break; }                    \
        case kF32: { using S = float; CALL; break; }                     \
        case kF16Dev: { using S = __half; CALL; break; }                 \
        case kBF16Dev: { using S = __nv_bfloat16; CALL; break; }         \
        default: return cudaErrorInvalidValue;                           \
    }

}  // namespace

long long reduce3_blocks(const LatticeParams& P) {
    return (long long)((P.nx + kB3 - 1) / kB3) * P.ny * P.nz;
}

cudaError_t launch_step3(int prec, const LatticeParams& P, const void* src, void* dst, cudaStream_t s) {
    if (prec == kF64) {
        k_stream_collide3_f64<<<grid3(P), kB3, 0, s>>>(P, static_cast<const double*>(src), static_cast<double*>(dst));
        return cudaGetLastError();
    }
    if (!P.sym5 || P.q1 != kQ1 || P.isothermal) return cudaErrorInvalidValue;
    switch (prec) {
        case kF32:
            k_stream_collide3<float><<<grid3(P), kB3, 0, s>>>(P, static_cast<const float*>(src), static_cast<float*>(dst));
            break;
        case kF16Dev:
            k_stream_collide3<__half><<<grid3(P), kB3, 0, s>>>(P, static_cast<const __half*>(src), static_cast<__half*>(dst));
            break;
        case kBF16Dev:
            k_stream_collide3<__nv_bfloat16><<<grid3(P), kB3, 0, s>>>(P, static_cast<const __nv_bfloat16*>(src),
                                                                     static_cast<__nv_bfloat16*>(dst));
            break;
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_init3(int prec, const LatticeParams& P, const double* rho, const double* ux, const double* uy,
                         const double* uz, const double* theta, void* f, cudaStream_t s) {
    PLBM_DISPATCH3(prec, (k_init3<S><<<grid3(P), kB3, 0, s>>>(P, rho, ux, uy, uz, theta, static_cast<S*>(f))));
    return cudaGetLastError();
}

cudaError_t launch_moments3(int prec, const LatticeParams& P, const void* f, double* rho, double* ux, double* uy,
                            double* uz, double* theta, cudaStream_t s) {
    PLBM_DISPATCH3(prec, (k_moments3<S><<<grid3(P), kB3, 0, s>>>(P, static_cast<const S*>(f), rho, ux, uy, uz, theta)));
    return cudaGetLastError();
}

cudaError_t launch_reduce3(int prec, const LatticeParams& P, const void* f, double* out, cudaStream_t s) {
    PLBM_DISPATCH3(prec, (k_reduce3<S><<<grid3(P), kB3, 0, s>>>(P, static_cast<const S*>(f))));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_finalize3<<<1, 256, 0, s>>>(P.partials, reduce3_blocks(P), out);
    return cudaGetLastError();
}

cudaError_t launch_get_pop3(int prec, const LatticeParams& P, const void* f, double* out, cudaStream_t s) {
    PLBM_DISPATCH3(prec, (k_get_pop3<S><<<grid3(P), kB3, 0, s>>>(P, static_cast<const S*>(f), out)));
    return cudaGetLastError();
}

cudaError_t launch_set_pop3(int prec, const LatticeParams& P, const double* in, void* f, cudaStream_t s) {
    PLBM_DISPATCH3(prec, (k_set_pop3<S><<<grid3(P), kB3, 0, s>>>(P, in, static_cast<S*>(f))));
    return cudaGetLastError();
}

}  // namespace plbm
