// Field-level kernels of the surrogate path: packing moments into FP32 NHWC
// fields, building normalised training pairs, applying a predicted change,
// FP64 conserved sums of field arrays, and the Chapman-Enskog reconstruction
// of populations from fields.
//
// Reconstruction.  For the stored (post-collision) state the first-order
// Chapman-Enskog population is
//     f_p = f^eq_p - ((1 - omega) / omega) D_p f^eq_p,   D_p = d_t + v_p . grad,
// (pre-collision non-equilibrium -(1/omega) D_p f^eq_p, relaxed once by the
// BGK step of Eq. eq:srt).  f^eq_p = rho r^x_i r^y_j (Eq. eq:rdr, Sec. 2.1), so
//     D_p f^eq_p = r^x r^y D rho + rho r^x' r^y D u_x + rho r^x r^y' D u_y
//                  + rho (r^x_th r^y + r^x r^y_th) D theta,
// with r' = C dmu/du, dmu_n/du = n mu_{n-1}, and r_th = C dmu/dtheta,
// dmu_n/dtheta = n (n - 1) mu_{n-2} / 2 (Gaussian moments).  Time derivatives
// come from the Euler equations of the ideal gas p = rho theta in d = 2
// (d_t rho = -div(rho u), d_t u = -u.grad u - grad p / rho,
// d_t theta = -u.grad theta - (2/d) theta div u); spatial derivatives are
// second-order central differences on the periodic grid.  Finally the
// non-equilibrium part is projected off span{w0, w0 v_x, w0 v_y, w0 |v|^2} so
// that mass, momentum and energy of the populations equal the fields exactly
// (to rounding).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "plbm_device.cuh"
#include "plbm_internal.h"

namespace plbm {

// fields_out[n][4] = (rho, ux, uy, theta) as FP32 from FP64 planes [n].
__global__ void k_pack_fields(const double* __restrict__ rho, const double* __restrict__ ux,
                              const double* __restrict__ uy, const double* __restrict__ th, long long n,
                              float4* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = make_float4((float)rho[i], (float)ux[i], (float)uy[i], (float)th[i]);
}

// SplitMix64 (Steele, Lea and Flood, 2014): the output function applied to z.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// Standard normal number of counter `ctr` under `seed`: the two halves of one
// 48-bit draw as uniforms u1 in (0, 1], u2 in [0, 1), then Box and Muller (1958):
// sqrt(-2 ln u1) cos(2 pi u2).
__device__ __forceinline__ float gauss_of(unsigned long long seed, unsigned long long ctr) {
    const unsigned long long h = splitmix64(seed ^ splitmix64(ctr));
    const float u1 = ((float)(h >> 40) + 1.0f) * (1.0f / 16777216.0f);
    const float u2 = (float)((h >> 16) & 0xffffffull) * (1.0f / 16777216.0f);
    return sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
}

// Training pair b: x[b] = (F[s0] - mean_in) / std_in + sigma n (bf16), y[b] = (F[s1] - F[s0] - mean_d) / std_d
// (fp32), F a stack of snapshots of `npix` nodes x 4 fields, pairs[b] = (s0, s1); n a standard normal number
// per input element (counter 4 i + field under `seed`), none when sigma = 0.
__global__ void k_assemble(const float4* __restrict__ snaps, long long npix, const int* __restrict__ pairs,
                           int B, float4 mean_in, float4 istd_in, float4 mean_d, float4 istd_d,
                           __nv_bfloat16* __restrict__ x, float4* __restrict__ y, float sigma,
                           unsigned long long seed) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npix * B) return;
    const int b = (int)(i / npix);
    const long long k = i - (long long)b * npix;
    const float4 a = snaps[(long long)pairs[2 * b] * npix + k];
    const float4 c = snaps[(long long)pairs[2 * b + 1] * npix + k];
    float4 n = make_float4(0.f, 0.f, 0.f, 0.f);
    if (sigma > 0.0f) {
        const unsigned long long c0 = 4ull * (unsigned long long)i;
        n = make_float4(sigma * gauss_of(seed, c0), sigma * gauss_of(seed, c0 + 1), sigma * gauss_of(seed, c0 + 2),
                        sigma * gauss_of(seed, c0 + 3));
    }
    __nv_bfloat16* xo = x + i * 4;
    xo[0] = __float2bfloat16_rn((a.x - mean_in.x) * istd_in.x + n.x);
    xo[1] = __float2bfloat16_rn((a.y - mean_in.y) * istd_in.y + n.y);
    xo[2] = __float2bfloat16_rn((a.z - mean_in.z) * istd_in.z + n.z);
    xo[3] = __float2bfloat16_rn((a.w - mean_in.w) * istd_in.w + n.w);
    y[i] = make_float4((c.x - a.x - mean_d.x) * istd_d.x, (c.y - a.y - mean_d.y) * istd_d.y,
                       (c.z - a.z - mean_d.z) * istd_d.z, (c.w - a.w - mean_d.w) * istd_d.w);
}

// Network input from current fields: x = (F - mean_in) / std_in (bf16).
__global__ void k_normalise(const float4* __restrict__ F, long long n, float4 mean_in, float4 istd_in,
                            __nv_bfloat16* __restrict__ x) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 a = F[i];
    __nv_bfloat16* xo = x + i * 4;
    xo[0] = __float2bfloat16_rn((a.x - mean_in.x) * istd_in.x);
    xo[1] = __float2bfloat16_rn((a.y - mean_in.y) * istd_in.y);
    xo[2] = __float2bfloat16_rn((a.z - mean_in.z) * istd_in.z);
    xo[3] = __float2bfloat16_rn((a.w - mean_in.w) * istd_in.w);
}

// F_new = F + delta * std_d + mean_d.
__global__ void k_apply_delta(const float4* __restrict__ F, const float4* __restrict__ d, long long n, float4 mean_d,
                              float4 std_d, float4* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 a = F[i], e = d[i];
    out[i] = make_float4(a.x + fmaf(e.x, std_d.x, mean_d.x), a.y + fmaf(e.y, std_d.y, mean_d.y),
                         a.z + fmaf(e.z, std_d.z, mean_d.z), a.w + fmaf(e.w, std_d.w, mean_d.w));
}

// Per-block FP64 sums over the fields of one lattice: mass, rho u_x, rho u_y,
// energy d rho theta + rho |u|^2 (d = 2); out[blk * 4 + k].
__global__ void k_field_sums(const float4* __restrict__ F, long long n, double* __restrict__ out) {
    __shared__ double sh[4][256];
    double s[4] = {0, 0, 0, 0};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float4 a = F[i];
        const double r = a.x, u = a.y, v = a.z, t = a.w;
        s[0] += r;
        s[1] += r * u;
        s[2] += r * v;
        s[3] += r * (2.0 * t + u * u + v * v);
    }
    for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] = s[k];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 4) out[blockIdx.x * 4 + threadIdx.x] = sh[threadIdx.x][0];
}

// The same for `nlat` lattices of n nodes each stored one after another:
// out[(lat * gridDim.x + blk) * 4 + k].  Each thread adds its nodes in FP32
// (a few per thread), then FP64 warp and block sums in a fixed order.
__global__ void __launch_bounds__(256) k_field_sums_batch(const float4* __restrict__ F, long long n,
                                                          double* __restrict__ out) {
    __shared__ double sh[8][4];
    const float4* Fl = F + (long long)blockIdx.y * n;
    float s[4] = {0.f, 0.f, 0.f, 0.f};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float4 a = Fl[i];
        s[0] += a.x;
        s[1] += a.x * a.y;
        s[2] += a.x * a.z;
        s[3] += a.x * (2.0f * a.w + a.y * a.y + a.z * a.z);
    }
    double d[4] = {s[0], s[1], s[2], s[3]};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < 4; ++k) d[k] += __shfl_xor_sync(0xffffffffu, d[k], o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int k = 0; k < 4; ++k) sh[warp][k] = d[k];
    __syncthreads();
    if (threadIdx.x < 4) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += sh[w][threadIdx.x];
        out[((long long)blockIdx.y * gridDim.x + blockIdx.x) * 4 + threadIdx.x] = t;
    }
}

// Relative drift of lattice b between the old and the predicted fields (FP64,
// partial sums added in a fixed order): max(|dM| / M, |dE| / E, |dJ| / (0.1 M)).
// One warp per lattice.
__global__ void k_field_drift(const double* __restrict__ so, const double* __restrict__ sn, int nblk, int nlat,
                              double* __restrict__ drift) {
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= nlat) return;
    double a[4] = {0, 0, 0, 0}, c[4] = {0, 0, 0, 0};
    for (int k = lane; k < nblk; k += 32)
        for (int j = 0; j < 4; ++j) {
            a[j] += so[((long long)b * nblk + k) * 4 + j];
            c[j] += sn[((long long)b * nblk + k) * 4 + j];
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            a[j] += __shfl_xor_sync(0xffffffffu, a[j], o);
            c[j] += __shfl_xor_sync(0xffffffffu, c[j], o);
        }
    if (lane == 0) {
        const double dm = fabs(c[0] - a[0]) / fabs(a[0]);
        const double de = fabs(c[3] - a[3]) / fabs(a[3]);
        const double dj = hypot(c[1] - a[1], c[2] - a[2]) / (0.1 * fabs(a[0]));
        drift[b] = fmax(dm, fmax(de, dj));
    }
}

// Conservative projection of predicted fields (option of the surrogate
// advance): per lattice, the uniform shifts of the conserved densities
// (rho, rho u_x, rho u_y, E = rho (2 theta + |u|^2)) that restore the old
// fields' totals, delta_k = (old_k - new_k) / n, from the per-block partial
// sums of k_field_sums_batch.  One warp per lattice.
__global__ void k_conserve_coef(const double* __restrict__ so, const double* __restrict__ sn, int nblk, int nlat,
                                long long n, float4* __restrict__ delta) {
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= nlat) return;
    double a[4] = {0, 0, 0, 0}, c[4] = {0, 0, 0, 0};
    for (int k = lane; k < nblk; k += 32)
        for (int j = 0; j < 4; ++j) {
            a[j] += so[((long long)b * nblk + k) * 4 + j];
            c[j] += sn[((long long)b * nblk + k) * 4 + j];
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            a[j] += __shfl_xor_sync(0xffffffffu, a[j], o);
            c[j] += __shfl_xor_sync(0xffffffffu, c[j], o);
        }
    if (lane == 0)
        delta[b] = make_float4((float)((a[0] - c[0]) / n), (float)((a[1] - c[1]) / n), (float)((a[2] - c[2]) / n),
                               (float)((a[3] - c[3]) / n));
}

// F <- fields of (rho + d0, rho u + (d1, d2), E + d3); a non-positive density or
// temperature becomes NaN, which the drift gate rejects.
__global__ void k_conserve_apply(float4* __restrict__ F, long long n, const float4* __restrict__ delta) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (i >= n) return;
    float4& a = F[(long long)b * n + i];
    const float4 d = delta[b];
    const float r = a.x + d.x;
    const float jx = fmaf(a.x, a.y, d.y), jy = fmaf(a.x, a.z, d.z);
    const float e = fmaf(a.x, 2.0f * a.w + a.y * a.y + a.z * a.z, d.w);
    const float ux = jx / r, uy = jy / r;
    const float th = 0.5f * (e / r - (ux * ux + uy * uy));
    const bool ok = r > 0.0f && th > 0.0f;
    a = ok ? make_float4(r, ux, uy, th) : make_float4(__int_as_float(0x7fc00000), 0.f, 0.f, 0.f);
}

struct CEConsts {
    float Ginv[16];   // inverse of G_jk = sum_p w0_p m_j(p) m_k(p), m = (1, v_x, v_y, |v|^2)
    float coef;       // (1 - omega) / omega
};

// Q1: the 1D velocity count when known at compile time (arrays then stay in
// registers), 0 for any q1 <= kMaxQ1.
// refs (batched launch, grid.z = lattice): lattice blockIdx.z writes refs[z].f from
// the fields at refs[z].index * nx * ny of F.
template <typename S, int Q1>
__global__ void k_ce_reconstruct(const __grid_constant__ LatticeParams P, const __grid_constant__ CEConsts K,
                                 const float4* __restrict__ F, S* __restrict__ f, const LatticeRef* __restrict__ refs) {
    constexpr int kQ1 = Q1 ? Q1 : kMaxQ1;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= P.nx) return;
    if (refs) {
        const LatticeRef r = refs[blockIdx.z];
        f = static_cast<S*>(r.f);
        F += r.index * P.nx * P.ny;
    }
    const int nx = P.nx, ny = P.ny;
    const int xp = x + 1 == nx ? 0 : x + 1, xm = x == 0 ? nx - 1 : x - 1;
    const int yp = y + 1 == ny ? 0 : y + 1, ym = y == 0 ? ny - 1 : y - 1;
    const float4 c = F[(long long)y * nx + x];
    const float4 e = F[(long long)y * nx + xp], w = F[(long long)y * nx + xm];
    const float4 n = F[(long long)yp * nx + x], s = F[(long long)ym * nx + x];
    const float rho = c.x, ux = c.y, uy = c.z, th = c.w;
    // central differences
    const float drx = 0.5f * (e.x - w.x), dry = 0.5f * (n.x - s.x);
    const float dux_x = 0.5f * (e.y - w.y), dux_y = 0.5f * (n.y - s.y);
    const float duy_x = 0.5f * (e.z - w.z), duy_y = 0.5f * (n.z - s.z);
    const float dth_x = 0.5f * (e.w - w.w), dth_y = 0.5f * (n.w - s.w);
    const float dp_x = 0.5f * (e.x * e.w - w.x * w.w), dp_y = 0.5f * (n.x * n.w - s.x * s.w);
    const float divu = dux_x + duy_y;
    const float inv_rho = 1.0f / rho;
    // Euler time derivatives (d = 2)
    const float dt_rho = -(ux * drx + uy * dry) - rho * divu;
    const float dt_ux = -(ux * dux_x + uy * dux_y) - dp_x * inv_rho;
    const float dt_uy = -(ux * duy_x + uy * duy_y) - dp_y * inv_rho;
    const float dt_th = -(ux * dth_x + uy * dth_y) - th * divu;
    // per-axis rule, its u- and theta-derivatives
    const int q1 = Q1 ? Q1 : P.q1;
    float r[2][kQ1], ru[2][kQ1], rt[2][kQ1];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const float u = a == 0 ? ux : uy;
        float mu[kQ1 + 1];
        mu[0] = 1.0f;
        mu[1] = u;
#pragma unroll
        for (int k = 1; k + 1 < kQ1; ++k)
            if (k + 1 < q1) mu[k + 1] = u * mu[k] + (float)k * th * mu[k - 1];
#pragma unroll
        for (int i = 0; i < kQ1; ++i) {
            if (i >= q1) break;
            float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f;
#pragma unroll
            for (int k = 0; k < kQ1; ++k) {
                if (k >= q1) break;
                const float cik = P.Cf[i * q1 + k] + P.Cf_lo[i * q1 + k];
                s0 += cik * mu[k];
                if (k >= 1) s1 += cik * (float)k * mu[k - 1];
                if (k >= 2) s2 += cik * 0.5f * (float)(k * (k - 1)) * mu[k - 2];
            }
            r[a][i] = s0;
            ru[a][i] = s1;
            rt[a][i] = s2;
        }
    }
    float fneq[kQ1 * kQ1], feq[kQ1 * kQ1];
    float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f;
#pragma unroll
    for (int i = 0; i < kQ1; ++i) {
        if (i >= q1) break;
        const float vx = (float)P.v[i];
#pragma unroll
        for (int j = 0; j < kQ1; ++j) {
            if (j >= q1) break;
            const float vy = (float)P.v[j];
            const int p = i * q1 + j;
            const float Drho = dt_rho + vx * drx + vy * dry;
            const float Dux = dt_ux + vx * dux_x + vy * dux_y;
            const float Duy = dt_uy + vx * duy_x + vy * duy_y;
            const float Dth = dt_th + vx * dth_x + vy * dth_y;
            const float D = r[0][i] * r[1][j] * Drho + rho * ru[0][i] * r[1][j] * Dux + rho * r[0][i] * ru[1][j] * Duy +
                            rho * (rt[0][i] * r[1][j] + r[0][i] * rt[1][j]) * Dth;
            const float fn = -K.coef * D;
            fneq[p] = fn;
            feq[p] = rho * r[0][i] * r[1][j];
            m0 += fn;
            m1 += vx * fn;
            m2 += vy * fn;
            m3 += (vx * vx + vy * vy) * fn;
        }
    }
    float cc[4];
    for (int k = 0; k < 4; ++k) cc[k] = K.Ginv[4 * k] * m0 + K.Ginv[4 * k + 1] * m1 + K.Ginv[4 * k + 2] * m2 + K.Ginv[4 * k + 3] * m3;
#pragma unroll
    for (int i = 0; i < kQ1; ++i) {
        if (i >= q1) break;
        const float vx = (float)P.v[i];
#pragma unroll
        for (int j = 0; j < kQ1; ++j) {
            if (j >= q1) break;
            const float vy = (float)P.v[j];
            const int p = i * q1 + j;
            const float proj = P.W0f[p] * (cc[0] + cc[1] * vx + cc[2] * vy + cc[3] * (vx * vx + vy * vy));
            if constexpr (Storage<S>::kDeviation) {
                Storage<S>::store(f + elem_index(P, p, x, y), (feq[p] - P.W0f[p]) + (fneq[p] - proj));
            } else {
                f[elem_index(P, p, x, y)] = (double)feq[p] + (double)(fneq[p] - proj);
            }
        }
    }
}

// ---------------------------------------------------------------------------
cudaError_t ce_pack_fields(const double* rho, const double* ux, const double* uy, const double* th, long long n,
                           float* out, cudaStream_t s) {
    k_pack_fields<<<(int)((n + 255) / 256), 256, 0, s>>>(rho, ux, uy, th, n, reinterpret_cast<float4*>(out));
    return cudaGetLastError();
}

cudaError_t ce_assemble(const float* snaps, long long npix, const int* pairs, int B, const float* mean_in,
                        const float* std_in, const float* mean_d, const float* std_d, void* x, float* y,
                        float sigma, unsigned long long seed, cudaStream_t s) {
    const float4 mi = make_float4(mean_in[0], mean_in[1], mean_in[2], mean_in[3]);
    const float4 si = make_float4(1.f / std_in[0], 1.f / std_in[1], 1.f / std_in[2], 1.f / std_in[3]);
    const float4 md = make_float4(mean_d[0], mean_d[1], mean_d[2], mean_d[3]);
    const float4 sd = make_float4(1.f / std_d[0], 1.f / std_d[1], 1.f / std_d[2], 1.f / std_d[3]);
    const long long n = npix * B;
    k_assemble<<<(int)((n + 255) / 256), 256, 0, s>>>(reinterpret_cast<const float4*>(snaps), npix, pairs, B, mi, si,
                                                       md, sd, static_cast<__nv_bfloat16*>(x),
                                                       reinterpret_cast<float4*>(y), sigma, seed);
    return cudaGetLastError();
}

cudaError_t ce_normalise(const float* F, long long n, const float* mean_in, const float* std_in, void* x,
                         cudaStream_t s) {
    const float4 mi = make_float4(mean_in[0], mean_in[1], mean_in[2], mean_in[3]);
    const float4 si = make_float4(1.f / std_in[0], 1.f / std_in[1], 1.f / std_in[2], 1.f / std_in[3]);
    k_normalise<<<(int)((n + 255) / 256), 256, 0, s>>>(reinterpret_cast<const float4*>(F), n, mi, si,
                                                        static_cast<__nv_bfloat16*>(x));
    return cudaGetLastError();
}

cudaError_t ce_apply_delta(const float* F, const float* d, long long n, const float* mean_d, const float* std_d,
                           float* out, cudaStream_t s) {
    const float4 md = make_float4(mean_d[0], mean_d[1], mean_d[2], mean_d[3]);
    const float4 sd = make_float4(std_d[0], std_d[1], std_d[2], std_d[3]);
    k_apply_delta<<<(int)((n + 255) / 256), 256, 0, s>>>(reinterpret_cast<const float4*>(F),
                                                          reinterpret_cast<const float4*>(d), n, md, sd,
                                                          reinterpret_cast<float4*>(out));
    return cudaGetLastError();
}

int ce_sum_blocks() { return 64; }

cudaError_t ce_conserve(const float* Fold, float* Fnew, long long n, int nlat, double* partial_old,
                        double* partial_new, float* delta, cudaStream_t s) {
    const dim3 grid(ce_sum_blocks(), nlat);
    k_field_sums_batch<<<grid, 256, 0, s>>>(reinterpret_cast<const float4*>(Fold), n, partial_old);
    k_field_sums_batch<<<grid, 256, 0, s>>>(reinterpret_cast<const float4*>(Fnew), n, partial_new);
    k_conserve_coef<<<(nlat + 3) / 4, 128, 0, s>>>(partial_old, partial_new, ce_sum_blocks(), nlat, n,
                                                   reinterpret_cast<float4*>(delta));
    k_conserve_apply<<<dim3((unsigned)((n + 255) / 256), nlat), 256, 0, s>>>(reinterpret_cast<float4*>(Fnew), n,
                                                                          reinterpret_cast<const float4*>(delta));
    return cudaGetLastError();
}

cudaError_t ce_field_drift(const float* Fold, const float* Fnew, long long n, int nlat, double* partial_old,
                           double* partial_new, double* drift, cudaStream_t s) {
    const dim3 grid(ce_sum_blocks(), nlat);
    k_field_sums_batch<<<grid, 256, 0, s>>>(reinterpret_cast<const float4*>(Fold), n, partial_old);
    k_field_sums_batch<<<grid, 256, 0, s>>>(reinterpret_cast<const float4*>(Fnew), n, partial_new);
    k_field_drift<<<(nlat + 3) / 4, 128, 0, s>>>(partial_old, partial_new, ce_sum_blocks(), nlat, drift);
    return cudaGetLastError();
}

cudaError_t ce_field_sums(const float* F, long long n, double* partial, cudaStream_t s) {
    k_field_sums<<<ce_sum_blocks(), 256, 0, s>>>(reinterpret_cast<const float4*>(F), n, partial);
    return cudaGetLastError();
}

static cudaError_t ce_reconstruct_batch_impl(int prec, const LatticeParams& P, const float* F, void* f,
                                             const LatticeRef* refs, int n, cudaStream_t s);

cudaError_t ce_reconstruct(int prec, const LatticeParams& P, const float* F, void* f, cudaStream_t s) {
    return ce_reconstruct_batch_impl(prec, P, F, f, nullptr, 1, s);
}

cudaError_t ce_reconstruct_batch(int prec, const LatticeParams& P, const float* F, const LatticeRef* refs, int n,
                                 cudaStream_t s) {
    if (n < 1 || n > 65535) return cudaErrorInvalidValue;
    return ce_reconstruct_batch_impl(prec, P, F, nullptr, refs, n, s);
}

static cudaError_t ce_reconstruct_batch_impl(int prec, const LatticeParams& P, const float* F, void* f,
                                             const LatticeRef* refs, int n, cudaStream_t s) {
    if (P.dim != 2) return cudaErrorInvalidValue;
    // G_jk = sum_p w0_p m_j m_k, m = (1, vx, vy, |v|^2), inverted in FP64 on the host.
    double G[4][4] = {{0}};
    for (int i = 0; i < P.q1; ++i)
        for (int j = 0; j < P.q1; ++j) {
            const double vx = P.v[i], vy = P.v[j];
            const double m[4] = {1.0, vx, vy, vx * vx + vy * vy};
            const double w = P.W0[i * P.q1 + j];
            for (int a = 0; a < 4; ++a)
                for (int b = 0; b < 4; ++b) G[a][b] += w * m[a] * m[b];
        }
    double A[4][8];
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 8; ++b) A[a][b] = b < 4 ? G[a][b] : (b - 4 == a ? 1.0 : 0.0);
    for (int col = 0; col < 4; ++col) {
        int piv = col;
        for (int r = col + 1; r < 4; ++r)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        for (int b = 0; b < 8; ++b) {
            const double t = A[col][b];
            A[col][b] = A[piv][b];
            A[piv][b] = t;
        }
        const double d = A[col][col];
        if (d == 0.0) return cudaErrorInvalidValue;
        for (int b = 0; b < 8; ++b) A[col][b] /= d;
        for (int r = 0; r < 4; ++r)
            if (r != col) {
                const double m = A[r][col];
                for (int b = 0; b < 8; ++b) A[r][b] -= m * A[col][b];
            }
    }
    CEConsts K;
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) K.Ginv[4 * a + b] = (float)A[a][4 + b];
    K.coef = (float)((1.0 - P.omega) / P.omega);
    dim3 grid((P.nx + 127) / 128, P.ny, n);
    const float4* Fv = reinterpret_cast<const float4*>(F);
    switch (prec) {
        case kF32:
            if (P.q1 == 5) k_ce_reconstruct<float, 5><<<grid, 128, 0, s>>>(P, K, Fv, static_cast<float*>(f), refs);
            else k_ce_reconstruct<float, 0><<<grid, 128, 0, s>>>(P, K, Fv, static_cast<float*>(f), refs);
            break;
        case kF16Dev:
            if (P.q1 == 5) k_ce_reconstruct<__half, 5><<<grid, 128, 0, s>>>(P, K, Fv, static_cast<__half*>(f), refs);
            else k_ce_reconstruct<__half, 0><<<grid, 128, 0, s>>>(P, K, Fv, static_cast<__half*>(f), refs);
            break;
        case kBF16Dev:
            if (P.q1 == 5)
                k_ce_reconstruct<__nv_bfloat16, 5><<<grid, 128, 0, s>>>(P, K, Fv, static_cast<__nv_bfloat16*>(f),
                                                                        refs);
            else
                k_ce_reconstruct<__nv_bfloat16, 0><<<grid, 128, 0, s>>>(P, K, Fv, static_cast<__nv_bfloat16*>(f),
                                                                        refs);
            break;
        case kF64:
            if (P.q1 == 5) k_ce_reconstruct<double, 5><<<grid, 128, 0, s>>>(P, K, Fv, static_cast<double*>(f), refs);
            else k_ce_reconstruct<double, 0><<<grid, 128, 0, s>>>(P, K, Fv, static_cast<double*>(f), refs);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace plbm
