// Device code of the PLBM stream-and-collide step (sm_103a).
//
// One thread updates one node.  Populations are SoA planes f[p][y][pitch].
// A step pulls f_p(x - v_p) for every population (Eq. eq:srt read as
// pull + collide on post-collision states), takes the moments, evaluates the
// Maxwell-Boltzmann moments mu_n(u, theta) by their recurrence, forms
// r_i = sum_j c_ij mu_{j-1} per axis (Eq. eq:rdr), the tensor-product
// equilibrium f^eq = rho r^x r^y (Sec. 2.1) and relaxes with omega.
//
// Two arithmetic cores:
//  * Direct (FP64 storage): moments of f, f^eq = rho r^x r^y,
//    f' = f + omega (f^eq - f).
//  * Deviation (FP32, FP16, BF16 storage, FP32 arithmetic): every population is
//    stored and handled as g = f - w0 with w0 = f^eq(1, 0, theta0) the rest
//    equilibrium.
//    Because the rule reproduces mu_0..mu_{q1-1} exactly (Eq. eq:rdr),
//    sum w0 = 1, sum v w0 = 0 and sum |v|^2 w0 = d theta0, so
//        rho - 1 = sum g,  rho u = sum v g,  d rho theta = d theta0 + sum |v|^2 g - rho |u|^2
//    and the equilibrium deviation is built from
//        dmu_n = mu_n(u, theta) - mu_n(0, theta0)   (recurrence below),
//        dr = C dmu,  f^eq - w0 = (rho - 1) w0 + rho (dr^x r^y + w^x dr^y)
//    which never subtracts two O(1) numbers.  Storing g instead of f also makes
//    the storage rounding proportional to |f - w0| rather than to |f|.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "plbm_internal.h"

namespace plbm {

// ---------------------------------------------------------------------------
// Storage traits: how a stored element becomes an arithmetic value.
// ---------------------------------------------------------------------------
template <typename S>
struct Storage;

template <>
struct Storage<double> {
    static constexpr bool kDeviation = false;
    static __device__ __forceinline__ double load(const double* p) { return __ldg(p); }
    static __device__ __forceinline__ void store(double* p, double v) { *p = v; }
    // FP64 value of the population f (for moments/diagnostics of the stored state)
    static __device__ __forceinline__ double to_f64(double s, double) { return s; }
    static __device__ __forceinline__ double from_f64(double f, double) { return f; }
};

template <>
struct Storage<float> {
    static constexpr bool kDeviation = true;   // stores g = f - w0 in FP32
    static __device__ __forceinline__ float load(const float* p) { return __ldg(p); }
    static __device__ __forceinline__ void store(float* p, float v) { *p = v; }
    static __device__ __forceinline__ double to_f64(float s, double w0) { return w0 + (double)s; }
    static __device__ __forceinline__ float from_f64(double f, double w0) { return (float)(f - w0); }
};

template <>
struct Storage<__half> {
    static constexpr bool kDeviation = true;   // stores g = f - w0
    static __device__ __forceinline__ float load(const __half* p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ void store(__half* p, float v) { *p = __float2half_rn(v); }
    static __device__ __forceinline__ double to_f64(__half s, double w0) {
        return w0 + (double)__half2float(s);
    }
    static __device__ __forceinline__ __half from_f64(double f, double w0) {
        return __double2half(f - w0);
    }
};

template <>
struct Storage<__nv_bfloat16> {
    static constexpr bool kDeviation = true;
    static __device__ __forceinline__ float load(const __nv_bfloat16* p) {
        return __bfloat162float(__ldg(p));
    }
    static __device__ __forceinline__ void store(__nv_bfloat16* p, float v) {
        *p = __float2bfloat16_rn(v);
    }
    static __device__ __forceinline__ double to_f64(__nv_bfloat16 s, double w0) {
        return w0 + (double)__bfloat162float(s);
    }
    static __device__ __forceinline__ __nv_bfloat16 from_f64(double f, double w0) {
        return __double2bfloat16(f - w0);
    }
};

// ---------------------------------------------------------------------------
// Per-node diagnostics accumulated by reducing launches.
// ---------------------------------------------------------------------------
struct NodeDiag {
    double mass, jx, jy, energy, rho_min, theta_min;
};

__device__ __forceinline__ void diag_zero(NodeDiag& d) {
    d.mass = d.jx = d.jy = d.energy = 0.0;
    d.rho_min = 1e300;
    d.theta_min = 1e300;
}

// Sets PLBM_STATUS_* bits for a node whose rho or theta is non-finite or
// non-positive.  Evaluated in the kernel's own precision (FP32 kernels never
// touch the FP64 pipe here).  NaN compares false, so it lands in the first test.
template <typename R>
__device__ __forceinline__ void flag_status(const LatticeParams& P, R rho, R theta) {
    const R big = (R)3.0e38f;
    if (!(rho > (R)0 && theta > (R)0 && rho < big && theta < big)) {
        unsigned bits = 0u;
        if (!(rho == rho) || !(theta == theta) || !(rho < big) || !(theta < big)) bits |= 1u;
        if (rho <= (R)0) bits |= 2u;
        if (theta <= (R)0) bits |= 4u;
        atomicOr(P.status, bits);
    }
}

// Float-float numbers: an FP32 pair hi + lo carried through error-free sums
// (TwoSum) and products (FMA), ~2^-48 relative: FP64-grade sums of FP32 data on
// the FP32 pipe (GB300's FP64 rate is two operations per SM per cycle).
struct FF {
    float hi, lo;
};
__device__ __forceinline__ FF ff_add(FF a, float b) {
    const float s = a.hi + b;
    const float t = s - a.hi;
    const float e = (a.hi - (s - t)) + (b - t);
    return {s, a.lo + e};
}
__device__ __forceinline__ FF ff_add(FF a, FF b) {
    const float s = a.hi + b.hi;
    const float t = s - a.hi;
    const float e = (a.hi - (s - t)) + (b.hi - t);
    return {s, (a.lo + b.lo) + e};
}
__device__ __forceinline__ FF ff_scale(FF a, float v) {
    const float p = a.hi * v;
    const float e = fmaf(a.hi, v, -p);
    return {p, fmaf(a.lo, v, e)};
}
__device__ __forceinline__ double ff_f64(FF a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ FF ff_shfl_down(FF a, int off) {
    return {__shfl_down_sync(0xffffffffu, a.hi, off), __shfl_down_sync(0xffffffffu, a.lo, off)};
}

// Per-thread diagnostics of 16/32-bit kernels: deviations from the rest state
// (mass - n, energy - n d theta0) in float-float, n the thread's node count.
struct NodeDiagF {
    FF dmass, jx, jy, denergy;
    float rho_min, theta_min, n;
};
__device__ __forceinline__ void diagf_zero(NodeDiagF& d) {
    d.dmass = d.jx = d.jy = d.denergy = FF{0.0f, 0.0f};
    d.rho_min = d.theta_min = 3.0e38f;
    d.n = 0.0f;
}

// Order-preserving int64 key of a double (total order, negatives included), so
// that FP64 minima reduce on the integer pipe.
__device__ __forceinline__ long long dkey(double v) {
    const long long b = __double_as_longlong(v);
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double dunkey(long long k) {
    return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffLL));
}
__device__ __forceinline__ long long kmin(long long a, long long b) { return a < b ? a : b; }

// Block reduction of NodeDiagF in float-float; thread 0 writes the same FP64
// record as block_reduce_diag (mass = n + dmass, energy = n d theta0 + denergy).
// DMIN: the minima are the caller's FP64 rho_min_d, theta_min_d (1e300 for no
// node), reduced as order-preserving integer keys, instead of the FP32 ones of d.
template <int NT, bool DMIN = false>
__device__ __forceinline__ void block_reduce_diagf(NodeDiagF d, double dtheta0, double* out, double rho_min_d = 0.0,
                                                   double theta_min_d = 0.0) {
    __shared__ float sh[11][NT / 32];
    __shared__ long long shk[2][NT / 32];
    long long kr = 0, kt = 0;
    if (DMIN) {
        kr = dkey(rho_min_d);
        kt = dkey(theta_min_d);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            kr = kmin(kr, __shfl_down_sync(0xffffffffu, kr, off));
            kt = kmin(kt, __shfl_down_sync(0xffffffffu, kt, off));
        }
        if ((threadIdx.x & 31) == 0) {
            shk[0][threadIdx.x >> 5] = kr;
            shk[1][threadIdx.x >> 5] = kt;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        d.dmass = ff_add(d.dmass, ff_shfl_down(d.dmass, off));
        d.jx = ff_add(d.jx, ff_shfl_down(d.jx, off));
        d.jy = ff_add(d.jy, ff_shfl_down(d.jy, off));
        d.denergy = ff_add(d.denergy, ff_shfl_down(d.denergy, off));
        d.rho_min = fminf(d.rho_min, __shfl_down_sync(0xffffffffu, d.rho_min, off));
        d.theta_min = fminf(d.theta_min, __shfl_down_sync(0xffffffffu, d.theta_min, off));
        d.n += __shfl_down_sync(0xffffffffu, d.n, off);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        sh[0][warp] = d.dmass.hi;
        sh[1][warp] = d.dmass.lo;
        sh[2][warp] = d.jx.hi;
        sh[3][warp] = d.jx.lo;
        sh[4][warp] = d.jy.hi;
        sh[5][warp] = d.jy.lo;
        sh[6][warp] = d.denergy.hi;
        sh[7][warp] = d.denergy.lo;
        sh[8][warp] = d.rho_min;
        sh[9][warp] = d.theta_min;
        sh[10][warp] = d.n;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        FF m{0.f, 0.f}, a{0.f, 0.f}, b{0.f, 0.f}, e{0.f, 0.f};
        float rmin = 3.0e38f, tmin = 3.0e38f, n = 0.0f;
        for (int w = 0; w < NT / 32; ++w) {
            m = ff_add(m, FF{sh[0][w], sh[1][w]});
            a = ff_add(a, FF{sh[2][w], sh[3][w]});
            b = ff_add(b, FF{sh[4][w], sh[5][w]});
            e = ff_add(e, FF{sh[6][w], sh[7][w]});
            rmin = fminf(rmin, sh[8][w]);
            tmin = fminf(tmin, sh[9][w]);
            n += sh[10][w];
        }
        out[0] = (double)n + ff_f64(m);
        out[1] = ff_f64(a);
        out[2] = ff_f64(b);
        out[3] = (double)n * dtheta0 + ff_f64(e);
        if (DMIN) {
            long long r = shk[0][0], t = shk[1][0];
            for (int w = 1; w < NT / 32; ++w) {
                r = kmin(r, shk[0][w]);
                t = kmin(t, shk[1][w]);
            }
            out[4] = dunkey(r);
            out[5] = dunkey(t);
        } else {
            out[4] = rmin < 3.0e38f ? (double)rmin : 1e300;
            out[5] = tmin < 3.0e38f ? (double)tmin : 1e300;
        }
    }
}

// Block reduction of NodeDiag; thread 0 writes kPartialStride doubles to out.
template <int NT>
__device__ __forceinline__ void block_reduce_diag(NodeDiag d, double* out) {
    __shared__ double sh[6][NT / 32];
    const unsigned full = 0xffffffffu;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        d.mass += __shfl_down_sync(full, d.mass, off);
        d.jx += __shfl_down_sync(full, d.jx, off);
        d.jy += __shfl_down_sync(full, d.jy, off);
        d.energy += __shfl_down_sync(full, d.energy, off);
        d.rho_min = fmin(d.rho_min, __shfl_down_sync(full, d.rho_min, off));
        d.theta_min = fmin(d.theta_min, __shfl_down_sync(full, d.theta_min, off));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        sh[0][warp] = d.mass;
        sh[1][warp] = d.jx;
        sh[2][warp] = d.jy;
        sh[3][warp] = d.energy;
        sh[4][warp] = d.rho_min;
        sh[5][warp] = d.theta_min;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double r[6] = {0, 0, 0, 0, 1e300, 1e300};
        for (int w = 0; w < NT / 32; ++w) {
            r[0] += sh[0][w];
            r[1] += sh[1][w];
            r[2] += sh[2][w];
            r[3] += sh[3][w];
            r[4] = fmin(r[4], sh[4][w]);
            r[5] = fmin(r[5], sh[5][w]);
        }
        for (int k = 0; k < 6; ++k) out[k] = r[k];
    }
}

// ---------------------------------------------------------------------------
// Source addresses of the pull: f_p(x - v_p) with periodic wrap or ghosts.
// ---------------------------------------------------------------------------
template <int Q1, int DIM>
struct PullIndex {
    int col[Q1];              // source column per x-velocity
    bool okx[Q1];             // false: the source lies in a fixed-end ghost
    bool leftx[Q1];           // ghost side when !okx
    long long row[DIM == 2 ? Q1 : 1];  // source row offset (elements) per y-velocity

    __device__ __forceinline__ void build(const LatticeParams& P, int x, int y) {
#pragma unroll
        for (int i = 0; i < Q1; ++i) {
            if (P.fixed_ends) {
                int s = x - P.v[i];
                okx[i] = (s >= 0) && (s < P.nx);
                leftx[i] = s < 0;
                col[i] = okx[i] ? s : 0;
            } else {
                int s = x + P.vxm[i];
                col[i] = (s >= P.nx) ? s - P.nx : s;
                okx[i] = true;
                leftx[i] = false;
            }
        }
        if (DIM == 2) {
#pragma unroll
            for (int j = 0; j < (DIM == 2 ? Q1 : 1); ++j) {
                int s = y + P.vym[j];
                s = (s >= P.ny) ? s - P.ny : s;
                row[j] = (long long)s * P.pitch;
            }
        } else {
            row[0] = 0;
        }
    }
};

// ---------------------------------------------------------------------------
// Direct FP64 core.
// ---------------------------------------------------------------------------
template <int Q1, int DIM>
struct DirectCore {
    static constexpr int Q = (DIM == 1) ? Q1 : Q1 * Q1;

    // f holds the pulled populations on entry and the post-collision ones on exit.
    static __device__ __forceinline__ void collide(double (&f)[Q], const LatticeParams& P,
                                                   double& rho_o, double& th_o, double& jx_o,
                                                   double& jy_o, double& e_o) {
        double S[Q1], T[Q1];
        if (DIM == 2) {
#pragma unroll
            for (int i = 0; i < Q1; ++i) {
                double s = 0.0;
#pragma unroll
                for (int j = 0; j < Q1; ++j) s += f[i * Q1 + j];
                S[i] = s;
            }
#pragma unroll
            for (int j = 0; j < Q1; ++j) {
                double t = 0.0;
#pragma unroll
                for (int i = 0; i < Q1; ++i) t += f[i * Q1 + j];
                T[j] = t;
            }
        } else {
#pragma unroll
            for (int i = 0; i < Q1; ++i) S[i] = f[i];
        }
        double rho = 0.0, jx = 0.0, ex = 0.0, jy = 0.0, ey = 0.0;
#pragma unroll
        for (int i = 0; i < Q1; ++i) {
            const double vi = (double)P.v[i];
            rho += S[i];
            jx += vi * S[i];
            ex += vi * vi * S[i];
            if (DIM == 2) {
                jy += vi * T[i];
                ey += vi * vi * T[i];
            }
        }
        const double inv = 1.0 / rho;
        const double ux = jx * inv, uy = jy * inv;
        double th = ((ex + ey) * inv - (ux * ux + uy * uy)) * (1.0 / DIM);
        rho_o = rho;
        th_o = th;
        jx_o = jx;
        jy_o = jy;
        e_o = ex + ey;
        if (P.isothermal) th = P.theta0;

        // mu_n(u, theta) by mu_{n+1} = u mu_n + n theta mu_{n-1}; r = C mu.
        double rx[Q1], ry[Q1];
        {
            double mu[Q1];
            mu[0] = 1.0;
            if (Q1 > 1) mu[1] = ux;
#pragma unroll
            for (int n = 1; n + 1 < Q1; ++n) mu[n + 1] = ux * mu[n] + (double)n * th * mu[n - 1];
#pragma unroll
            for (int i = 0; i < Q1; ++i) {
                double r = 0.0;
#pragma unroll
                for (int n = 0; n < Q1; ++n) r += P.C[i * Q1 + n] * mu[n];
                rx[i] = rho * r;  // rho folded into the x factor
            }
        }
        if (DIM == 2) {
            double mu[Q1];
            mu[0] = 1.0;
            if (Q1 > 1) mu[1] = uy;
#pragma unroll
            for (int n = 1; n + 1 < Q1; ++n) mu[n + 1] = uy * mu[n] + (double)n * th * mu[n - 1];
#pragma unroll
            for (int i = 0; i < Q1; ++i) {
                double r = 0.0;
#pragma unroll
                for (int n = 0; n < Q1; ++n) r += P.C[i * Q1 + n] * mu[n];
                ry[i] = r;
            }
        }
        const double om = P.omega;
#pragma unroll
        for (int i = 0; i < Q1; ++i) {
            if (DIM == 2) {
#pragma unroll
                for (int j = 0; j < Q1; ++j) {
                    const double feq = rx[i] * ry[j];
                    f[i * Q1 + j] = f[i * Q1 + j] + om * (feq - f[i * Q1 + j]);
                }
            } else {
                f[i] = f[i] + om * (rx[i] - f[i]);
            }
        }
    }
};

// ---------------------------------------------------------------------------
// Deviation FP32 core (see the file header for the algebra).
// ---------------------------------------------------------------------------
template <int Q1, int DIM>
struct DeviationCore {
    static constexpr int Q = (DIM == 1) ? Q1 : Q1 * Q1;

    // dmu_n = mu_n(u, theta) - mu_n(0, theta0), dr = C dmu, for one axis.
    static __device__ __forceinline__ void axis(const LatticeParams& P, float u, float th,
                                                float dth, float (&dr)[Q1]) {
        float dmu[Q1];
        dmu[0] = 0.0f;
        if (Q1 > 1) dmu[1] = u;
#pragma unroll
        for (int n = 1; n + 1 < Q1; ++n) {
            const float fn = (float)n;
            dmu[n + 1] = u * (P.mu0f[n] + dmu[n]) + fn * th * dmu[n - 1] + fn * dth * P.mu0f[n - 1];
        }
        // C carried as Cf + Cf_lo: a single FP32 rounding of c_ij would break the
        // moment identities of Eq. (eq:rdr) by ~1e-8 in a fixed direction, which
        // the collision turns into a systematic momentum source.
#pragma unroll
        for (int i = 0; i < Q1; ++i) {
            float r = 0.0f, rl = 0.0f;
#pragma unroll
            for (int n = 1; n < Q1; ++n) {
                r = fmaf(P.Cf[i * Q1 + n], dmu[n], r);
                rl = fmaf(P.Cf_lo[i * Q1 + n], dmu[n], rl);
            }
            dr[i] = r + rl;
        }
    }

    // g holds pulled deviations on entry and post-collision deviations on exit.
    static __device__ __forceinline__ void collide(float (&g)[Q], const LatticeParams& P,
                                                   float& drho_o, float& th_o, float& jx_o,
                                                   float& jy_o, float& e_o) {
        float S[Q1], T[Q1];
        if (DIM == 2) {
#pragma unroll
            for (int i = 0; i < Q1; ++i) {
                float s = 0.0f;
#pragma unroll
                for (int j = 0; j < Q1; ++j) s += g[i * Q1 + j];
                S[i] = s;
            }
#pragma unroll
            for (int j = 0; j < Q1; ++j) {
                float t = 0.0f;
#pragma unroll
                for (int i = 0; i < Q1; ++i) t += g[i * Q1 + j];
                T[j] = t;
            }
        } else {
#pragma unroll
            for (int i = 0; i < Q1; ++i) S[i] = g[i];
        }
        float drho = 0.0f, jx = 0.0f, ex = 0.0f, jy = 0.0f, ey = 0.0f;
#pragma unroll
        for (int i = 0; i < Q1; ++i) {
            const float vi = (float)P.v[i];
            drho += S[i];
            jx += vi * S[i];
            ex += vi * vi * S[i];
            if (DIM == 2) {
                jy += vi * T[i];
                ey += vi * vi * T[i];
            }
        }
        const float rho = 1.0f + drho;
        const float inv = 1.0f / rho;
        const float ux = jx * inv, uy = jy * inv;
        const float dthp = (((ex + ey) - (float)DIM * P.theta0f * drho) * inv - (ux * ux + uy * uy)) *
                           (1.0f / (float)DIM);
        drho_o = drho;
        th_o = P.theta0f + dthp;
        jx_o = jx;
        jy_o = jy;
        e_o = ex + ey;
        const float dth = P.isothermal ? 0.0f : dthp;
        const float th = P.theta0f + dth;

        float drx[Q1];
        axis(P, ux, th, dth, drx);
        const float om = P.omegaf;
        if (DIM == 2) {
            float dry[Q1], ry[Q1];
            axis(P, uy, th, dth, dry);
#pragma unroll
            for (int j = 0; j < Q1; ++j) ry[j] = P.w1f[j] + dry[j];
#pragma unroll
            for (int i = 0; i < Q1; ++i) {
                const float a = rho * drx[i];
                const float b = rho * P.w1f[i];
#pragma unroll
                for (int j = 0; j < Q1; ++j) {
                    const int p = i * Q1 + j;
                    const float geq = drho * P.W0f[p] + (a * ry[j] + b * dry[j]);
                    g[p] = g[p] + om * (geq - g[p]);
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < Q1; ++i) {
                const float geq = drho * P.w1f[i] + rho * drx[i];
                g[i] = g[i] + om * (geq - g[i]);
            }
        }
    }
};

// ---------------------------------------------------------------------------
// One node of the fused stream-and-collide step: pull, collide, store; the
// node's contribution to the diagnostics when REDUCE (d for FP64 storage, df
// for 16/32-bit storage).  Shared by the single-lattice kernel and the batched
// persistent kernel, so both give bit-identical states.
// ---------------------------------------------------------------------------
template <typename S, int Q1, int DIM, bool REDUCE>
__device__ __forceinline__ void node_update(const LatticeParams& P, const S* __restrict__ src,
                                            S* __restrict__ dst, int x, int y, NodeDiag& d, NodeDiagF& df) {
    constexpr int Q = (DIM == 1) ? Q1 : Q1 * Q1;
    PullIndex<Q1, DIM> ix;
    ix.build(P, x, y);
    const long long here = (long long)y * P.pitch + x;
    if constexpr (!Storage<S>::kDeviation && sizeof(S) == 8) {
        // FP64: direct core
        double f[Q];
#pragma unroll
        for (int i = 0; i < Q1; ++i) {
#pragma unroll
            for (int j = 0; j < (DIM == 2 ? Q1 : 1); ++j) {
                const int p = (DIM == 2) ? i * Q1 + j : i;
                f[p] = ix.okx[i] ? Storage<S>::load(src + p * P.plane + ix.row[j] + ix.col[i])
                                 : (ix.leftx[i] ? P.ghostL[p] : P.ghostR[p]);
            }
        }
        double rho, th, jx, jy, e;
        DirectCore<Q1, DIM>::collide(f, P, rho, th, jx, jy, e);
        flag_status<double>(P, rho, th);
        if (REDUCE) {
            d.mass = rho;
            d.jx = jx;
            d.jy = jy;
            d.energy = e;
            d.rho_min = rho;
            d.theta_min = th;
        }
#pragma unroll
        for (int p = 0; p < Q; ++p) Storage<S>::store(dst + p * P.plane + here, f[p]);
    } else {
        // FP32 arithmetic on deviations g = f - w0
        float g[Q];
#pragma unroll
        for (int i = 0; i < Q1; ++i) {
#pragma unroll
            for (int j = 0; j < (DIM == 2 ? Q1 : 1); ++j) {
                const int p = (DIM == 2) ? i * Q1 + j : i;
                if (ix.okx[i]) {
                    float s = Storage<S>::load(src + p * P.plane + ix.row[j] + ix.col[i]);
                    g[p] = Storage<S>::kDeviation ? s : s - P.W0f[p];
                } else {
                    g[p] = ix.leftx[i] ? P.ghostLg[p] : P.ghostRg[p];
                }
            }
        }
        float drho, th, jx, jy, e;
        DeviationCore<Q1, DIM>::collide(g, P, drho, th, jx, jy, e);
        flag_status<float>(P, 1.0f + drho, th);
        if (REDUCE) {
            df.dmass = FF{drho, 0.0f};
            df.jx = FF{jx, 0.0f};
            df.jy = FF{jy, 0.0f};
            df.denergy = FF{e, 0.0f};
            df.rho_min = 1.0f + drho;
            df.theta_min = th;
            df.n = 1.0f;
        }
#pragma unroll
        for (int p = 0; p < Q; ++p) {
            const float out = Storage<S>::kDeviation ? g[p] : g[p] + P.W0f[p];
            Storage<S>::store(dst + p * P.plane + here, out);
        }
    }
}

// ---------------------------------------------------------------------------
// The fused stream-and-collide kernel.
// grid = (ceil(nx / blockDim.x), ny), blockDim.x threads along x (kBlockX when
// REDUCE, whose per-block records assume it).
// ---------------------------------------------------------------------------
template <typename S, int Q1, int DIM, bool REDUCE>
__global__ void __launch_bounds__(kBlockX)
k_stream_collide(const __grid_constant__ LatticeParams P, const S* __restrict__ src,
                 S* __restrict__ dst) {
    const int x = blockIdx.x * (REDUCE ? kBlockX : (int)blockDim.x) + threadIdx.x;
    const int y = blockIdx.y;

    NodeDiag d;       // FP64 storage
    NodeDiagF df;     // 16/32-bit storage
    if (REDUCE) {
        diag_zero(d);
        diagf_zero(df);
    }
    if (x < P.nx) node_update<S, Q1, DIM, REDUCE>(P, src, dst, x, y, d, df);
    if (REDUCE) {
        const int blk = blockIdx.y * gridDim.x + blockIdx.x;
        if constexpr (!Storage<S>::kDeviation && sizeof(S) == 8)
            block_reduce_diag<kBlockX>(d, P.partials + (long long)blk * kPartialStride);
        else
            block_reduce_diagf<kBlockX>(df, (double)DIM * P.theta0, P.partials + (long long)blk * kPartialStride);
    }
}

// ---------------------------------------------------------------------------
// Batched persistent step over 2D lattices in the plain layout (one node per
// thread): odd row counts, FP64 storage, isothermal models and velocity sets
// other than (0, +-a, +-b), which the row-paired batched kernel does not take.
// A tile is kBlockX nodes of one row of one lattice; all such lattices' tiles
// form one list that CTA c walks as c, c + G, c + 2G, ... (G CTAs), reading
// each tile's lattice from tile_inst and that lattice's parameters from the
// device table (cached by L1).  Per node it runs node_update, as the
// single-lattice kernel does.
// ---------------------------------------------------------------------------
template <typename S, int Q1>
__global__ void __launch_bounds__(kBlockX)
k_batch_node(const LatticeParams* __restrict__ inst, const NodeSpan* __restrict__ span, int total_tiles,
             int parity, const unsigned short* __restrict__ tile_inst) {
    NodeDiag d;
    NodeDiagF df;
    for (int t = blockIdx.x; t < total_tiles; t += gridDim.x) {
        const int i = tile_inst[t];
        const NodeSpan sp = span[i];
        const LatticeParams& P = inst[i];
        const int local = t - sp.tile_begin;
        const int y = local / sp.tiles_x;
        const int x = (local - y * sp.tiles_x) * kBlockX + threadIdx.x;
        if (x < sp.nx)
            node_update<S, Q1, 2, false>(P, static_cast<const S*>(sp.f[parity]), static_cast<S*>(sp.f[parity ^ 1]),
                                         x, y, d, df);
    }
}

inline int device_sm_count() {
    static int n = 0;
    if (!n) {
        int d = 0;
        cudaGetDevice(&d);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d) != cudaSuccess || n < 1) n = 1;
    }
    return n;
}

template <typename S>
cudaError_t launch_step_t(const LatticeParams& P, const void* src, void* dst, bool reduce,
                          cudaStream_t stream) {
    if (P.paired) return cudaErrorInvalidValue;  // row-paired layouts use k_stream_collide_pair
    // Small lattices (fewer than two blocks per SM): 32-thread blocks spread the
    // nodes over four times as many SMs (GB300's FP64 rate per SM is low).
    int bx = kBlockX;
    if (!reduce && (long long)((P.nx + kBlockX - 1) / kBlockX) * P.ny < 2LL * device_sm_count()) bx = 32;
    dim3 grid((P.nx + bx - 1) / bx, P.ny);
    dim3 block(bx);
    const S* s = static_cast<const S*>(src);
    S* t = static_cast<S*>(dst);
#define PLBM_LAUNCH(Q1v, DIMv)                                                              \
    if (P.q1 == Q1v && P.dim == DIMv) {                                                     \
        if (reduce)                                                                         \
            k_stream_collide<S, Q1v, DIMv, true><<<grid, block, 0, stream>>>(P, s, t);      \
        else                                                                                \
            k_stream_collide<S, Q1v, DIMv, false><<<grid, block, 0, stream>>>(P, s, t);     \
        return cudaGetLastError();                                                          \
    }
    PLBM_LAUNCH(3, 1)
    PLBM_LAUNCH(4, 1)
    PLBM_LAUNCH(5, 1)
    PLBM_LAUNCH(6, 1)
    PLBM_LAUNCH(7, 1)
    PLBM_LAUNCH(8, 1)
    PLBM_LAUNCH(3, 2)
    PLBM_LAUNCH(4, 2)
    PLBM_LAUNCH(5, 2)
    PLBM_LAUNCH(6, 2)
    PLBM_LAUNCH(7, 2)
    PLBM_LAUNCH(8, 2)
#undef PLBM_LAUNCH
    return cudaErrorInvalidValue;
}

// Batched plain-layout step of every lattice of one (precision, q1) group.
template <typename S>
cudaError_t launch_batch_node_t(int q1, const LatticeParams* inst, const NodeSpan* span, int total_tiles,
                                int ctas, int parity, const unsigned short* tile_inst, cudaStream_t stream) {
    switch (q1) {
        case 3: k_batch_node<S, 3><<<ctas, kBlockX, 0, stream>>>(inst, span, total_tiles, parity, tile_inst); break;
        case 4: k_batch_node<S, 4><<<ctas, kBlockX, 0, stream>>>(inst, span, total_tiles, parity, tile_inst); break;
        case 5: k_batch_node<S, 5><<<ctas, kBlockX, 0, stream>>>(inst, span, total_tiles, parity, tile_inst); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename S>
cudaError_t batch_node_occupancy_t(int q1, int* blocks_per_sm) {
    switch (q1) {
        case 3: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_batch_node<S, 3>, kBlockX, 0);
        case 4: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_batch_node<S, 4>, kBlockX, 0);
        case 5: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_batch_node<S, 5>, kBlockX, 0);
    }
    return cudaErrorInvalidValue;
}

}  // namespace plbm
