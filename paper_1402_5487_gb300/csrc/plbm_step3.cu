// Three-dimensional lattices (Sec. 2.1: D3 models are the tensor product of
// three 1D rules with one scalar theta), periodic in x, y and z.
//
// Population p = (a * q1 + b) * q1 + c has velocity (v[a], v[b], v[c]); storage
// [q][nz][ny][pitch] (row index z * ny + y of elem_index).  The rest equilibrium
// is the product w0_p = w_a w_b w_c of the 1D rest weights.
//
// k_stream_collide3<S> (FP32 arithmetic; FP16 or BF16 storage of the deviation
// g = f - w0 on the plain layout; symmetric five-velocity sets (0, +-a, +-b),
// D3Q125; k_stream_collide3_split below is the FP32 kernel, the same update
// with a node's populations spread over five warps):
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
// k_stream_collide3_zpair<S> (FP16 or BF16 storage, even nz): the same update
// on the z-paired layout, where nodes (x, y, z) and (x, y, z + nz/2) sit side by
// side.  One thread updates both: each of the 125 pulls is one aligned 4-byte
// load of the two 16-bit deviations (kept packed in one register until the
// collision), each store one 4-byte store, and the arithmetic runs on the two
// nodes as the lanes of packed FP32x2 instructions.  Pull across the z wrap:
// node z = r reads z - v_z; when r - v_z leaves [0, nz/2) the source pair row is
// r - v_z -+ nz/2 and holds the two nodes in swapped lane order.
// k_stream_collide3_f64: FP64 storage of f, any q1 <= 5, thermal or isothermal,
// the plain formulas (an ALU-bound path).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "plbm_device.cuh"
#include "plbm_pair.cuh"

namespace plbm {

namespace {

constexpr int kB3 = 128;       // threads per block along x
constexpr int kQ1 = 5;         // D3Q125
constexpr int kQ3 = kQ1 * kQ1 * kQ1;

__device__ __forceinline__ int wrap_add(int i, int d, int n) {
    const int s = i + d;
    return s >= n ? s - n : s;
}

// Element offset of node (x, y, z) within a population plane (plain or z-paired layout).
__device__ __forceinline__ long long node3(const LatticeParams& P, int x, int y, int z) {
    if (P.zpaired) {
        const int hi = z >= P.half_nz;
        const int r = hi ? z - P.half_nz : z;
        return ((long long)r * P.ny + y) * 2 * P.pitch + 2LL * x + hi;
    }
    return ((long long)z * P.ny + y) * P.pitch + x;
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
        for (int b = 0; b < kQ1; ++b) {
            float R = 0.0f;   // R_ab = sum_c g; S_a = sum_b R_ab, T_b = sum_a R_ab
#pragma unroll
            for (int c = 0; c < kQ1; ++c) {
                const float v = g[(a * kQ1 + b) * kQ1 + c];
                R += v;
                Uc[c] += v;
            }
            Sa[a] += R;
            Tb[b] += R;
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
    // g' = (1 - omega) g + omega (f^eq - w0), omega (f^eq - w0) = X_a P_bc + W_a Q_bc with
    // X_a = omega (rho r^x_a - w_a) = omega ((rho - 1) w_a + rho dr^x_a), W_a = omega w_a.
    const float om = P.omegaf;
    float X[kQ1];
#pragma unroll
    for (int a = 0; a < kQ1; ++a) X[a] = om * fmaf(drho, P.w1f[a], rho * drx[a]);
    const float keep = 1.0f - om;
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
                const float d = fmaf(X[a], Pbc, (om * P.w1f[a]) * Qbc);
                Storage<S>::store(dst + (long long)p * P.plane + here, fmaf(keep, g[p], d));
            }
        }
}

// The same update with the 125 populations of a node split over five warps:
// warp a of a CTA takes the 25 populations (a, b, c) of the 32 nodes
// x0 .. x0 + 31 (lane = node), so a thread holds 25 values instead of 125 and
// far more warps fit per SM.  Each warp forms its partial sums (S_a, and T_b,
// U_c over its own a) into shared memory; warp 0 completes the moments of the
// 32 nodes and the x rule; warp a then forms row b = a of the factor table
// P_bc = r^y_b r^z_c, Q_bc = dr^y_b r^z_c + w_b dr^z_c, which every warp reads
// (three barriers per CTA).
constexpr int kSplitNodes = 32;
constexpr int kSplitThreads = kSplitNodes * kQ1;   // 160

template <typename S>
__global__ void __launch_bounds__(kSplitThreads) k_stream_collide3_split(const __grid_constant__ LatticeParams P,
                                                                         const S* __restrict__ src,
                                                                         S* __restrict__ dst) {
    __shared__ float sS[kQ1][kSplitNodes];
    __shared__ float sT[kQ1][kQ1][kSplitNodes];   // [warp a][b][node]
    __shared__ float sU[kQ1][kQ1][kSplitNodes];   // [warp a][c][node]
    __shared__ float sM[5][kSplitNodes];          // drho, ux, uy, uz, dth
    __shared__ float sDx[kQ1][kSplitNodes];       // dr^x_a
    __shared__ float sP[kQ1][kQ1][kSplitNodes];   // P_bc = r^y_b r^z_c
    __shared__ float sQ[kQ1][kQ1][kSplitNodes];   // Q_bc = dr^y_b r^z_c + w_b dr^z_c
    const int a = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x = blockIdx.x * kSplitNodes + lane;
    const int y = blockIdx.y, z = blockIdx.z;
    const bool active = x < P.nx;
    int xa = 0, yr[kQ1], zr[kQ1];
    float g[kQ1 * kQ1];
    if (active) {
        xa = wrap_add(x, P.vxm[a], P.nx);
#pragma unroll
        for (int i = 0; i < kQ1; ++i) {
            yr[i] = wrap_add(y, P.vym[i], P.ny) * P.pitch;
            zr[i] = wrap_add(z, P.vzm[i], P.nz) * P.ny * P.pitch;
        }
        const long long pa = (long long)a * kQ1 * kQ1 * P.plane;
#pragma unroll
        for (int b = 0; b < kQ1; ++b)
#pragma unroll
            for (int c = 0; c < kQ1; ++c)
                g[b * kQ1 + c] = Storage<S>::load(src + pa + (long long)(b * kQ1 + c) * P.plane + (zr[c] + yr[b] + xa));
        float Sa = 0.0f, Uc[kQ1];
#pragma unroll
        for (int c = 0; c < kQ1; ++c) Uc[c] = 0.0f;
#pragma unroll
        for (int b = 0; b < kQ1; ++b) {
            float T = 0.0f;
#pragma unroll
            for (int c = 0; c < kQ1; ++c) {
                T += g[b * kQ1 + c];
                Uc[c] += g[b * kQ1 + c];
            }
            sT[a][b][lane] = T;
            Sa += T;
        }
        sS[a][lane] = Sa;
#pragma unroll
        for (int c = 0; c < kQ1; ++c) sU[a][c][lane] = Uc[c];
    }
    __syncthreads();
    if (a == 0 && active) {
        float drho = 0.0f, jx = 0.0f, jy = 0.0f, jz = 0.0f, de = 0.0f;
#pragma unroll
        for (int i = 0; i < kQ1; ++i) {
            const float vi = (float)P.v[i];
            float Ti = 0.0f, Ui = 0.0f;
#pragma unroll
            for (int w = 0; w < kQ1; ++w) {
                Ti += sT[w][i][lane];
                Ui += sU[w][i][lane];
            }
            const float Si = sS[i][lane];
            drho += Si;
            jx += vi * Si;
            jy += vi * Ti;
            jz += vi * Ui;
            de += vi * vi * (Si + Ti + Ui);
        }
        const float rho = 1.0f + drho;
        const float ir = 1.0f / rho;
        const float ux = jx * ir, uy = jy * ir, uz = jz * ir;
        const float dth = ((de - 3.0f * P.theta0f * drho) * ir - (ux * ux + uy * uy + uz * uz)) * (1.0f / 3.0f);
        flag_status<float>(P, rho, P.theta0f + dth);
        sM[0][lane] = drho;
        sM[1][lane] = uy;
        sM[2][lane] = uz;
        sM[4][lane] = dth;
        float drx[kQ1];
        axis_dev(P, ux, dth, drx);
#pragma unroll
        for (int i = 0; i < kQ1; ++i) sDx[i][lane] = drx[i];
    }
    __syncthreads();
    // warp a forms row b = a of the factor table for its 32 nodes
    if (active) {
        const float dth = sM[4][lane];
        float dry[kQ1], drz[kQ1];
        axis_dev(P, sM[1][lane], dth, dry);
        axis_dev(P, sM[2][lane], dth, drz);
        const int b = a;
#pragma unroll
        for (int c = 0; c < kQ1; ++c) {
            const float rzc = P.w1f[c] + drz[c];
            sP[b][c][lane] = (P.w1f[b] + dry[b]) * rzc;
            sQ[b][c][lane] = dry[b] * rzc + P.w1f[b] * drz[c];
        }
    }
    __syncthreads();
    if (!active) return;
    const float drho = sM[0][lane];
    const float rho = 1.0f + drho;
    const float om = P.omegaf;
    const float X = om * fmaf(drho, P.w1f[a], rho * sDx[a][lane]);
    const float Wa = om * P.w1f[a];
    const float keep = 1.0f - om;
    const long long here = ((long long)z * P.ny + y) * P.pitch + x;
    const long long pa = (long long)a * kQ1 * kQ1 * P.plane;
#pragma unroll
    for (int b = 0; b < kQ1; ++b)
#pragma unroll
        for (int c = 0; c < kQ1; ++c) {
            const float d = fmaf(X, sP[b][c][lane], Wa * sQ[b][c][lane]);
            Storage<S>::store(dst + pa + (long long)(b * kQ1 + c) * P.plane + here, fmaf(keep, g[b * kQ1 + c], d));
        }
}

// Two packed 16-bit deviations <-> float2 (lane x = the node in the lower half).
template <typename S>
struct Pack2;

// unpack_again converts a second time in the collision (an asm statement, so the
// compiler keeps the 125 packed registers instead of 250 converted ones).
template <>
struct Pack2<__half> {
    static __device__ __forceinline__ float2 unpack(unsigned r) {
        __half2 h;
        memcpy(&h, &r, 4);
        return __half22float2(h);
    }
    static __device__ __forceinline__ float2 unpack_again(unsigned r) {
        float2 v;
        asm volatile("{\n\t.reg .f16 lo, hi;\n\tmov.b32 {lo, hi}, %2;\n\tcvt.f32.f16 %0, lo;\n\tcvt.f32.f16 %1, hi;\n\t}"
                     : "=f"(v.x), "=f"(v.y) : "r"(r));
        return v;
    }
    static __device__ __forceinline__ unsigned pack(float2 v) {
        const __half2 h = __float22half2_rn(v);
        unsigned r;
        memcpy(&r, &h, 4);
        return r;
    }
};

template <>
struct Pack2<__nv_bfloat16> {
    static __device__ __forceinline__ float2 unpack(unsigned r) {
        return make_float2(__uint_as_float(r << 16), __uint_as_float(r & 0xffff0000u));
    }
    static __device__ __forceinline__ float2 unpack_again(unsigned r) {
        unsigned lo, hi;
        asm volatile("shl.b32 %0, %2, 16;\n\tand.b32 %1, %2, 0xffff0000;" : "=r"(lo), "=r"(hi) : "r"(r));
        return make_float2(__uint_as_float(lo), __uint_as_float(hi));
    }
    static __device__ __forceinline__ unsigned pack(float2 v) {
        const __nv_bfloat162 h = __float22bfloat162_rn(v);
        unsigned r;
        memcpy(&r, &h, 4);
        return r;
    }
};

// axis_dev on both nodes of a pair.
__device__ __forceinline__ void axis_dev2(const LatticeParams& P, float2 u, float2 dth, float2 (&dr)[kQ1]) {
    const float2 th0 = f2s(P.theta0f);
    const float2 u2 = mul2(u, u);
    const float2 th = add2(th0, dth);
    const float2 dm1 = u;
    const float2 dm2 = add2(u2, dth);
    const float2 dm3 = mul2(u, fma2(f2s(3.0f), th, u2));
    const float2 dm4 = fma2(u2, fma2(f2s(6.0f), th, u2), mul2(mul2(f2s(3.0f), dth), add2(th, th0)));
    const float2 Ob = mul2(fma2(f2s(-P.sa2), dm1, dm3), f2s(P.kOb));
    const float2 Oa = mul2(fma2(f2s(-2.0f * P.sb), Ob, dm1), f2s(P.kOa));
    const float2 Eb = mul2(fma2(f2s(-P.sa2), dm2, dm4), f2s(P.kEb));
    const float2 Ea = mul2(fma2(f2s(-2.0f * P.sb2), Eb, dm2), f2s(P.kEa));
    dr[0] = mul2(f2s(-2.0f), add2(Ea, Eb));
    dr[1] = add2(Ea, Oa);
    dr[2] = sub2(Ea, Oa);
    dr[3] = add2(Eb, Ob);
    dr[4] = sub2(Eb, Ob);
}

// Both nodes of pair row r at column x.  WRAP: some pull of z crosses the wrap
// (r < max|v| or r >= nz/2 - max|v|), so the lanes of those loads are swapped;
// pair rows away from the wrap (all but 2 max|v| of them) take the WRAP = false
// copy without the per-load lane test.
template <typename S, bool WRAP>
__device__ __forceinline__ void zpair_update(const LatticeParams& P, const unsigned* __restrict__ s32,
                                             unsigned* __restrict__ d32, int x, int y, int r) {
    const int H = P.half_nz;
    int xs[kQ1], ys[kQ1], zr[kQ1];
    bool sw[kQ1];
#pragma unroll
    for (int i = 0; i < kQ1; ++i) {
        xs[i] = wrap_add(x, P.vxm[i], P.nx);
        ys[i] = wrap_add(y, P.vym[i], P.ny);
        const int zs = r - P.v[i];             // |v| <= nz/2 (checked on the host)
        sw[i] = zs < 0 || zs >= H;
        zr[i] = zs < 0 ? zs + H : (zs >= H ? zs - H : zs);
    }
    // Offsets in pairs fit 32 bits (the host sends larger lattices to the plain kernel).
    const unsigned plane = (unsigned)(P.plane >> 1);   // pairs per population plane
    unsigned g[kQ3];
#pragma unroll
    for (int b = 0; b < kQ1; ++b)
#pragma unroll
        for (int c = 0; c < kQ1; ++c) {
            const unsigned row = ((unsigned)zr[c] * P.ny + ys[b]) * P.pitch;   // in pairs
#pragma unroll
            for (int a = 0; a < kQ1; ++a) {
                const int p = (a * kQ1 + b) * kQ1 + c;
                const unsigned v = __ldg(s32 + (p * plane + row + xs[a]));
                g[p] = (WRAP && sw[c]) ? __byte_perm(v, 0u, 0x1032) : v;
            }
        }
    // Row sums: R_ab = sum_c g, S_a = sum_b R_ab, T_b = sum_a R_ab, U_c = sum_ab g.
    float2 Sa[kQ1], Tb[kQ1], Uc[kQ1];
#pragma unroll
    for (int i = 0; i < kQ1; ++i) Sa[i] = Tb[i] = Uc[i] = f2s(0.0f);
#pragma unroll
    for (int a = 0; a < kQ1; ++a)
#pragma unroll
        for (int b = 0; b < kQ1; ++b) {
            float2 R = f2s(0.0f);
#pragma unroll
            for (int c = 0; c < kQ1; ++c) {
                const float2 v = Pack2<S>::unpack(g[(a * kQ1 + b) * kQ1 + c]);
                R = add2(R, v);
                Uc[c] = add2(Uc[c], v);
            }
            Sa[a] = add2(Sa[a], R);
            Tb[b] = add2(Tb[b], R);
        }
    float2 drho = f2s(0.0f), jx = drho, jy = drho, jz = drho, de = drho;
#pragma unroll
    for (int i = 0; i < kQ1; ++i) {
        const float2 vi = f2s((float)P.v[i]);
        drho = add2(drho, Sa[i]);
        jx = fma2(vi, Sa[i], jx);
        jy = fma2(vi, Tb[i], jy);
        jz = fma2(vi, Uc[i], jz);
        de = fma2(mul2(vi, vi), add2(add2(Sa[i], Tb[i]), Uc[i]), de);
    }
    const float2 rho = add2(f2s(1.0f), drho);
    const float2 ir = f2(1.0f / rho.x, 1.0f / rho.y);
    const float2 ux = mul2(jx, ir), uy = mul2(jy, ir), uz = mul2(jz, ir);
    const float2 uu = fma2(ux, ux, fma2(uy, uy, mul2(uz, uz)));
    const float2 dth = mul2(sub2(mul2(fma2(f2s(-3.0f * P.theta0f), drho, de), ir), uu), f2s(1.0f / 3.0f));
    flag_status<float>(P, rho.x, P.theta0f + dth.x);
    flag_status<float>(P, rho.y, P.theta0f + dth.y);
    float2 drx[kQ1], dry[kQ1], drz[kQ1];
    axis_dev2(P, ux, dth, drx);
    axis_dev2(P, uy, dth, dry);
    axis_dev2(P, uz, dth, drz);
    // g' = (1 - omega) g + omega (f^eq - w0), with omega folded into the x factors:
    // omega (f^eq - w0) = X_a P_bc + W_a Q_bc, X_a = omega (rho r^x_a - w_a), W_a = omega w_a.
    const float2 om = f2s(P.omegaf);
    float2 X[kQ1];
#pragma unroll
    for (int a = 0; a < kQ1; ++a) X[a] = mul2(om, fma2(drho, f2s(P.w1f[a]), mul2(rho, drx[a])));
    const float2 keep = f2s(1.0f - P.omegaf);
    const unsigned here = ((unsigned)r * P.ny + y) * P.pitch + x;   // in pairs
#pragma unroll
    for (int b = 0; b < kQ1; ++b)
#pragma unroll
        for (int c = 0; c < kQ1; ++c) {
            const float2 rzc = add2(f2s(P.w1f[c]), drz[c]);
            const float2 Pbc = mul2(add2(f2s(P.w1f[b]), dry[b]), rzc);
            const float2 Qbc = fma2(dry[b], rzc, mul2(f2s(P.w1f[b]), drz[c]));
#pragma unroll
            for (int a = 0; a < kQ1; ++a) {
                const int p = (a * kQ1 + b) * kQ1 + c;
                const float2 gp = Pack2<S>::unpack_again(g[p]);
                const float2 d = fma2(X[a], Pbc, mul2(f2s(P.omegaf * P.w1f[a]), Qbc));
                d32[p * plane + here] = Pack2<S>::pack(fma2(keep, gp, d));   // 32-bit index
            }
        }
}

// 64-thread CTAs with no minimum-residency hint: the same 8 warps per SM as
// 128-thread CTAs with a hint of two, fewer spilled registers and a finer
// refill of the SM as CTAs finish (1,614 / 1,597 us against 1,688 / 1,688 us
// per FP16 / BF16 step at 256^3; 32-thread CTAs 1,668 / 1,659 us).
constexpr int kZpairBlock = 64;

template <typename S>
__global__ void __launch_bounds__(kZpairBlock) k_stream_collide3_zpair(const __grid_constant__ LatticeParams P,
                                                                      const S* __restrict__ src,
                                                                      S* __restrict__ dst) {
    const int x = blockIdx.x * kZpairBlock + threadIdx.x;
    const int y = blockIdx.y, r = blockIdx.z;   // pair row r: nodes z = r and z = r + nz/2
    if (x >= P.nx) return;
    bool wrap = false;
#pragma unroll
    for (int i = 0; i < kQ1; ++i) wrap |= (r - P.v[i] < 0) || (r - P.v[i] >= P.half_nz);
    const unsigned* s32 = reinterpret_cast<const unsigned*>(src);
    unsigned* d32 = reinterpret_cast<unsigned*>(dst);
    if (wrap)
        zpair_update<S, true>(P, s32, d32, x, y, r);
    else
        zpair_update<S, false>(P, s32, d32, x, y, r);
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

// FP64, compile-time q1 (3 or 5), in two passes over the pulled values so that
// no thread holds all q1^3 of them: the first forms the row sums
// R_ab = sum_c f, S_a, T_b, U_c; the second loads them again (L1/L2 hits) and
// writes f' = (1 - omega) f + (omega rho r^x_a r^y_b) r^z_c.  The same formulas
// as k_stream_collide3_f64 (moments, C mu rule), with the sums factorised.
__device__ __forceinline__ double ldg_again(const double* p) {
    double v;
    asm volatile("ld.global.nc.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}

template <int Q1>
__device__ __forceinline__ void rule_q(const LatticeParams& P, double u, double th, double (&r)[Q1]) {
    double mu[Q1];
    mu[0] = 1.0;
    mu[1] = u;
#pragma unroll
    for (int n = 1; n + 1 < Q1; ++n) mu[n + 1] = u * mu[n] + (double)n * th * mu[n - 1];
#pragma unroll
    for (int i = 0; i < Q1; ++i) {
        double t = 0.0;
#pragma unroll
        for (int n = 0; n < Q1; ++n) t += P.C[i * Q1 + n] * mu[n];
        r[i] = t;
    }
}

template <int Q1>
__global__ void __launch_bounds__(kB3) k_stream_collide3_f64q(const __grid_constant__ LatticeParams P,
                                                              const double* __restrict__ src,
                                                              double* __restrict__ dst) {
    const int x = blockIdx.x * kB3 + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= P.nx) return;
    // element offsets within a plane fit 32 bits (a plane is at most the device memory / 2 q^3 sizeof)
    int xs[Q1], yr[Q1], zr[Q1];
#pragma unroll
    for (int i = 0; i < Q1; ++i) {
        xs[i] = wrap_add(x, P.vxm[i], P.nx);
        yr[i] = wrap_add(y, P.vym[i], P.ny) * P.pitch;
        zr[i] = wrap_add(z, P.vzm[i], P.nz) * P.ny * P.pitch;
    }
    double Sa[Q1], Tb[Q1], Uc[Q1];
#pragma unroll
    for (int i = 0; i < Q1; ++i) Sa[i] = Tb[i] = Uc[i] = 0.0;
#pragma unroll
    for (int a = 0; a < Q1; ++a)
#pragma unroll
        for (int b = 0; b < Q1; ++b) {
            double R = 0.0;
#pragma unroll
            for (int c = 0; c < Q1; ++c) {
                const int p = (a * Q1 + b) * Q1 + c;
                const double v = __ldg(src + (long long)p * P.plane + (zr[c] + yr[b] + xs[a]));
                R += v;
                Uc[c] += v;
            }
            Sa[a] += R;
            Tb[b] += R;
        }
    double m0 = 0.0, mx = 0.0, my = 0.0, mz = 0.0, en = 0.0;
#pragma unroll
    for (int i = 0; i < Q1; ++i) {
        const double vi = (double)P.v[i];
        m0 += Sa[i];
        mx += vi * Sa[i];
        my += vi * Tb[i];
        mz += vi * Uc[i];
        en += vi * vi * (Sa[i] + Tb[i] + Uc[i]);
    }
    const double ux = mx / m0, uy = my / m0, uz = mz / m0;
    const double th = (en / m0 - (ux * ux + uy * uy + uz * uz)) / 3.0;
    flag_status<double>(P, m0, th);
    const double the = P.isothermal ? P.theta0 : th;
    double ra[Q1], rb[Q1], rc[Q1];
    rule_q<Q1>(P, ux, the, ra);
    rule_q<Q1>(P, uy, the, rb);
    rule_q<Q1>(P, uz, the, rc);
    const double om = P.omega, keep = 1.0 - om;
    const long long here = ((long long)z * P.ny + y) * P.pitch + x;
    long long plane2 = P.plane;   // fresh index terms: the second pass recomputes its addresses
    asm volatile("" : "+l"(plane2));
#pragma unroll
    for (int i = 0; i < Q1; ++i) asm volatile("" : "+r"(xs[i]), "+r"(yr[i]), "+r"(zr[i]));
#pragma unroll
    for (int a = 0; a < Q1; ++a)
#pragma unroll
        for (int b = 0; b < Q1; ++b) {
            const double X = om * m0 * ra[a] * rb[b];
#pragma unroll
            for (int c = 0; c < Q1; ++c) {
                const int p = (a * Q1 + b) * Q1 + c;
                const double f = ldg_again(src + (long long)p * plane2 + (zr[c] + yr[b] + xs[a]));
                dst[(long long)p * plane2 + here] = fma(keep, f, X * rc[c]);
            }
        }
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
    const long long here = node3(P, x, y, z);
    for (int p = 0; p < P.q; ++p) f[(long long)p * P.plane + here] = Storage<S>::from_f64(fe[p], w0_3(P, p));
}

template <typename S>
__global__ void k_moments3(const __grid_constant__ LatticeParams P, const S* __restrict__ f, double* rho,
                           double* ux, double* uy, double* uz, double* theta) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= P.nx) return;
    const long long here = node3(P, x, y, z);
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
        const long long here = node3(P, x, y, z);
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

// The same record for 16/32-bit storage with q1 = 5 on the FP32 pipe: row sums
// of the stored deviations in float-float (R_ab = sum_c g, S_a, T_b, U_c),
// mass - 1, j, E - 3 theta0 per node, block sums in float-float, and the FP64
// minima of rho and theta reduced as order-preserving integer keys.
template <typename S>
__global__ void __launch_bounds__(kB3) k_reduce3_dev(const __grid_constant__ LatticeParams P, const S* __restrict__ f) {
    __shared__ float sh[11][kB3 / 32];
    __shared__ long long shk[2][kB3 / 32];
    const int x = blockIdx.x * kB3 + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    FF dm{0.f, 0.f}, jx = dm, jy = dm, jz = dm, de = dm;
    float n = 0.0f;
    long long kr = dkey(1e300), kt = dkey(1e300);
    if (x < P.nx) {
        const long long here = node3(P, x, y, z);
        FF Sa[kQ1], Tb[kQ1], Uc[kQ1];
#pragma unroll
        for (int i = 0; i < kQ1; ++i) Sa[i] = Tb[i] = Uc[i] = FF{0.f, 0.f};
#pragma unroll
        for (int a = 0; a < kQ1; ++a)
#pragma unroll
            for (int b = 0; b < kQ1; ++b) {
                FF R{0.f, 0.f};
#pragma unroll
                for (int c = 0; c < kQ1; ++c) {
                    const float g = Storage<S>::load(f + (long long)((a * kQ1 + b) * kQ1 + c) * P.plane + here);
                    R = ff_add(R, g);
                    Uc[c] = ff_add(Uc[c], g);
                }
                Sa[a] = ff_add(Sa[a], R);
                Tb[b] = ff_add(Tb[b], R);
            }
#pragma unroll
        for (int i = 0; i < kQ1; ++i) {
            const float vi = (float)P.v[i];
            dm = ff_add(dm, Sa[i]);
            jx = ff_add(jx, ff_scale(Sa[i], vi));
            jy = ff_add(jy, ff_scale(Tb[i], vi));
            jz = ff_add(jz, ff_scale(Uc[i], vi));
            de = ff_add(de, ff_scale(ff_scale(ff_add(ff_add(Sa[i], Tb[i]), Uc[i]), vi), vi));
        }
        const double rho = 1.0 + ff_f64(dm);
        const double ir = 1.0 / rho;
        const double ux = ff_f64(jx) * ir, uy = ff_f64(jy) * ir, uz = ff_f64(jz) * ir;
        const double th = ((3.0 * P.theta0 + ff_f64(de)) * ir - (ux * ux + uy * uy + uz * uz)) / 3.0;
        flag_status<double>(P, rho, th);
        n = 1.0f;
        kr = dkey(rho);
        kt = dkey(th);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        dm = ff_add(dm, ff_shfl_down(dm, off));
        jx = ff_add(jx, ff_shfl_down(jx, off));
        jy = ff_add(jy, ff_shfl_down(jy, off));
        jz = ff_add(jz, ff_shfl_down(jz, off));
        de = ff_add(de, ff_shfl_down(de, off));
        n += __shfl_down_sync(0xffffffffu, n, off);
        kr = kmin(kr, __shfl_down_sync(0xffffffffu, kr, off));
        kt = kmin(kt, __shfl_down_sync(0xffffffffu, kt, off));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        const FF v[5] = {dm, jx, jy, jz, de};
        for (int k = 0; k < 5; ++k) {
            sh[2 * k][warp] = v[k].hi;
            sh[2 * k + 1][warp] = v[k].lo;
        }
        sh[10][warp] = n;
        shk[0][warp] = kr;
        shk[1][warp] = kt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        FF t[5] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        float nn = 0.0f;
        long long r = shk[0][0], q = shk[1][0];
        for (int w = 0; w < kB3 / 32; ++w) {
            for (int k = 0; k < 5; ++k) t[k] = ff_add(t[k], FF{sh[2 * k][w], sh[2 * k + 1][w]});
            nn += sh[10][w];
            r = kmin(r, shk[0][w]);
            q = kmin(q, shk[1][w]);
        }
        const long long blk = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        double* out = P.partials + blk * kPartialStride;
        out[0] = (double)nn + ff_f64(t[0]);
        out[1] = ff_f64(t[1]);
        out[2] = ff_f64(t[2]);
        out[3] = (double)nn * 3.0 * P.theta0 + ff_f64(t[4]);
        out[4] = dunkey(r);
        out[5] = dunkey(q);
        out[6] = ff_f64(t[3]);
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
    const long long here = node3(P, x, y, z);
    const long long vol = (long long)P.nx * P.ny * P.nz;
    const long long n = ((long long)z * P.ny + y) * P.nx + x;
    for (int p = 0; p < P.q; ++p) out[p * vol + n] = Storage<S>::to_f64(f[(long long)p * P.plane + here], w0_3(P, p));
}

template <typename S>
__global__ void k_set_pop3(const __grid_constant__ LatticeParams P, const double* __restrict__ in, S* __restrict__ f) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= P.nx) return;
    const long long here = node3(P, x, y, z);
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
        const double* a = static_cast<const double*>(src);
        double* b = static_cast<double*>(dst);
        if (P.q1 == 5)
            k_stream_collide3_f64q<5><<<grid3(P), kB3, 0, s>>>(P, a, b);
        else if (P.q1 == 3)
            k_stream_collide3_f64q<3><<<grid3(P), kB3, 0, s>>>(P, a, b);
        else
            k_stream_collide3_f64<<<grid3(P), kB3, 0, s>>>(P, a, b);
        return cudaGetLastError();
    }
    if (!P.sym5 || P.q1 != kQ1 || P.isothermal) return cudaErrorInvalidValue;
    if (P.zpaired) {
        const dim3 g((P.nx + kZpairBlock - 1) / kZpairBlock, P.ny, P.half_nz);
        if (prec == kF16Dev)
            k_stream_collide3_zpair<__half><<<g, kZpairBlock, 0, s>>>(P, static_cast<const __half*>(src),
                                                                       static_cast<__half*>(dst));
        else if (prec == kBF16Dev)
            k_stream_collide3_zpair<__nv_bfloat16><<<g, kZpairBlock, 0, s>>>(
                P, static_cast<const __nv_bfloat16*>(src), static_cast<__nv_bfloat16*>(dst));
        else
            return cudaErrorInvalidValue;
        return cudaGetLastError();
    }
    switch (prec) {
        case kF32:
            k_stream_collide3_split<float><<<dim3((P.nx + kSplitNodes - 1) / kSplitNodes, P.ny, P.nz), kSplitThreads, 0,
                                              s>>>(P, static_cast<const float*>(src), static_cast<float*>(dst));
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
    if (prec != kF64 && P.q1 == kQ1) {
        switch (prec) {
            case kF32: k_reduce3_dev<float><<<grid3(P), kB3, 0, s>>>(P, static_cast<const float*>(f)); break;
            case kF16Dev: k_reduce3_dev<__half><<<grid3(P), kB3, 0, s>>>(P, static_cast<const __half*>(f)); break;
            case kBF16Dev:
                k_reduce3_dev<__nv_bfloat16><<<grid3(P), kB3, 0, s>>>(P, static_cast<const __nv_bfloat16*>(f));
                break;
            default: return cudaErrorInvalidValue;
        }
    } else {
        PLBM_DISPATCH3(prec, (k_reduce3<S><<<grid3(P), kB3, 0, s>>>(P, static_cast<const S*>(f))));
    }
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
