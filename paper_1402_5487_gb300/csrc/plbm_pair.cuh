// Fast stream-and-collide for 2D symmetric five-velocity sets
// (D2Q25 = D1Q5 x D1Q5 with v = (0, a, -a, b, -b), Sec. 2.4 and Sec. 4),
// periodic, FP32 / FP16 / BF16 deviation storage, FP32 arithmetic.
//
// Each thread updates the two nodes (x, r) and (x, r + ny/2), which the
// row-paired layout stores side by side: every pull f_p(x - v_p) of both
// nodes is one aligned 8-byte (FP32) or 4-byte (16-bit) vector load, and every
// store one vector store.  The two nodes travel through the collision as the
// two lanes of float2 values, so the arithmetic issues as Blackwell packed
// FP32x2 instructions (fma/add/mul .f32x2).
//
// Pull across the y wrap: node (x, r) reads row s = (r - v_y) mod ny and node
// (x, r + H) reads (s + H) mod ny.  When s < H the pair row s holds them in
// lane order; when s >= H the pair row s - H holds them swapped.
//
// Equilibrium in constraint form.  For v = (0, +-a, +-b) the deviation
// dr = r(u, theta) - r(0, theta0) of Eq. (eq:rdr) splits into an odd part
// (O_a for +-a, O_b for +-b) and an even part (E_0, E_a, E_b) fixed by the
// moment identities sum v^n dr = dmu_n (n = 0..4):
//   O_b = (dmu_3 - a^2 dmu_1) / (2b(b^2 - a^2)),   O_a = (dmu_1 - 2b O_b) / (2a),
//   E_b = (dmu_4 - a^2 dmu_2) / (2b^2(b^2 - a^2)), E_a = (dmu_2 - 2b^2 E_b) / (2a^2),
//   E_0 = -2 (E_a + E_b),   dr_(+-a) = E_a +- O_a,   dr_(+-b) = E_b +- O_b.
// Written this way the conserved moments (n = 0, 1, 2) hold up to the rounding
// of the last operations, whatever the rounding of the constant factors, so
// FP32 collisions conserve mass, momentum and energy without a systematic drift.
#pragma once

#include <type_traits>

#include "plbm_device.cuh"
#include "plbm_internal.h"

namespace plbm {

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 f2s(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, f2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// The same operations on one node (plain layout): each is the single-lane form of
// the packed one above, correctly rounded and never contracted, so a node gets
// bit for bit the same result whichever layout and kernel update it.
__device__ __forceinline__ float add2(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub2(float a, float b) { return __fadd_rn(a, -b); }
__device__ __forceinline__ float mul2(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fma2(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <class V>
__device__ __forceinline__ V splat(float a);
template <>
__device__ __forceinline__ float2 splat<float2>(float a) { return f2s(a); }
template <>
__device__ __forceinline__ float splat<float>(float a) { return a; }
__device__ __forceinline__ float2 neg2(float2 a) { return f2(-a.x, -a.y); }
__device__ __forceinline__ float neg2(float a) { return -a; }
__device__ __forceinline__ float2 rcp2(float2 a) { return f2(__frcp_rn(a.x), __frcp_rn(a.y)); }
__device__ __forceinline__ float rcp2(float a) { return __frcp_rn(a); }

// Storage of one node pair.
template <typename S>
struct PairStore;

template <>
struct PairStore<float> {
    using V = float2;
    static constexpr bool kReconvert = false;
    static __device__ __forceinline__ void store(V* p, float2 v) { *p = v; }
    static __device__ __forceinline__ V raw(const V* p) { return __ldg(p); }
    static __device__ __forceinline__ V swap(V v) { return f2(v.y, v.x); }
    static __device__ __forceinline__ float2 cvt(V v) { return v; }
    static __device__ __forceinline__ float2 cvt_again(V v) { return v; }
};

// FP16 pairs are converted once, at the load.  BF16 pairs stay packed in
// registers between the moment sums and the collision (kReconvert): cvt_again
// converts a second time through an asm statement, which the compiler cannot
// merge with the first conversion, so 25 packed registers are live across the
// equilibrium instead of 50 converted ones and seven CTAs fit per SM.  For FP16,
// whose conversion costs more, the same measured slower (56.7 k against 58.4 k
// MLUPS at 2048^2); for BF16 it gains 1.7 % (60.1 k against 59.1 k).
template <>
struct PairStore<__half> {
    using V = __half2;
    static constexpr bool kReconvert = false;
    static __device__ __forceinline__ void store(V* p, float2 v) { *p = __float22half2_rn(v); }
    static __device__ __forceinline__ V raw(const V* p) { return __ldg(p); }
    static __device__ __forceinline__ V swap(V v) { return __lowhigh2highlow(v); }
    static __device__ __forceinline__ float2 cvt(V v) { return __half22float2(v); }
    static __device__ __forceinline__ float2 cvt_again(V v) { return cvt(v); }
};

template <>
struct PairStore<__nv_bfloat16> {
    using V = __nv_bfloat162;
    static constexpr bool kReconvert = true;
    static __device__ __forceinline__ void store(V* p, float2 v) { *p = __float22bfloat162_rn(v); }
    static __device__ __forceinline__ V raw(const V* p) { return __ldg(p); }
    static __device__ __forceinline__ V swap(V v) { return __lowhigh2highlow(v); }
    static __device__ __forceinline__ float2 cvt(V v) { return __bfloat1622float2(v); }
    static __device__ __forceinline__ float2 cvt_again(V v) {
        unsigned r, lo, hi;
        memcpy(&r, &v, 4);
        asm volatile("shl.b32 %0, %2, 16;\n\tand.b32 %1, %2, 0xffff0000;" : "=r"(lo), "=r"(hi) : "r"(r));
        return f2(__uint_as_float(lo), __uint_as_float(hi));
    }
};

// dmu_1..dmu_4 = mu_n(u, theta) - mu_n(0, theta0) from mu_{n+1} = u mu_n + n theta mu_{n-1}
// with mu(0, theta0) = (1, 0, theta0, 0, 3 theta0^2), then dr by the constraint form.
// V = float2: the two nodes of a pair; V = float: one node.
template <class V>
__device__ __forceinline__ void sym5_axis(const PairParams& P, V u, V th, V dth, V (&dr)[5]) {
    const V th0 = splat<V>(P.theta0f);
    const V d1 = u;
    const V d2 = fma2(u, u, dth);
    const V d3 = mul2(u, add2(add2(th0, d2), add2(th, th)));
    const V d4 = fma2(u, d3, mul2(splat<V>(3.0f), fma2(th, d2, mul2(dth, th0))));
    const V Ob = mul2(fma2(splat<V>(-P.sa2), d1, d3), splat<V>(P.kOb));
    const V Oa = mul2(fma2(splat<V>(-2.0f * P.sb), Ob, d1), splat<V>(P.kOa));
    const V Eb = mul2(fma2(splat<V>(-P.sa2), d2, d4), splat<V>(P.kEb));
    const V Ea = mul2(fma2(splat<V>(-2.0f * P.sb2), Eb, d2), splat<V>(P.kEa));
    dr[0] = mul2(splat<V>(-2.0f), add2(Ea, Eb));
    dr[1] = add2(Ea, Oa);
    dr[2] = sub2(Ea, Oa);
    dr[3] = add2(Eb, Ob);
    dr[4] = sub2(Eb, Ob);
}

// sum(p), col(p): pulled deviation p of the node(s), read for the moment sums
// and for the collision; out: post-collision deviations.  Returns rho and theta
// (for the status check and reductions).
template <class V, class GetSum, class GetCol>
__device__ __forceinline__ void sym5_collide(const PairParams& P, GetSum sum, GetCol col, V (&out)[25], V& rho_o,
                                             V& th_o, V& drho_o, V& jx_o, V& jy_o, V& e_o) {
    V S[5], T[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        S[i] = add2(add2(sum(5 * i), sum(5 * i + 1)), add2(add2(sum(5 * i + 2), sum(5 * i + 3)), sum(5 * i + 4)));
    }
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        T[j] = add2(add2(sum(j), sum(5 + j)), add2(add2(sum(10 + j), sum(15 + j)), sum(20 + j)));
    }
    const V a = splat<V>(P.sa), b = splat<V>(P.sb), a2 = splat<V>(P.sa2), b2 = splat<V>(P.sb2);
    const V drho = add2(add2(S[0], S[1]), add2(add2(S[2], S[3]), S[4]));
    const V jx = fma2(a, sub2(S[1], S[2]), mul2(b, sub2(S[3], S[4])));
    const V ex = fma2(a2, add2(S[1], S[2]), mul2(b2, add2(S[3], S[4])));
    const V jy = fma2(a, sub2(T[1], T[2]), mul2(b, sub2(T[3], T[4])));
    const V ey = fma2(a2, add2(T[1], T[2]), mul2(b2, add2(T[3], T[4])));
    const V rho = add2(splat<V>(1.0f), drho);
    const V inv = rcp2(rho);
    const V ux = mul2(jx, inv), uy = mul2(jy, inv);
    const V uu = fma2(ux, ux, mul2(uy, uy));
    // 2 rho theta = 2 theta0 + sum |v|^2 g - rho |u|^2  =>  theta - theta0:
    const V dth = mul2(splat<V>(0.5f), fma2(fma2(splat<V>(-2.0f * P.theta0f), drho, add2(ex, ey)), inv, neg2(uu)));
    const V th = add2(splat<V>(P.theta0f), dth);
    rho_o = rho;
    th_o = th;
    drho_o = drho;
    jx_o = jx;
    jy_o = jy;
    e_o = add2(ex, ey);

    V dx[5], dy[5];
    sym5_axis(P, ux, th, dth, dx);
    sym5_axis(P, uy, th, dth, dy);

    // g' = (1 - omega) g + omega (f^eq - w0) with
    // f^eq - w0 = drho w_i w_j + rho (dx_i r^y_j + w_i dy_j),  r^y_j = w_j + dy_j:
    //   g'_ij = (1 - omega) g_ij + A_i r^y_j + w_i Y_j,
    //   A_i = omega rho dx_i,  Y_j = omega (rho dy_j + drho w_j).
    const V om = splat<V>(P.omegaf);
    const V orho = mul2(om, rho);
    const V odrho = mul2(om, drho);
    const V keep = splat<V>(1.0f - P.omegaf);
    V ry[5], Y[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        ry[j] = add2(splat<V>(P.w1f[j]), dy[j]);
        Y[j] = fma2(orho, dy[j], mul2(odrho, splat<V>(P.w1f[j])));
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const V A = mul2(orho, dx[i]);
        const V w = splat<V>(P.w1f[i]);
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            const int p = 5 * i + j;
            out[p] = fma2(keep, col(p), fma2(A, ry[j], mul2(w, Y[j])));
        }
    }
}

__device__ __forceinline__ bool healthy2(float2 rho, float2 th) {
    // false for NaN, infinities and non-positive values (NaN compares false)
    return (rho.x > 0.0f) & (rho.y > 0.0f) & (th.x > 0.0f) & (th.y > 0.0f) &
           (rho.x < 3.0e38f) & (rho.y < 3.0e38f) & (th.x < 3.0e38f) & (th.y < 3.0e38f);
}

// The 25 pulls of a node pair (lane order fixed up across the y wrap), each
// passed through conv on its way into dst.
template <typename PS, typename T, class Conv>
__device__ __forceinline__ void pull25(const typename PS::V* __restrict__ src, long long plane2,
                                       const unsigned (&row)[5], const unsigned (&col)[5], const bool (&swp)[5],
                                       bool any_swap, T (&dst)[25], Conv conv) {
    if (!any_swap) {
#pragma unroll
        for (int i = 0; i < 5; ++i)
#pragma unroll
            for (int j = 0; j < 5; ++j) {
                const int p = 5 * i + j;
                dst[p] = conv(PS::raw(src + p * plane2 + (row[j] + col[i])));
            }
    } else {
#pragma unroll
        for (int i = 0; i < 5; ++i)
#pragma unroll
            for (int j = 0; j < 5; ++j) {
                const int p = 5 * i + j;
                const typename PS::V a = PS::raw(src + p * plane2 + (row[j] + col[i]));
                dst[p] = conv(swp[j] ? PS::swap(a) : a);
            }
    }
}

// Collision and store of the node pair (x, r) and (x, r + ny/2) of one lattice,
// x < nx; pull(v, conv) fills v[p] with conv(pulled pair p) in lane order.
template <typename S, bool REDUCE, class Pull>
__device__ __forceinline__ void pair_update(const PairParams& P, Pull pull, typename PairStore<S>::V* __restrict__ dst,
                                            int x, int r, NodeDiagF& d) {
    using PS = PairStore<S>;
    float2 rho, th, drho, jx, jy, e;
    float2 o[25];
    if constexpr (PS::kReconvert) {
        typename PS::V v[25];
        pull(v, [](typename PS::V a) { return a; });
        sym5_collide<float2>(P, [&](int p) { return PS::cvt(v[p]); }, [&](int p) { return PS::cvt_again(v[p]); },
                             o, rho, th, drho, jx, jy, e);
    } else {
        pull(o, [](typename PS::V a) { return PS::cvt(a); });
        sym5_collide<float2>(P, [&](int p) { return o[p]; }, [&](int p) { return o[p]; }, o, rho, th, drho, jx, jy,
                             e);
    }
    if (!healthy2(rho, th)) {
        unsigned bits = 0u;
        bits |= (!(rho.x == rho.x) || !(rho.y == rho.y) || !(th.x == th.x) || !(th.y == th.y) ||
                 !(rho.x < 3.0e38f) || !(rho.y < 3.0e38f) || !(th.x < 3.0e38f) || !(th.y < 3.0e38f))
                    ? 1u : 0u;
        bits |= (rho.x <= 0.0f || rho.y <= 0.0f) ? 2u : 0u;
        bits |= (th.x <= 0.0f || th.y <= 0.0f) ? 4u : 0u;
        atomicOr(P.status, bits);
    }
    if (REDUCE) {   // two nodes: deviations from the rest state in float-float
        d.dmass = ff_add(FF{drho.x, 0.0f}, drho.y);
        d.jx = ff_add(FF{jx.x, 0.0f}, jx.y);
        d.jy = ff_add(FF{jy.x, 0.0f}, jy.y);
        d.denergy = ff_add(FF{e.x, 0.0f}, e.y);
        d.rho_min = fminf(rho.x, rho.y);
        d.theta_min = fminf(th.x, th.y);
        d.n = 2.0f;
    }
    const unsigned here = (unsigned)(r * P.pitch + x);
#pragma unroll
    for (int p = 0; p < 25; ++p) PS::store(dst + p * P.plane2 + here, o[p]);
}

// Pull addresses of the node pair (x, r): col[i] = (x - v_x,i) mod nx, row[j] =
// pitch times the pair row that holds (r - v_y,j) mod ny; bit j of the result is
// set when that pair row holds the two nodes swapped (pulls across the y wrap).
__device__ __forceinline__ unsigned pair_pull_index(const PairParams& P, int x, int r, unsigned (&row)[5],
                                                    unsigned (&col)[5]) {
    const int H = P.half_ny;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const int s = x + P.vxm[i];
        col[i] = (unsigned)((s >= P.nx) ? s - P.nx : s);
    }
    unsigned swp = 0u;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        int s = r + P.vym[j];
        s = (s >= P.ny) ? s - P.ny : s;
        const bool w = s >= H;
        swp |= (w ? 1u : 0u) << j;
        row[j] = (unsigned)((w ? s - H : s) * P.pitch);
    }
    return swp;
}

// One thread's work: nodes (x, r) and (x, r + ny/2) of one lattice, x < nx.
template <typename S, bool REDUCE>
__device__ __forceinline__ void pair_node(const PairParams& P, const typename PairStore<S>::V* __restrict__ src,
                                          typename PairStore<S>::V* __restrict__ dst, int x, int r,
                                          NodeDiagF& d) {
    using PS = PairStore<S>;
    unsigned col[5], row[5];
    const unsigned m = pair_pull_index(P, x, r, row, col);
    bool swp[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) swp[j] = (m >> j) & 1u;
    pair_update<S, REDUCE>(
        P, [&](auto& v, auto conv) { pull25<PS>(src, P.plane2, row, col, swp, m != 0u, v, conv); }, dst, x, r, d);
}

// ---------------------------------------------------------------------------
// FP16 pairs, two tiles per thread.  A thread that updates one node pair keeps
// only its 25 x 4 bytes of pulls in flight and then computes with none; FP16
// pairs, converted at the load (94 registers), fit only 20 warps per SM, too few
// to cover the DRAM latency that way.  Here a thread issues the pulls of two
// node pairs (tiles t and t + 1 of kPair2Block x-consecutive pairs of a pair
// row, t = pair row * tiles_x + tile column) before it collides the first, so
// the second pair's loads stay in flight through the first pair's arithmetic:
// 125 registers, 16 warps per SM, each with twice the bytes outstanding.  The
// arithmetic is pair_update's, so the state is bit-identical to the one-pair
// kernel's.  (Measured at 2048^2: 67.7 against 71.7 us per step.  The same for
// BF16 pairs, kept packed at 72 registers and 28 warps per SM, measured slower,
// 76.7 against 69.7 us, and so did staging the pulls through shared memory
// with 4-byte cp.async for either type, 79-84 us.)
// ---------------------------------------------------------------------------
constexpr int kPair2Block = 64;

template <typename S>
__global__ void __launch_bounds__(kPair2Block)
k_stream_collide_pair2(const __grid_constant__ PairParams P, const typename PairStore<S>::V* __restrict__ src,
                       typename PairStore<S>::V* __restrict__ dst, int tiles_x, int ntiles) {
    using PS = PairStore<S>;
    using V = typename PS::V;
    const int t0 = 2 * blockIdx.x;
    const int ra = t0 / tiles_x;
    const int xa = (t0 - ra * tiles_x) * kPair2Block + threadIdx.x;
    int rb = 0, xb = P.nx;
    if (t0 + 1 < ntiles) {
        rb = (t0 + 1) / tiles_x;
        xb = (t0 + 1 - rb * tiles_x) * kPair2Block + threadIdx.x;
    }
    V va[25], vb[25];
    unsigned ma = 0u, mb = 0u;
    auto load = [&](int x, int r, V (&v)[25]) {
        unsigned col[5], row[5];
        const unsigned m = pair_pull_index(P, x, r, row, col);
#pragma unroll
        for (int i = 0; i < 5; ++i)
#pragma unroll
            for (int j = 0; j < 5; ++j) v[5 * i + j] = PS::raw(src + (5 * i + j) * P.plane2 + (row[j] + col[i]));
        return m;
    };
    if (xa < P.nx) ma = load(xa, ra, va);
    if (xb < P.nx) mb = load(xb, rb, vb);
    NodeDiagF d;
    auto update = [&](const V (&v)[25], unsigned m, int x, int r) {
        pair_update<S, false>(
            P,
            [&](auto& o, auto conv) {
#pragma unroll
                for (int i = 0; i < 5; ++i)
#pragma unroll
                    for (int j = 0; j < 5; ++j) {
                        const int p = 5 * i + j;
                        o[p] = conv(((m >> j) & 1u) ? PS::swap(v[p]) : v[p]);
                    }
            },
            dst, x, r, d);
    };
    if (xa < P.nx) update(va, ma, xa, ra);
    if (xb < P.nx) update(vb, mb, xb, rb);
}

// One node (x, y) of a lattice in the plain layout (storage [25][ny][pitch], plane
// elements per population), with the single-node forms of the pair arithmetic:
// the same result as the row-paired kernels give the node.
template <typename S>
struct Scalar16;
template <>
struct Scalar16<float> {
    static __device__ __forceinline__ float load(const float* p) { return __ldg(p); }
    static __device__ __forceinline__ void store(float* p, float v) { *p = v; }
};
template <>
struct Scalar16<__half> {
    static __device__ __forceinline__ float load(const __half* p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ void store(__half* p, float v) { *p = __float2half_rn(v); }
};
template <>
struct Scalar16<__nv_bfloat16> {
    static __device__ __forceinline__ float load(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
    static __device__ __forceinline__ void store(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
};

template <typename S, bool REDUCE>
__device__ __forceinline__ void sym5_node(const PairParams& P, const S* __restrict__ src, S* __restrict__ dst,
                                          int x, int y, NodeDiagF& d) {
    unsigned col[5], row[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const int s = x + P.vxm[i];
        col[i] = (unsigned)((s >= P.nx) ? s - P.nx : s);
        int t = y + P.vym[i];
        t = (t >= P.ny) ? t - P.ny : t;
        row[i] = (unsigned)t * (unsigned)P.pitch;
    }
    const long long plane = P.plane2;   // elements per population plane (plain layout)
    float g[25];
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            const int p = 5 * i + j;
            g[p] = Scalar16<S>::load(src + p * plane + (row[j] + col[i]));
        }
    float rho, th, drho, jx, jy, e;
    sym5_collide<float>(P, [&](int p) { return g[p]; }, [&](int p) { return g[p]; }, g, rho, th, drho, jx, jy, e);
    if (!((rho > 0.0f) & (th > 0.0f) & (rho < 3.0e38f) & (th < 3.0e38f))) {
        unsigned bits = (!(rho == rho) || !(th == th) || !(rho < 3.0e38f) || !(th < 3.0e38f)) ? 1u : 0u;
        bits |= rho <= 0.0f ? 2u : 0u;
        bits |= th <= 0.0f ? 4u : 0u;
        atomicOr(P.status, bits);
    }
    if (REDUCE) {
        d.dmass = FF{drho, 0.0f};
        d.jx = FF{jx, 0.0f};
        d.jy = FF{jy, 0.0f};
        d.denergy = FF{e, 0.0f};
        d.rho_min = rho;
        d.theta_min = th;
        d.n = 1.0f;
    }
    const unsigned here = (unsigned)y * (unsigned)P.pitch + (unsigned)x;
#pragma unroll
    for (int p = 0; p < 25; ++p) Scalar16<S>::store(dst + p * plane + here, g[p]);
}

// grid = (ceil(nx / blockDim.x), ny), one node per thread (blockDim.x = kBlockX when REDUCE).
template <typename S, bool REDUCE>
__global__ void __launch_bounds__(kBlockX)
k_stream_collide_sym5(const __grid_constant__ PairParams P, const S* __restrict__ src, S* __restrict__ dst) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    NodeDiagF d;
    if (REDUCE) diagf_zero(d);
    if (x < P.nx) sym5_node<S, REDUCE>(P, src, dst, x, blockIdx.y, d);
    if (REDUCE) {
        const int blk = blockIdx.y * gridDim.x + blockIdx.x;
        block_reduce_diagf<kBlockX>(d, 2.0 * P.theta0, P.partials + (long long)blk * kPartialStride);
    }
}

// Resident CTAs per SM the register allocation aims at: seven 128-thread CTAs
// (at most 72 registers) for BF16 pairs, kept packed; none (0) for the others
// and for the steps that also reduce the diagnostics.  An explicit 1 is not
// the same as none: it let FP32 and FP16 grow from 94 to 112 registers.
template <typename S>
struct PairMinBlocks {
    static constexpr int value = PairStore<S>::kReconvert ? 7 : 0;
};

// grid = (ceil(nx / kBlockX), ny / 2); thread (x, r) owns nodes (x, r) and (x, r + ny/2).
template <typename S, bool REDUCE>
__global__ void __launch_bounds__(kBlockX, REDUCE ? 0 : PairMinBlocks<S>::value)
k_stream_collide_pair(const __grid_constant__ PairParams P,
                      const typename PairStore<S>::V* __restrict__ src,
                      typename PairStore<S>::V* __restrict__ dst) {
    const int x = blockIdx.x * kBlockX + threadIdx.x;
    NodeDiagF d;
    if (REDUCE) diagf_zero(d);
    if (x < P.nx) pair_node<S, REDUCE>(P, src, dst, x, blockIdx.y, d);
    if (REDUCE) {
        const int blk = blockIdx.y * gridDim.x + blockIdx.x;
        block_reduce_diagf<kBlockX>(d, 2.0 * P.theta0, P.partials + (long long)blk * kPartialStride);
    }
}

// Plain-layout symmetric five-velocity lattices (odd ny, or PLBM_FLAG_PLAIN_LAYOUT):
// one node per thread; small lattices take 32-thread blocks (more SMs busy).
template <typename S>
cudaError_t launch_step_sym5_t(const LatticeParams& L, const void* src, void* dst, bool reduce,
                               cudaStream_t stream) {
    const PairParams P = pair_params(L);
    int bx = kBlockX;
    if (!reduce && (long long)((P.nx + kBlockX - 1) / kBlockX) * P.ny < 2LL * device_sm_count()) bx = 32;
    dim3 grid((P.nx + bx - 1) / bx, P.ny);
    const S* s = static_cast<const S*>(src);
    S* t = static_cast<S*>(dst);
    if (reduce)
        k_stream_collide_sym5<S, true><<<grid, kBlockX, 0, stream>>>(P, s, t);
    else
        k_stream_collide_sym5<S, false><<<grid, bx, 0, stream>>>(P, s, t);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_step_pair_t(const LatticeParams& L, const void* src, void* dst, bool reduce,
                               cudaStream_t stream) {
    using V = typename PairStore<S>::V;
    const PairParams P = pair_params(L);
    dim3 grid((P.nx + kBlockX - 1) / kBlockX, P.half_ny);
    const V* s = static_cast<const V*>(src);
    V* t = static_cast<V*>(dst);
    if constexpr (std::is_same<S, __half>::value) {
        if (!reduce) {
            const int tiles_x = (P.nx + kPair2Block - 1) / kPair2Block;
            const int ntiles = tiles_x * P.half_ny;
            k_stream_collide_pair2<S><<<(ntiles + 1) / 2, kPair2Block, 0, stream>>>(P, s, t, tiles_x, ntiles);
            return cudaGetLastError();
        }
    }
    if (reduce)
        k_stream_collide_pair<S, true><<<grid, kBlockX, 0, stream>>>(P, s, t);
    else
        k_stream_collide_pair<S, false><<<grid, kBlockX, 0, stream>>>(P, s, t);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Batched persistent step: every instance of a batch advances one step in one
// launch.  The instances' tiles (BX threads x one pair row, or x one row for a
// lattice in the plain layout) form one global list; CTA c walks the contiguous range [c * per_cta, (c + 1) * per_cta), so it
// meets few instance boundaries and keeps the current instance's PairParams in
// shared memory.  `parity` selects which of each instance's two arrays is read.
// ---------------------------------------------------------------------------
// One thread's node(s) of a tile of the batched sweep: a node pair of pair row r
// (row-paired lattices) or node (x, r) (plain layout, odd ny).
template <typename S>
__device__ __forceinline__ void batch_tile_node(const PairParams& sp, int parity, int x, int r, NodeDiagF& d) {
    using V = typename PairStore<S>::V;
    if (sp.paired)
        pair_node<S, false>(sp, static_cast<const V*>(sp.f[parity]), static_cast<V*>(sp.f[parity ^ 1]), x, r, d);
    else
        sym5_node<S, false>(sp, static_cast<const S*>(sp.f[parity]), static_cast<S*>(sp.f[parity ^ 1]), x, r, d);
}

template <typename S, int BX>
__global__ void __launch_bounds__(BX)
k_batch_pair(const PairParams* __restrict__ inst, int ninst, int total_tiles, int per_cta, int parity,
             const unsigned short* __restrict__ tile_inst) {
    using V = typename PairStore<S>::V;
    __shared__ PairParams sp;
    __shared__ int s_inst;
    constexpr int kWords = (int)(sizeof(PairParams) / sizeof(int));
    NodeDiagF d;
    if (tile_inst) {
        // Interleaved order: CTA c takes tiles c, c + G, c + 2G, ... (G CTAs), so the
        // tiles in flight at any moment are neighbours in memory, as in a plain grid.
        int cur = -1;
        int t = blockIdx.x;
        int i_next = t < total_tiles ? tile_inst[t] : 0;
        for (; t < total_tiles; t += gridDim.x) {
            const int i = i_next;
            if (t + (int)gridDim.x < total_tiles) i_next = tile_inst[t + gridDim.x];
            if (i != cur) {  // block-uniform
                __syncthreads();
                for (int k = threadIdx.x; k < kWords; k += BX)
                    reinterpret_cast<int*>(&sp)[k] = reinterpret_cast<const int*>(&inst[i])[k];
                __syncthreads();
                cur = i;
            }
            const int local = t - sp.tile_begin;
            const int r = local / sp.tiles_x;
            const int x = (local - r * sp.tiles_x) * BX + threadIdx.x;
            if (x < sp.nx) batch_tile_node<S>(sp, parity, x, r, d);
        }
        return;
    }
    const int t0 = blockIdx.x * per_cta;
    const int t1 = min(t0 + per_cta, total_tiles);
    if (t0 >= t1) return;
    // first instance containing t0 (binary search over tile_begin)
    if (threadIdx.x == 0) {
        int lo = 0, hi = ninst - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (inst[mid].tile_begin <= t0) lo = mid; else hi = mid - 1;
        }
        s_inst = lo;
    }
    __syncthreads();
    int i = s_inst;
    int next_begin = (i + 1 < ninst) ? inst[i + 1].tile_begin : total_tiles;
    static_assert(sizeof(PairParams) % sizeof(int) == 0, "PairParams copy granularity");
    for (int k = threadIdx.x; k < kWords; k += BX)
        reinterpret_cast<int*>(&sp)[k] = reinterpret_cast<const int*>(&inst[i])[k];
    __syncthreads();
    for (int t = t0; t < t1; ++t) {
        if (t >= next_begin) {  // block-uniform: move to the instance holding tile t
            while (t >= next_begin) {
                ++i;
                next_begin = (i + 1 < ninst) ? inst[i + 1].tile_begin : total_tiles;
            }
            __syncthreads();
            for (int k = threadIdx.x; k < kWords; k += BX)
                reinterpret_cast<int*>(&sp)[k] = reinterpret_cast<const int*>(&inst[i])[k];
            __syncthreads();
        }
        const int local = t - sp.tile_begin;
        const int r = local / sp.tiles_x;
        const int x = (local - r * sp.tiles_x) * BX + threadIdx.x;
        if (x < sp.nx) batch_tile_node<S>(sp, parity, x, r, d);
    }
}

template <typename S>
cudaError_t launch_batch_pair_t(const PairParams* inst, int ninst, int total_tiles, int block_x, int ctas,
                                int parity, const unsigned short* tile_inst, cudaStream_t stream) {
    const int per_cta = (total_tiles + ctas - 1) / ctas;
    switch (block_x) {
        case 64: k_batch_pair<S, 64><<<ctas, 64, 0, stream>>>(inst, ninst, total_tiles, per_cta, parity, tile_inst); break;
        case 128: k_batch_pair<S, 128><<<ctas, 128, 0, stream>>>(inst, ninst, total_tiles, per_cta, parity, tile_inst); break;
        case 256: k_batch_pair<S, 256><<<ctas, 256, 0, stream>>>(inst, ninst, total_tiles, per_cta, parity, tile_inst); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename S>
cudaError_t batch_occupancy_t(int block_x, int* blocks_per_sm) {
    switch (block_x) {
        case 64: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_batch_pair<S, 64>, 64, 0);
        case 128: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_batch_pair<S, 128>, 128, 0);
        case 256: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_batch_pair<S, 256>, 256, 0);
    }
    return cudaErrorInvalidValue;
}

}  // namespace plbm
