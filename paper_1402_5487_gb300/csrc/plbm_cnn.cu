// Kernels of the learned surrogate: 3x3 convolutions with circular padding on
// NHWC activations, their gradients, loss and optimiser.
//
// The surrogate is a 6-layer CNN (4 -> 64, 4 x (64 -> 64), 64 -> 4 channels)
// mapping (rho, u_x, u_y, theta) of a periodic lattice to the change of those
// fields K lattice steps later.  It is not in the paper; it is a throughput
// service built around the paper's solver, which generates its training data
// and stays the fallback.
//
//  * 64 -> 64 layers: implicit GEMM on the tensor cores with mma.sync
//    m16n8k16 BF16 x BF16 -> FP32 (M = output pixels, N = 64 output channels,
//    K = 9 taps x 64 input channels).  Weights (72 KB) stay in shared memory for
//    the life of a persistent CTA; the three input rows of each 128-pixel tile
//    are staged with cp.async into a double buffer while the previous tile runs.
//    Shared rows of 128 bytes are XOR-swizzled in 16-byte chunks so that the
//    eight row addresses of every ldmatrix hit distinct banks.
//  * Backward data of a 64 -> 64 layer is the same forward kernel with the
//    taps flipped and the channel axes of the weights swapped, epilogue
//    multiplying by the ReLU mask of the layer input.
//  * Weight gradients of 64 -> 64 layers: one warp per tap accumulates the
//    64 x 64 block X_shift^T dY over the CTA's pixels with mma.sync; per-CTA
//    partial sums are reduced in a fixed order.
//  * The thin 4 -> 64 and 64 -> 4 layers (and their gradients) run on the CUDA
//    cores in FP32.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "plbm_internal.h"

namespace plbm {
namespace cnn {

constexpr int kC = 64;            // hidden channels
constexpr int kTile = 128;        // output pixels per tile (one row segment)
constexpr int kRowPix = kTile + 2;
constexpr int kThreadsMid = 256;  // 8 warps: 4 pixel slabs x 2 channel halves
constexpr int kWBytes = 9 * kC * kC * 2;             // 73728
constexpr int kInBytes = 3 * kRowPix * kC * 2;       // 49920
constexpr int kMidSmem = kWBytes + 2 * kInBytes;     // 173568

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(gmem));
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(smem)), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldsm_x4(unsigned addr, unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned addr, unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}
__device__ __forceinline__ void mma_bf16(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Byte offset of 16-byte chunk c (0..7) of 128-byte row `row` with the XOR swizzle.
__device__ __forceinline__ int swz(int row, int c) { return (row * 8 + (c ^ (row & 7))) * 16; }

struct ConvShape {
    int B, H, W;
};

// ---------------------------------------------------------------------------
// 64 -> 64 convolution, forward (mode 0: + bias, ReLU if relu; mode 1: no bias,
// output multiplied by (mask > 0)).  X, Y, mask: NHWC bf16; Wt: [tap][ci][co] bf16;
// bias: fp32[64].
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreadsMid, 1)
k_conv64_fwd(ConvShape S, const __nv_bfloat16* __restrict__ X, const __nv_bfloat16* __restrict__ Wt,
             const float* __restrict__ bias, const __nv_bfloat16* __restrict__ mask, __nv_bfloat16* __restrict__ Y,
             int mode, int relu) {
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* sW = smem;
    unsigned char* sIn = smem + kWBytes;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 3, wn = warp >> 2;
    const int tiles_x = S.W / kTile;
    const int ntiles = S.B * S.H * tiles_x;

    // weights: 9*64 rows of 128 bytes
    for (int i = tid; i < 9 * kC * 8; i += kThreadsMid) {
        const int row = i >> 3, c = i & 7;
        cp_async16(sW + swz(row, c), Wt + (size_t)row * kC + c * 8);
    }
    auto load_tile = [&](int t, int buf) {
        const int b = t / (S.H * tiles_x);
        const int rem = t - b * S.H * tiles_x;
        const int y = rem / tiles_x;
        const int x0 = (rem - y * tiles_x) * kTile;
        unsigned char* dst = sIn + buf * kInBytes;
        for (int i = tid; i < 3 * kRowPix * 8; i += kThreadsMid) {
            const int c = i & 7;
            const int pr = i >> 3;              // r * kRowPix + p
            const int r = pr / kRowPix, p = pr - r * kRowPix;
            int yy = y + r - 1;
            yy += (yy < 0) ? S.H : 0;
            yy -= (yy >= S.H) ? S.H : 0;
            int xx = x0 + p - 1;
            xx += (xx < 0) ? S.W : 0;
            xx -= (xx >= S.W) ? S.W : 0;
            const __nv_bfloat16* src = X + (((size_t)b * S.H + yy) * S.W + xx) * kC + c * 8;
            cp_async16(dst + r * kRowPix * 128 + swz(p, c), src);
        }
    };
    int t = blockIdx.x;
    if (t < ntiles) load_tile(t, 0);
    cp_async_commit();
    int buf = 0;
    for (; t < ntiles; t += gridDim.x) {
        const int tn = t + gridDim.x;
        if (tn < ntiles) load_tile(tn, buf ^ 1);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();

        float acc[2][4][4];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.0f;

        const unsigned char* in = sIn + buf * kInBytes;
#pragma unroll 1
        for (int tap = 0; tap < 9; ++tap) {
            const int ky = tap / 3, kx = tap - ky * 3;
            const unsigned char* rowp = in + ky * kRowPix * 128;
#pragma unroll
            for (int kc = 0; kc < 4; ++kc) {  // 16 input channels per step
                unsigned a[2][4];
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    const int j = lane >> 3;
                    const int p = wm * 32 + mt * 16 + (lane & 7) + 8 * (j & 1) + kx;
                    const int c = kc * 2 + (j >> 1);
                    ldsm_x4(smem_u32(rowp + swz(p, c)), a[mt][0], a[mt][1], a[mt][2], a[mt][3]);
                }
                unsigned bf[4][2];
#pragma unroll
                for (int np = 0; np < 2; ++np) {  // two n8 tiles per ldmatrix
                    const int krow = tap * kC + kc * 16 + (lane & 7) + 8 * ((lane >> 3) & 1);
                    const int c = wn * 4 + np * 2 + (lane >> 4);
                    ldsm_x4_t(smem_u32(sW + swz(krow, c)), bf[np * 2][0], bf[np * 2][1], bf[np * 2 + 1][0],
                              bf[np * 2 + 1][1]);
                }
#pragma unroll
                for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                    for (int nt = 0; nt < 4; ++nt)
                        mma_bf16(acc[mt][nt], a[mt][0], a[mt][1], a[mt][2], a[mt][3], bf[nt][0], bf[nt][1]);
            }
        }
        // epilogue
        const int b = t / (S.H * tiles_x);
        const int rem = t - b * S.H * tiles_x;
        const int y = rem / tiles_x;
        const int x0 = (rem - y * tiles_x) * kTile;
        const int g = lane >> 2, q = lane & 3;
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int x = x0 + wm * 32 + mt * 16 + g + 8 * h;
                const size_t pix = ((size_t)b * S.H + y) * S.W + x;
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) {
                    const int co = wn * 32 + nt * 8 + 2 * q;
                    float v0 = acc[mt][nt][2 * h], v1 = acc[mt][nt][2 * h + 1];
                    if (mode == 0) {
                        v0 += bias[co];
                        v1 += bias[co + 1];
                        if (relu) {
                            v0 = fmaxf(v0, 0.0f);
                            v1 = fmaxf(v1, 0.0f);
                        }
                    } else {
                        const __nv_bfloat162 mk = *reinterpret_cast<const __nv_bfloat162*>(mask + pix * kC + co);
                        v0 = __bfloat162float(mk.x) > 0.0f ? v0 : 0.0f;
                        v1 = __bfloat162float(mk.y) > 0.0f ? v1 : 0.0f;
                    }
                    *reinterpret_cast<__nv_bfloat162*>(Y + pix * kC + co) = __floats2bfloat162_rn(v0, v1);
                }
            }
        __syncthreads();  // the buffer is refilled by the next iteration's prefetch
        buf ^= 1;
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// 64 -> 64 weight gradient.  Warp w (w < 9) owns tap w and accumulates
// dW[tap][ci][co] = sum_pixels X[pix + shift][ci] dY[pix][co] for the CTA's
// tiles; warp 9 also sums dY per channel for the bias.  Partials per CTA:
// partial[cta][tap][ci][co] (fp32), partial_b[cta][co].
// ---------------------------------------------------------------------------
constexpr int kThreadsWg = 320;  // 10 warps
constexpr int kDyBytes = kTile * kC * 2;  // 16384
constexpr int kWgSmem = 2 * (kInBytes + kDyBytes);

__global__ void __launch_bounds__(kThreadsWg, 1)
k_conv64_wgrad(ConvShape S, const __nv_bfloat16* __restrict__ X, const __nv_bfloat16* __restrict__ dY,
               float* __restrict__ partial, float* __restrict__ partial_b) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tiles_x = S.W / kTile;
    const int ntiles = S.B * S.H * tiles_x;
    auto load_tile = [&](int t, int buf) {
        const int b = t / (S.H * tiles_x);
        const int rem = t - b * S.H * tiles_x;
        const int y = rem / tiles_x;
        const int x0 = (rem - y * tiles_x) * kTile;
        unsigned char* dIn = smem + buf * (kInBytes + kDyBytes);
        unsigned char* dG = dIn + kInBytes;
        for (int i = tid; i < 3 * kRowPix * 8; i += kThreadsWg) {
            const int c = i & 7;
            const int pr = i >> 3;
            const int r = pr / kRowPix, p = pr - r * kRowPix;
            int yy = y + r - 1;
            yy += (yy < 0) ? S.H : 0;
            yy -= (yy >= S.H) ? S.H : 0;
            int xx = x0 + p - 1;
            xx += (xx < 0) ? S.W : 0;
            xx -= (xx >= S.W) ? S.W : 0;
            cp_async16(dIn + r * kRowPix * 128 + swz(p, c), X + (((size_t)b * S.H + yy) * S.W + xx) * kC + c * 8);
        }
        for (int i = tid; i < kTile * 8; i += kThreadsWg) {
            const int c = i & 7, p = i >> 3;
            cp_async16(dG + swz(p, c), dY + (((size_t)b * S.H + y) * S.W + x0 + p) * kC + c * 8);
        }
    };
    float acc[4][8][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.0f;
    float bsum = 0.0f;  // warp 9, lanes 0..31: channels lane and lane + 32

    float bsum2 = 0.0f;
    int t = blockIdx.x;
    if (t < ntiles) load_tile(t, 0);
    cp_async_commit();
    int buf = 0;
    for (; t < ntiles; t += gridDim.x) {
        const int tn = t + gridDim.x;
        if (tn < ntiles) load_tile(tn, buf ^ 1);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        const unsigned char* in = smem + buf * (kInBytes + kDyBytes);
        const unsigned char* gy = in + kInBytes;
        if (warp < 9) {
            const int ky = warp / 3, kx = warp - ky * 3;
            const unsigned char* rowp = in + ky * kRowPix * 128;
#pragma unroll 1
            for (int ks = 0; ks < kTile / 16; ++ks) {  // 16 pixels per k step
                unsigned a[4][4];
#pragma unroll
                for (int mt = 0; mt < 4; ++mt) {  // 16 input channels per m tile
                    const int j = lane >> 3;
                    const int p = ks * 16 + (lane & 7) + 8 * (j >> 1) + kx;
                    const int c = mt * 2 + (j & 1);
                    ldsm_x4_t(smem_u32(rowp + swz(p, c)), a[mt][0], a[mt][1], a[mt][2], a[mt][3]);
                }
#pragma unroll
                for (int np = 0; np < 4; ++np) {
                    unsigned b0, b1, b2, b3;
                    const int p = ks * 16 + (lane & 7) + 8 * ((lane >> 3) & 1);
                    const int c = np * 2 + (lane >> 4);
                    ldsm_x4_t(smem_u32(gy + swz(p, c)), b0, b1, b2, b3);
#pragma unroll
                    for (int mt = 0; mt < 4; ++mt) {
                        mma_bf16(acc[mt][np * 2], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b0, b1);
                        mma_bf16(acc[mt][np * 2 + 1], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b2, b3);
                    }
                }
            }
        } else {
            // bias gradient: lane owns channels lane and lane + 32
            for (int p = 0; p < kTile; ++p) {
                const __nv_bfloat16* row = reinterpret_cast<const __nv_bfloat16*>(gy + swz(p, lane >> 3));
                const __nv_bfloat16* row2 = reinterpret_cast<const __nv_bfloat16*>(gy + swz(p, (lane + 32) >> 3));
                bsum += __bfloat162float(row[lane & 7]);
                bsum2 += __bfloat162float(row2[lane & 7]);
            }
        }
        __syncthreads();
        buf ^= 1;
    }
    cp_async_wait<0>();
    if (warp < 9) {
        float* out = partial + ((size_t)blockIdx.x * 9 + warp) * kC * kC;
        const int g = lane >> 2, q = lane & 3;
#pragma unroll
        for (int mt = 0; mt < 4; ++mt)
#pragma unroll
            for (int nt = 0; nt < 8; ++nt)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int ci = mt * 16 + g + 8 * h;
                    const int co = nt * 8 + 2 * q;
                    out[ci * kC + co] = acc[mt][nt][2 * h];
                    out[ci * kC + co + 1] = acc[mt][nt][2 * h + 1];
                }
    } else {
        partial_b[(size_t)blockIdx.x * kC + lane] = bsum;
        partial_b[(size_t)blockIdx.x * kC + lane + 32] = bsum2;
    }
}

// out[j] = sum_c partial[c * n + j] in a fixed order: block = 32 consecutive j;
// warp w sums the parts c of its contiguous eighth (in order, four loads in
// flight), and lane j adds the eight warps' sums in warp order.  The blocks past
// the first (n + 31) / 32 do the same for a second array (partial2, n2, out2),
// so that a weight gradient and its bias gradient take one launch.
__global__ void __launch_bounds__(256) k_sum_partials(const float* __restrict__ partial, int nparts, int n,
                                                      float* __restrict__ out, const float* __restrict__ partial2,
                                                      int n2, float* __restrict__ out2) {
    __shared__ float sh[8][33];
    int blk = blockIdx.x;
    const int nb1 = (n + 31) / 32;
    if (blk >= nb1) {
        partial = partial2;
        n = n2;
        out = out2;
        blk -= nb1;
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = blk * 32 + lane;
    const int per = (nparts + 7) / 8;
    const int c0 = w * per, c1 = min(nparts, c0 + per);
    float s = 0.0f;
    if (j < n) {
        int c = c0;
        for (; c + 4 <= c1; c += 4) {
            const float a0 = partial[(size_t)c * n + j], a1 = partial[(size_t)(c + 1) * n + j];
            const float a2 = partial[(size_t)(c + 2) * n + j], a3 = partial[(size_t)(c + 3) * n + j];
            s += a0;
            s += a1;
            s += a2;
            s += a3;
        }
        for (; c < c1; ++c) s += partial[(size_t)c * n + j];
    }
    sh[w][lane] = s;
    __syncthreads();
    if (w == 0 && j < n) {
        float t = sh[0][lane];
#pragma unroll
        for (int k = 1; k < 8; ++k) t += sh[k][lane];
        out[j] = t;
    }
}

// The same sums, four consecutive j per thread (float4; n, n2 multiples of 4):
// a block covers 128 j, so the loads in flight are 16 bytes wide.  Per j the
// order of the additions is the one of k_sum_partials.
__global__ void __launch_bounds__(256) k_sum_partials4(const float4* __restrict__ partial, int nparts, int n4,
                                                       float4* __restrict__ out, const float4* __restrict__ partial2,
                                                       int n24, float4* __restrict__ out2) {
    __shared__ float4 sh[8][32];
    int blk = blockIdx.x;
    const int nb1 = (n4 + 31) / 32;
    if (blk >= nb1) {
        partial = partial2;
        n4 = n24;
        out = out2;
        blk -= nb1;
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = blk * 32 + lane;
    const int per = (nparts + 7) / 8;
    const int c0 = w * per, c1 = min(nparts, c0 + per);
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    auto add = [](float4& a, const float4 b) {
        a.x += b.x;
        a.y += b.y;
        a.z += b.z;
        a.w += b.w;
    };
    if (j < n4) {
        int c = c0;
        for (; c + 8 <= c1; c += 8) {
            float4 a[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) a[k] = __ldg(partial + (size_t)(c + k) * n4 + j);
#pragma unroll
            for (int k = 0; k < 8; ++k) add(s, a[k]);
        }
        for (; c < c1; ++c) add(s, __ldg(partial + (size_t)c * n4 + j));
    }
    sh[w][lane] = s;
    __syncthreads();
    if (w == 0 && j < n4) {
        float4 t = sh[0][lane];
#pragma unroll
        for (int k = 1; k < 8; ++k) add(t, sh[k][lane]);
        out[j] = t;
    }
}

// ---------------------------------------------------------------------------
// Thin layers on the CUDA cores (FP32 arithmetic, weights fp32 [tap][ci][co]).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ float to_f(T v);
template <>
__device__ __forceinline__ float to_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

__device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// 4 -> 64: tile = 128 pixels of one row, thread = pixel.  The 36 inputs of a
// pixel sit in registers, the weights are read as broadcast float4 from shared
// memory, and the 64 outputs per pixel leave through a swizzled shared tile so
// that the global stores are 16-byte and coalesced.
// mode 0: + bias, ReLU if relu; mode 1: no bias, times (mask > 0).
constexpr int kInFwdSmem = 9 * 4 * 64 * 4 + kTile * 64 * 2;

template <typename TI>
__global__ void __launch_bounds__(128)
k_thin_in_fwd(ConvShape S, const TI* __restrict__ X, const float* __restrict__ Wf, const float* __restrict__ bias,
              const __nv_bfloat16* __restrict__ mask, __nv_bfloat16* __restrict__ Y, int mode, int relu) {
    extern __shared__ __align__(16) unsigned char dsm[];
    float* sW = reinterpret_cast<float*>(dsm);
    unsigned char* sOut = dsm + 9 * 4 * 64 * 4;
    const int tiles_x = S.W / kTile;
    const int t = blockIdx.x;
    const int b = t / (S.H * tiles_x);
    const int rem = t - b * S.H * tiles_x;
    const int y = rem / tiles_x;
    const int x0 = (rem - y * tiles_x) * kTile;
    for (int i = threadIdx.x; i < 9 * 4 * 64; i += 128) sW[i] = Wf[i];
    const int px = threadIdx.x, x = x0 + px;
    float in[36];
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
        const int yy = wrap(y + tap / 3 - 1, S.H), xx = wrap(x + tap % 3 - 1, S.W);
        const TI* xp = X + (((size_t)b * S.H + yy) * S.W + xx) * 4;
#pragma unroll
        for (int i = 0; i < 4; ++i) in[tap * 4 + i] = to_f<TI>(xp[i]);
    }
    __syncthreads();
    float2 acc[32];   // output channels (2j, 2j + 1): packed FP32x2 FMAs, the same roundings as scalar ones
#pragma unroll
    for (int j = 0; j < 32; ++j)
        acc[j] = (mode == 0) ? make_float2(bias[2 * j], bias[2 * j + 1]) : make_float2(0.0f, 0.0f);
#pragma unroll
    for (int k = 0; k < 36; ++k) {
        const float2 xv = make_float2(in[k], in[k]);
        const float4* w = reinterpret_cast<const float4*>(sW + k * 64);
#pragma unroll
        for (int o4 = 0; o4 < 16; ++o4) {
            const float4 ww = w[o4];
            acc[2 * o4] = __ffma2_rn(xv, make_float2(ww.x, ww.y), acc[2 * o4]);
            acc[2 * o4 + 1] = __ffma2_rn(xv, make_float2(ww.z, ww.w), acc[2 * o4 + 1]);
        }
    }
    const size_t pix = ((size_t)b * S.H + y) * S.W + x;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        float v[8];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[2 * k] = acc[4 * c + k].x;
            v[2 * k + 1] = acc[4 * c + k].y;
        }
        if (mode == 0) {
            if (relu)
#pragma unroll
                for (int k = 0; k < 8; ++k) v[k] = fmaxf(v[k], 0.0f);
        } else {
            const uint4 mk = *reinterpret_cast<const uint4*>(mask + pix * 64 + 8 * c);
            const __nv_bfloat16* m = reinterpret_cast<const __nv_bfloat16*>(&mk);
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = __bfloat162float(m[k]) > 0.0f ? v[k] : 0.0f;
        }
        uint4 o;
        __nv_bfloat162* ob = reinterpret_cast<__nv_bfloat162*>(&o);
#pragma unroll
        for (int k = 0; k < 4; ++k) ob[k] = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
        *reinterpret_cast<uint4*>(sOut + swz(px, c)) = o;
    }
    __syncthreads();
    // coalesced copy-out: the tile's 128 pixels x 128 bytes are contiguous in global memory
    uint4* dst = reinterpret_cast<uint4*>(Y + (((size_t)b * S.H + y) * S.W + x0) * 64);
    for (int i = threadIdx.x; i < kTile * 8; i += 128) {
        const int p = i >> 3, c = i & 7;
        dst[i] = *reinterpret_cast<const uint4*>(sOut + swz(p, c));
    }
}

// 64 -> 4 (+ bias, fp32 output): tile = 128 pixels of one row; the three input rows
// are staged in shared memory (16-byte chunks XOR-swizzled by pixel), thread =
// pixel, one 16-byte store per thread.
constexpr int kOutSmem = 9 * 64 * 4 * 4 + 3 * kRowPix * 64 * 2;

__global__ void __launch_bounds__(128)
k_thin_out_fwd(ConvShape S, const __nv_bfloat16* __restrict__ X, const float* __restrict__ Wf,
               const float* __restrict__ bias, float* __restrict__ Y) {
    extern __shared__ __align__(16) unsigned char dsm[];
    float* sW = reinterpret_cast<float*>(dsm);
    unsigned char* sX = dsm + 9 * 64 * 4 * 4;
    const int tiles_x = S.W / kTile;
    const int t = blockIdx.x;
    const int b = t / (S.H * tiles_x);
    const int rem = t - b * S.H * tiles_x;
    const int y = rem / tiles_x;
    const int x0 = (rem - y * tiles_x) * kTile;
    for (int i = threadIdx.x; i < 9 * 64 * 4; i += 128) sW[i] = Wf[i];
    for (int i = threadIdx.x; i < 3 * kRowPix * 8; i += 128) {
        const int c = i & 7, pr = i >> 3, r = pr / kRowPix, p = pr - r * kRowPix;
        const int yy = wrap(y + r - 1, S.H), xx = wrap(x0 + p - 1, S.W);
        *reinterpret_cast<uint4*>(sX + r * kRowPix * 128 + swz(p, c)) =
            *reinterpret_cast<const uint4*>(X + (((size_t)b * S.H + yy) * S.W + xx) * 64 + 8 * c);
    }
    __syncthreads();
    const int px = threadIdx.x;
    float4 acc = make_float4(bias[0], bias[1], bias[2], bias[3]);
#pragma unroll 1
    for (int tap = 0; tap < 9; ++tap) {
        const int ky = tap / 3, kx = tap % 3;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const uint4 raw = *reinterpret_cast<const uint4*>(sX + ky * kRowPix * 128 + swz(px + kx, c));
            const __nv_bfloat16* xv = reinterpret_cast<const __nv_bfloat16*>(&raw);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const float a = __bfloat162float(xv[k]);
                const float4 w = *reinterpret_cast<const float4*>(sW + (tap * 64 + 8 * c + k) * 4);
                acc.x = fmaf(a, w.x, acc.x);
                acc.y = fmaf(a, w.y, acc.y);
                acc.z = fmaf(a, w.z, acc.z);
                acc.w = fmaf(a, w.w, acc.w);
            }
        }
    }
    reinterpret_cast<float4*>(Y)[((size_t)b * S.H + y) * S.W + x0 + px] = acc;
}

// Weight gradient of a thin layer, X with CX channels (bf16), dY with CG channels
// (TG), one of CX, CG equal to 64 and the other to 4.  Thread (tap, a), a < 64,
// accumulates the 4 entries of dW[tap][.][.] along the narrow axis over the CTA's
// 128-pixel tiles; threads with tap 0 also sum dY for the bias.  Each tile's
// three input rows and its dY row are staged with cp.async into one of two
// shared-memory stages while the previous tile is summed, so the copies of a
// tile are all in flight at once and overlap the arithmetic.
// partial[cta][tap][ci][co], partial_b[cta][co].
template <int CX, int CG, typename TG>
constexpr int thin_wgrad_stage() { return 3 * kRowPix * CX * 2 + kTile * CG * (int)sizeof(TG); }
template <int CX, int CG, typename TG>
constexpr int thin_wgrad_smem() { return 2 * thin_wgrad_stage<CX, CG, TG>(); }

template <int CX, int CG, typename TG>
__device__ __forceinline__ void thin_wgrad_stage_in(ConvShape S, const __nv_bfloat16* __restrict__ X,
                                                    const TG* __restrict__ dY, int t, unsigned char* st) {
    const int tiles_x = S.W / kTile;
    const int b = t / (S.H * tiles_x);
    const int rem = t - b * S.H * tiles_x;
    const int y = rem / tiles_x;
    const int x0 = (rem - y * tiles_x) * kTile;
    auto sX = reinterpret_cast<__nv_bfloat16 (*)[kRowPix][CX]>(st);
    auto sG = reinterpret_cast<TG (*)[CG]>(st + 3 * kRowPix * CX * 2);
    if (CX == 64) {   // 16-byte pieces: 8 channels of one pixel
        for (int i = threadIdx.x; i < 3 * kRowPix * 8; i += blockDim.x) {
            const int q = i & 7, pr = i >> 3, r = pr / kRowPix, p = pr - r * kRowPix;
            cp_async16(&sX[r][p][8 * q],
                       X + (((size_t)b * S.H + wrap(y + r - 1, S.H)) * S.W + wrap(x0 + p - 1, S.W)) * CX + 8 * q);
        }
    } else {          // 8-byte pieces: the 4 channels of one pixel
        for (int i = threadIdx.x; i < 3 * kRowPix; i += blockDim.x) {
            const int r = i / kRowPix, p = i - r * kRowPix;
            cp_async8(&sX[r][p][0],
                      X + (((size_t)b * S.H + wrap(y + r - 1, S.H)) * S.W + wrap(x0 + p - 1, S.W)) * CX);
        }
    }
    constexpr int GV = 16 / (int)sizeof(TG);  // dY values per 16-byte piece
    for (int i = threadIdx.x; i < kTile * (CG / GV); i += blockDim.x) {
        const int q = i % (CG / GV), p = i / (CG / GV);
        cp_async16(&sG[p][GV * q], dY + (((size_t)b * S.H + y) * S.W + x0 + p) * CG + GV * q);
    }
    cp_async_commit();
}

template <int CX, int CG, typename TG>
__global__ void __launch_bounds__(576)
k_thin_wgrad(ConvShape S, const __nv_bfloat16* __restrict__ X, const TG* __restrict__ dY, float* __restrict__ partial,
             float* __restrict__ partial_b) {
    static_assert((CX == 64 && CG == 4) || (CX == 4 && CG == 64), "thin layer shapes");
    extern __shared__ __align__(16) unsigned char dsm[];
    constexpr int kStage = thin_wgrad_stage<CX, CG, TG>();
    const int tap = threadIdx.x / 64, a = threadIdx.x % 64;
    const int ky = tap / 3, kx = tap % 3;
    const int ntiles = S.B * S.H * (S.W / kTile);
    float2 acc01 = make_float2(0.f, 0.f), acc23 = acc01;   // packed FP32x2 FMAs
    float bacc = 0.0f;
    int stage = 0;
    if ((int)blockIdx.x < ntiles) thin_wgrad_stage_in<CX, CG, TG>(S, X, dY, blockIdx.x, dsm);
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        // the other stage was last read in the previous iteration, behind its closing barrier
        if (t + (int)gridDim.x < ntiles) {
            thin_wgrad_stage_in<CX, CG, TG>(S, X, dY, t + gridDim.x, dsm + (stage ^ 1) * kStage);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        auto sX = reinterpret_cast<const __nv_bfloat16 (*)[kRowPix][CX]>(dsm + stage * kStage);
        auto sG = reinterpret_cast<const TG (*)[CG]>(dsm + stage * kStage + 3 * kRowPix * CX * 2);
#pragma unroll 4
        for (int p = 0; p < kTile; ++p) {
            if (CX == 64) {  // a = ci, narrow axis = co (dY fp32, 4 values)
                const float x1 = __bfloat162float(sX[ky][p + kx][a]);
                const float2 xv = make_float2(x1, x1);
                const float2 g01 = make_float2(to_f<TG>(sG[p][0]), to_f<TG>(sG[p][1]));
                const float2 g23 = make_float2(to_f<TG>(sG[p][2]), to_f<TG>(sG[p][3]));
                acc01 = __ffma2_rn(xv, g01, acc01);
                acc23 = __ffma2_rn(xv, g23, acc23);
                if (tap == 0 && a < 4) bacc += to_f<TG>(sG[p][a]);
            } else {  // a = co, narrow axis = ci
                const float g1 = to_f<TG>(sG[p][a]);
                const float2 g = make_float2(g1, g1);
                const uint2 raw = *reinterpret_cast<const uint2*>(&sX[ky][p + kx][0]);
                const __nv_bfloat162* xv = reinterpret_cast<const __nv_bfloat162*>(&raw);
                acc01 = __ffma2_rn(__bfloat1622float2(xv[0]), g, acc01);
                acc23 = __ffma2_rn(__bfloat1622float2(xv[1]), g, acc23);
                if (tap == 0) bacc += g1;
            }
        }
        __syncthreads();
        stage ^= 1;
    }
    float* out = partial + (size_t)blockIdx.x * 9 * CX * CG + (size_t)tap * CX * CG;
    const float acc[4] = {acc01.x, acc01.y, acc23.x, acc23.y};
    if (CX == 64) {
#pragma unroll
        for (int o = 0; o < 4; ++o) out[a * CG + o] = acc[o];
        if (tap == 0 && a < 4) partial_b[(size_t)blockIdx.x * CG + a] = bacc;
    } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) out[i * CG + a] = acc[i];
        if (tap == 0) partial_b[(size_t)blockIdx.x * CG + a] = bacc;
    }
}

// 64 -> 4 weight gradient (FP32 upstream gradient): 256 threads, thread (ci =
// t mod 64, group g = t / 64) takes input channel ci over the pixels 32 g ..
// 32 g + 31 of every tile and keeps all 36 sums dW[tap][ci][0..3] in registers:
// per pixel three new inputs (one per row, a sliding window over kx) and one
// broadcast float4 of dY feed 18 packed FMAs, against 4 multiply-adds per
// thread and pixel when every (tap, ci) had a thread of its own.  The four
// groups' sums are added in a fixed order at the end.  Stages and layout as
// k_thin_wgrad<64, 4, float>.
__global__ void __launch_bounds__(256)
k_thin_wgrad_64x4(ConvShape S, const __nv_bfloat16* __restrict__ X, const float* __restrict__ dY,
                  float* __restrict__ partial, float* __restrict__ partial_b) {
    extern __shared__ __align__(16) unsigned char dsm[];
    constexpr int kStage = thin_wgrad_stage<64, 4, float>();
    const int ci = threadIdx.x & 63, g = threadIdx.x >> 6;
    const int ntiles = S.B * S.H * (S.W / kTile);
    float2 acc[9][2];   // [tap][co pair]
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[k][0] = acc[k][1] = make_float2(0.f, 0.f);
    float4 bacc = make_float4(0.f, 0.f, 0.f, 0.f);
    int stage = 0;
    if ((int)blockIdx.x < ntiles) thin_wgrad_stage_in<64, 4, float>(S, X, dY, blockIdx.x, dsm);
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        if (t + (int)gridDim.x < ntiles) {
            thin_wgrad_stage_in<64, 4, float>(S, X, dY, t + gridDim.x, dsm + (stage ^ 1) * kStage);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        auto sX = reinterpret_cast<const __nv_bfloat16 (*)[kRowPix][64]>(dsm + stage * kStage);
        auto sG = reinterpret_cast<const float4*>(dsm + stage * kStage + 3 * kRowPix * 64 * 2);
        const int p0 = 32 * g;
        float x[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            x[r][0] = __bfloat162float(sX[r][p0][ci]);
            x[r][1] = __bfloat162float(sX[r][p0 + 1][ci]);
        }
#pragma unroll
        for (int p = p0; p < p0 + 32; ++p) {
#pragma unroll
            for (int r = 0; r < 3; ++r) x[r][2] = __bfloat162float(sX[r][p + 2][ci]);
            const float4 d = sG[p];
            const float2 d01 = make_float2(d.x, d.y), d23 = make_float2(d.z, d.w);
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int kx = 0; kx < 3; ++kx) {
                    const float2 xv = make_float2(x[r][kx], x[r][kx]);
                    acc[r * 3 + kx][0] = __ffma2_rn(xv, d01, acc[r * 3 + kx][0]);
                    acc[r * 3 + kx][1] = __ffma2_rn(xv, d23, acc[r * 3 + kx][1]);
                }
            if (ci == 0) {
                bacc.x += d.x;
                bacc.y += d.y;
                bacc.z += d.z;
                bacc.w += d.w;
            }
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                x[r][0] = x[r][1];
                x[r][1] = x[r][2];
            }
        }
        __syncthreads();
        stage ^= 1;
    }
    // the four groups' sums in a fixed order: red[g][ci][tap * 4 + co]
    float* red = reinterpret_cast<float*>(dsm);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        float* r = red + ((size_t)g * 64 + ci) * 36 + 4 * k;
        r[0] = acc[k][0].x;
        r[1] = acc[k][0].y;
        r[2] = acc[k][1].x;
        r[3] = acc[k][1].y;
    }
    float* redb = red + 4 * 64 * 36;
    if (ci == 0) {
        redb[4 * g + 0] = bacc.x;
        redb[4 * g + 1] = bacc.y;
        redb[4 * g + 2] = bacc.z;
        redb[4 * g + 3] = bacc.w;
    }
    __syncthreads();
    float* out = partial + (size_t)blockIdx.x * 9 * 64 * 4;   // [tap][ci][co]
    for (int i = threadIdx.x; i < 9 * 64 * 4; i += 256) {
        const int co = i & 3, c = (i >> 2) & 63, tap = i >> 8;
        const int j = c * 36 + 4 * tap + co;
        out[i] = ((red[j] + red[64 * 36 + j]) + red[2 * 64 * 36 + j]) + red[3 * 64 * 36 + j];
    }
    if (threadIdx.x < 4)
        partial_b[(size_t)blockIdx.x * 4 + threadIdx.x] =
            ((redb[threadIdx.x] + redb[4 + threadIdx.x]) + redb[8 + threadIdx.x]) + redb[12 + threadIdx.x];
}



// Per-sample, per-channel mean error m[b][c] = mean over the npix pixels of
// pred - target (NHWC [B][npix][4]); one block per sample.
__global__ void k_mean_err(const float* __restrict__ pred, const float* __restrict__ target, long long npix,
                           float* __restrict__ m) {
    __shared__ float sh[4][256];
    const long long base = (long long)blockIdx.x * npix * 4;
    float a[4] = {0.f, 0.f, 0.f, 0.f};
    for (long long i = threadIdx.x; i < npix; i += blockDim.x)
#pragma unroll
        for (int c = 0; c < 4; ++c) a[c] += pred[base + i * 4 + c] - target[base + i * 4 + c];
#pragma unroll
    for (int c = 0; c < 4; ++c) sh[c][threadIdx.x] = a[c];
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k)
#pragma unroll
            for (int c = 0; c < 4; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x < 4) m[blockIdx.x * 4 + threadIdx.x] = sh[threadIdx.x][0] / (float)npix;
}

// Loss (1/n) sum (pred - target)^2 + lam mean_{b,c} m[b][c]^2 (fp32, n = B npix 4
// values; m from k_mean_err, or NULL for lam = 0) and its gradient
// 2 (pred - target) / n + 2 lam m[b][c] / n; per-block partial sums of squares
// (the first term).  The second term drives the lattice-mean error of every
// predicted field, which the surrogate's drift gate measures, towards zero.
__global__ void k_mse(const float* __restrict__ pred, const float* __restrict__ target, long long n,
                      long long npix, const float* __restrict__ m, float lam, float* __restrict__ grad,
                      float* __restrict__ partial) {
    __shared__ float sh[256];
    float s = 0.0f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float d = pred[i] - target[i];
        const float dm = m ? lam * m[(i / (npix * 4)) * 4 + (i & 3)] : 0.0f;
        grad[i] = 2.0f * (d + dm) / (float)n;
        s += d * d;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

// The same four elements (one pixel) at a time, for 16-byte aligned pred, target
// and grad; per element the same arithmetic as k_mse.
__global__ void k_mse4(const float4* __restrict__ pred, const float4* __restrict__ target, long long n,
                       long long npix, const float4* __restrict__ m, float lam, float4* __restrict__ grad,
                       uint2* __restrict__ grad16, float* __restrict__ partial) {
    __shared__ float sh[256];
    float s = 0.0f;
    const long long n4 = n / 4;
    const float fn = (float)n;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x) {
        const float4 p = __ldg(pred + i), t = __ldg(target + i);
        const float4 d = make_float4(p.x - t.x, p.y - t.y, p.z - t.z, p.w - t.w);
        float4 dm = make_float4(0.f, 0.f, 0.f, 0.f);
        if (m) {
            const float4 mm = m[i / npix];
            dm = make_float4(lam * mm.x, lam * mm.y, lam * mm.z, lam * mm.w);
        }
        const float4 g = make_float4(2.0f * (d.x + dm.x) / fn, 2.0f * (d.y + dm.y) / fn, 2.0f * (d.z + dm.z) / fn,
                                     2.0f * (d.w + dm.w) / fn);
        grad[i] = g;
        if (grad16) {   // the same gradient in bf16 (round to nearest), for the tensor-core backward pass
            const __nv_bfloat162 a = __floats2bfloat162_rn(g.x, g.y), b = __floats2bfloat162_rn(g.z, g.w);
            grad16[i] = make_uint2(*reinterpret_cast<const uint32_t*>(&a), *reinterpret_cast<const uint32_t*>(&b));
        }
        s += d.x * d.x;
        s += d.y * d.y;
        s += d.z * d.z;
        s += d.w * d.w;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

// Adam (Kingma & Ba): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
// p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       long long n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void k_f32_to_bf16(const float* __restrict__ a, long long n, __nv_bfloat16* __restrict__ b) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = __float2bfloat16_rn(a[i]);
}


}  // namespace cnn

// ---------------------------------------------------------------------------
// Launchers (plbm_internal.h).
// ---------------------------------------------------------------------------
static int g_sms = 0;

static int sm_count() {
    if (!g_sms) {
        int d = 0;
        cudaGetDevice(&d);
        cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, d);
        if (g_sms <= 0) g_sms = 1;
    }
    return g_sms;
}

cudaError_t cnn_conv64_fwd(int B, int H, int W, const void* X, const void* Wt, const float* bias, const void* mask,
                           void* Y, int mode, int relu, cudaStream_t s) {
    if (W % cnn::kTile) return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(cnn::k_conv64_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             cnn::kMidSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int ntiles = B * H * (W / cnn::kTile);
    const int grid = ntiles < sm_count() ? ntiles : sm_count();
    cnn::k_conv64_fwd<<<grid, cnn::kThreadsMid, cnn::kMidSmem, s>>>(
        cnn::ConvShape{B, H, W}, static_cast<const __nv_bfloat16*>(X), static_cast<const __nv_bfloat16*>(Wt), bias,
        static_cast<const __nv_bfloat16*>(mask), static_cast<__nv_bfloat16*>(Y), mode, relu);
    return cudaGetLastError();
}

int cnn_wgrad64_parts(int B, int H, int W) {
    const int ntiles = B * H * (W / cnn::kTile);
    return ntiles < sm_count() ? ntiles : sm_count();
}

cudaError_t cnn_sum_partials(const float* partial, int nparts, int n, float* out, cudaStream_t s) {
    cnn::k_sum_partials<<<(n + 31) / 32, 256, 0, s>>>(partial, nparts, n, out, nullptr, 0, nullptr);
    return cudaGetLastError();
}

cudaError_t cnn_sum_partials2(const float* partial, int n, float* out, const float* partial2, int n2, float* out2,
                              int nparts, cudaStream_t s) {
    const bool vec = n % 4 == 0 && n2 % 4 == 0 &&
                     (reinterpret_cast<uintptr_t>(partial) | reinterpret_cast<uintptr_t>(out) |
                      reinterpret_cast<uintptr_t>(partial2) | reinterpret_cast<uintptr_t>(out2)) % 16 == 0;
    if (vec) {
        const int n4 = n / 4, n24 = n2 / 4;
        cnn::k_sum_partials4<<<(n4 + 31) / 32 + (n24 + 31) / 32, 256, 0, s>>>(
            reinterpret_cast<const float4*>(partial), nparts, n4, reinterpret_cast<float4*>(out),
            reinterpret_cast<const float4*>(partial2), n24, reinterpret_cast<float4*>(out2));
    } else {
        cnn::k_sum_partials<<<(n + 31) / 32 + (n2 + 31) / 32, 256, 0, s>>>(partial, nparts, n, out, partial2, n2, out2);
    }
    return cudaGetLastError();
}

cudaError_t cnn_conv64_wgrad(int B, int H, int W, const void* X, const void* dY, float* partial, float* partial_b,
                             float* dW, float* db, cudaStream_t s) {
    if (W % cnn::kTile) return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(cnn::k_conv64_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             cnn::kWgSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int grid = cnn_wgrad64_parts(B, H, W);
    cnn::k_conv64_wgrad<<<grid, cnn::kThreadsWg, cnn::kWgSmem, s>>>(
        cnn::ConvShape{B, H, W}, static_cast<const __nv_bfloat16*>(X), static_cast<const __nv_bfloat16*>(dY), partial,
        partial_b);
    const int n = 9 * cnn::kC * cnn::kC;
    return cnn_sum_partials2(partial, n, dW, partial_b, cnn::kC, db, grid, s);
}

// Thin layer dispatch: (ci, co, ti, to) with ti/to 0 = bf16, 1 = fp32.
cudaError_t cnn_conv_thin_fwd(int ci, int co, int ti, int to, int B, int H, int W, const void* X, const float* Wf,
                              const float* bias, const void* mask, void* Y, int mode, int relu, cudaStream_t s) {
    cnn::ConvShape S{B, H, W};
    const __nv_bfloat16* mk = static_cast<const __nv_bfloat16*>(mask);
    if (ci == 4 && co == 64 && to == 0) {
        if (W % cnn::kTile) return cudaErrorInvalidValue;
        const int grid = B * H * (W / cnn::kTile);
        if (ti == 0)
            cnn::k_thin_in_fwd<__nv_bfloat16><<<grid, 128, cnn::kInFwdSmem, s>>>(
                S, static_cast<const __nv_bfloat16*>(X), Wf, bias, mk, static_cast<__nv_bfloat16*>(Y), mode, relu);
        else
            cnn::k_thin_in_fwd<float><<<grid, 128, cnn::kInFwdSmem, s>>>(
                S, static_cast<const float*>(X), Wf, bias, mk, static_cast<__nv_bfloat16*>(Y), mode, relu);
    } else if (ci == 64 && co == 4 && ti == 0 && to == 1 && mode == 0 && !relu) {
        if (W % cnn::kTile) return cudaErrorInvalidValue;
        static bool attr = false;
        if (!attr) {
            cudaError_t e = cudaFuncSetAttribute(cnn::k_thin_out_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 cnn::kOutSmem);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        const int grid = B * H * (W / cnn::kTile);
        cnn::k_thin_out_fwd<<<grid, 128, cnn::kOutSmem, s>>>(S, static_cast<const __nv_bfloat16*>(X), Wf, bias,
                                                             static_cast<float*>(Y));
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

int cnn_thin_parts(int B, int H, int W, int* pix_per_block) {
    const int ntiles = B * H * (W / cnn::kTile);
    const int parts = ntiles < 2 * sm_count() ? ntiles : 2 * sm_count();
    if (pix_per_block) *pix_per_block = cnn::kTile;
    return parts;
}

cudaError_t cnn_conv_thin_wgrad(int ci, int co, int tx, int tg, int B, int H, int W, const void* X, const void* dY,
                                float* partial, float* partial_b, float* dW, float* db, cudaStream_t s) {
    if (W % cnn::kTile || tx != 0) return cudaErrorInvalidValue;
    const int parts = cnn_thin_parts(B, H, W, nullptr);
    cnn::ConvShape S{B, H, W};
    const __nv_bfloat16* Xb = static_cast<const __nv_bfloat16*>(X);
    if (ci == 4 && co == 64 && tg == 0) {
        constexpr int sm = cnn::thin_wgrad_smem<4, 64, __nv_bfloat16>();
        static bool attr = false;
        if (!attr) {
            cudaError_t e = cudaFuncSetAttribute(cnn::k_thin_wgrad<4, 64, __nv_bfloat16>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        cnn::k_thin_wgrad<4, 64, __nv_bfloat16><<<parts, 576, sm, s>>>(S, Xb, static_cast<const __nv_bfloat16*>(dY),
                                                                      partial, partial_b);
    } else if (ci == 64 && co == 4 && tg == 1) {
        constexpr int sm = cnn::thin_wgrad_smem<64, 4, float>();
        static_assert(sm >= (4 * 64 * 36 + 16) * 4, "reduction area within the stages");
        static bool attr = false;
        if (!attr) {
            cudaError_t e = cudaFuncSetAttribute(cnn::k_thin_wgrad_64x4, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        cnn::k_thin_wgrad_64x4<<<parts, 256, sm, s>>>(S, Xb, static_cast<const float*>(dY), partial, partial_b);
    } else {
        return cudaErrorInvalidValue;
    }
    const int n = 9 * ci * co;
    return cnn_sum_partials2(partial, n, dW, partial_b, co, db, parts, s);
}



cudaError_t cnn_mse(const float* pred, const float* target, long long n, long long npix, float lam, float* merr,
                    float* grad, void* grad16, float* partial, int parts, cudaStream_t s) {
    if (lam != 0.0f) {
        cnn::k_mean_err<<<(int)(n / (npix * 4)), 256, 0, s>>>(pred, target, npix, merr);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const bool vec = n % 4 == 0 && (reinterpret_cast<uintptr_t>(pred) | reinterpret_cast<uintptr_t>(target) |
                                    reinterpret_cast<uintptr_t>(grad) | reinterpret_cast<uintptr_t>(merr)) % 16 == 0 &&
                     reinterpret_cast<uintptr_t>(grad16) % 8 == 0;
    if (vec) {
        cnn::k_mse4<<<parts, 256, 0, s>>>(reinterpret_cast<const float4*>(pred), reinterpret_cast<const float4*>(target),
                                          n, npix, lam != 0.0f ? reinterpret_cast<const float4*>(merr) : nullptr, lam,
                                          reinterpret_cast<float4*>(grad), static_cast<uint2*>(grad16), partial);
        return cudaGetLastError();
    }
    cnn::k_mse<<<parts, 256, 0, s>>>(pred, target, n, npix, lam != 0.0f ? merr : nullptr, lam, grad, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !grad16) return e;
    return cnn_to_bf16(grad, n, grad16, s);
}

cudaError_t cnn_adam(float* p, const float* g, float* m, float* v, long long n, float lr, float b1, float b2, float eps,
                     int t, cudaStream_t s) {
    const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
    cnn::k_adam<<<(int)((n + 255) / 256), 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t cnn_to_bf16(const float* a, long long n, void* b, cudaStream_t s) {
    cnn::k_f32_to_bf16<<<(int)((n + 255) / 256), 256, 0, s>>>(a, n, static_cast<__nv_bfloat16*>(b));
    return cudaGetLastError();
}


}  // namespace plbm
