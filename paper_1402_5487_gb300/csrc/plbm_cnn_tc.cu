// 64 -> 64 circular 3x3 convolution on the 5th-generation tensor cores
// (tcgen05.mma, accumulators in tensor memory), sm_103a.
//
// Implicit GEMM per tile of 128 output pixels of one row: D[128 x 64] =
// sum over 9 taps and 4 K-steps of A_tap[128 x 16] B_tap[16 x 64], with
// A_tap the input pixels shifted by the tap (K-major: 64 channels = one
// 128-byte row per pixel) and B_tap the tap's weights (K-major: one 128-byte
// row per output channel).  Every operand tile starts on a 1024-byte boundary
// and is stored with the 128-byte swizzle (16-byte chunk index XOR row % 8), the
// layout the shared-memory matrix descriptors name; the three horizontal taps
// of a row get their own shifted copy of the input so that no tile starts
// inside a swizzle period.
//
// One elected thread issues the 36 MMAs of a tile and commits them to an
// mbarrier; all 256 threads then read the 128 x 64 FP32 accumulator from
// tensor memory (warp w: lanes 32 (w % 4).., columns 32 (w / 4)..) and run the
// epilogue.  Waits are bounded: on a timeout the kernel records it in *err,
// stops issuing work, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "plbm_internal.h"

namespace plbm {
namespace tc {

constexpr int kC = 64;
constexpr int kTile = 128;
constexpr int kThreads = 256;
constexpr int kATile = kTile * 128;       // 16 KB per tap
constexpr int kBTile = kC * 128;          // 8 KB per tap
constexpr int kSmemA = 9 * kATile;        // 147456
constexpr int kSmemB = 9 * kBTile;        // 73728
constexpr int kSmem = kSmemA + kSmemB + 1024 + 64;  // + alignment slack + barrier/tmem slot
constexpr unsigned kTmemCols = 64;
constexpr long long kSpinLimit = 1LL << 26;

__device__ __forceinline__ uint32_t s2u(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ int swz(int row, int c) { return (row * 8 + (c ^ (row & 7))) * 16; }

__device__ __forceinline__ void cp_async16(uint32_t smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem), "l"(gmem));
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);          // start address
    d |= (uint64_t)1 << 16;                          // leading byte offset (unused with swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset
    d |= (uint64_t)1 << 46;                          // descriptor version
    d |= (uint64_t)2 << 61;                          // 128-byte swizzle
    return d;
}

// Instruction descriptor of kind::f16: D fp32, A and B bf16, both K-major, N = 64, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kC >> 3) << 17) |
                            ((uint32_t)(kTile >> 4) << 24);

__device__ __forceinline__ void mma_issue(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate));
}

__device__ __forceinline__ bool wait_parity(uint32_t bar, uint32_t parity) {
    for (long long i = 0; i < kSpinLimit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity));
        if (done) return true;
    }
    return false;
}

// mode 0: Y = relu?(conv(X) + bias); mode 1: Y = conv(X) * (mask > 0).  Wk: K-major
// weights [tap][n][k] bf16 (n = output channel, k = input channel).
__global__ void __launch_bounds__(kThreads, 1)
k_conv64_tc(int B, int H, int W, const __nv_bfloat16* __restrict__ X, const __nv_bfloat16* __restrict__ Wk,
            const float* __restrict__ bias, const __nv_bfloat16* __restrict__ mask, __nv_bfloat16* __restrict__ Y,
            int mode, int relu, unsigned* __restrict__ err) {
    extern __shared__ unsigned char dsm_raw[];
    // 1024-byte aligned operand area
    const uint32_t raw = s2u(dsm_raw);
    const uint32_t pad = (1024 - (raw & 1023)) & 1023;
    unsigned char* base = dsm_raw + pad;
    const uint32_t sA = raw + pad;
    const uint32_t sB = sA + kSmemA;
    unsigned char* slot = base + kSmemA + kSmemB;
    const uint32_t bar = s2u(slot);
    volatile uint32_t* tmem_slot = reinterpret_cast<volatile uint32_t*>(slot + 16);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(slot + 32);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_x = W / kTile;
    const int ntiles = B * H * tiles_x;

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
        *abort_flag = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(s2u(slot + 16)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    // weights: 9 taps x 64 rows x 8 chunks
    for (int i = tid; i < 9 * kC * 8; i += kThreads) {
        const int c = i & 7, row = i >> 3;  // row = tap * 64 + n
        cp_async16(sB + swz(row, c), Wk + (size_t)row * kC + c * 8);
    }
    asm volatile("cp.async.wait_all;\n" ::);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    const uint32_t tmem = *tmem_slot;

    uint32_t phase = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int b = t / (H * tiles_x);
        const int rem = t - b * H * tiles_x;
        const int y = rem / tiles_x;
        const int x0 = (rem - y * tiles_x) * kTile;
        // A tiles: tap (ky, kx) row r holds input pixel (y + ky - 1, x0 + r + kx - 1)
        for (int i = tid; i < 9 * kTile * 8; i += kThreads) {
            const int c = i & 7, rr = i >> 3, tap = rr >> 7, r = rr & (kTile - 1);
            const int ky = tap / 3, kx = tap - 3 * ky;
            int yy = y + ky - 1;
            yy += (yy < 0) ? H : 0;
            yy -= (yy >= H) ? H : 0;
            int xx = x0 + r + kx - 1;
            xx += (xx < 0) ? W : 0;
            xx -= (xx >= W) ? W : 0;
            cp_async16(sA + tap * kATile + swz(r, c), X + (((size_t)b * H + yy) * W + xx) * kC + c * 8);
        }
        asm volatile("cp.async.wait_all;\n" ::);
        asm volatile("fence.proxy.async.shared::cta;\n" ::);
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
            uint32_t acc = 0;
            for (int tap = 0; tap < 9; ++tap)
                for (int k = 0; k < 4; ++k) {
                    mma_issue(tmem, smem_desc(sA + tap * kATile + k * 32), smem_desc(sB + tap * kBTile + k * 32), acc);
                    acc = 1;
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar));
        }
        const bool ok = wait_parity(bar, phase);
        phase ^= 1;
        if (!ok) *abort_flag = 1;
        __syncthreads();
        if (*abort_flag) break;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
        // accumulator rows 32 (warp % 4) + lane, columns 32 (warp / 4) .. + 31
        uint32_t v[32];
        const uint32_t taddr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(32 * (warp >> 2));
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
              "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
              "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
        const int px = 32 * (warp & 3) + lane;
        const int cb = 32 * (warp >> 2);
        const size_t pix = ((size_t)b * H + y) * W + x0 + px;
#pragma unroll
        for (int q = 0; q < 4; ++q) {  // 8 channels per 16-byte store
            float f[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) f[k] = __uint_as_float(v[8 * q + k]);
            if (mode == 0) {
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    f[k] += bias[cb + 8 * q + k];
                    if (relu) f[k] = fmaxf(f[k], 0.0f);
                }
            } else {
                const uint4 mk = *reinterpret_cast<const uint4*>(mask + pix * kC + cb + 8 * q);
                const __nv_bfloat16* m = reinterpret_cast<const __nv_bfloat16*>(&mk);
#pragma unroll
                for (int k = 0; k < 8; ++k) f[k] = __bfloat162float(m[k]) > 0.0f ? f[k] : 0.0f;
            }
            uint4 o;
            __nv_bfloat162* ob = reinterpret_cast<__nv_bfloat162*>(&o);
#pragma unroll
            for (int k = 0; k < 4; ++k) ob[k] = __floats2bfloat162_rn(f[2 * k], f[2 * k + 1]);
            *reinterpret_cast<uint4*>(Y + pix * kC + cb + 8 * q) = o;
        }
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
        __syncthreads();
    }
    if (*abort_flag && tid == 0) atomicOr(err, 1u);
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols));
    }
}

// K-major weight layouts from W[tap][ci][co] (bf16):
// forward: Wk[tap][co][ci] = W[tap][ci][co]; backward data: Wk[tap][ci][co] = W[8 - tap][ci][co].
__global__ void k_weights_kmajor(const __nv_bfloat16* __restrict__ W, __nv_bfloat16* __restrict__ Wf,
                                 __nv_bfloat16* __restrict__ Wb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 9 * kC * kC) return;
    const int co = i % kC, ci = (i / kC) % kC, tap = i / (kC * kC);
    const __nv_bfloat16 w = W[i];
    Wf[(tap * kC + co) * kC + ci] = w;
    Wb[((8 - tap) * kC + ci) * kC + co] = w;
}

}  // namespace tc

static int tc_sms() {
    static int n = 0;
    if (!n) {
        int d = 0;
        cudaGetDevice(&d);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d);
        if (n <= 0) n = 1;
    }
    return n;
}

cudaError_t cnn_conv64_tc(int B, int H, int W, const void* X, const void* Wk, const float* bias, const void* mask,
                          void* Y, int mode, int relu, unsigned* err, cudaStream_t s) {
    if (W % tc::kTile) return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(tc::k_conv64_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::kSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int ntiles = B * H * (W / tc::kTile);
    const int grid = ntiles < tc_sms() ? ntiles : tc_sms();
    tc::k_conv64_tc<<<grid, tc::kThreads, tc::kSmem, s>>>(
        B, H, W, static_cast<const __nv_bfloat16*>(X), static_cast<const __nv_bfloat16*>(Wk), bias,
        static_cast<const __nv_bfloat16*>(mask), static_cast<__nv_bfloat16*>(Y), mode, relu, err);
    return cudaGetLastError();
}

cudaError_t cnn_weights_kmajor(const void* W, void* Wf, void* Wb, cudaStream_t s) {
    tc::k_weights_kmajor<<<(9 * 64 * 64 + 255) / 256, 256, 0, s>>>(
        static_cast<const __nv_bfloat16*>(W), static_cast<__nv_bfloat16*>(Wf), static_cast<__nv_bfloat16*>(Wb));
    return cudaGetLastError();
}

}  // namespace plbm
