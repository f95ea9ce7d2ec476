// Circular 3x3 convolutions of the surrogate on the 5th-generation tensor
// cores (tcgen05.mma, accumulators in tensor memory), sm_103a.
//
// Implicit GEMM per tile of 128 output pixels of one row segment:
// D[128 x N] = sum over 9 taps (ky, kx) and 4 K-steps of A[128 x 16] B[16 x N],
// A = input pixels shifted by the tap, B = the tap's weights.
//
// k_conv_ring<N, MODE, BITS> (64 input channels: the 64 -> 64 layers and the
// 64 -> 4 output layer with N = 16, four columns used; BITS: a forward pass that
// also records each pixel's ReLU bits, one uint64_t, for the backward pass, whose
// MODE 1 reads them instead of the 128-byte activations) is warp-specialised and
// pipelined:
//   * the CTA's tile range is cut into two streams, each with its own warps,
//     row slots, accumulators and staging tile (below, per stream);
//   * two loader warps stage input row segments (pixels x0 - 1 .. x0 + 128,
//     wrapped) into the stream's ring of shared-memory slots: lane 0 issues
//     eight TMA tile copies (cp.async.bulk.tensor, one per 16-byte channel
//     chunk) of the 128 pixels x0 .. x0 + 127, completing on the slot's
//     mbarrier by byte count, and 16 lanes copy the two wrapped halo pixels and
//     arrive on it.
//     A CTA owns a run of consecutive output rows of one column of tiles, so
//     each input row is loaded once;
//   * one issuing thread walks the input rows in order.  Input row y_in feeds
//     the output rows y_in + 1, y_in, y_in - 1 through the taps ky = 0, 1, 2;
//     with the weights of the three taps (ky, kx) stacked along N and the
//     accumulators of consecutive output rows in descending TMEM columns, the
//     three products of one (kx, K-step) are one MMA of N = 3 x 64, 12 MMAs per
//     input row, and A, the shifted input row, is read from shared memory once
//     per input row instead of three times per output row.  Commits hand each
//     finished accumulator to the epilogue and each consumed row slot back to
//     the loaders;
//   * four epilogue warps read the accumulator (warp w owns TMEM lanes
//     32 (w % 4) ..), hand it back and, for N = 64, write the tile's outputs into a shared
//     staging tile in the 128-byte swizzle that one TMA store sends out.  The
//     threads' own stores (128 bytes per pixel, pixels 128 bytes apart: 32 L1
//     wavefronts per warp instruction) held up the MMAs' operand reads.
// The row slots use the no-swizzle K-major layout with one plane per 16-byte
// channel chunk (pixel p, chunk c at c * plane + 16 p): 8-row core matrices are
// contiguous 128-byte blocks, so the tap shift kx is a 16 * kx byte offset of
// the descriptor start.  The weights use the 128-byte swizzle (1024-byte
// aligned 8-row atoms).
//
// k_conv_in_tc is the 4 -> 64 input layer: the 36 products of a pixel (9 taps
// x 4 channels) are gathered into one K = 48 row (zero padded) and three MMAs
// make the tile.
//
// k_wgrad_tc, k_wgrad_in_tc and k_wgrad_out_tc are the weight gradients of the
// 64 -> 64 layers, the 4 -> 64 input layer and the 64 -> 4 output layer: the
// reduction over pixels is the K dimension, both operands MN-major.
//
// Every wait is bounded by the global timer: on a timeout a kernel records it
// in *err, stops issuing work, waits (bounded) for the MMAs it issued, frees
// its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstdint>

#include "plbm_internal.h"

namespace plbm {
namespace tc {

constexpr int kC = 64;
constexpr int kTile = 128;
constexpr unsigned long long kTimeoutNs = 2000000000ull;  // 2 s: default wait budget and the drain bound

__device__ __forceinline__ uint32_t s2u(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ int swz(int row, int c) { return (row * 8 + (c ^ (row & 7))) * 16; }
__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

__device__ __forceinline__ uint64_t gtime() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}
__device__ __forceinline__ void cp_async16(uint32_t smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem), "l"(gmem) : "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }

__device__ __forceinline__ void bar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint32_t bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}\n" ::"r"(bar) : "memory");
}
// One potentially blocking test of the phase: the thread may be suspended (up
// to the hint, 10 ms) until the phase completes, so waiting warps do not take
// issue slots from the warps that work.
__device__ __forceinline__ bool bar_try(uint32_t bar, uint32_t parity, uint32_t hint_ns = 10000000u) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity), "r"(hint_ns)
        : "memory");
    return done != 0;
}
// Budgets below this are checked on every poll with non-blocking tests (a
// suspended try_wait may outlast a short hint); the default budget takes the
// suspending path.
constexpr unsigned long long kShortBudgetNs = 10000000ull;
__device__ __forceinline__ bool bar_test(uint32_t bar, uint32_t parity);
// Wait for the phase of parity `parity` of `bar`; false once budget_ns have
// passed (which sets *abort) or when another role has already set *abort.
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity, volatile int* abort,
                                         unsigned long long budget_ns) {
    if (budget_ns < kShortBudgetNs) {
        const uint64_t t0 = gtime();
        for (;;) {
            if (bar_test(bar, parity)) return true;
            if (*abort) return false;
            if (gtime() - t0 > budget_ns) {
                *abort = 1;
                return false;
            }
        }
    }
    if (bar_try(bar, parity)) return true;
    const uint64_t t0 = gtime();
    for (;;) {
        if (bar_try(bar, parity)) return true;
        if (*abort) return false;
        if (gtime() - t0 > budget_ns) {
            *abort = 1;
            return false;
        }
    }
}
// Non-blocking test of the phase, for the MMA issuer: it must not be suspended
// while the tensor pipe could take more work.  Its shared-memory reads queue
// behind the tensor cores' operand reads, so the issuer tests several phases
// at once (test_many) instead of one per tile.
__device__ __forceinline__ bool bar_test(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}
__device__ __forceinline__ bool bar_spin(uint32_t bar, uint32_t parity, volatile int* abort,
                                         unsigned long long budget_ns) {
    if (bar_test(bar, parity)) return true;
    const uint64_t t0 = gtime();
    const uint32_t every = budget_ns < kShortBudgetNs ? 0u : 255u;   // short budgets: check every poll
    for (uint32_t i = 1;; ++i) {
        if (bar_test(bar, parity)) return true;
        if ((i & every) == 0) {
            if (*abort) return false;
            if (gtime() - t0 > budget_ns) {
                *abort = 1;
                return false;
            }
        }
    }
}
// Tests of up to 4 barrier phases issued together; returns how many of them, in
// order, have completed.  Each queried phase must be at most one ahead of a
// phase known to be complete on the same barrier (a parity test cannot tell a
// phase from the one two before it).
__device__ __forceinline__ int test_many(const uint32_t (&bars)[4], const uint32_t (&par)[4], int n) {
    uint32_t d[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) d[k] = k < n ? (bar_test(bars[k], par[k]) ? 1u : 0u) : 0u;
    int c = 0;
    while (c < n && d[c]) ++c;
    return c;
}
// The same without looking at *abort, bounded by the fixed kTimeoutNs whatever
// the wait budget (used to drain issued MMAs before freeing TMEM).
__device__ __forceinline__ bool bar_wait_drain(uint32_t bar, uint32_t parity) {
    const uint64_t t0 = gtime();
    for (;;) {
        if (bar_try(bar, parity)) return true;
        if (gtime() - t0 > kTimeoutNs) return false;
    }
}

__device__ __forceinline__ void bar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}\n" ::"r"(bar),
                 "r"(bytes)
                 : "memory");
}
// TMA tile copy of a 5D box to shared memory, completing `bar` by byte count.
__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            int c4, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
        "%6}], [%7];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
        : "memory");
}

// TMA tile store of a 2D box from shared memory (bulk async group of this thread).
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int c0, int c1, uint32_t src) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];\n" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(c0), "r"(c1), "r"(src)
                 : "memory");
}
// Named barrier `id` over `n` threads that also returns the OR of their predicates.
__device__ __forceinline__ bool bar_or(int id, int n, bool pred) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "barrier.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(id), "r"(n)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ void bar_named(int id, int n) { asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(n) : "memory"); }

__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                 : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t slot_addr, uint32_t cols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(slot_addr), "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t tmem, uint32_t cols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(cols) : "memory");
}

// Shared-memory matrix descriptors (K-major).
// 128-byte swizzle: 8-row atoms of 1024 bytes (stride byte offset 1024).
__device__ __forceinline__ uint64_t desc_sw128(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// No swizzle: 8 rows x 16 bytes core matrices; `kstride` bytes between the two
// core matrices of a K = 16 step (leading byte offset), 128 bytes between
// 8-row groups (stride byte offset).
__device__ __forceinline__ uint64_t desc_plain(uint32_t addr, uint32_t kstride) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(kstride >> 4) << 16) | ((uint64_t)(128 >> 4) << 32) |
           ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: D fp32, A and B bf16, both K-major, M = 128.
template <int N>
struct Idesc {
    static constexpr uint32_t value = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
                                      ((uint32_t)(kTile >> 4) << 24);
};

// The same for N known at run time (a multiple of 16, 16..256).
__device__ __forceinline__ uint32_t idesc_n(uint32_t n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((uint32_t)(kTile >> 4) << 24);
}
__device__ __forceinline__ void mma_n(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

template <int N>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(Idesc<N>::value), "r"(accumulate)
        : "memory");
}

#define PLBM_TMEM_LD32(v, base, addr)                                                                               \
    asm volatile(                                                                                                   \
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"            \
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"                                \
        : "=r"(v[base + 0]), "=r"(v[base + 1]), "=r"(v[base + 2]), "=r"(v[base + 3]), "=r"(v[base + 4]),           \
          "=r"(v[base + 5]), "=r"(v[base + 6]), "=r"(v[base + 7]), "=r"(v[base + 8]), "=r"(v[base + 9]),           \
          "=r"(v[base + 10]), "=r"(v[base + 11]), "=r"(v[base + 12]), "=r"(v[base + 13]), "=r"(v[base + 14]),      \
          "=r"(v[base + 15]), "=r"(v[base + 16]), "=r"(v[base + 17]), "=r"(v[base + 18]), "=r"(v[base + 19]),      \
          "=r"(v[base + 20]), "=r"(v[base + 21]), "=r"(v[base + 22]), "=r"(v[base + 23]), "=r"(v[base + 24]),      \
          "=r"(v[base + 25]), "=r"(v[base + 26]), "=r"(v[base + 27]), "=r"(v[base + 28]), "=r"(v[base + 29]),      \
          "=r"(v[base + 30]), "=r"(v[base + 31])                                                                    \
        : "r"(addr)                                                                                                 \
        : "memory")

// The 64 outputs of pixel px (its TMEM lane's 64 accumulator columns) into a
// shared tile of 128 pixels x 128 bytes in the 128-byte swizzle of a TMA box
// (16-byte chunk q of pixel p at p * 128 + (q ^ (p mod 8)) * 16): the 32 lanes
// of a warp store 512 bytes per instruction without bank conflicts.  Mode 0:
// relu?(acc + bias); with want_bits the return value holds the pixel's ReLU bits
// (bit c: stored bf16 output c > 0, i.e. its bit pattern h has 1 <= h <= 0x7F80,
// +inf included, NaN not).  Mode 1: acc where bit c of mbits is set, else 0.
__device__ __forceinline__ uint64_t stage64(const uint32_t (&v)[64], int mode, int relu, const float* __restrict__ bias,
                                            uint64_t mbits, bool want_bits, uint32_t stage, int px) {
    uint32_t bits[2] = {0u, 0u};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        float f[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) f[k] = __uint_as_float(v[8 * q + k]);
        if (mode == 0) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                f[k] += bias[8 * q + k];
                if (relu) f[k] = fmaxf(f[k], 0.0f);
            }
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) f[k] = (mbits >> (8 * q + k)) & 1u ? f[k] : 0.0f;
        }
        const uint32_t a = stage + (uint32_t)px * 128u + (uint32_t)((q ^ (px & 7)) * 16);
        uint32_t o[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(f[2 * k], f[2 * k + 1]);
            o[k] = *reinterpret_cast<const uint32_t*>(&h);
        }
        if (mode == 0 && want_bits) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                bits[q >> 2] |= (uint32_t)(((o[k] & 0xFFFFu) - 1u) < 0x7F80u) << (8 * (q & 3) + 2 * k);
                bits[q >> 2] |= (uint32_t)(((o[k] >> 16) - 1u) < 0x7F80u) << (8 * (q & 3) + 2 * k + 1);
            }
        }
        asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};\n" ::"r"(a), "r"(o[0]), "r"(o[1]), "r"(o[2]), "r"(o[3])
                     : "memory");
    }
    return (uint64_t)bits[1] << 32 | bits[0];
}

// ---------------------------------------------------------------------------
// Ring-staged convolution with 64 input channels.
// MODE 0: Y bf16 [.][64] = relu?(conv + bias)    (N = 64)
// MODE 1: Y bf16 [.][64] = conv * relu bit       (N = 64, backward data)
// MODE 2: Y fp32 [.][4]  = conv + bias           (N = 16, output columns 0..3)
// Wk: bf16 [9 taps][N][64], K-major.
// ---------------------------------------------------------------------------
// Streams: the CTA works on the two halves of its tile range at once, each with
// its own issuer, row slots, accumulators (256 TMEM columns) and epilogue warps,
// so that one issuer's barrier tests and set-up between rows overlap the other
// stream's MMAs.  At B = 16 a 64 -> 64 layer takes 71.8 us with two streams and
// 106.7 us with one (8 row slots, 8 accumulators).
constexpr int kStreams = 2;
constexpr int kLoadersPer = 2;         // loader warps per stream
constexpr int kLoaders = kStreams * kLoadersPer;
constexpr int kIssuers = kStreams;     // warp kLoaders + q issues the MMAs of stream q
constexpr int kEpiWarps = 4;           // epilogue warps per stream
constexpr int kRingThreads = 32 * (kLoaders + kIssuers + kStreams * kEpiWarps);
constexpr int kSegPix = kTile + 2;     // staged pixels per input row: x0 - 1 .. x0 + 128
// One 16-byte channel chunk of every staged pixel (pixel p at 16 p).  A plane
// starts 112 bytes into a 128-byte line, so pixel 1 (x0), the destination of
// the TMA copy, is 128-byte aligned; planes are 17 lines apart.
constexpr int kPlane = 17 * 128;       // 2176 bytes >= 130 pixels x 16 bytes
constexpr int kPlaneOff = 112;
constexpr int kSeg = 8 * kPlane;       // 17408 bytes per staged row
static_assert(kSegPix * 16 <= kPlane && (kPlaneOff + 16) % 128 == 0 && kSeg % 128 == 0, "row slot layout");
constexpr int kRingS = 3;              // row slots per stream (slots kRingS q ..)
constexpr int kRing = kStreams * kRingS;
// A loader waits for the release of the row kRingS before its own; the row it
// loaded before that one is at most kRingS rows back, so that release's
// previous phase has completed and a parity test cannot be fooled.
static_assert(kLoadersPer <= kRingS, "loader lag within the row ring");
constexpr int kHaloLanes = 16;         // two wrapped pixels x 8 chunks
constexpr uint32_t kRowTxBytes = 8 * kTile * 16;  // the eight TMA boxes of a row
constexpr int kRingBytes = kRing * kSeg + kPlaneOff;
constexpr int kRingSOff = ((kRingBytes + 1023) / 1024) * 1024;  // output staging tiles after the ring
constexpr int kStageBytes = kTile * kC * 2;                      // 128 pixels x 64 bf16 (N = 64 modes)
template <int N>
__host__ __device__ constexpr int ring_woff() { return kRingSOff + (N == 64 ? kStreams * kStageBytes : 0); }
constexpr int kRingBarBytes = 512 + 256;  // barriers, TMEM slot, abort flag, then 64 fp32 biases
template <int N>
constexpr int ring_smem() { return 1024 + ring_woff<N>() + 9 * N * 128 + kRingBarBytes; }
static_assert(ring_smem<64>() <= 232448, "ring kernel shared memory within the 227 KB a CTA may use");
constexpr uint32_t kRingTmemCols = 512;
constexpr uint32_t kStreamCols = kRingTmemCols / kStreams;   // stream q: columns kStreamCols q ..
constexpr int kAccS = (int)kStreamCols / 64;                 // accumulators per stream, N columns each
// Accumulator of the stream's tile u: descending, so that the tiles of output
// rows y + 1, y, y - 1 (consecutive u) sit in ascending TMEM columns.
__device__ __forceinline__ uint32_t acc_slot(uint32_t u) { return (uint32_t)(kAccS - (int)(u % kAccS)) % kAccS; }

// barrier slots (8 bytes each) after the weights: per row slot a full and an
// empty barrier, per stream and accumulator a full and an empty barrier, per
// issuer a drain barrier
constexpr int kBarFull = 0, kBarEmpty = kRing, kBarTFull = 2 * kRing, kBarTEmpty = kBarTFull + kStreams * kAccS,
              kBarDrain = kBarTEmpty + kStreams * kAccS, kBarCount = kBarDrain + kIssuers;
static_assert(kBarCount * 8 + 16 <= 512, "barrier area below the biases");

// Tiles t = ((b * tiles_x + xt) * H + y); a CTA takes a contiguous range, which
// splits into strips of consecutive rows y of one column (b, xt).
struct Strip {
    int b, x0, y0, n;
};
__device__ __forceinline__ Strip strip_at(int t, int t1, int H, int tiles_x) {
    const int col = t / H, y0 = t - col * H;
    Strip s;
    s.b = col / tiles_x;
    s.x0 = (col - s.b * tiles_x) * kTile;
    s.y0 = y0;
    s.n = min(t1 - t, H - y0);
    return s;
}

// tmX views X as the 5D tensor [B][H][W][8 chunks][8 channels] (innermost last)
// with a box of 128 pixels x 1 chunk.
template <int N, int MODE, bool BITS>
__global__ void __launch_bounds__(kRingThreads, 1)
k_conv_ring(int B, int H, int W, const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY,
            const __nv_bfloat16* __restrict__ X, const __nv_bfloat16* __restrict__ Wk, const float* __restrict__ bias,
            uint64_t* __restrict__ rbits, void* __restrict__ Yv, int relu, const TcErr err) {
    static_assert((N == 64 && MODE < 2) || (N == 16 && MODE == 2), "ring conv shapes");
    static_assert(!BITS || MODE == 0, "ReLU bits come from the forward pass");
    static_assert(kAccS * N <= (int)kStreamCols, "a stream's accumulators fit its share of the TMEM columns");
    extern __shared__ unsigned char dsm_raw[];
    const uint32_t raw = s2u(dsm_raw);
    const uint32_t pad = (1024 - (raw & 1023)) & 1023;
    unsigned char* base = dsm_raw + pad;
    const uint32_t sRing = raw + pad;
    const uint32_t sW = sRing + ring_woff<N>();
    unsigned char* bars_p = base + ring_woff<N>() + 9 * N * 128;
    const uint32_t bars = s2u(bars_p);
    volatile uint32_t* tmem_slot = reinterpret_cast<volatile uint32_t*>(bars_p + kBarCount * 8);
    volatile int* abortp = reinterpret_cast<volatile int*>(bars_p + kBarCount * 8 + 8);
    float* sbias = reinterpret_cast<float*>(bars_p + 512);
    auto bar = [&](int i) { return bars + 8u * (uint32_t)i; };

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_x = W / kTile;
    const int ntiles = B * H * tiles_x;
    const int per = (ntiles + gridDim.x - 1) / gridDim.x;
    const int t_begin = min(ntiles, (int)blockIdx.x * per);
    const int t_end = min(ntiles, t_begin + per);
    // stream q: tiles [tq0(q), tq1(q)), the CTA's range cut into kStreams parts
    auto tq0 = [&](int q) { return t_begin + (int)((long long)(t_end - t_begin) * q / kStreams); };
    auto tq1 = [&](int q) { return t_begin + (int)((long long)(t_end - t_begin) * (q + 1) / kStreams); };

    if (tid == 0) {
        for (int i = 0; i < kRing; ++i) {
            bar_init(bar(kBarFull + i), 1 + kHaloLanes);
            bar_init(bar(kBarEmpty + i), 1);
        }
        for (int i = 0; i < kStreams * kAccS; ++i) {
            bar_init(bar(kBarTFull + i), 1);
            bar_init(bar(kBarTEmpty + i), 32 * kEpiWarps);
        }
        for (int i = 0; i < kIssuers; ++i) bar_init(bar(kBarDrain + i), 1);
        *abortp = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == kLoaders) tmem_alloc(s2u(bars_p + kBarCount * 8), kRingTmemCols);
    for (int i = tid; i < 9 * N * 8; i += kRingThreads) {  // weights: 9 N rows of 8 chunks, swizzled
        const int c = i & 7, row = i >> 3;
        const int tap = row / N, n = row - tap * N, ky = tap / 3, kx = tap - 3 * ky;
        cp_async16(sW + swz((kx * 3 + ky) * N + n, c), Wk + (size_t)row * kC + c * 8);
    }
    if (MODE != 1 && tid < (MODE == 2 ? 4 : 64)) sbias[tid] = bias[tid];
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp < kLoaders) {
        // ---- loaders: stream q = warp / 2 loads its rows k = warp mod 2, + 2, ...
        // (rows y0 - 1 .. y0 + n of every strip, in order) into its row slots
        // 4 q + k mod 4.  Lane 0 arms the slot's full barrier with the TMA byte
        // count and issues the eight chunk copies; lanes 0..15 copy the halo
        // pixels x0 - 1 and x0 + 128 (wrapped) and arrive after a proxy fence.
        // Nothing waits for the TMA data here: the issuer does. ----
        const int q = warp / kLoadersPer, r = warp % kLoadersPer;
        if (lane == 0) asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&tmX)) : "memory");
        uint32_t k = 0;
        bool ok = true;
        for (int t = tq0(q); t < tq1(q) && ok;) {
            const Strip s = strip_at(t, tq1(q), H, tiles_x);
            for (int j = 0; j < s.n + 2; ++j, ++k) {
                if ((int)(k % kLoadersPer) != r) continue;
                const int slot = q * kRingS + (int)(k % kRingS);
                const uint32_t par = ((k / kRingS) & 1) ^ 1;
                if (!bar_wait(bar(kBarEmpty + slot), par, abortp, err.wait_ns)) {
                    ok = false;
                    break;
                }
                const int yy = wrapi(s.y0 - 1 + j, H);
                const uint32_t seg = sRing + (uint32_t)slot * kSeg + kPlaneOff;
                const uint32_t full = bar(kBarFull + slot);
                if (lane == 0) {
                    bar_arrive_expect_tx(full, kRowTxBytes);
#pragma unroll
                    for (int c = 0; c < 8; ++c) tma_load_5d(seg + c * kPlane + 16, &tmX, 0, c, s.x0, yy, s.b, full);
                }
                if (lane < kHaloLanes) {
                    // halo chunks by the threads (loads, shared stores, a proxy fence and
                    // an arrival): 16-byte bulk copies cost more
                    const int right = lane >> 3, c = lane & 7;
                    const int xx = wrapi(right ? s.x0 + kTile : s.x0 - 1, W);
                    const uint4 v = __ldg(reinterpret_cast<const uint4*>(
                        X + (((size_t)s.b * H + yy) * (size_t)W + xx) * kC + c * 8));
                    const uint32_t dst = seg + c * kPlane + (right ? 16 * (kSegPix - 1) : 0);
                    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};\n" ::"r"(dst), "r"(v.x), "r"(v.y),
                                 "r"(v.z), "r"(v.w)
                                 : "memory");
                    fence_async_smem();
                    bar_arrive(full);
                }
            }
            t += s.n;
        }
    } else if (warp < kLoaders + kIssuers) {
        const int q = warp - kLoaders;
        if (lane == 0) {
            // ---- MMA issuer of stream q.  Input row e of a strip of n output rows
            // (pixel row y0 - 1 + e) feeds the strip's tiles i = e - ky through the
            // taps ky in [ky_lo, ky_hi]: with the weights of the three taps (ky, kx)
            // stacked along N (shared-memory rows (kx * 3 + ky) N + n) and the
            // accumulators of consecutive tiles in descending TMEM columns, one
            // MMA of up to 3 N columns per (kx, K-step) feeds all three, and A, the
            // shifted input row, is read once per input row.  Tile i = e opens
            // (zeroes its accumulator) with the first MMA of row e; tile i = e - 2
            // is complete after row e. ----
            const uint64_t a0 = desc_plain(sRing + kPlaneOff, kPlane);
            const uint64_t b0 = desc_sw128(sW);
            const uint32_t cols = tmem + kStreamCols * (uint32_t)q;
            uint32_t k = 0, T0 = 0, freed = 0;
            bool ok = true, issued = false;
            for (int t = tq0(q); t < tq1(q) && ok;) {
                const Strip s = strip_at(t, tq1(q), H, tiles_x);
                for (int e = 0; e < s.n + 2; ++e, ++k) {
                    const uint32_t row_slot = q * kRingS + k % kRingS;
                    ok = bar_spin(bar(kBarFull + row_slot), (k / kRingS) & 1, abortp, err.wait_ns);
                    const int ky_lo = max(0, e - (s.n - 1)), ky_hi = min(2, e);
                    if (ok && ky_lo == 0 && T0 + e >= (uint32_t)kAccS) {
                        // tile T0 + e reuses the accumulator of tile T0 + e - kAccS; the
                        // epilogue releases the tiles in order
                        const uint32_t want = T0 + e - kAccS;
                        if (freed <= want) {
                            ok = bar_spin(bar(kBarTEmpty + q * kAccS + acc_slot(want)), (want / kAccS) & 1, abortp,
                                          err.wait_ns);
                            freed = want + 1;
                        }
                    }
                    if (!ok) break;
                    tc_after_sync();
                    // The MMAs of one (kx, K-step), as segments of taps ky: the opening
                    // product of tile e alone, otherwise as many taps as fit before
                    // the accumulators wrap around the stream's columns (at most
                    // three segments); f = 0 for the first (kx, K-step), 1 for the rest.
                    const uint32_t s_lo = acc_slot(T0 + e - ky_lo);
                    const uint64_t arow = a0 + ((row_slot * kSeg) >> 4);
                    if (ky_lo == 0 && ky_hi == 2 && s_lo + 2 < (uint32_t)kAccS) {
                        // an interior row whose three accumulators do not wrap (the common
                        // case): the opening product, then one MMA of 3 N columns each
                        const uint32_t d = cols + s_lo * N;
                        const uint32_t i1 = idesc_n(N), i2 = idesc_n(2 * N), i3 = idesc_n(3 * N);
#pragma unroll
                        for (int kx = 0; kx < 3; ++kx)
#pragma unroll
                            for (int ks = 0; ks < 4; ++ks) {
                                const uint64_t a = arow + ((kx * 16 + ks * 2 * kPlane) >> 4);
                                const uint64_t b = b0 + ((kx * 3 * N * 128 + ks * 32) >> 4);
                                if (kx == 0 && ks == 0) {
                                    mma_n(d, a, b, i1, 0u);
                                    mma_n(d + N, a, b + ((N * 128) >> 4), i2, 1u);
                                } else {
                                    mma_n(d, a, b, i3, 1u);
                                }
                            }
                    } else if (ky_lo == 0 && ky_hi == 2) {
                        // an interior row whose accumulators wrap: the first w taps at
                        // s_lo, the rest from column 0 (the opening product alone)
                        const uint32_t w = (uint32_t)kAccS - s_lo;   // 1 or 2
                        const uint32_t d = cols + s_lo * N;
                        const uint32_t i1 = idesc_n(N), iw = idesc_n(w * N), ir = idesc_n((3 - w) * N);
                        const uint32_t bw = (w * N * 128) >> 4;
#pragma unroll
                        for (int kx = 0; kx < 3; ++kx)
#pragma unroll
                            for (int ks = 0; ks < 4; ++ks) {
                                const uint64_t a = arow + ((kx * 16 + ks * 2 * kPlane) >> 4);
                                const uint64_t b = b0 + ((kx * 3 * N * 128 + ks * 32) >> 4);
                                if (kx == 0 && ks == 0) {
                                    mma_n(d, a, b, i1, 0u);
                                    if (w == 2) mma_n(d + N, a, b + ((N * 128) >> 4), i1, 1u);
                                } else {
                                    mma_n(d, a, b, iw, 1u);
                                }
                                mma_n(cols, a, b + bw, ir, 1u);
                            }
                    } else {
                        uint32_t sd[2][3], sb[2][3], si[2][3], sa[2][3];
                        bool sv[2][3];
#pragma unroll
                        for (int f = 0; f < 2; ++f) {
                            int kk = ky_lo;
#pragma unroll
                            for (int j = 0; j < 3; ++j) {
                                sv[f][j] = kk <= ky_hi;
                                const bool open = f == 0 && kk == 0;
                                const uint32_t sl = (s_lo + (uint32_t)(kk - ky_lo)) % kAccS;
                                const int end = min(open ? 0 : ky_hi, kk + (int)(kAccS - 1 - sl));
                                sd[f][j] = cols + sl * N;
                                sb[f][j] = (uint32_t)(kk * N * 128) >> 4;
                                si[f][j] = idesc_n((uint32_t)(end - kk + 1) * N);
                                sa[f][j] = open ? 0u : 1u;
                                kk = end + 1;
                            }
                        }
#pragma unroll
                        for (int kx = 0; kx < 3; ++kx)
#pragma unroll
                            for (int ks = 0; ks < 4; ++ks) {
                                const uint64_t a = arow + ((kx * 16 + ks * 2 * kPlane) >> 4);
                                const uint64_t b = b0 + ((kx * 3 * N * 128 + ks * 32) >> 4);
                                const int f = (kx == 0 && ks == 0) ? 0 : 1;
#pragma unroll
                                for (int j = 0; j < 3; ++j)
                                    if (sv[f][j]) mma_n(sd[f][j], a, b + sb[f][j], si[f][j], sa[f][j]);
                            }
                    }
                    if (e >= 2) tc_commit(bar(kBarTFull + q * kAccS + acc_slot(T0 + e - 2)));
                    tc_commit(bar(kBarEmpty + row_slot));
                    issued = true;
                }
                if (!ok) break;
                T0 += s.n;
                t += s.n;
            }
            // every MMA issued has completed before the accumulators are released
            if (issued) {
                tc_commit(bar(kBarDrain + q));
                if (!bar_wait_drain(bar(kBarDrain + q), 0)) *abortp = 1;
            }
        }
        __syncwarp();
    } else {
        // ---- epilogue of stream q: 4 warps, TMEM lanes 32 (warp % 4) .. + 31.  For
        // N = 64 the tile's outputs go through the stream's staging tile (128-byte
        // swizzle) and leave as one TMA store; the four warps decide together
        // whether to go on (a barrier that ORs their wait results). ----
        const int q = (warp - kLoaders - kIssuers) / kEpiWarps;
        const int quad = warp & 3;
        const int px = 32 * quad + lane;
        const bool leader = (warp - kLoaders - kIssuers) % kEpiWarps == 0 && lane == 0;
        const int nb = 1 + q;   // named barrier of the group
        const uint32_t sStage = sRing + kRingSOff + (uint32_t)q * kStageBytes;
        uint32_t u = 0;
        bool ok = true;
        for (int t = tq0(q); t < tq1(q) && ok;) {
            const Strip s = strip_at(t, tq1(q), H, tiles_x);
            for (int i = 0; i < s.n; ++i, ++u) {
                const uint32_t acc = acc_slot(u);
                const size_t pix = ((size_t)s.b * H + s.y0 + i) * W + s.x0 + px;
                // backward data: the pixel's ReLU bits, loaded while the MMAs run
                const uint64_t mb = MODE == 1 ? __ldg(rbits + pix) : 0ull;
                const bool got = bar_wait(bar(kBarTFull + q * kAccS + acc), (u / kAccS) & 1, abortp, err.wait_ns);
                if (bar_or(nb, 32 * kEpiWarps, !got || *abortp)) {
                    ok = false;
                    break;
                }
                tc_after_sync();
                const uint32_t taddr = tmem + ((uint32_t)(32 * quad) << 16) + kStreamCols * q + acc * N;
                if (MODE == 2) {
                    uint32_t v[4];
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];\n"
                                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
                                 : "r"(taddr)
                                 : "memory");
                    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                    tc_before_sync();
                    bar_arrive(bar(kBarTEmpty + q * kAccS + acc));
                    float4 o;
                    o.x = __uint_as_float(v[0]) + sbias[0];
                    o.y = __uint_as_float(v[1]) + sbias[1];
                    o.z = __uint_as_float(v[2]) + sbias[2];
                    o.w = __uint_as_float(v[3]) + sbias[3];
                    reinterpret_cast<float4*>(Yv)[pix] = o;   // 16 bytes per pixel: coalesced
                } else {
                    uint32_t v[64];
                    PLBM_TMEM_LD32(v, 0, taddr);
                    PLBM_TMEM_LD32(v, 32, taddr + 32);
                    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                    tc_before_sync();
                    bar_arrive(bar(kBarTEmpty + q * kAccS + acc));
                    // the previous tile's store has finished reading the staging tile
                    if (leader) asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
                    bar_named(nb, 32 * kEpiWarps);
                    const uint64_t bits = stage64(v, MODE, relu, sbias, mb, BITS, sStage, px);
                    if (BITS) rbits[pix] = bits;   // forward: the ReLU bits for the backward pass
                    fence_async_smem();
                    bar_named(nb, 32 * kEpiWarps);
                    if (leader) {
                        tma_store_2d(&tmY, 0, (int)(pix - px), sStage);
                        asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
                    }
                }
            }
            t += s.n;
        }
        // every store has left the staging tile and reached global memory
        if (leader) asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
    }
    __syncthreads();
    if (tid == 0 && *abortp) {
        atomicOr(err.flag, 1u);
        // TMA copies the loaders issued may not have been waited for: give them
        // time to land (they are plain copies) before the shared memory is released
        const uint64_t t0 = gtime();
        while (gtime() - t0 < 20000000ull) {
        }
    }
    __syncthreads();
    if (warp == kLoaders) {
        tc_after_sync();
        tmem_free(tmem, kRingTmemCols);
    }
}

// ---------------------------------------------------------------------------
// 4 -> 64 input layer: Y bf16 [.][64] = relu?(conv(X) + bias), X bf16 [.][4]
// (mode 0; rbits, when given, receives each pixel's ReLU bits); the same kernel
// computes the output layer's backward data, Y = conv(X) * relu bit with X =
// bf16 upstream gradient [.][4], the flipped weights and the bits rbits of the
// forward pass (mode 1).
// A row of a pixel: K = tap * 4 + ci for the 36 products, zero to K = 48, in the
// no-swizzle chunk-planar layout (6 planes of 128 pixels x 16 bytes).
// Win: bf16 [6 chunks][64 n][8], the same layout for B (plane = 64 x 16 bytes).
// One tile at a time per CTA; several CTAs per SM overlap.  Once a tile's MMAs
// are done, its A region holds the tile's outputs in the 128-byte swizzle of a
// TMA box, and one TMA store writes them (coalesced, off the threads).
// ---------------------------------------------------------------------------
constexpr int kInThreads = 128;
constexpr int kInPlanes = 6;
constexpr int kInA = kInPlanes * kTile * 16;  // 12288
constexpr int kInAS = kTile * kC * 2;         // 16384: A, then the output staging tile
constexpr int kInB = kInPlanes * kC * 16;     // 6144
constexpr int kInBar = 64 + 256;  // barriers, TMEM slot, abort flag, 64 fp32 biases
constexpr int kInSmem = 26 * 1024;  // A/staging, B, barriers and padding that caps residency at 8 CTAs per SM
static_assert(kInA <= kInAS && 1024 + kInAS + kInB + kInBar <= kInSmem, "input-layer shared memory");
constexpr uint32_t kInTmemCols = 64;

template <int MODE, bool BITS>
__global__ void __launch_bounds__(kInThreads)
k_conv_in_tc(int B, int H, int W, const __nv_bfloat16* __restrict__ X, const __nv_bfloat16* __restrict__ Win,
             const float* __restrict__ bias, uint64_t* __restrict__ rbits,
             const __grid_constant__ CUtensorMap tmY, int relu, const TcErr err) {
    static_assert(MODE == 0 || (MODE == 1 && !BITS), "ReLU bits come from the forward pass");
    constexpr int mode = MODE;
    extern __shared__ unsigned char dsm_raw[];
    const uint32_t raw = s2u(dsm_raw);
    const uint32_t pad = (1024 - (raw & 1023)) & 1023;   // the staging tile's swizzle wants 1024-byte alignment
    unsigned char* base = dsm_raw + pad;
    const uint32_t sA = raw + pad;
    const uint32_t sB = sA + kInAS;
    unsigned char* bars_p = base + kInAS + kInB;
    const uint32_t bar_mma = s2u(bars_p), bar_drain = bar_mma + 8;
    volatile uint32_t* tmem_slot = reinterpret_cast<volatile uint32_t*>(bars_p + 16);
    volatile int* abortp = reinterpret_cast<volatile int*>(bars_p + 24);
    float* sbias = reinterpret_cast<float*>(bars_p + 64);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_x = W / kTile;
    const int ntiles = B * H * tiles_x;
    if (tid < 64) sbias[tid] = mode == 0 ? bias[tid] : 0.0f;
    if (tid == 0) {
        bar_init(bar_mma, 1);
        bar_init(bar_drain, 1);
        *abortp = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) tmem_alloc(s2u(bars_p + 16), kInTmemCols);
    for (int i = tid; i < kInB / 16; i += kInThreads)
        *reinterpret_cast<uint4*>(base + kInAS + 16 * i) = reinterpret_cast<const uint4*>(Win)[i];
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = *tmem_slot;
    const uint64_t adesc = desc_plain(sA, kTile * 16);
    const uint64_t bdesc = desc_plain(sB, kC * 16);

    // the gathered inputs of the next tile are loaded while the current tile's MMAs run
    auto gather = [&](int t, uint2 (&g)[9]) {
        const int b = t / (H * tiles_x);
        const int rem = t - b * H * tiles_x;
        const int y = rem / tiles_x;
        const int x = (rem - y * tiles_x) * kTile + tid;
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            const int yy = wrapi(y + tap / 3 - 1, H), xx = wrapi(x + tap % 3 - 1, W);
            g[tap] = *reinterpret_cast<const uint2*>(X + (((size_t)b * H + yy) * W + xx) * 4);
        }
    };
    uint2 g[9];
    if ((int)blockIdx.x < ntiles) gather(blockIdx.x, g);
    uint32_t phase = 0;
    bool issued = false;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int b = t / (H * tiles_x);
        const int rem = t - b * H * tiles_x;
        const int y = rem / tiles_x;
        const int x0 = (rem - y * tiles_x) * kTile;
        const size_t pix = ((size_t)b * H + y) * W + x0 + tid;
        const uint64_t mb = mode == 1 ? __ldg(rbits + pix) : 0ull;   // backward data: the pixel's ReLU bits
        // the previous tile's store has finished reading the region A is written to
        if (tid == 0) asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
        __syncthreads();
        *reinterpret_cast<uint4*>(base + 5 * kTile * 16 + tid * 16) = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int c = 0; c < 4; ++c)
            *reinterpret_cast<uint4*>(base + c * kTile * 16 + tid * 16) =
                make_uint4(g[2 * c].x, g[2 * c].y, g[2 * c + 1].x, g[2 * c + 1].y);
        *reinterpret_cast<uint4*>(base + 4 * kTile * 16 + tid * 16) = make_uint4(g[8].x, g[8].y, 0u, 0u);
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc_after_sync();
#pragma unroll
            for (int ks = 0; ks < 3; ++ks)
                mma<64>(tmem, adesc + ((ks * 2 * kTile * 16) >> 4), bdesc + ((ks * 2 * kC * 16) >> 4), ks != 0);
            tc_commit(bar_mma);
            issued = true;
        }
        if (t + (int)gridDim.x < ntiles) gather(t + gridDim.x, g);
        if (!bar_wait(bar_mma, phase, abortp, err.wait_ns)) *abortp = 1;
        phase ^= 1;
        __syncthreads();
        if (*abortp) break;
        tc_after_sync();
        uint32_t v[64];
        const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16);
        PLBM_TMEM_LD32(v, 0, taddr);
        PLBM_TMEM_LD32(v, 32, taddr + 32);
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        tc_before_sync();
        const uint64_t bits = stage64(v, mode, relu, sbias, mb, BITS, sA, tid);
        if (BITS) rbits[pix] = bits;
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            tma_store_2d(&tmY, 0, (int)(((size_t)b * H + y) * W + x0), sA);
            asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
        }
    }
    if (tid == 0) asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
    if (tid == 0 && issued) {  // drain before the accumulator is released
        tc_commit(bar_drain);
        if (!bar_wait_drain(bar_drain, 0)) *abortp = 1;
    }
    __syncthreads();
    if (tid == 0 && *abortp) atomicOr(err.flag, 1u);
    if (warp == 0) {
        tc_after_sync();
        tmem_free(tmem, kInTmemCols);
    }
    (void)lane;
}

// ---------------------------------------------------------------------------
// 64 -> 64 weight gradient: dW[tap][ci][co] = sum over pixels of
// X[pixel shifted by the tap][ci] dY[pixel][co], bias gradient db[co] = sum dY.
// Rows of 128 pixels (input rows with their two halo pixels x0 - 1, x0 + 128)
// are staged in the chunk-planar no-swizzle layout (chunk c of pixel s at plane
// c, byte 16 s), which is the MN-major canonical layout for both operands: A =
// X^T (M = channels, K = pixels) and B = dY (K = pixels, N = channels), 8-pixel
// K blocks 128 bytes apart (leading byte offset) and 8-channel blocks one plane
// apart (stride byte offset).  Planes of consecutive rows follow each other, so
// two rows stack into one operand of 128 channels.
//
// Step r multiplies the input rows (r, r + 1) (M = 128) by the dY rows (r, r + 1)
// (N = 128): per K step of 16 pixels and tap column kx one MMA of 128 x 128 x 16
// into the kx-th 128-column TMEM accumulator.  Input row r + i meets dY row r + j
// in tap ky = i - j + 1: quadrant (0, 0) is ky = 1, (0, 1) ky = 0, (1, 0) ky = 2,
// and (1, 1) is ky = 1 again (not read out).  A CTA takes a contiguous range of
// output rows in column order (t = (b * W / 128 + xt) * H + y); a run of n rows
// y .. y + n - 1 of one column takes the n + 1 steps r = y - 1 .. y + n - 1 with
// the dY rows y - 1 and y + n taken as zero, so that every output row meets its
// three input rows once in quadrants (0, 0), (0, 1), (1, 0).  Each input row and
// dY row is staged once, as fill f = 0, 1, ... of the CTA into row slot f mod
// kWpR of two rings (input, dY); slot kWpR is a second copy of slot 0, so that
// the rows of every step are two adjacent slots of each ring.  The CTA writes
// its partial sums partial[cta][tap][ci][co], partial_b[cta][co] at the end.
// ---------------------------------------------------------------------------
constexpr int kWgRowPix = kTile + 2;
// X planes 17 lines apart, pixel 0 of a plane 112 bytes into a line, so that pixel
// 1 (x0), the destination of the TMA box, is 128-byte aligned
constexpr int kWgPlaneX = 17 * 128;             // 2176 >= 130 pixels x 16 bytes
constexpr int kWgXOff = 112;
constexpr int kWgPlaneG = kTile * 16;           // 2048
constexpr int kWpR = 5;                         // row slots of each ring
constexpr int kWpD = 8;                         // commit barriers of the steps
constexpr int kWpXSlot = 8 * kWgPlaneX;         // 17408: one input row
constexpr int kWpGSlot = 8 * kWgPlaneG;         // 16384: one dY row
constexpr int kWpG = (kWpR + 1) * kWpXSlot + 128;               // dY ring (after slot kWpR and the offset)
constexpr int kWpBars = kWpG + (kWpR + 1) * kWpGSlot;           // barriers, TMEM slot, bias sums
constexpr int kWpSmem = 128 + kWpBars + 512;
// Per fill: 8 TMA boxes of 128 input pixels (the 16 halo chunks of 16 bytes are
// copied by the threads) and 8 boxes of the dY row (none for a zero dY row).
constexpr uint32_t kWpRowTx = 8 * kTile * 16;
static_assert(kWpXSlot % 128 == 0 && kWpG % 128 == 0 && kWpSmem <= 232448, "weight-gradient rings");
constexpr uint32_t kWgTmemCols = 512;
// kind::f16, D fp32, A and B bf16, both MN-major (bits 15, 16), N = 64, M = 128.
constexpr uint32_t kIdescWg = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((64u >> 3) << 17) |
                              ((128u >> 4) << 24);
// The same with N = 128.
constexpr uint32_t kIdescWp = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((128u >> 3) << 17) |
                              ((128u >> 4) << 24);

__device__ __forceinline__ uint64_t desc_mn(uint32_t addr, uint32_t mn_stride) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(mn_stride >> 4) << 32) |
           ((uint64_t)1 << 46);
}
__device__ __forceinline__ void mma_wg(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(kIdescWg), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_wp(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(kIdescWp), "r"(accumulate)
        : "memory");
}

// The CTA's output rows come as runs within one column: run of n rows from (b,
// x0, y), n = min(H - y, rows left).
struct WpRun {
    int b, x0, y, n;
};
__device__ __forceinline__ WpRun wp_run(int t, int left, int H, int tiles_x) {
    const int col = t / H;
    WpRun r;
    r.y = t - col * H;
    r.b = col / tiles_x;
    r.x0 = (col - r.b * tiles_x) * kTile;
    r.n = min(H - r.y, left);
    return r;
}

// Warp roles: lane 0 of warp 0 issues the MMAs, warp 1 stages the rows, warps 2
// and 3 sum dY for the bias gradient.  They hand slots over through mbarriers
// only: full[s] (fill in row slot s landed, input row and dY row), done[t mod
// kWpD] (the MMAs of steps up to t are done: tcgen05.commit tracks every earlier
// MMA of the thread), bias[s] (both bias warps have read the dY row of slot s).
constexpr int kWgsThreads = 128;

__global__ void __launch_bounds__(kWgsThreads, 1)
k_wgrad_tc(int B, int H, int W, const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmG,
           const __nv_bfloat16* __restrict__ X, float* __restrict__ partial, float* __restrict__ partial_b,
           const TcErr err) {
    extern __shared__ unsigned char dsm_raw[];
    const uint32_t raw = s2u(dsm_raw);
    const uint32_t pad = (128 - (raw & 127)) & 127;
    unsigned char* base = dsm_raw + pad;
    const uint32_t sbase = raw + pad;
    unsigned char* bars_p = base + kWpBars;
    // done[kWpD], drain, TMEM slot, abort flag, full[kWpR], bias[kWpR]; 64 bias sums at 256
    const uint32_t bar_done0 = s2u(bars_p), bar_drain = bar_done0 + 8 * kWpD;
    unsigned char* slot_p = bars_p + 8 * kWpD + 8;
    volatile uint32_t* tmem_slot = reinterpret_cast<volatile uint32_t*>(slot_p);
    volatile int* abortp = reinterpret_cast<volatile int*>(slot_p + 4);
    const uint32_t bar_full0 = bar_drain + 16;
    const uint32_t bar_bias0 = bar_full0 + 8 * kWpR;
    float* red = reinterpret_cast<float*>(bars_p + 256);
    static_assert(8 * kWpD + 16 + 16 * kWpR <= 256, "weight-gradient barriers");
    const uint32_t sX = sbase + kWgXOff, sG = sbase + kWpG;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_x = W / kTile;
    const long long ntiles = (long long)B * H * tiles_x;
    const int t0 = (int)(ntiles * blockIdx.x / gridDim.x);
    const int ntl = (int)(ntiles * (blockIdx.x + 1) / gridDim.x) - t0;   // >= 1: the grid is at most ntiles
    if (tid == 0) {
        for (int k = 0; k < kWpD; ++k) bar_init(bar_done0 + 8 * k, 1);
        for (int k = 0; k < kWpR; ++k) {
            bar_init(bar_full0 + 8 * k, 1 + 8);
            bar_init(bar_bias0 + 8 * k, 64);
        }
        bar_init(bar_drain, 1);
        *abortp = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) tmem_alloc(s2u(slot_p), kWgTmemCols);
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 1) {
        // ---- staging: per fill, lane c < 8 stages chunk plane c of the input row
        // (TMA box for pixels x0 .. x0 + 127, loads and shared stores for the two
        // halo pixels) and zeroes plane c of a zero dY row, then fences and
        // arrives; lanes 24..31 issue the dY boxes ----
        if (lane == 0) asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&tmX)) : "memory");
        int lastuse[kWpR];   // the last step that reads the fill in each slot
#pragma unroll
        for (int k = 0; k < kWpR; ++k) lastuse[k] = -1;
        // the fill in hand: fill j of the run that starts at output row t0 + i; the
        // halo chunks of the next fill are loaded while this one is staged, so that
        // their latency is not paid fill after fill
        int i = 0, j = 0, f = 0, t = 0;   // t: the first step of the run
        WpRun run = wp_run(t0, ntl, H, tiles_x);
        uint4 lft = make_uint4(0u, 0u, 0u, 0u), rgt = lft;
        auto halo = [&](const WpRun& r, int jj, int c) {
            const size_t row = ((size_t)r.b * H + wrapi(r.y - 1 + jj, H)) * W;
            lft = __ldg(reinterpret_cast<const uint4*>(X + (row + wrapi(r.x0 - 1, W)) * kC + 8 * c));
            rgt = __ldg(reinterpret_cast<const uint4*>(X + (row + wrapi(r.x0 + kTile, W)) * kC + 8 * c));
        };
        if (lane < 8) halo(run, 0, lane);
        for (;;) {
            const int sl = f % kWpR;
            if (f >= kWpR) {   // the slot's previous fill: its last step's MMAs done, its dY summed
                int u = -1;
#pragma unroll
                for (int k = 0; k < kWpR; ++k)
                    if (k == sl) u = lastuse[k];
                if (!bar_wait(bar_done0 + 8 * (u % kWpD), (uint32_t)(u / kWpD) & 1u, abortp, err.wait_ns) ||
                    !bar_wait(bar_bias0 + 8 * sl, (uint32_t)((f - kWpR) / kWpR) & 1u, abortp, err.wait_ns))
                    break;
            }
            const bool zero = j == 0 || j == run.n + 1;   // dY rows y - 1 and y + n
            const int xr = wrapi(run.y - 1 + j, H), gr = run.y - 1 + j;
            const int ncopy = sl == 0 ? 2 : 1;
            const uint32_t full = bar_full0 + 8 * sl;
            if (lane == 0) bar_arrive_expect_tx(full, (uint32_t)ncopy * (zero ? kWpRowTx : 2 * kWpRowTx));
            __syncwarp();
            if (lane < 8) {
                const int c = lane;
                for (int dup = 0; dup < ncopy; ++dup) {
                    const int s = dup ? kWpR : sl;
                    const uint32_t plane = sX + (uint32_t)(s * kWpXSlot + c * kWgPlaneX);
                    tma_load_5d(plane + 16, &tmX, 0, c, run.x0, xr, run.b, full);
                }
                for (int dup = 0; dup < ncopy; ++dup) {
                    const int s = dup ? kWpR : sl;
                    const uint32_t plane = sX + (uint32_t)(s * kWpXSlot + c * kWgPlaneX);
                    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};\n" ::"r"(plane), "r"(lft.x), "r"(lft.y),
                                 "r"(lft.z), "r"(lft.w)
                                 : "memory");
                    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};\n" ::"r"(plane + 16 * (kWgRowPix - 1)),
                                 "r"(rgt.x), "r"(rgt.y), "r"(rgt.z), "r"(rgt.w)
                                 : "memory");
                    if (zero) {
                        const uint32_t gp = sG + (uint32_t)(s * kWpGSlot + c * kWgPlaneG);
                        for (int e = 0; e < kWgPlaneG / 16; ++e)
                            asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};\n" ::"r"(gp + 16 * e), "r"(0u)
                                         : "memory");
                    }
                }
                fence_async_smem();
                bar_arrive(full);
            } else if (lane >= 24 && !zero) {
                const int c = lane - 24;
                for (int dup = 0; dup < ncopy; ++dup)
                    tma_load_5d(sG + (uint32_t)((dup ? kWpR : sl) * kWpGSlot + c * kWgPlaneG), &tmG, 0, c, run.x0, gr,
                                run.b, full);
            }
            // fill j of the run is read by its steps j - 1 and j (0 .. n)
#pragma unroll
            for (int k = 0; k < kWpR; ++k)
                if (k == sl) lastuse[k] = t + min(j, run.n);
            ++f;
            if (++j == run.n + 2) {   // the next run
                t += run.n + 1;
                i += run.n;
                if (i >= ntl) break;
                run = wp_run(t0 + i, ntl - i, H, tiles_x);
                j = 0;
            }
            if (lane < 8) halo(run, j, lane);
        }
        // after an abort, the copies already issued land before the CTA exits:
        // each slot's last fill completes its barrier (every fill arms all of its arrivals)
        if (lane == 0 && *abortp)
            for (int k = 0; k < kWpR; ++k) {
                const int fl = (f - 1) - (((f - 1) - k) % kWpR + kWpR) % kWpR;
                if (fl >= 0) bar_wait_drain(bar_full0 + 8 * k, (uint32_t)(fl / kWpR) & 1u);
            }
    } else if (warp == 0) {
        if (lane == 0) {
            int fbase = 0, t = 0, waited = -1;
            bool ok = true;
            for (int i = 0; i < ntl && ok;) {
                const WpRun run = wp_run(t0 + i, ntl - i, H, tiles_x);
                for (int k = 0; k <= run.n && ok; ++k, ++t) {
                    const int a = fbase + k;   // the step's fills a, a + 1
                    for (int fw = waited + 1; fw <= a + 1 && ok; ++fw) {
                        if (fw < a) continue;
                        ok = bar_spin(bar_full0 + 8 * (fw % kWpR), (uint32_t)(fw / kWpR) & 1u, abortp, err.wait_ns);
                    }
                    if (!ok) break;
                    waited = a + 1;
                    tc_after_sync();
                    // descriptors of the step: constant offsets (start-address field, byte
                    // offset / 16, no carry: shared addresses < 256 KB) of two bases
                    const uint64_t da = desc_mn(sX + (uint32_t)((a % kWpR) * kWpXSlot), kWgPlaneX);
                    const uint64_t dg = desc_mn(sG + (uint32_t)((a % kWpR) * kWpGSlot), kWgPlaneG);
                    const uint32_t acc0 = t > 0 ? 1u : 0u;
#pragma unroll
                    for (int ks = 0; ks < kTile / 16; ++ks)
#pragma unroll
                        for (int kx = 0; kx < 3; ++kx)
                            mma_wp(tmem + (uint32_t)(kx * 128), da + (uint64_t)(16 * ks + kx), dg + (uint64_t)(16 * ks),
                                   ks > 0 ? 1u : acc0);
                    tc_commit(bar_done0 + 8 * (t % kWpD));
                }
                fbase += run.n + 2;
                i += run.n;
            }
            if (t > 0) {   // every issued MMA done before the accumulators are read or released
                tc_commit(bar_drain);
                if (!bar_wait_drain(bar_drain, 0)) *abortp = 1;
            }
        }
        __syncwarp();
    } else {
        // ---- bias: warp 2 + h sums the dY planes 4 h .. 4 h + 3 of every real dY row ----
        const int h = warp - 2;
        float bsum[4][8];   // planes 4 h + pl (channels 8 (4 h + pl) + e), pixels lane + 32 j
#pragma unroll
        for (int pl = 0; pl < 4; ++pl)
#pragma unroll
            for (int e = 0; e < 8; ++e) bsum[pl][e] = 0.0f;
        int f = 0;
        bool ok = true;
        for (int i = 0; i < ntl && ok;) {
            const WpRun run = wp_run(t0 + i, ntl - i, H, tiles_x);
            for (int j = 0; j < run.n + 2; ++j, ++f) {
                const int sl = f % kWpR;
                if (!bar_wait(bar_full0 + 8 * sl, (uint32_t)(f / kWpR) & 1u, abortp, err.wait_ns)) {
                    ok = false;
                    break;
                }
                if (j >= 1 && j <= run.n) {
#pragma unroll
                    for (int pl = 0; pl < 4; ++pl) {
                        const unsigned char* g = base + kWpG + sl * kWpGSlot + (4 * h + pl) * kWgPlaneG;
#pragma unroll
                        for (int jj = 0; jj < kTile / 32; ++jj) {
                            const uint4 r = *reinterpret_cast<const uint4*>(g + 16 * (lane + 32 * jj));
                            const __nv_bfloat162* hv = reinterpret_cast<const __nv_bfloat162*>(&r);
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const float2 v = __bfloat1622float2(hv[e]);
                                bsum[pl][2 * e] += v.x;
                                bsum[pl][2 * e + 1] += v.y;
                            }
                        }
                    }
                }
                bar_arrive(bar_bias0 + 8 * sl);
            }
            i += run.n;
        }
#pragma unroll
        for (int pl = 0; pl < 4; ++pl)
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                float v = bsum[pl][e];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) red[8 * (4 * h + pl) + e] = v;
            }
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (!*abortp) {
        // warp w reads TMEM lanes 32 w .. 32 w + 31: lanes < 64 are input row r (i = 0):
        // columns 0..63 tap ky = 1, 64..127 ky = 0; lanes >= 64 (i = 1): columns 0..63 ky = 2
        const int L = 32 * warp + lane;
        const int ci = L & 63;
#pragma unroll 1
        for (int kx = 0; kx < 3; ++kx)
#pragma unroll 1
            for (int jc = 0; jc < 2; ++jc) {
                if (warp >= 2 && jc == 1) continue;   // quadrant (1, 1): ky = 1 again
                uint32_t v[64];
                const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(kx * 128 + jc * 64);
                PLBM_TMEM_LD32(v, 0, taddr);
                PLBM_TMEM_LD32(v, 32, taddr + 32);
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                const int ky = L < 64 ? (jc == 0 ? 1 : 0) : 2;
                float4* out =
                    reinterpret_cast<float4*>(partial + (((size_t)blockIdx.x * 9 + ky * 3 + kx) * kC + ci) * kC);
#pragma unroll
                for (int c4 = 0; c4 < 16; ++c4)
                    out[c4] = make_float4(__uint_as_float(v[4 * c4]), __uint_as_float(v[4 * c4 + 1]),
                                          __uint_as_float(v[4 * c4 + 2]), __uint_as_float(v[4 * c4 + 3]));
            }
        if (tid < kC) partial_b[(size_t)blockIdx.x * kC + tid] = red[tid];
    }
    tc_before_sync();
    __syncthreads();
    if (tid == 0 && *abortp) atomicOr(err.flag, 1u);
    if (warp == 0) {
        tc_after_sync();
        tmem_free(tmem, kWgTmemCols);
    }
}

// ---------------------------------------------------------------------------
// 4 -> 64 input-layer weight gradient: dW[tap][ci][co] = sum over pixels of
// X[pixel shifted by the tap][ci] dY[pixel][co].  M = (tap, ci) = 36 rows, padded
// to 128: per tile the 9 taps x 4 channels of each pixel are gathered into chunk
// planes 0..4 (row m = 4 tap + ci in plane m / 8; planes 5..15 and the upper half
// of plane 4 stay zero); dY (B: K = pixels, N = 64) arrives by TMA in the
// chunk-planar layout.  One MMA of 128 x 64 x 16 per 16 pixels into one
// accumulator summed over the CTA's tiles.  Warps: 0 issues the MMAs (lane 0),
// 1 issues the dY copies, 2..5 gather A (one pixel a thread) and then sum the
// stage's dY for db (warp w: planes 2 (w - 2), 2 (w - 2) + 1).  Barriers per
// stage k: xfull (dY landed), afull (A gathered), done (MMAs done), bias (dY
// summed).  Partials per CTA: partial[cta][tap][ci][co], partial_b[cta][co].
// ---------------------------------------------------------------------------
constexpr int kWiThreads = 192;
constexpr int kWiStages = 4;
constexpr int kWiA = 16 * kWgPlaneG;              // 32 KB: 16 planes of 128 pixels x 16 bytes
constexpr int kWiStage = kWiA + 8 * kWgPlaneG;    // + dY
constexpr int kWiBars = kWiStages * kWiStage;
constexpr int kWiSmem = 128 + kWiBars + 256 + 64 * 4;
constexpr uint32_t kWiTmemCols = 64;
static_assert(kWiSmem <= 232448, "input-layer weight-gradient stages");

__global__ void __launch_bounds__(kWiThreads, 1)
k_wgrad_in_tc(int B, int H, int W, const __nv_bfloat16* __restrict__ X, const __grid_constant__ CUtensorMap tmG,
              float* __restrict__ partial, float* __restrict__ partial_b, const TcErr err) {
    extern __shared__ unsigned char dsm_raw[];
    const uint32_t raw = s2u(dsm_raw);
    const uint32_t pad = (128 - (raw & 127)) & 127;
    unsigned char* base = dsm_raw + pad;
    const uint32_t sbase = raw + pad;
    unsigned char* bars_p = base + kWiBars;
    // xfull[k] 8 k, afull[k] 32 + 8 k, done[k] 64 + 8 k, bias[k] 96 + 8 k, drain 128, TMEM slot 136, abort 140
    const uint32_t bar_x0 = s2u(bars_p), bar_a0 = bar_x0 + 32, bar_d0 = bar_x0 + 64, bar_b0 = bar_x0 + 96;
    const uint32_t bar_drain = bar_x0 + 128;
    volatile uint32_t* tmem_slot = reinterpret_cast<volatile uint32_t*>(bars_p + 136);
    volatile int* abortp = reinterpret_cast<volatile int*>(bars_p + 140);
    float* red = reinterpret_cast<float*>(bars_p + 256);   // 64 bias sums
    static_assert(kWiStages == 4, "barrier layout");

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_x = W / kTile;
    const int ntiles = B * H * tiles_x;
    const int ntl = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    // zero the A planes of every stage once: the gathers write planes 0..4 only
    // (plane 4: the first 8 bytes of each pixel, tap 8)
    for (int i = tid; i < kWiStages * kWiA / 16; i += kWiThreads) {
        const int k = i / (kWiA / 16), j = i - k * (kWiA / 16);
        *reinterpret_cast<uint4*>(base + k * kWiStage + 16 * j) = make_uint4(0u, 0u, 0u, 0u);
    }
    fence_async_smem();
    if (tid == 0) {
        for (int k = 0; k < kWiStages; ++k) {
            bar_init(bar_x0 + 8 * k, 1);
            bar_init(bar_a0 + 8 * k, 128);
            bar_init(bar_d0 + 8 * k, 1);
            bar_init(bar_b0 + 8 * k, 128);
        }
        bar_init(bar_drain, 1);
        *abortp = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) tmem_alloc(s2u(bars_p + 136), kWiTmemCols);
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = *tmem_slot;
    float bsum[2][8];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int e = 0; e < 8; ++e) bsum[h][e] = 0.0f;

    if (warp == 1) {
        if (lane == 0) asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&tmG)) : "memory");
        int it = 0;
        for (; it < ntl; ++it) {
            const int k = it % kWiStages;
            if (it >= kWiStages) {   // the stage's previous tile: MMAs done and dY summed
                const uint32_t par = (uint32_t)(it / kWiStages - 1) & 1u;
                if (!bar_wait(bar_d0 + 8 * k, par, abortp, err.wait_ns) ||
                    !bar_wait(bar_b0 + 8 * k, par, abortp, err.wait_ns))
                    break;
            }
            const int t = (int)blockIdx.x + it * (int)gridDim.x;
            const int b = t / (H * tiles_x);
            const int rem = t - b * H * tiles_x;
            const int y = rem / tiles_x;
            const int x0 = (rem - y * tiles_x) * kTile;
            if (lane == 0) bar_arrive_expect_tx(bar_x0 + 8 * k, 8 * kWgPlaneG);
            __syncwarp();
            if (lane < 8)
                tma_load_5d(sbase + (uint32_t)(k * kWiStage + kWiA + lane * kWgPlaneG), &tmG, 0, lane, x0, y, b,
                            bar_x0 + 8 * k);
        }
        if (lane == 0 && *abortp)   // copies already issued land before the CTA exits
            for (int k = 0; k < kWiStages; ++k) {
                const int j = (it - 1) - (((it - 1) - k) % kWiStages + kWiStages) % kWiStages;
                if (j >= 0) bar_wait_drain(bar_x0 + 8 * k, (uint32_t)(j / kWiStages) & 1u);
            }
    } else if (warp == 0) {
        if (lane == 0) {
            int issued = 0;
            for (int it = 0; it < ntl; ++it) {
                const int k = it % kWiStages;
                const uint32_t par = (uint32_t)(it / kWiStages) & 1u;
                if (!bar_spin(bar_a0 + 8 * k, par, abortp, err.wait_ns) ||
                    !bar_spin(bar_x0 + 8 * k, par, abortp, err.wait_ns))
                    break;
                tc_after_sync();
                const uint32_t sA = sbase + (uint32_t)(k * kWiStage), sG = sA + kWiA;
#pragma unroll
                for (int ks = 0; ks < kTile / 16; ++ks)
                    mma_wg(tmem, desc_mn(sA + 16 * 16 * ks, kWgPlaneG), desc_mn(sG + 16 * 16 * ks, kWgPlaneG),
                           (it > 0 || ks > 0) ? 1u : 0u);
                tc_commit(bar_d0 + 8 * k);
                ++issued;
            }
            if (issued > 0) {
                tc_commit(bar_drain);
                if (!bar_wait_drain(bar_drain, 0)) *abortp = 1;
            }
        }
        __syncwarp();
    } else {
        const int q = tid - 64;       // gather: pixel q of the tile
        const int pw = warp - 2;      // bias: dY planes 2 pw, 2 pw + 1
        for (int it = 0; it < ntl; ++it) {
            const int k = it % kWiStages;
            if (it >= kWiStages &&
                !bar_wait(bar_d0 + 8 * k, (uint32_t)(it / kWiStages - 1) & 1u, abortp, err.wait_ns))
                break;
            const int t = (int)blockIdx.x + it * (int)gridDim.x;
            const int b = t / (H * tiles_x);
            const int rem = t - b * H * tiles_x;
            const int y = rem / tiles_x;
            const int x0 = (rem - y * tiles_x) * kTile;
            uint2 v[9];   // every load in flight before the first shared store
#pragma unroll
            for (int tap = 0; tap < 9; ++tap) {
                const int yy = wrapi(y + tap / 3 - 1, H), xx = wrapi(x0 + q + tap % 3 - 1, W);
                v[tap] = __ldg(reinterpret_cast<const uint2*>(X + (((size_t)b * H + yy) * W + xx) * 4));
            }
            const uint32_t st = sbase + (uint32_t)(k * kWiStage) + 16 * q;
#pragma unroll
            for (int tap = 0; tap < 9; ++tap)
                asm volatile("st.shared.v2.u32 [%0], {%1, %2};\n" ::"r"(st + (tap >> 1) * kWgPlaneG + 8 * (tap & 1)),
                             "r"(v[tap].x), "r"(v[tap].y)
                             : "memory");
            fence_async_smem();
            bar_arrive(bar_a0 + 8 * k);
            // bias: this stage's dY once it has landed
            if (!bar_wait(bar_x0 + 8 * k, (uint32_t)(it / kWiStages) & 1u, abortp, err.wait_ns)) break;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const unsigned char* g = base + k * kWiStage + kWiA + (2 * pw + h) * kWgPlaneG;
#pragma unroll
                for (int j = 0; j < kTile / 32; ++j) {
                    const uint4 r = *reinterpret_cast<const uint4*>(g + 16 * (lane + 32 * j));
                    const __nv_bfloat162* hv = reinterpret_cast<const __nv_bfloat162*>(&r);
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float2 f = __bfloat1622float2(hv[e]);
                        bsum[h][2 * e] += f.x;
                        bsum[h][2 * e + 1] += f.y;
                    }
                }
            }
            bar_arrive(bar_b0 + 8 * k);
        }
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const bool ok = !*abortp && ntl > 0;
    if (warp >= 4) {   // TMEM lanes 0..63 (warps 4, 5) hold rows m = 4 tap + ci < 36
        const int m = 32 * (warp - 4) + lane;
        uint32_t v[64];
        const uint32_t taddr = tmem + ((uint32_t)(32 * (warp - 4)) << 16);
        PLBM_TMEM_LD32(v, 0, taddr);
        PLBM_TMEM_LD32(v, 32, taddr + 32);
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        if (ok && m < 36) {
            float4* out = reinterpret_cast<float4*>(partial + ((size_t)blockIdx.x * 36 + m) * kC);
#pragma unroll
            for (int c4 = 0; c4 < 16; ++c4)
                out[c4] = make_float4(__uint_as_float(v[4 * c4]), __uint_as_float(v[4 * c4 + 1]),
                                      __uint_as_float(v[4 * c4 + 2]), __uint_as_float(v[4 * c4 + 3]));
        }
    }
    if (warp >= 2) {   // per warp and lane: channels 8 (2 pw + h) + e
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                float v = bsum[h][e];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) red[8 * (2 * (warp - 2) + h) + e] = v;
            }
    }
    tc_before_sync();
    __syncthreads();
    if (ok && tid < kC) partial_b[(size_t)blockIdx.x * kC + tid] = red[tid];
    if (tid == 0 && *abortp) atomicOr(err.flag, 1u);
    if (warp == 0) {
        tc_after_sync();
        tmem_free(tmem, kWiTmemCols);
    }
}





// ---------------------------------------------------------------------------
// 64 -> 4 output-layer weight gradient on tcgen05: dW[tap][ci][co] = sum over
// pixels of X[y + ky - 1][x + kx - 1][ci] dY[y][x][co], db[co] = sum dY.  The
// same sum taken over the input pixel (y', x') = (y + ky - 1, x + kx - 1) pairs
// X[y'][x'] with dY[y' - ky + 1][x' - kx + 1], so a tile of two input rows
// (y0, y0 + 1) x 128 pixels is one M = 128 operand (A = X^T: (row, ci) x pixels,
// staged by TMA in the chunk-planar layout, with no halo), and the shifted
// upstream gradients of dY rows y0 - 1 .. y0 + 2 form B: K = pixels, N = (j,
// kx, co) = 4 rows x 3 shifts x 4 channels = 48 columns.  Row y' = y0 + r of X
// meets dY row y = y0 - 1 + j in tap ky = y' - y + 1 = r - j + 2 when that lies
// in 0..2 (3 of the 4 rows j for either r).  dY is FP32: B carries it as a bf16 pair
// hi + lo (hi = bf16(dY), lo = bf16(dY - hi)) in columns 0..47 and 48..95, so
// that the products keep FP32 accuracy (N = 96).  X rows past the lattice (odd
// H) are zero (TMA out-of-range fill).
// Warps: 0 issues the MMAs (lane 0), 1 issues the TMA copies of X, 2..5 build B
// (one pixel a thread) and sum dY for db, then read the accumulators.
// ---------------------------------------------------------------------------
constexpr int kWoThreads = 192;
constexpr int kWoStages = 3;
constexpr int kWoX = 16 * kWgPlaneG;                 // 32 KB: 2 rows x 8 chunk planes of 128 pixels
constexpr int kWoStage = kWoX + 12 * kWgPlaneG;      // + B: 12 planes of 8 columns
constexpr int kWoBars = kWoStages * kWoStage;
constexpr int kWoSmem = 128 + kWoBars + 128;
constexpr uint32_t kWoTmemCols = 128;
static_assert(kWoSmem <= 232448 && 9 * kC * 4 * 4 <= kWoBars, "output-layer weight-gradient stages");
// kind::f16, D fp32, A and B bf16, both MN-major, N = 96, M = 128.
constexpr uint32_t kIdescWo = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((96u >> 3) << 17) |
                              ((128u >> 4) << 24);

__global__ void __launch_bounds__(kWoThreads, 1)
k_wgrad_out_tc(int B, int H, int W, const __grid_constant__ CUtensorMap tmX, const float* __restrict__ dY,
               float* __restrict__ partial, float* __restrict__ partial_b, const TcErr err) {
    extern __shared__ unsigned char dsm_raw[];
    const uint32_t raw = s2u(dsm_raw);
    const uint32_t pad = (128 - (raw & 127)) & 127;
    unsigned char* base = dsm_raw + pad;
    const uint32_t sbase = raw + pad;
    unsigned char* bars_p = base + kWoBars;
    // xfull[k] at 8 k, bfull[k] at 24 + 8 k, done[k] at 48 + 8 k, drain 72, TMEM slot 80, abort flag 84
    const uint32_t bar_x0 = s2u(bars_p), bar_b0 = bar_x0 + 24, bar_d0 = bar_x0 + 48, bar_drain = bar_x0 + 72;
    volatile uint32_t* tmem_slot = reinterpret_cast<volatile uint32_t*>(bars_p + 80);
    volatile int* abortp = reinterpret_cast<volatile int*>(bars_p + 84);
    static_assert(kWoStages == 3, "barrier layout");

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_x = W / kTile, hp = (H + 1) / 2;
    const int ntiles = B * hp * tiles_x;
    const int ntl = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    if (tid == 0) {
        for (int k = 0; k < kWoStages; ++k) {
            bar_init(bar_x0 + 8 * k, 1);
            bar_init(bar_b0 + 8 * k, 128);
            bar_init(bar_d0 + 8 * k, 1);
        }
        bar_init(bar_drain, 1);
        *abortp = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) tmem_alloc(s2u(bars_p + 80), kWoTmemCols);
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = *tmem_slot;
    float bacc[4] = {0.f, 0.f, 0.f, 0.f};

    if (warp == 1) {
        if (lane == 0) asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&tmX)) : "memory");
        int it = 0;
        for (; it < ntl; ++it) {
            const int k = it % kWoStages;
            if (it >= kWoStages &&
                !bar_wait(bar_d0 + 8 * k, (uint32_t)(it / kWoStages - 1) & 1u, abortp, err.wait_ns))
                break;
            const int t = (int)blockIdx.x + it * (int)gridDim.x;
            const int b = t / (hp * tiles_x);
            const int rem = t - b * hp * tiles_x;
            const int y0 = 2 * (rem / tiles_x);
            const int x0 = (rem % tiles_x) * kTile;
            if (lane == 0) bar_arrive_expect_tx(bar_x0 + 8 * k, (uint32_t)kWoX);
            __syncwarp();
            if (lane < 16)   // plane (r, c) of row y0 + r; row H (odd H) is out of range: zeros
                tma_load_5d(sbase + (uint32_t)(k * kWoStage + lane * kWgPlaneG), &tmX, 0, lane & 7, x0,
                            y0 + (lane >> 3), b, bar_x0 + 8 * k);
        }
        if (lane == 0 && *abortp)   // copies already issued land before the CTA exits
            for (int k = 0; k < kWoStages; ++k) {
                const int j = (it - 1) - (((it - 1) - k) % kWoStages + kWoStages) % kWoStages;
                if (j >= 0) bar_wait_drain(bar_x0 + 8 * k, (uint32_t)(j / kWoStages) & 1u);
            }
    } else if (warp == 0) {
        if (lane == 0) {
            int issued = 0;
            for (int it = 0; it < ntl; ++it) {
                const int k = it % kWoStages;
                const uint32_t par = (uint32_t)(it / kWoStages) & 1u;
                if (!bar_spin(bar_x0 + 8 * k, par, abortp, err.wait_ns) ||
                    !bar_spin(bar_b0 + 8 * k, par, abortp, err.wait_ns))
                    break;
                tc_after_sync();
                const uint32_t sA = sbase + (uint32_t)(k * kWoStage), sB = sA + kWoX;
#pragma unroll
                for (int ks = 0; ks < kTile / 16; ++ks) {
                    const uint64_t a = desc_mn(sA + 256 * ks, kWgPlaneG), bd = desc_mn(sB + 256 * ks, kWgPlaneG);
                    asm volatile(
                        "{\n\t.reg .pred p;\n\t"
                        "setp.ne.u32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                        "l"(a), "l"(bd), "r"(kIdescWo), "r"((it > 0 || ks > 0) ? 1u : 0u)
                        : "memory");
                }
                tc_commit(bar_d0 + 8 * k);
                ++issued;
            }
            if (issued > 0) {
                tc_commit(bar_drain);
                if (!bar_wait_drain(bar_drain, 0)) *abortp = 1;
            }
        }
        __syncwarp();
    } else {
        // B builders: thread q = pixel q of the tile; column n = 48 h + 12 j + 4 kx + co
        const int q = tid - 64;
        for (int it = 0; it < ntl; ++it) {
            const int k = it % kWoStages;
            if (it >= kWoStages &&
                !bar_wait(bar_d0 + 8 * k, (uint32_t)(it / kWoStages - 1) & 1u, abortp, err.wait_ns))
                break;
            const int t = (int)blockIdx.x + it * (int)gridDim.x;
            const int b = t / (hp * tiles_x);
            const int rem = t - b * hp * tiles_x;
            const int y0 = 2 * (rem / tiles_x);
            const int x0 = (rem % tiles_x) * kTile;
            const uint32_t sB = sbase + (uint32_t)(k * kWoStage + kWoX) + 16 * q;
            float4 d[4][3];   // every load in flight before the first shared store
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int yj = ((y0 - 1 + j) % H + H) % H;
                const float4* row = reinterpret_cast<const float4*>(dY) + ((size_t)b * H + yj) * W;
#pragma unroll
                for (int kx = 0; kx < 3; ++kx) d[j][kx] = __ldg(row + wrapi(x0 + q - kx + 1, W));
            }
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int kx = 0; kx < 3; ++kx) {
                    const float4 e = d[j][kx];
                    const __nv_bfloat162 h01 = __floats2bfloat162_rn(e.x, e.y), h23 = __floats2bfloat162_rn(e.z, e.w);
                    const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
                    const __nv_bfloat162 l01 = __floats2bfloat162_rn(e.x - f01.x, e.y - f01.y);
                    const __nv_bfloat162 l23 = __floats2bfloat162_rn(e.z - f23.x, e.w - f23.y);
                    const int n = 12 * j + 4 * kx;   // hi at n, lo at 48 + n
                    const uint32_t dh = sB + (uint32_t)((n >> 3) * kWgPlaneG + 2 * (n & 7));
                    const uint32_t dl = sB + (uint32_t)(((48 + n) >> 3) * kWgPlaneG + 2 * ((48 + n) & 7));
                    asm volatile("st.shared.v2.u32 [%0], {%1, %2};\n" ::"r"(dh),
                                 "r"(*reinterpret_cast<const uint32_t*>(&h01)),
                                 "r"(*reinterpret_cast<const uint32_t*>(&h23))
                                 : "memory");
                    asm volatile("st.shared.v2.u32 [%0], {%1, %2};\n" ::"r"(dl),
                                 "r"(*reinterpret_cast<const uint32_t*>(&l01)),
                                 "r"(*reinterpret_cast<const uint32_t*>(&l23))
                                 : "memory");
                    if (kx == 1 && (j == 1 || (j == 2 && y0 + 1 < H))) {   // the tile's own dY rows, once each
                        bacc[0] += e.x;
                        bacc[1] += e.y;
                        bacc[2] += e.z;
                        bacc[3] += e.w;
                    }
                }
            fence_async_smem();
            bar_arrive(bar_b0 + 8 * k);
        }
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    // red[tap][ci][co] (the stages are free: every MMA is done), redb[q][co]
    float* red = reinterpret_cast<float*>(base);
    float* redb = red + 9 * kC * 4;
    const bool ok = !*abortp && ntl > 0;
    uint32_t v[96];
    if (warp >= 2) {
        const int L = 32 * (warp & 3) + lane;   // TMEM lane: row r = L / 64, channel ci = L mod 64
        const uint32_t taddr = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
        PLBM_TMEM_LD32(v, 0, taddr);
        PLBM_TMEM_LD32(v, 32, taddr + 32);
        PLBM_TMEM_LD32(v, 64, taddr + 64);
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        if (L < 64 && ok)   // row y0: tap ky = 2 - j
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int n = 0; n < 12; ++n)
                    red[((2 - j) * 3 + n / 4) * kC * 4 + L * 4 + (n & 3)] =
                        __uint_as_float(v[12 * j + n]) + __uint_as_float(v[48 + 12 * j + n]);
        const int qq = tid - 64;
#pragma unroll
        for (int c = 0; c < 4; ++c) redb[qq * 4 + c] = bacc[c];
    }
    __syncthreads();
    if (warp >= 2 && ok) {
        const int L = 32 * (warp & 3) + lane;
        if (L >= 64) {   // row y0 + 1: tap ky = 3 - j, added to row y0's part
            const int ci = L - 64;
            float* out = partial + (size_t)blockIdx.x * 9 * kC * 4;
#pragma unroll
            for (int j = 1; j < 4; ++j)
#pragma unroll
                for (int n = 0; n < 12; ++n) {
                    const int i = ((3 - j) * 3 + n / 4) * kC * 4 + ci * 4 + (n & 3);
                    out[i] = red[i] + (__uint_as_float(v[12 * j + n]) + __uint_as_float(v[48 + 12 * j + n]));
                }
        }
        if (tid - 64 < 4) {
            const int c = tid - 64;
            float sum = 0.0f;
            for (int i = 0; i < 128; ++i) sum += redb[i * 4 + c];
            partial_b[(size_t)blockIdx.x * 4 + c] = sum;
        }
    }
    tc_before_sync();
    __syncthreads();
    if (tid == 0 && *abortp) atomicOr(err.flag, 1u);
    if (warp == 0) {
        tc_after_sync();
        tmem_free(tmem, kWoTmemCols);
    }
}


// Every derived weight array of the surrogate from the FP32 master weights p in
// one launch: pr = bf16-rounded p;
// for the 64 -> 64 layers l = 1..4 the bf16 weights [tap][ci][co], their
// backward-data form [8 - tap][co][ci] and the two K-major tensor-core layouts;
// the output layer's backward-data weights w6flip[tap][co][ci] = pr[8 - tap][ci][co]
// (FP32); and the tensor-core layouts of the input layer, of w6flip and of the
// output layer.  One thread per output element.
struct RefreshArgs {
    const float* p;
    long long np;
    long long woff[6];
    float* pr;
    __nv_bfloat16* wbf;
    __nv_bfloat16* wflip;
    __nv_bfloat16* wtc;
    float* w6flip;
    __nv_bfloat16* win;
    __nv_bfloat16* win6;
    __nv_bfloat16* wout;
};
constexpr int kW64 = 9 * kC * kC;

__global__ void k_refresh_weights(const RefreshArgs a) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const float* p = a.p;
    if (i < a.np) {
        a.pr[i] = __bfloat162float(__float2bfloat16_rn(p[i]));
        return;
    }
    i -= a.np;
    if (i < 4 * kW64) {   // source element (tap, ci, co) of layer l
        const int l = (int)(i / kW64), e = (int)(i % kW64);
        const int co = e % kC, ci = (e / kC) % kC, tap = e / (kC * kC);
        const __nv_bfloat16 w = __float2bfloat16_rn(p[a.woff[l + 1] + e]);
        a.wbf[(size_t)l * kW64 + e] = w;
        a.wflip[(size_t)l * kW64 + ((8 - tap) * kC + co) * kC + ci] = w;
        a.wtc[(size_t)(2 * l) * kW64 + (tap * kC + co) * kC + ci] = w;
        a.wtc[(size_t)(2 * l + 1) * kW64 + ((8 - tap) * kC + ci) * kC + co] = w;
        return;
    }
    i -= 4 * kW64;
    const float* w5 = p + a.woff[5];
    const float* w0 = p + a.woff[0];
    auto r = [](float v) { return __bfloat162float(__float2bfloat16_rn(v)); };
    if (i < 9 * 4 * kC) {   // w6flip[(tap * 4 + co) * 64 + ci]
        const int ci = (int)i % kC, co = ((int)i / kC) % 4, tap = (int)i / (4 * kC);
        a.w6flip[i] = r(w5[((8 - tap) * kC + ci) * 4 + co]);
        return;
    }
    i -= 9 * 4 * kC;
    if (i < 2 * kInPlanes * kC * 8) {   // win, then win6: [plane c][n][8], k = 8 c + j < 36
        const bool six = i >= kInPlanes * kC * 8;
        const int e = (int)(six ? i - kInPlanes * kC * 8 : i);
        const int j = e % 8, n = (e / 8) % kC, c = e / (8 * kC);
        const int k = 8 * c + j;
        float v = 0.0f;
        if (k < 36) v = six ? r(w5[((8 - (k >> 2)) * kC + n) * 4 + (k & 3)]) : r(w0[k * kC + n]);
        (six ? a.win6 : a.win)[e] = __float2bfloat16_rn(v);
        return;
    }
    i -= 2 * kInPlanes * kC * 8;
    if (i < 9 * 16 * kC) {   // wout[tap][n][ci], n < 4
        const int ci = (int)i % kC, n = ((int)i / kC) % 16, tap = (int)i / (16 * kC);
        a.wout[i] = __float2bfloat16_rn(n < 4 ? w5[(tap * kC + ci) * 4 + n] : 0.0f);
    }
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

// Tensor map of a bf16 NHWC activation with 64 channels as [B][H][W][8][8]
// (box: 8 channels x 1 chunk x 128 pixels), for the ring loaders' TMA copies.
static cudaError_t encode_act_map(CUtensorMap* map, const void* X, int B, int H, int W) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q{};
        void* fn = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    if (reinterpret_cast<uintptr_t>(X) % 16) return cudaErrorMisalignedAddress;
    const cuuint64_t dims[5] = {8, 8, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
    const cuuint64_t strides[4] = {16, 128, (cuuint64_t)W * 128, (cuuint64_t)H * W * 128};
    const cuuint32_t box[5] = {8, 1, (cuuint32_t)tc::kTile, 1, 1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(X), dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Tensor map of a bf16 NHWC output with 64 channels as [pixels][64] (box: 64
// channels x 128 pixels, 128-byte swizzle), for the ring epilogue's TMA stores.
static cudaError_t encode_out_map(CUtensorMap* map, void* Y, long long npix) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q{};
        void* fn = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    if (reinterpret_cast<uintptr_t>(Y) % 16) return cudaErrorMisalignedAddress;
    const cuuint64_t dims[2] = {64, (cuuint64_t)npix};
    const cuuint64_t strides[1] = {128};
    const cuuint32_t box[2] = {64, (cuuint32_t)tc::kTile};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, Y, dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int N, int MODE, bool BITS = false>
static cudaError_t launch_ring(int B, int H, int W, const void* X, const void* Wk, const float* bias,
                               uint64_t* rbits, void* Y, int relu, TcErr err, cudaStream_t s) {
    if (W % tc::kTile || H < 1 || B < 1) return cudaErrorInvalidValue;
    if (MODE == 1 && !rbits) return cudaErrorInvalidValue;
    CUtensorMap map, mapY;
    cudaError_t em = encode_act_map(&map, X, B, H, W);
    if (em != cudaSuccess) return em;
    if (N == 64) {
        em = encode_out_map(&mapY, Y, (long long)B * H * W);
        if (em != cudaSuccess) return em;
    } else {
        mapY = map;   // not used by the 64 -> 4 layer (fp32 stores from the threads)
    }
    constexpr int smem = tc::ring_smem<N>();
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(tc::k_conv_ring<N, MODE, BITS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int ntiles = B * H * (W / tc::kTile);
    const int grid = ntiles < tc_sms() ? ntiles : tc_sms();
    tc::k_conv_ring<N, MODE, BITS><<<grid, tc::kRingThreads, smem, s>>>(
        B, H, W, map, mapY, static_cast<const __nv_bfloat16*>(X), static_cast<const __nv_bfloat16*>(Wk), bias, rbits,
        Y, relu, err);
    return cudaGetLastError();
}

cudaError_t cnn_conv64_tc(int B, int H, int W, const void* X, const void* Wk, const float* bias, uint64_t* rbits,
                          void* Y, int mode, int relu, TcErr err, cudaStream_t s) {
    if (mode == 0 && rbits) return launch_ring<64, 0, true>(B, H, W, X, Wk, bias, rbits, Y, relu, err, s);
    if (mode == 0) return launch_ring<64, 0>(B, H, W, X, Wk, bias, nullptr, Y, relu, err, s);
    return launch_ring<64, 1>(B, H, W, X, Wk, bias, rbits, Y, relu, err, s);
}

cudaError_t cnn_conv_out_tc(int B, int H, int W, const void* X, const void* Wo, const float* bias, float* Y,
                            TcErr err, cudaStream_t s) {
    return launch_ring<16, 2>(B, H, W, X, Wo, bias, nullptr, Y, 0, err, s);
}

template <int MODE, bool BITS>
static cudaError_t launch_in(int B, int H, int W, const void* X, const void* Win, const float* bias, uint64_t* rbits,
                             void* Y, int relu, TcErr err, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(tc::k_conv_in_tc<MODE, BITS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             tc::kInSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    CUtensorMap mapY;
    cudaError_t em = encode_out_map(&mapY, Y, (long long)B * H * W);
    if (em != cudaSuccess) return em;
    const int ntiles = B * H * (W / tc::kTile);
    const int grid = ntiles < 8 * tc_sms() ? ntiles : 8 * tc_sms();
    tc::k_conv_in_tc<MODE, BITS><<<grid, tc::kInThreads, tc::kInSmem, s>>>(
        B, H, W, static_cast<const __nv_bfloat16*>(X), static_cast<const __nv_bfloat16*>(Win), bias, rbits, mapY, relu,
        err);
    return cudaGetLastError();
}

cudaError_t cnn_conv_in_tc(int B, int H, int W, const void* X, const void* Win, const float* bias, uint64_t* rbits,
                           void* Y, int mode, int relu, TcErr err, cudaStream_t s) {
    if ((mode == 0 && !bias) || (mode == 1 && !rbits) || mode < 0 || mode > 1) return cudaErrorInvalidValue;
    if (W % tc::kTile || H < 1 || B < 1) return cudaErrorInvalidValue;
    if (mode == 1) return launch_in<1, false>(B, H, W, X, Win, bias, rbits, Y, relu, err, s);
    if (rbits) return launch_in<0, true>(B, H, W, X, Win, bias, rbits, Y, relu, err, s);
    return launch_in<0, false>(B, H, W, X, Win, bias, nullptr, Y, relu, err, s);
}

cudaError_t cnn_conv64_wgrad_tc(int B, int H, int W, const void* X, const void* dY, float* partial, float* partial_b,
                                float* dW, float* db, TcErr err, cudaStream_t s) {
    if (W % tc::kTile || H < 1 || B < 1) return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(tc::k_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::kWpSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    CUtensorMap mapX, mapG;
    cudaError_t em = encode_act_map(&mapX, X, B, H, W);
    if (em == cudaSuccess) em = encode_act_map(&mapG, dY, B, H, W);
    if (em != cudaSuccess) return em;
    const int grid = cnn_wgrad64_parts(B, H, W);   // one CTA per SM at most (the partial buffers' size)
    tc::k_wgrad_tc<<<grid, tc::kWgsThreads, tc::kWpSmem, s>>>(B, H, W, mapX, mapG, static_cast<const __nv_bfloat16*>(X),
                                                             partial, partial_b, err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cnn_sum_partials2(partial, 9 * tc::kC * tc::kC, dW, partial_b, tc::kC, db, grid, s);
}

cudaError_t cnn_conv_in_wgrad_tc(int B, int H, int W, const void* X, const void* dY, float* partial, float* partial_b,
                                 float* dW, float* db, TcErr err, cudaStream_t s) {
    if (W % tc::kTile || H < 1 || B < 1) return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        cudaError_t e =
            cudaFuncSetAttribute(tc::k_wgrad_in_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::kWiSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    if (reinterpret_cast<uintptr_t>(X) % 8) return cudaErrorMisalignedAddress;
    CUtensorMap mapG;
    cudaError_t em = encode_act_map(&mapG, dY, B, H, W);
    if (em != cudaSuccess) return em;
    const int grid = cnn_wgrad64_parts(B, H, W);   // at most one CTA per SM: within the partial buffers
    tc::k_wgrad_in_tc<<<grid, tc::kWiThreads, tc::kWiSmem, s>>>(B, H, W, static_cast<const __nv_bfloat16*>(X), mapG,
                                                                partial, partial_b, err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cnn_sum_partials2(partial, 9 * 4 * tc::kC, dW, partial_b, tc::kC, db, grid, s);
}





cudaError_t cnn_conv_out_wgrad_tc(int B, int H, int W, const void* X, const float* dY, float* partial,
                                  float* partial_b, float* dW, float* db, TcErr err, cudaStream_t s) {
    if (W % tc::kTile || H < 1 || B < 1) return cudaErrorInvalidValue;
    if (reinterpret_cast<uintptr_t>(dY) % 16) return cudaErrorMisalignedAddress;
    static bool attr = false;
    if (!attr) {
        cudaError_t e =
            cudaFuncSetAttribute(tc::k_wgrad_out_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::kWoSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    CUtensorMap mapX;
    cudaError_t em = encode_act_map(&mapX, X, B, H, W);
    if (em != cudaSuccess) return em;
    const int ntiles = B * ((H + 1) / 2) * (W / tc::kTile);
    const int grid = ntiles < tc_sms() ? ntiles : tc_sms();   // within the partial buffers (one part per SM)
    tc::k_wgrad_out_tc<<<grid, tc::kWoThreads, tc::kWoSmem, s>>>(B, H, W, mapX, dY, partial, partial_b, err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cnn_sum_partials2(partial, 9 * tc::kC * 4, dW, partial_b, 4, db, grid, s);
}


cudaError_t cnn_refresh_weights(const float* p, long long np, const long long* woff, float* pr, void* wbf,
                                void* wflip, void* wtc, float* w6flip, void* win, void* win6, void* wout,
                                cudaStream_t s) {
    tc::RefreshArgs a;
    a.p = p;
    a.np = np;
    for (int l = 0; l < 6; ++l) a.woff[l] = woff[l];
    a.pr = pr;
    a.wbf = static_cast<__nv_bfloat16*>(wbf);
    a.wflip = static_cast<__nv_bfloat16*>(wflip);
    a.wtc = static_cast<__nv_bfloat16*>(wtc);
    a.w6flip = w6flip;
    a.win = static_cast<__nv_bfloat16*>(win);
    a.win6 = static_cast<__nv_bfloat16*>(win6);
    a.wout = static_cast<__nv_bfloat16*>(wout);
    const long long n = np + 4LL * tc::kW64 + 9 * 4 * tc::kC + 2 * tc::kInPlanes * tc::kC * 8 + 9 * 16 * tc::kC;
    tc::k_refresh_weights<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace plbm
