// Internal declarations shared by the host library and the CUDA translation
// units of libplbm.  Not part of the public ABI (see include/plbm.h).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "plbm.h"

namespace plbm {

constexpr int kMaxQ1 = 8;
constexpr int kMaxQ = kMaxQ1 * kMaxQ1;
constexpr int kBlockX = 128;       // threads per block along x in the step kernels
constexpr int kPartialStride = 8;  // doubles per block in the reduction scratch
constexpr int kPitchAlign = 64;    // row pitch is a multiple of this many elements

enum Prec { kF64 = 0, kF32 = 1, kF16Dev = 2, kBF16Dev = 3 };

// Everything a step kernel needs about one lattice, passed by value as a
// __grid_constant__ kernel parameter (it lives in the constant bank, so the
// c_ij, velocities and rest weights are broadcast reads).
struct LatticeParams {
    int nx, ny, pitch, dim;
    long long plane;        // elements between population planes (= pitch * ny)
    int q1, q;
    int fixed_ends;         // 1: ghost populations outside 0 <= x < nx
    int isothermal;         // 1: theta in f^eq held at theta0
    int paired;             // 1: row-paired layout (see elem_index), 2D even ny only
    int half_ny;            // ny / 2 when paired
    int sym5;               // 1: q1 = 5 with v = (0, a, -a, b, -b), a, b > 0, a != b
    int v[kMaxQ1];          // integer velocities
    int vxm[kMaxQ1];        // (-v) mod nx, in [0, nx): source column = x + vxm (- nx)
    int vym[kMaxQ1];        // (-v) mod ny, in [0, ny)
    int nz;                 // 3D: nodes along z (1 otherwise); rows of elem_index are z * ny + y
    int zpaired;            // 3D z-paired layout (16-bit storage, even nz): nodes (x, y, z) and
                            // (x, y, z + nz/2) side by side, row (z mod nz/2) * ny + y
    int half_nz;            // nz / 2 when zpaired
    int vzm[kMaxQ1];        // (-v) mod nz, in [0, nz)
    double omega, theta0;
    float omegaf, theta0f;
    double C[kMaxQ1 * kMaxQ1];   // C[i*q1 + n] multiplies mu_n in r_i (Eq. eq:rdr)
    float Cf[kMaxQ1 * kMaxQ1];   // FP32 part of C ...
    float Cf_lo[kMaxQ1 * kMaxQ1];// ... and the FP32 remainder C - Cf (coefficients to ~2^-48)
    // Symmetric five-velocity sets: factors of the constraint form of the rule
    // (odd part from sum v r = mu_1, sum v^3 r = mu_3; even part from
    // sum r = mu_0, sum v^2 r = mu_2, sum v^4 r = mu_4).
    float sa, sb, sa2, sb2;      // a, b, a^2, b^2
    float kOa, kOb, kEa, kEb;    // 1/(2a), 1/(2b(b^2-a^2)), 1/(2a^2), 1/(2b^2(b^2-a^2))
    float w1f[kMaxQ1];           // 1D rest weights r_i(0, theta0)
    float mu0f[kMaxQ1];          // mu_n(0, theta0)
    float W0f[kMaxQ];            // rest equilibrium w0_p (product of 1D weights in 2D)
    double W0[kMaxQ];            // the same in FP64
    double w1[kMaxQ1];           // 1D rest weights in FP64
    double ghostL[kMaxQ], ghostR[kMaxQ];    // f^eq of the end states (f-space, FP64)
    float ghostLg[kMaxQ], ghostRg[kMaxQ];   // the same as deviations from w0 (FP32)
    unsigned* status;            // device status word (PLBM_STATUS_* bits)
    double* partials;            // reduction scratch, kPartialStride doubles per block
};

// Where a lattice of a batch in the plain layout sits: its two population
// arrays and its first tile in the batch's tile list (tiles_x tiles per row).
struct NodeSpan {
    void* f[2];
    int nx, tiles_x, tile_begin, pad_;
};

// Compact parameters of the row-paired kernel (one lattice).  The batched
// runner keeps one per instance in device memory and caches it in shared memory.
struct PairParams {
    int nx, ny, half_ny, pitch;   // pitch in elements of one row (pairs per pair row)
    long long plane2;             // pairs per population plane (= half_ny * pitch)
    int vxm[5], vym[5];
    float sa, sb, sa2, sb2, kOa, kOb, kEa, kEb;
    float w1f[5];
    float omegaf, theta0f;
    double theta0;
    unsigned* status;
    double* partials;
    void* f[2];                   // population arrays (batched runner; unused by single launches)
    int tile_begin, tiles_x;      // batched runner: first global tile, tiles per pair row (per row, plain)
    int paired;                   // 1: row-paired layout, plane2 in pairs; 0: plain, plane2 in elements
};

// Rows of tiles of a lattice in the batched runner: pair rows or rows.
inline int tile_rows(const PairParams& Q) { return Q.paired ? Q.half_ny : Q.ny; }

inline PairParams pair_params(const LatticeParams& P) {
    PairParams Q{};
    Q.nx = P.nx;
    Q.ny = P.ny;
    Q.half_ny = P.half_ny;
    Q.pitch = P.pitch;
    Q.paired = P.paired;
    Q.plane2 = P.paired ? (long long)P.half_ny * P.pitch : P.plane;
    for (int i = 0; i < 5; ++i) {
        Q.vxm[i] = P.vxm[i];
        Q.vym[i] = P.vym[i];
        Q.w1f[i] = P.w1f[i];
    }
    Q.sa = P.sa;
    Q.sb = P.sb;
    Q.sa2 = P.sa2;
    Q.sb2 = P.sb2;
    Q.kOa = P.kOa;
    Q.kOb = P.kOb;
    Q.kEa = P.kEa;
    Q.kEb = P.kEb;
    Q.omegaf = P.omegaf;
    Q.theta0f = P.theta0f;
    Q.theta0 = P.theta0;
    Q.status = P.status;
    Q.partials = P.partials;
    return Q;
}

// max |lambda| of the one-step operator linearised at f^eq(1, (ux, 0), theta0),
// over an nk x nk grid of wave vectors (plbm_stability.cpp).  With stop_above > 0
// the search may stop at the first |lambda| above it (the result is then a lower
// bound that exceeds stop_above).
double spectral_radius(int dim, int q1, const int* v, const double* C, double omega, double theta0,
                       bool isothermal, double ux, int nk, double stop_above);

// Error flag of the tensor-core kernels and the budget of each of their bounded
// waits: a wait that runs longer sets *flag, and the kernel stops issuing work,
// drains the MMAs it issued (a fixed 2 s bound, whatever the budget), frees its
// tensor memory and returns.
struct TcErr {
    unsigned* flag;
    unsigned long long wait_ns;
};

// Surrogate kernels (plbm_cnn.cu, plbm_ce.cu).
cudaError_t cnn_conv64_fwd(int B, int H, int W, const void* X, const void* Wt, const float* bias, const void* mask,
                           void* Y, int mode, int relu, cudaStream_t s);
int cnn_wgrad64_parts(int B, int H, int W);
cudaError_t cnn_conv64_wgrad(int B, int H, int W, const void* X, const void* dY, float* partial, float* partial_b,
                             float* dW, float* db, cudaStream_t s);
cudaError_t cnn_conv64_wgrad_tc(int B, int H, int W, const void* X, const void* dY, float* partial, float* partial_b,
                                float* dW, float* db, TcErr err, cudaStream_t s);
cudaError_t cnn_sum_partials(const float* partial, int nparts, int n, float* out, cudaStream_t s);
// Two partial-sum reductions (a weight gradient and its bias gradient) in one launch.
cudaError_t cnn_sum_partials2(const float* partial, int n, float* out, const float* partial2, int n2, float* out2,
                              int nparts, cudaStream_t s);
cudaError_t cnn_conv_in_wgrad_tc(int B, int H, int W, const void* X, const void* dY, float* partial, float* partial_b,
                                 float* dW, float* db, TcErr err, cudaStream_t s);
// Every derived weight array of the surrogate from the FP32 master weights p (np
// values, layer l's weights at woff[l], 6 layers) in one launch: pr (bf16-rounded
// p), wbf / wflip (4 x 9*64*64 bf16), wtc (8 x 9*64*64 bf16), w6flip (FP32), and
// the tensor-core layouts win, win6, wout.
cudaError_t cnn_refresh_weights(const float* p, long long np, const long long* woff, float* pr, void* wbf,
                                void* wflip, void* wtc, float* w6flip, void* win, void* win6, void* wout,
                                cudaStream_t s);
// Output-layer (64 -> 4) weight and bias gradients on tcgen05 from the bf16 activations X and the FP32
// upstream gradient dY ([B][H][W][4], 16-byte aligned).
cudaError_t cnn_conv_out_wgrad_tc(int B, int H, int W, const void* X, const float* dY, float* partial,
                                  float* partial_b, float* dW, float* db, TcErr err, cudaStream_t s);
cudaError_t cnn_conv_thin_fwd(int ci, int co, int ti, int to, int B, int H, int W, const void* X, const float* Wf,
                              const float* bias, const void* mask, void* Y, int mode, int relu, cudaStream_t s);
int cnn_thin_parts(int B, int H, int W, int* pix_per_block);
cudaError_t cnn_conv_thin_wgrad(int ci, int co, int tx, int tg, int B, int H, int W, const void* X, const void* dY,
                                float* partial, float* partial_b, float* dW, float* db, cudaStream_t s);
// ReLU bits rbits: one uint64_t per pixel, bit c set when the stored bf16 output
// channel c of a forward ReLU layer is > 0.  mode 0 (forward) writes them when
// rbits is not null; mode 1 (backward data, Y = conv(X) * bit) reads them.
cudaError_t cnn_conv64_tc(int B, int H, int W, const void* X, const void* Wk, const float* bias, uint64_t* rbits,
                          void* Y, int mode, int relu, TcErr err, cudaStream_t s);
cudaError_t cnn_conv_out_tc(int B, int H, int W, const void* X, const void* Wo, const float* bias, float* Y,
                            TcErr err, cudaStream_t s);
// mode 0: Y = relu?(conv(X) + bias) (the 4 -> 64 input layer; ReLU bits to rbits
// when given); mode 1: Y = conv(X) * bit (the 64 -> 4 output layer's backward data,
// X = its bf16 upstream gradient, Win from the flipped weights, rbits required).
cudaError_t cnn_conv_in_tc(int B, int H, int W, const void* X, const void* Win, const float* bias, uint64_t* rbits,
                           void* Y, int mode, int relu, TcErr err, cudaStream_t s);
// grad16 (optional): the gradient also in bf16.
cudaError_t cnn_mse(const float* pred, const float* target, long long n, long long npix, float lam, float* merr,
                    float* grad, void* grad16, float* partial, int parts, cudaStream_t s);
cudaError_t cnn_adam(float* p, const float* g, float* m, float* v, long long n, float lr, float b1, float b2, float eps,
                     int t, cudaStream_t s);
cudaError_t cnn_to_bf16(const float* a, long long n, void* b, cudaStream_t s);
cudaError_t ce_pack_fields(const double* rho, const double* ux, const double* uy, const double* th, long long n,
                           float* out, cudaStream_t s);
cudaError_t ce_assemble(const float* snaps, long long npix, const int* pairs, int B, const float* mean_in,
                        const float* std_in, const float* mean_d, const float* std_d, void* x, float* y,
                        float sigma, unsigned long long seed, cudaStream_t s);
cudaError_t ce_normalise(const float* F, long long n, const float* mean_in, const float* std_in, void* x,
                         cudaStream_t s);
cudaError_t ce_apply_delta(const float* F, const float* d, long long n, const float* mean_d, const float* std_d,
                           float* out, cudaStream_t s);
int ce_sum_blocks();
cudaError_t ce_field_sums(const float* F, long long n, double* partial, cudaStream_t s);
cudaError_t ce_reconstruct(int prec, const LatticeParams& P, const float* F, void* f, cudaStream_t s);
// A lattice of a batched launch over lattices of one model (the same
// LatticeParams but for the arrays): its population array and its index in the
// field stacks (fields of lattice `index` start at index * nx * ny).
struct LatticeRef {
    void* f;
    long long index;
};
// ce_reconstruct for n lattices in one launch (grid.z = lattice): refs in device memory.
cudaError_t ce_reconstruct_batch(int prec, const LatticeParams& P, const float* F, const LatticeRef* refs, int n,
                                 cudaStream_t s);
// Shift the predicted fields of nlat lattices so that their global mass,
// momentum and energy equal the old fields' (delta: 4 floats per lattice).
cudaError_t ce_conserve(const float* Fold, float* Fnew, long long n, int nlat, double* partial_old,
                        double* partial_new, float* delta, cudaStream_t s);
cudaError_t ce_field_drift(const float* Fold, const float* Fnew, long long n, int nlat, double* partial_old,
                           double* partial_new, double* drift, cudaStream_t s);

// Internals of a live handle for the surrogate path (plbm_host.cpp).
struct HandleView {
    const LatticeParams* P;
    void* f_cur;
    void* f_next;      // the other population array
    int* cur;          // index of the current array (0/1)
    int prec;
    cudaStream_t stream;
    long long* steps;
};
bool handle_view(void* h, HandleView* out);
// Whether plbm_create gives this descriptor the row-paired layout.
bool desc_row_paired(const plbm_desc* d);

// Records the error text returned by plbm_last_error(NULL) for this thread.
void set_thread_error(const char* msg);

// Launchers implemented in the CUDA translation units.  All are asynchronous
// on `stream` and return the launch error.
cudaError_t launch_step(int prec, const LatticeParams& P, const void* src, void* dst,
                        bool reduce, cudaStream_t stream);
// Rows [y0, y1) (y1 < 0: to the last row); field pointers index the whole lattice.
// Batched step of 2D lattices in the plain layout, all of precision prec and
// q1 velocities per axis (q1 = 3, 4 or 5): tiles of kBlockX nodes of one row.
cudaError_t launch_batch_node(int prec, int q1, const LatticeParams* inst, const NodeSpan* span, int total_tiles,
                              int ctas, int parity, const unsigned short* tile_inst, cudaStream_t stream);
cudaError_t batch_node_occupancy(int prec, int q1, int* blocks_per_sm);
cudaError_t launch_init(int prec, const LatticeParams& P, const double* rho, const double* ux,
                        const double* uy, const double* theta, void* f, cudaStream_t stream, int y0 = 0,
                        int y1 = -1);
cudaError_t launch_moments(int prec, const LatticeParams& P, const void* f, double* rho,
                           double* ux, double* uy, double* theta, cudaStream_t stream, int y0 = 0,
                           int y1 = -1);
// Up to five FP64 field arrays of n values; rho and theta index the fields that
// must be positive (-1: none).  Null pointers are not allowed in field[0..count).
struct FieldSet {
    const double* field[5];
    int count, rho, theta;
};
// Sets PLBM_STATUS_* bits in *status for non-finite values, rho <= 0, theta <= 0.
cudaError_t launch_check_fields(const FieldSet& F, long long n, unsigned* status, cudaStream_t stream);
// Three-dimensional lattices (plbm_step3.cu): storage [q][nz][ny][pitch].
long long reduce3_blocks(const LatticeParams& P);
cudaError_t launch_step3(int prec, const LatticeParams& P, const void* src, void* dst, cudaStream_t s);
cudaError_t launch_init3(int prec, const LatticeParams& P, const double* rho, const double* ux, const double* uy,
                         const double* uz, const double* theta, void* f, cudaStream_t s);
cudaError_t launch_moments3(int prec, const LatticeParams& P, const void* f, double* rho, double* ux, double* uy,
                            double* uz, double* theta, cudaStream_t s);
cudaError_t launch_reduce3(int prec, const LatticeParams& P, const void* f, double* out, cudaStream_t s);
cudaError_t launch_get_pop3(int prec, const LatticeParams& P, const void* f, double* out, cudaStream_t s);
cudaError_t launch_set_pop3(int prec, const LatticeParams& P, const double* in, void* f, cudaStream_t s);
cudaError_t launch_moments_pack(int prec, const LatticeParams& P, const void* f, float* F, void* x,
                                const float* mean_in, const float* std_in, cudaStream_t stream);
// launch_moments_pack for n lattices of one model in one launch; F and x are the
// stacks, lattice r writes at r.index * nx * ny.
cudaError_t launch_moments_pack_batch(int prec, const LatticeParams& P, const LatticeRef* refs, int n, float* F,
                                      void* x, const float* mean_in, const float* std_in, cudaStream_t stream);
// Per-block partial sums of the stored state, then one deterministic final pass
// writing out[0..5] = mass, jx, jy, energy, rho_min, theta_min.
cudaError_t launch_reduce_state(int prec, const LatticeParams& P, const void* f, double* out,
                                cudaStream_t stream);
// Final pass over the partials written by a reducing step kernel.
cudaError_t launch_finalize(const LatticeParams& P, int nblocks, double* out, cudaStream_t stream);
cudaError_t launch_get_populations(int prec, const LatticeParams& P, const void* f, double* out,
                                   cudaStream_t stream);
cudaError_t launch_set_populations(int prec, const LatticeParams& P, const double* in, void* f,
                                   cudaStream_t stream);

// Batched persistent step over the instances of `inst` (device array, tile_begin
// ascending); block_x in {64, 128, 256}; ctas persistent CTAs.
// Persistent batched step.  tile_inst == nullptr: CTA c walks the contiguous tile
// range [c * per_cta, (c + 1) * per_cta); otherwise the tiles c, c + ctas, ...
// with tile_inst[t] the instance of global tile t.
cudaError_t launch_batch(int prec, const PairParams* inst, int ninst, int total_tiles, int block_x,
                         int ctas, int parity, const unsigned short* tile_inst, cudaStream_t stream);
cudaError_t batch_occupancy(int prec, int block_x, int* blocks_per_sm);

// Number of blocks of a step launch (row-paired kernels cover two rows per block row).
inline int step_blocks(const LatticeParams& P) {
    return ((P.nx + kBlockX - 1) / kBlockX) * (P.paired ? P.half_ny : P.ny);
}

// Number of blocks of a reduction over the stored state (one node per thread).
inline int reduce_blocks(const LatticeParams& P) {
    return ((P.nx + kBlockX - 1) / kBlockX) * P.ny;
}

// Element index of population p at node (x, y) in a population array.
// Plain layout:  p * plane + y * pitch + x.
// Row-paired layout (2D, even ny, H = ny / 2): nodes (x, r) and (x, r + H) sit
// next to each other, so one aligned 2-element vector holds both:
//                p * plane + (y mod H) * 2 * pitch + 2 x + (y >= H).
__host__ __device__ inline long long elem_index(const LatticeParams& P, int p, int x, int y) {
    if (P.paired) {
        const int hi = y >= P.half_ny;
        const int r = hi ? y - P.half_ny : y;
        return (long long)p * P.plane + (long long)r * 2 * P.pitch + 2LL * x + hi;
    }
    return (long long)p * P.plane + (long long)y * P.pitch + x;
}

}  // namespace plbm
