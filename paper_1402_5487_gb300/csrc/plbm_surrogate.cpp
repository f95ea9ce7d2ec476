// Learned surrogate: network state, training step, inference and the advance
// of lattices by K steps with Chapman-Enskog reconstruction and LBM fallback.
//
// Network: 6 convolutions 3x3 with circular padding, channels 4 -> 64 -> 64 ->
// 64 -> 64 -> 64 -> 4, ReLU after the first five, BF16 activations and
// weights with FP32 accumulation, FP32 master weights and Adam state.  Input:
// normalised (rho, u_x, u_y, theta) of a periodic lattice; output: the
// normalised change of those fields over K lattice steps.
//
// Flat parameter layout (FP32): for each layer, W[3][3][cin][cout] then b[cout].
#include "plbm.h"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "plbm_internal.h"

namespace {

constexpr int kLayers = 6;
constexpr int kCin[kLayers] = {4, 64, 64, 64, 64, 64};
constexpr int kCout[kLayers] = {64, 64, 64, 64, 64, 4};

struct Sur {
    int Bm = 0, H = 0, W = 0;
    cudaStream_t stream = nullptr;
    bool owns_stream = false;
    long long woff[kLayers], boff[kLayers], nparams = 0;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    float* pr = nullptr;            // parameters rounded to bf16 precision (fp32 storage)
    void* wbf = nullptr;            // bf16 weights of layers 1..4 (64 -> 64), 4 x 9*64*64
    void* wflip = nullptr;          // their backward-data form
    float* w6flip = nullptr;        // backward-data weights of the last layer (4 -> 64)
    void* wtc = nullptr;            // K-major bf16 weights for tcgen05: 4 layers x (forward, backward data)
    void* win = nullptr;            // first layer (4 -> 64) for tcgen05: bf16 [6][64][8]
    void* win6 = nullptr;           // the last layer's backward-data weights in the same layout
    void* dout16 = nullptr;         // bf16 copy of the upstream gradient of the output [pix][4]
    uint64_t* rbits = nullptr;      // ReLU bits of the hidden layers 0..4 (tensor-core path), 5 x [pix]
    void* wout = nullptr;           // last layer (64 -> 4) for tcgen05: bf16 [9][16][64]
    unsigned* derr = nullptr;       // device flag: a bounded wait in a tensor-core kernel ran out
    unsigned long long wait_ns = 2000000000ull;  // budget of each of those waits
    int use_tc = 1;                 // forward convolutions and 64 -> 64 backward data: 1 tcgen05, 0 mma.sync / CUDA cores
    int conserve = 0;               // 1: project predicted fields onto the old global sums before the drift gate
    float mean_penalty = 0.0f;      // weight of the lattice-mean error term of the training loss
    void* act[kLayers] = {nullptr}; // act[0..4] bf16 [B][H][W][64]; act[5] fp32 [B][H][W][4]
    void* dz[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // dL/d(pre-activation) of layers 1..5
    float* dout = nullptr;
    float *part = nullptr, *part_b = nullptr;
    float* loss_part = nullptr;
    float* host_loss = nullptr;
    int adam_t = 0;
    float norm[16] = {0, 0, 0, 0, 1, 1, 1, 1, 0, 0, 0, 0, 1, 1, 1, 1};  // mean_in, std_in, mean_d, std_d
    // advance scratch
    float *Fold = nullptr, *Fnew = nullptr;
    void* xin = nullptr;
    double* planes = nullptr;
    double* sums = nullptr;         // per-block FP64 field sums: old fields, then predicted fields
    double* host_sums = nullptr;
    double* drift = nullptr;        // device: drift of every lattice of the last advance
    plbm::PairParams* fb_table = nullptr;  // device: batched fallback of row-paired lattices
    unsigned short* fb_tile_inst = nullptr;  // device: lattice of every fallback tile (interleaved order)
    plbm::LatticeRef* dref = nullptr;   // device: lattices of the batched moments and reconstruction launches
    plbm::LatticeRef* href = nullptr;   // pinned host copy (2 x max_batch: moments, then reconstruction)
    int sms = 0;
    std::vector<double> last_drift;
    std::vector<unsigned short> fb_tiles;  // host copy of fb_tile_inst (kept for the async copy)
    cudaEvent_t ev = nullptr;
    char err[512] = "";
};

void serr(Sur* s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    plbm::set_thread_error(buf);
    if (s) std::snprintf(s->err, sizeof s->err, "%s", buf);
}

#define SCK(call)                                                              \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) {                                               \
            serr(s, "%s failed: %s", #call, cudaGetErrorString(e_));           \
            return PLBM_E_CUDA;                                                \
        }                                                                      \
    } while (0)

// splitmix64 and Box-Muller: a fully specified generator, so the initial
// weights are the same on every host.
uint64_t splitmix(uint64_t& x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
double uniform01(uint64_t& st) { return ((splitmix(st) >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
double normal(uint64_t& st) {
    const double u1 = uniform01(st), u2 = uniform01(st);
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

void free_sur(Sur* s) {
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    void* bufs[] = {s->p, s->g, s->m, s->v, s->pr, s->wbf, s->wflip, s->w6flip, s->dz[0], s->dz[1], s->dz[2],
                    s->dz[3], s->dz[4], s->dout, s->part, s->part_b, s->loss_part, s->Fold, s->Fnew, s->xin,
                    s->planes, s->sums, s->wtc, s->derr, s->win, s->win6, s->dout16, s->wout, s->drift, s->fb_table, s->fb_tile_inst,
                    s->dref, s->rbits};
    for (void* b : bufs)
        if (b) cudaFree(b);
    for (void* a : s->act)
        if (a) cudaFree(a);
    if (s->host_loss) cudaFreeHost(s->host_loss);
    if (s->host_sums) cudaFreeHost(s->host_sums);
    if (s->href) cudaFreeHost(s->href);
    if (s->ev) cudaEventDestroy(s->ev);
    if (s->owns_stream) cudaStreamDestroy(s->stream);
    delete s;
}

// Whether two lattices share every parameter the per-lattice kernels of an
// advance read (all but their arrays, status word and reduction scratch).
bool same_model(const plbm::LatticeParams& a, const plbm::LatticeParams& b) {
    plbm::LatticeParams x = a, y = b;
    x.status = y.status = nullptr;
    x.partials = y.partials = nullptr;
    return std::memcmp(&x, &y, sizeof x) == 0;
}

void* wtc_fwd(Sur* s, int l) { return static_cast<char*>(s->wtc) + (size_t)(2 * (l - 1)) * 9 * 64 * 64 * 2; }
void* wtc_bwd(Sur* s, int l) { return static_cast<char*>(s->wtc) + (size_t)(2 * (l - 1) + 1) * 9 * 64 * 64 * 2; }
// ReLU bits of hidden layer l (output of layer l, 0..4): one uint64_t per pixel
uint64_t* rbits_of(Sur* s, int l) { return s->rbits + (size_t)l * s->Bm * s->H * s->W; }

// Rounded copies, bf16 weights and backward-data weights from the FP32 master weights.
plbm_status refresh_weights(Sur* s) {
    SCK(plbm::cnn_refresh_weights(s->p, s->nparams, s->woff, s->pr, s->wbf, s->wflip, s->wtc, s->w6flip, s->win,
                                  s->win6, s->wout, s->stream));
    return PLBM_OK;
}

// keep_bits: the tensor-core path also records the ReLU bits of every hidden
// layer for a backward pass.
plbm_status forward(Sur* s, int B, const void* x, bool keep_bits = false) {
    const int H = s->H, W = s->W;
    if (s->use_tc) {
        SCK(plbm::cnn_conv_in_tc(B, H, W, x, s->win, s->p + s->boff[0], keep_bits ? rbits_of(s, 0) : nullptr,
                                 s->act[0], 0, 1,
                                 plbm::TcErr{s->derr, s->wait_ns}, s->stream));
    } else {
        SCK(plbm::cnn_conv_thin_fwd(4, 64, 0, 0, B, H, W, x, s->pr + s->woff[0], s->p + s->boff[0], nullptr,
                                    s->act[0], 0, 1, s->stream));
    }
    for (int l = 1; l <= 4; ++l) {
        if (s->use_tc) {
            SCK(plbm::cnn_conv64_tc(B, H, W, s->act[l - 1], wtc_fwd(s, l), s->p + s->boff[l],
                                    keep_bits ? rbits_of(s, l) : nullptr, s->act[l], 0, 1,
                                    plbm::TcErr{s->derr, s->wait_ns}, s->stream));
        } else {
            const char* wb = static_cast<const char*>(s->wbf) + (size_t)(l - 1) * 9 * 64 * 64 * 2;
            SCK(plbm::cnn_conv64_fwd(B, H, W, s->act[l - 1], wb, s->p + s->boff[l], nullptr, s->act[l], 0, 1,
                                     s->stream));
        }
    }
    if (s->use_tc) {
        SCK(plbm::cnn_conv_out_tc(B, H, W, s->act[4], s->wout, s->p + s->boff[5], static_cast<float*>(s->act[5]),
                                  plbm::TcErr{s->derr, s->wait_ns}, s->stream));
    } else {
        SCK(plbm::cnn_conv_thin_fwd(64, 4, 0, 1, B, H, W, s->act[4], s->pr + s->woff[5], s->p + s->boff[5], nullptr,
                                    s->act[5], 0, 0, s->stream));
    }
    return PLBM_OK;
}

// Gradients of every parameter into s->g for the upstream gradient dout of the
// output.  dz[k] keeps dL/dZ of layer k + 1 (Z = convolution output before ReLU).
// dout16_ready: s->dout16 already holds dout in bf16 (written with the loss).
plbm_status backward(Sur* s, int B, const void* x, const float* dout, bool dout16_ready = false) {
    const int H = s->H, W = s->W;
    // last layer (64 -> 4): weights, then dZ_5 = (conv^T dout) * (A_5 > 0)
    if (s->use_tc && reinterpret_cast<uintptr_t>(dout) % 16 == 0)
        SCK(plbm::cnn_conv_out_wgrad_tc(B, H, W, s->act[4], dout, s->part, s->part_b, s->g + s->woff[5],
                                        s->g + s->boff[5], plbm::TcErr{s->derr, s->wait_ns}, s->stream));
    else
        SCK(plbm::cnn_conv_thin_wgrad(64, 4, 0, 1, B, H, W, s->act[4], dout, s->part, s->part_b, s->g + s->woff[5],
                                      s->g + s->boff[5], s->stream));
    if (s->use_tc) {   // tcgen05, on the bf16-rounded upstream gradient (the other layers' gradients are bf16 too)
        if (!dout16_ready) SCK(plbm::cnn_to_bf16(dout, (long long)B * H * W * 4, s->dout16, s->stream));
        SCK(plbm::cnn_conv_in_tc(B, H, W, s->dout16, s->win6, nullptr, rbits_of(s, 4), s->dz[4], 1, 0,
                                 plbm::TcErr{s->derr, s->wait_ns}, s->stream));
    } else {
        SCK(plbm::cnn_conv_thin_fwd(4, 64, 1, 0, B, H, W, dout, s->w6flip, nullptr, s->act[4], s->dz[4], 1, 0,
                                    s->stream));
    }
    for (int l = 4; l >= 1; --l) {
        if (s->use_tc)
            SCK(plbm::cnn_conv64_wgrad_tc(B, H, W, s->act[l - 1], s->dz[l], s->part, s->part_b, s->g + s->woff[l],
                                          s->g + s->boff[l], plbm::TcErr{s->derr, s->wait_ns}, s->stream));
        else
            SCK(plbm::cnn_conv64_wgrad(B, H, W, s->act[l - 1], s->dz[l], s->part, s->part_b, s->g + s->woff[l],
                                       s->g + s->boff[l], s->stream));
        if (s->use_tc) {
            SCK(plbm::cnn_conv64_tc(B, H, W, s->dz[l], wtc_bwd(s, l), nullptr, rbits_of(s, l - 1), s->dz[l - 1], 1, 0,
                                    plbm::TcErr{s->derr, s->wait_ns}, s->stream));
        } else {
            const char* wf = static_cast<const char*>(s->wflip) + (size_t)(l - 1) * 9 * 64 * 64 * 2;
            SCK(plbm::cnn_conv64_fwd(B, H, W, s->dz[l], wf, nullptr, s->act[l - 1], s->dz[l - 1], 1, 0, s->stream));
        }
    }
    if (s->use_tc)
        SCK(plbm::cnn_conv_in_wgrad_tc(B, H, W, x, s->dz[0], s->part, s->part_b, s->g + s->woff[0],
                                       s->g + s->boff[0], plbm::TcErr{s->derr, s->wait_ns}, s->stream));
    else
        SCK(plbm::cnn_conv_thin_wgrad(4, 64, 0, 0, B, H, W, x, s->dz[0], s->part, s->part_b, s->g + s->woff[0],
                                      s->g + s->boff[0], s->stream));
    return PLBM_OK;
}

Sur* as_sur(plbm_surrogate h) { return reinterpret_cast<Sur*>(h); }

}  // namespace

extern "C" {

int plbm_sur_num_params(void) {
    long long n = 0;
    for (int l = 0; l < kLayers; ++l) n += 9LL * kCin[l] * kCout[l] + kCout[l];
    return (int)n;
}

plbm_status plbm_sur_create(int max_batch, int H, int W, unsigned long long seed, void* stream, plbm_surrogate* out) {
    if (!out || max_batch < 1 || max_batch > 65535 || H < 3 || W < 128 || W % 128) {
        serr(nullptr, "plbm_sur_create: need 1 <= max_batch <= 65535, H >= 3 and W a multiple of 128");
        return PLBM_E_ARG;
    }
    *out = nullptr;
    Sur* s = new (std::nothrow) Sur();
    if (!s) return PLBM_E_NOMEM;
    s->Bm = max_batch;
    s->H = H;
    s->W = W;
    if (stream) {
        s->stream = static_cast<cudaStream_t>(stream);
    } else {
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
            serr(s, "cudaStreamCreate failed");
            delete s;
            return PLBM_E_CUDA;
        }
        s->owns_stream = true;
    }
    long long off = 0;
    for (int l = 0; l < kLayers; ++l) {
        s->woff[l] = off;
        off += 9LL * kCin[l] * kCout[l];
        s->boff[l] = off;
        off += kCout[l];
    }
    s->nparams = off;
    const size_t np = (size_t)off * sizeof(float);
    const size_t pix = (size_t)max_batch * H * W;
    int pb = 0;
    const int thin_parts = plbm::cnn_thin_parts(max_batch, H, W, &pb);
    const int mid_parts = plbm::cnn_wgrad64_parts(max_batch, H, W);
    const size_t part_n = std::max((size_t)mid_parts * 9 * 64 * 64, (size_t)thin_parts * 9 * 64 * 4);
    const size_t partb_n = (size_t)std::max(mid_parts, thin_parts) * 64;
    struct A {
        void** p;
        size_t n;
    } allocs[] = {
        {(void**)&s->p, np}, {(void**)&s->g, np}, {(void**)&s->m, np}, {(void**)&s->v, np}, {(void**)&s->pr, np},
        {&s->wbf, 4 * 9 * 64 * 64 * 2}, {&s->wflip, 4 * 9 * 64 * 64 * 2}, {(void**)&s->w6flip, 9 * 4 * 64 * 4},
        {&s->dz[0], pix * 64 * 2}, {&s->dz[1], pix * 64 * 2}, {&s->dz[2], pix * 64 * 2},
        {&s->dz[3], pix * 64 * 2}, {&s->dz[4], pix * 64 * 2}, {(void**)&s->dout, pix * 4 * 4},
        {(void**)&s->part, part_n * 4}, {(void**)&s->part_b, partb_n * 4}, {(void**)&s->loss_part, (size_t)(1024 + 4 * max_batch) * 4},
        {(void**)&s->Fold, pix * 4 * 4}, {(void**)&s->Fnew, pix * 4 * 4}, {&s->xin, pix * 4 * 2},
        {(void**)&s->planes, (size_t)H * W * 4 * 8}, {(void**)&s->sums, (size_t)max_batch * 2 * 64 * 4 * 8},
        {&s->wtc, 8 * 9 * 64 * 64 * 2}, {(void**)&s->derr, 256}, {&s->win, 6 * 64 * 8 * 2},
        {&s->win6, 6 * 64 * 8 * 2}, {&s->dout16, pix * 4 * 2},
        {&s->wout, 9 * 16 * 64 * 2}, {(void**)&s->drift, (size_t)max_batch * 24 + 16},
        {(void**)&s->fb_table, (size_t)max_batch * sizeof(plbm::PairParams)},
        {(void**)&s->fb_tile_inst, (size_t)max_batch * ((W + 127) / 128) * ((H + 1) / 2) * sizeof(unsigned short) + 256},
        {(void**)&s->dref, (size_t)2 * max_batch * sizeof(plbm::LatticeRef)},
        {(void**)&s->rbits, 5 * pix * 8},
    };
    for (auto& a : allocs) {
        if (cudaMalloc(a.p, a.n) != cudaSuccess) {
            serr(s, "cudaMalloc of %zu bytes failed", a.n);
            free_sur(s);
            return PLBM_E_NOMEM;
        }
    }
    for (int l = 0; l < 5; ++l) {
        if (cudaMalloc(&s->act[l], pix * 64 * 2) != cudaSuccess) {
            serr(s, "cudaMalloc of activations failed");
            free_sur(s);
            return PLBM_E_NOMEM;
        }
    }
    if (cudaMalloc(&s->act[5], pix * 4 * 4) != cudaSuccess ||
        cudaMallocHost((void**)&s->host_loss, 1024 * 4) != cudaSuccess ||
        cudaMallocHost((void**)&s->host_sums, (size_t)max_batch * 2 * 64 * 4 * 8) != cudaSuccess ||
        cudaMallocHost((void**)&s->href, (size_t)2 * max_batch * sizeof(plbm::LatticeRef)) != cudaSuccess) {
        serr(s, "allocation failed");
        free_sur(s);
        return PLBM_E_NOMEM;
    }
    {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, dev);
        if (s->sms < 1) s->sms = 1;
    }
    if (cudaEventCreateWithFlags(&s->ev, cudaEventDisableTiming) != cudaSuccess) {
        serr(s, "cudaEventCreate failed");
        free_sur(s);
        return PLBM_E_CUDA;
    }
    if (cudaMemsetAsync(s->derr, 0, 256, s->stream) != cudaSuccess) {
        serr(s, "cudaMemset failed");
        free_sur(s);
        return PLBM_E_CUDA;
    }
    // He initialisation (normal, std sqrt(2 / fan_in)); the last layer scaled by 0.1 so
    // that an untrained network predicts almost no change.  Biases zero.
    std::vector<float> h(off, 0.0f);
    uint64_t st = seed * 0x2545F4914F6CDD1DULL + 12345;
    for (int l = 0; l < kLayers; ++l) {
        const double sd = std::sqrt(2.0 / (9.0 * kCin[l])) * (l == kLayers - 1 ? 0.1 : 1.0);
        for (long long k = 0; k < 9LL * kCin[l] * kCout[l]; ++k) h[s->woff[l] + k] = (float)(sd * normal(st));
    }
    plbm_surrogate out_h = reinterpret_cast<plbm_surrogate>(s);
    plbm_status r = plbm_sur_set_params(out_h, h.data());
    if (r != PLBM_OK) {
        free_sur(s);
        return r;
    }
    *out = out_h;
    return PLBM_OK;
}

plbm_status plbm_sur_destroy(plbm_surrogate h) {
    free_sur(as_sur(h));
    return PLBM_OK;
}

plbm_status plbm_sur_set_params(plbm_surrogate h, const float* params) {
    Sur* s = as_sur(h);
    if (!s || !params) return PLBM_E_ARG;
    SCK(cudaMemcpyAsync(s->p, params, s->nparams * 4, cudaMemcpyHostToDevice, s->stream));
    SCK(cudaMemsetAsync(s->m, 0, s->nparams * 4, s->stream));
    SCK(cudaMemsetAsync(s->v, 0, s->nparams * 4, s->stream));
    s->adam_t = 0;
    plbm_status r = refresh_weights(s);
    if (r != PLBM_OK) return r;
    SCK(cudaStreamSynchronize(s->stream));
    return PLBM_OK;
}

plbm_status plbm_sur_get_params(plbm_surrogate h, float* params, float* grads) {
    Sur* s = as_sur(h);
    if (!s) return PLBM_E_ARG;
    if (params) SCK(cudaMemcpyAsync(params, s->p, s->nparams * 4, cudaMemcpyDeviceToHost, s->stream));
    if (grads) SCK(cudaMemcpyAsync(grads, s->g, s->nparams * 4, cudaMemcpyDeviceToHost, s->stream));
    SCK(cudaStreamSynchronize(s->stream));
    return PLBM_OK;
}

plbm_status plbm_sur_set_option(plbm_surrogate h, int option, int value) {
    Sur* s = as_sur(h);
    if (!s) return PLBM_E_ARG;
    if (option == PLBM_SUR_OPT_TENSOR_PATH && (value == 0 || value == 1)) {
        s->use_tc = value;
        return PLBM_OK;
    }
    if (option == PLBM_SUR_OPT_CONSERVE && (value == 0 || value == 1)) {
        s->conserve = value;
        return PLBM_OK;
    }
    if (option == PLBM_SUR_OPT_WAIT_NS && value >= 1) {
        s->wait_ns = (unsigned long long)value;
        return PLBM_OK;
    }
    serr(s, "unknown option %d or value %d", option, value);
    return PLBM_E_ARG;
}

plbm_status plbm_sur_set_mean_penalty(plbm_surrogate h, float lambda) {
    Sur* s = as_sur(h);
    if (!s || !(lambda >= 0.0f) || !(lambda < 1e30f)) {
        serr(s, "mean penalty must be finite and >= 0");
        return PLBM_E_ARG;
    }
    s->mean_penalty = lambda;
    return PLBM_OK;
}

plbm_status plbm_sur_check(plbm_surrogate h) {
    Sur* s = as_sur(h);
    if (!s) return PLBM_E_ARG;
    unsigned e = 0;
    SCK(cudaMemcpyAsync(&e, s->derr, sizeof e, cudaMemcpyDeviceToHost, s->stream));
    SCK(cudaStreamSynchronize(s->stream));
    if (e) {
        SCK(cudaMemsetAsync(s->derr, 0, sizeof e, s->stream));  // reported once
        SCK(cudaStreamSynchronize(s->stream));
        serr(s, "a bounded wait of a tensor-core kernel ran out: the pass was abandoned, its results are invalid");
        return PLBM_E_TIMEOUT;
    }
    return PLBM_OK;
}

plbm_status plbm_sur_set_norm(plbm_surrogate h, const float* mean_in, const float* std_in, const float* mean_d,
                              const float* std_d) {
    Sur* s = as_sur(h);
    if (!s || !mean_in || !std_in || !mean_d || !std_d) return PLBM_E_ARG;
    for (int k = 0; k < 4; ++k) {
        if (!(std_in[k] > 0.0f) || !(std_d[k] > 0.0f)) {
            serr(s, "standard deviations must be > 0");
            return PLBM_E_ARG;
        }
        s->norm[k] = mean_in[k];
        s->norm[4 + k] = std_in[k];
        s->norm[8 + k] = mean_d[k];
        s->norm[12 + k] = std_d[k];
    }
    return PLBM_OK;
}

plbm_status plbm_sur_forward(plbm_surrogate h, int B, const void* x, float* out) {
    Sur* s = as_sur(h);
    if (!s || !x || B < 1 || B > s->Bm) return PLBM_E_ARG;
    plbm_status r = forward(s, B, x);
    if (r != PLBM_OK) return r;
    if (out) SCK(cudaMemcpyAsync(out, s->act[5], (size_t)B * s->H * s->W * 16, cudaMemcpyDeviceToDevice, s->stream));
    return PLBM_OK;
}

plbm_status plbm_sur_backward(plbm_surrogate h, int B, const void* x, const float* dout) {
    Sur* s = as_sur(h);
    if (!s || !x || !dout || B < 1 || B > s->Bm) return PLBM_E_ARG;
    plbm_status r = forward(s, B, x, true);
    if (r != PLBM_OK) return r;
    return backward(s, B, x, dout);
}

plbm_status plbm_sur_copy(plbm_surrogate h, int kind, int layer, int B, void* dst) {
    Sur* s = as_sur(h);
    if (!s || !dst || B < 1 || B > s->Bm) return PLBM_E_ARG;
    const size_t pix = (size_t)B * s->H * s->W;
    const void* src = nullptr;
    size_t bytes = 0;
    if (kind == 0 && layer >= 1 && layer <= 5) {
        src = s->act[layer - 1];
        bytes = pix * 64 * 2;
    } else if (kind == 0 && layer == 6) {
        src = s->act[5];
        bytes = pix * 4 * 4;
    } else if (kind == 1 && layer >= 1 && layer <= 5) {
        src = s->dz[layer - 1];
        bytes = pix * 64 * 2;
    } else {
        serr(s, "plbm_sur_copy: kind 0 takes layers 1..6, kind 1 layers 1..5");
        return PLBM_E_ARG;
    }
    SCK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s->stream));
    SCK(cudaStreamSynchronize(s->stream));
    return PLBM_OK;
}

plbm_status plbm_sur_train_step(plbm_surrogate h, int B, const void* x, const float* target, float lr, float* loss) {
    Sur* s = as_sur(h);
    if (!s || !x || !target || B < 1 || B > s->Bm || !(lr > 0.0f)) return PLBM_E_ARG;
    plbm_status r = forward(s, B, x, true);
    if (r != PLBM_OK) return r;
    const long long n = (long long)B * s->H * s->W * 4;
    const int parts = 1024;   // the loss partials (loss_part[0 .. 1023])
    SCK(plbm::cnn_mse(static_cast<const float*>(s->act[5]), target, n, (long long)s->H * s->W, s->mean_penalty,
                      s->loss_part + 1024, s->dout, s->use_tc ? s->dout16 : nullptr, s->loss_part, parts, s->stream));
    r = backward(s, B, x, s->dout, s->use_tc);
    if (r != PLBM_OK) return r;
    ++s->adam_t;
    SCK(plbm::cnn_adam(s->p, s->g, s->m, s->v, s->nparams, lr, 0.9f, 0.999f, 1e-8f, s->adam_t, s->stream));
    r = refresh_weights(s);
    if (r != PLBM_OK) return r;
    if (loss) {
        SCK(cudaMemcpyAsync(s->host_loss, s->loss_part, parts * 4, cudaMemcpyDeviceToHost, s->stream));
        SCK(cudaStreamSynchronize(s->stream));
        double t = 0.0;
        for (int k = 0; k < parts; ++k) t += s->host_loss[k];
        *loss = (float)(t / (double)n);
    }
    return PLBM_OK;
}

plbm_status plbm_sur_pack_fields(const double* rho, const double* ux, const double* uy, const double* theta,
                                 long long n, float* out, void* stream) {
    if (!rho || !ux || !uy || !theta || !out || n < 1) return PLBM_E_ARG;
    cudaError_t e = plbm::ce_pack_fields(rho, ux, uy, theta, n, out, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? PLBM_OK : PLBM_E_CUDA;
}

plbm_status plbm_sur_assemble(plbm_surrogate h, const float* snaps, long long npix, const int* pairs, int B, void* x,
                              float* y) {
    return plbm_sur_assemble_noise(h, snaps, npix, pairs, B, x, y, 0.0f, 0ull);
}

plbm_status plbm_sur_assemble_noise(plbm_surrogate h, const float* snaps, long long npix, const int* pairs, int B,
                                    void* x, float* y, float sigma, unsigned long long seed) {
    Sur* s = as_sur(h);
    if (!s || !snaps || !pairs || !x || !y || B < 1) return PLBM_E_ARG;
    if (!(sigma >= 0.0f) || !(sigma < 1e30f)) {
        serr(s, "input noise sigma must be finite and >= 0");
        return PLBM_E_ARG;
    }
    SCK(plbm::ce_assemble(snaps, npix, pairs, B, s->norm, s->norm + 4, s->norm + 8, s->norm + 12, x, y, sigma, seed,
                          s->stream));
    return PLBM_OK;
}

plbm_status plbm_sur_advance(plbm_surrogate h, plbm_handle* hs, int n, int K, double tol, int* fell_back) {
    Sur* s = as_sur(h);
    if (!s || !hs || n < 1 || n > s->Bm || K < 1) return PLBM_E_ARG;
    const long long npix = (long long)s->H * s->W;
    std::vector<plbm::HandleView> views(n);
    for (int b = 0; b < n; ++b) {
        if (!plbm::handle_view(hs[b], &views[b])) {
            serr(s, "handle %d is not initialised or in an error state", b);
            return PLBM_E_STATE;
        }
        const plbm::LatticeParams& P = *views[b].P;
        if (P.dim != 2 || P.nx != s->W || P.ny != s->H || P.fixed_ends) {
            serr(s, "handle %d: the surrogate takes periodic %d x %d lattices", b, s->W, s->H);
            return PLBM_E_ARG;
        }
    }
    // Lattices of one model (the same parameters but for their arrays) take the
    // per-lattice kernels below in one launch each (grid.z = lattice).
    bool one_model = n > 1;
    for (int b = 1; b < n && one_model; ++b) one_model = views[b].prec == views[0].prec && same_model(*views[b].P, *views[0].P);
    // 1. fields and network input of every lattice, on the surrogate's stream
    //    once the lattice's own stream has reached this point
    for (int b = 0; b < n; ++b) {
        SCK(cudaEventRecord(s->ev, views[b].stream));
        SCK(cudaStreamWaitEvent(s->stream, s->ev, 0));
        if (!one_model)
            SCK(plbm::launch_moments_pack(views[b].prec, *views[b].P, views[b].f_cur, s->Fold + (size_t)b * npix * 4,
                                          static_cast<char*>(s->xin) + (size_t)b * npix * 4 * 2, s->norm,
                                          s->norm + 4, s->stream));
    }
    if (one_model) {
        for (int b = 0; b < n; ++b) s->href[b] = plbm::LatticeRef{views[b].f_cur, b};
        SCK(cudaMemcpyAsync(s->dref, s->href, (size_t)n * sizeof(plbm::LatticeRef), cudaMemcpyHostToDevice,
                            s->stream));
        SCK(plbm::launch_moments_pack_batch(views[0].prec, *views[0].P, s->dref, n, s->Fold, s->xin, s->norm,
                                            s->norm + 4, s->stream));
    }
    // 2. network, predicted fields, drift of the conserved sums
    plbm_status r = forward(s, n, s->xin);
    if (r != PLBM_OK) return r;
    SCK(plbm::ce_apply_delta(s->Fold, static_cast<const float*>(s->act[5]), npix * n, s->norm + 8, s->norm + 12,
                             s->Fnew, s->stream));
    const size_t half = (size_t)s->Bm * plbm::ce_sum_blocks() * 4;
    if (s->conserve)
        SCK(plbm::ce_conserve(s->Fold, s->Fnew, npix, n, s->sums, s->sums + half,
                              reinterpret_cast<float*>(s->drift + ((s->Bm + 1) & ~1)), s->stream));
    SCK(plbm::ce_field_drift(s->Fold, s->Fnew, npix, n, s->sums, s->sums + half, s->drift, s->stream));
    SCK(cudaMemcpyAsync(s->host_sums, s->drift, (size_t)n * 8, cudaMemcpyDeviceToHost, s->stream));
    SCK(cudaStreamSynchronize(s->stream));
    s->last_drift.assign(s->host_sums, s->host_sums + n);
    // 3. accepted lattices: Chapman-Enskog populations on the surrogate's stream,
    //    which the lattice's stream then waits for; the others run K LBM steps
    bool any = false;
    int nacc = 0;
    for (int b = 0; b < n; ++b) {
        const bool fall = !(s->last_drift[b] <= tol);
        if (fell_back) fell_back[b] = fall ? 1 : 0;
        if (fall) continue;
        if (one_model)
            s->href[s->Bm + nacc++] = plbm::LatticeRef{views[b].f_cur, b};
        else
            SCK(plbm::ce_reconstruct(views[b].prec, *views[b].P, s->Fnew + (size_t)b * npix * 4, views[b].f_cur,
                                     s->stream));
        *views[b].steps += K;
        any = true;
    }
    if (nacc > 0) {
        SCK(cudaMemcpyAsync(s->dref + s->Bm, s->href + s->Bm, (size_t)nacc * sizeof(plbm::LatticeRef),
                            cudaMemcpyHostToDevice, s->stream));
        SCK(plbm::ce_reconstruct_batch(views[0].prec, *views[0].P, s->Fnew, s->dref + s->Bm, nacc, s->stream));
    }
    // Fallback lattices in the row-paired layout (one precision) take K steps
    // together, one persistent launch per step over all of them (the batched
    // runner's kernel); any other fallback lattice steps on its own.
    std::vector<int> batched, single;
    int bprec = -1;
    for (int b = 0; b < n; ++b) {
        if (s->last_drift[b] <= tol) continue;
        const plbm::LatticeParams& P = *views[b].P;
        if (P.paired && (bprec < 0 || views[b].prec == bprec)) {
            bprec = views[b].prec;
            batched.push_back(b);
        } else {
            single.push_back(b);
        }
    }
    if (batched.size() < 2) {
        single.insert(single.end(), batched.begin(), batched.end());
        batched.clear();
    }
    if (!batched.empty()) {
        constexpr int kBX = 128;
        std::vector<plbm::PairParams> table(batched.size());
        int tiles = 0;
        for (size_t k = 0; k < batched.size(); ++k) {
            const plbm::HandleView& v = views[batched[k]];
            plbm::PairParams Q = plbm::pair_params(*v.P);
            Q.f[0] = v.f_cur;
            Q.f[1] = v.f_next;
            Q.tiles_x = (Q.nx + kBX - 1) / kBX;
            Q.tile_begin = tiles;
            tiles += Q.tiles_x * plbm::tile_rows(Q);
            table[k] = Q;
        }
        // interleaved tile order (the batched runner's default): lattice of every tile
        s->fb_tiles.assign((size_t)tiles, 0);
        for (size_t k = 0; k < table.size(); ++k)
            std::fill(s->fb_tiles.begin() + table[k].tile_begin,
                      s->fb_tiles.begin() + table[k].tile_begin + table[k].tiles_x * plbm::tile_rows(table[k]),
                      (unsigned short)k);
        SCK(cudaMemcpyAsync(s->fb_table, table.data(), sizeof(plbm::PairParams) * table.size(),
                            cudaMemcpyHostToDevice, s->stream));
        SCK(cudaMemcpyAsync(s->fb_tile_inst, s->fb_tiles.data(), sizeof(unsigned short) * s->fb_tiles.size(),
                            cudaMemcpyHostToDevice, s->stream));
        int occ = 1;
        if (plbm::batch_occupancy(bprec, kBX, &occ) != cudaSuccess || occ < 1) occ = 1;
        const int ctas = s->sms * (occ < 3 ? occ : 3);   // the sweep's tuned shape: 128 threads, 3 CTAs per SM
        for (int k = 0; k < K; ++k)
            SCK(plbm::launch_batch(bprec, s->fb_table, (int)table.size(), tiles, kBX, ctas, k & 1,
                                   s->fb_tile_inst, s->stream));
        for (int b : batched) {
            if (K & 1) *views[b].cur ^= 1;
            *views[b].steps += K;
        }
        any = true;
    }
    if (any) SCK(cudaEventRecord(s->ev, s->stream));
    for (int b = 0; b < n; ++b)
        if (s->last_drift[b] <= tol || std::find(batched.begin(), batched.end(), b) != batched.end())
            SCK(cudaStreamWaitEvent(views[b].stream, s->ev, 0));
    for (int b : single) {
        r = plbm_step(hs[b], K);
        if (r != PLBM_OK) return r;
    }
    return PLBM_OK;
}

plbm_status plbm_sur_last_drift(plbm_surrogate h, double* out, int n) {
    Sur* s = as_sur(h);
    if (!s || !out || n < 0 || (size_t)n > s->last_drift.size()) return PLBM_E_ARG;
    for (int b = 0; b < n; ++b) out[b] = s->last_drift[b];
    return PLBM_OK;
}

const char* plbm_sur_last_error(plbm_surrogate h) {
    Sur* s = as_sur(h);
    return s ? s->err : plbm_last_error(nullptr);
}

}  // extern "C"
