// Host side of libplbm: descriptor validation, FP64 coefficients, the
// positivity gate, device memory and the extern "C" entry points of plbm.h.
#include "plbm.h"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "plbm_internal.h"

using plbm::LatticeParams;

namespace {

thread_local char g_thread_error[512] = "";

struct Handle {
    plbm_desc desc{};
    int v[plbm::kMaxQ1]{};
    LatticeParams P{};
    int prec = 0;
    size_t elem = 0;
    size_t pop_bytes = 0;      // one population array
    size_t ws_bytes = 0;
    char* ws = nullptr;        // device workspace base
    bool owns_ws = false;
    void* f[2] = {nullptr, nullptr};
    int cur = 0;
    double* partials = nullptr;
    double* result = nullptr;  // 8 doubles on the device
    unsigned* status = nullptr;
    double* host_buf = nullptr; // pinned: 8 result doubles + status word
    cudaStream_t stream = nullptr;
    long long steps = 0;
    plbm_status sticky = PLBM_OK;
    bool initialised = false;
    bool in_batch = false;     // owned by a plbm_batch: not destroyable on its own
    // Host-pointer init/moments: a staging buffer kept after first use, and a copy
    // stream that overlaps the transfer of one band of rows with the kernel on another.
    void* stage = nullptr;
    size_t stage_bytes = 0;
    cudaStream_t xfer = nullptr;
    cudaEvent_t xev[8] = {};
    // Small lattices: kGraphSteps steps captured once per starting array and replayed.
    cudaGraphExec_t sgraph[2] = {nullptr, nullptr};
    cudaStream_t cap = nullptr;                // private stream the graphs are captured on
    char err[512] = "";
};

constexpr int kGraphSteps = 32;                 // even: a replay leaves the current array unchanged
constexpr long long kGraphMaxNodes = 1 << 18;   // above this the GPU, not the launches, sets the pace

constexpr int kXferChunks = 8;       // row bands of a pipelined host transfer
constexpr size_t kXferMinNodes = 1u << 18;   // smaller lattices move in one band

void set_err(Handle* h, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    std::snprintf(g_thread_error, sizeof g_thread_error, "%s", buf);
    if (h) std::snprintf(h->err, sizeof h->err, "%s", buf);
}

size_t align_up(size_t n, size_t a) { return (n + a - 1) / a * a; }

size_t elem_size(int prec) {
    switch (prec) {
        case PLBM_F64: return 8;
        case PLBM_F32: return 4;
        case PLBM_F16DEV:
        case PLBM_BF16DEV: return 2;
    }
    return 0;
}

// Coefficients of Eq. (eq:rdr): row i holds the monomial coefficients of the
// Lagrange polynomial L_i(v) = prod_{j != i} (v - v_j) / prod_{j != i} (v_i - v_j),
// i.e. C = V^{-1} of the Appendix.  The numerator is expanded factor by factor.
bool lagrange_coefficients(int q1, const int* v, double* C) {
    for (int i = 0; i < q1; ++i) {
        double poly[plbm::kMaxQ1 + 1] = {1.0};
        int deg = 0;
        double den = 1.0;
        for (int j = 0; j < q1; ++j) {
            if (j == i) continue;
            if (v[j] == v[i]) return false;
            // poly <- poly * (v - v_j)
            for (int k = deg + 1; k >= 1; --k) poly[k] = poly[k - 1] - (double)v[j] * poly[k];
            poly[0] = -(double)v[j] * poly[0];
            ++deg;
            den *= (double)(v[i] - v[j]);
        }
        for (int n = 0; n < q1; ++n) C[i * q1 + n] = poly[n] / den;
    }
    return true;
}

// Maxwell-Boltzmann raw moments mu_0..mu_{q1-1} (Gaussian, mean u, variance theta).
void mb_moments(double u, double theta, int q1, double* mu) {
    mu[0] = 1.0;
    if (q1 > 1) mu[1] = u;
    for (int n = 1; n + 1 < q1; ++n) mu[n + 1] = u * mu[n] + n * theta * mu[n - 1];
}

void rule_1d(int q1, const double* C, double u, double theta, double* r) {
    double mu[plbm::kMaxQ1];
    mb_moments(u, theta, q1, mu);
    for (int i = 0; i < q1; ++i) {
        double s = 0.0;
        for (int n = 0; n < q1; ++n) s += C[i * q1 + n] * mu[n];
        r[i] = s;
    }
}

void feq_host(int dim, int q1, const double* C, double rho, double ux, double uy, double th,
              double* out) {
    double rx[plbm::kMaxQ1], ry[plbm::kMaxQ1];
    rule_1d(q1, C, ux, th, rx);
    if (dim == 1) {
        for (int i = 0; i < q1; ++i) out[i] = rho * rx[i];
        return;
    }
    rule_1d(q1, C, uy, th, ry);
    for (int i = 0; i < q1; ++i)
        for (int j = 0; j < q1; ++j) out[i * q1 + j] = rho * rx[i] * ry[j];
}

bool finite_pos(double a) { return std::isfinite(a) && a > 0.0; }

plbm_status validate(const plbm_desc* d, Handle* h) {
    if (!d) { set_err(h, "descriptor is NULL"); return PLBM_E_ARG; }
    if (d->dim < 1 || d->dim > 3) { set_err(h, "dim must be 1, 2 or 3 (got %d)", d->dim); return PLBM_E_ARG; }
    if (d->q1 < 3 || d->q1 > PLBM_MAX_Q1 || (d->dim == 3 && d->q1 > 5)) {
        set_err(h, "q1 must lie in [3, %d] (3D: [3, 5]) (got %d)", PLBM_MAX_Q1, d->q1);
        return PLBM_E_ARG;
    }
    if (!d->v) { set_err(h, "velocity array is NULL"); return PLBM_E_ARG; }
    for (int i = 0; i < d->q1; ++i) {
        if (d->v[i] < -64 || d->v[i] > 64) { set_err(h, "|v| must be <= 64"); return PLBM_E_ARG; }
        for (int j = 0; j < i; ++j)
            if (d->v[i] == d->v[j]) { set_err(h, "velocities must be distinct"); return PLBM_E_ARG; }
    }
    if (!(d->omega >= 0.0 && d->omega < 2.0)) {
        set_err(h, "omega must lie in [0, 2) (got %g)", d->omega);
        return PLBM_E_ARG;
    }
    if (!finite_pos(d->theta0)) { set_err(h, "theta0 must be finite and > 0"); return PLBM_E_ARG; }
    if (d->nx < 1 || d->ny < 1) { set_err(h, "nx, ny must be >= 1"); return PLBM_E_ARG; }
    if (d->dim == 1 && d->ny != 1) { set_err(h, "ny must be 1 in 1D"); return PLBM_E_ARG; }
    if (d->ny > 65535) { set_err(h, "ny must be <= 65535"); return PLBM_E_ARG; }
    const long long nz = d->dim == 3 ? d->nz : 1;
    if (d->dim == 3) {
        if (d->nz < 1 || d->nz > 65535) { set_err(h, "nz must lie in [1, 65535] in 3D"); return PLBM_E_ARG; }
        if (d->bc != PLBM_PERIODIC) { set_err(h, "3D lattices are periodic"); return PLBM_E_ARG; }
        const int* v = d->v;
        const bool sym5 = d->q1 == 5 && v && v[0] == 0 && v[1] > 0 && v[2] == -v[1] && v[3] > 0 && v[4] == -v[3] &&
                          v[1] != v[3];
        if (d->prec != PLBM_F64 && (!sym5 || (d->flags & PLBM_FLAG_ISOTHERMAL))) {
            set_err(h, "3D with 16/32-bit storage needs a thermal set v = (0, a, -a, b, -b)");
            return PLBM_E_ARG;
        }
    }
    if ((long long)d->nx * d->ny * nz > (1LL << 31)) { set_err(h, "grid too large"); return PLBM_E_ARG; }
    if (elem_size(d->prec) == 0) { set_err(h, "unknown precision %d", (int)d->prec); return PLBM_E_ARG; }
    if (d->bc != PLBM_PERIODIC && d->bc != PLBM_FIXED_ENDS) { set_err(h, "unknown boundary"); return PLBM_E_ARG; }
    if (d->bc == PLBM_FIXED_ENDS) {
        if (!d->left_state || !d->right_state) { set_err(h, "fixed ends need both end states"); return PLBM_E_ARG; }
        for (const double* s : {d->left_state, d->right_state}) {
            if (!finite_pos(s[0]) || !std::isfinite(s[1]) || !finite_pos(s[2])) {
                set_err(h, "end states need rho > 0, finite u, theta > 0");
                return PLBM_E_ARG;
            }
        }
    }
    if (d->check_every < 0) { set_err(h, "check_every must be >= 0"); return PLBM_E_ARG; }
    if (!(d->u_max >= 0.0) || !std::isfinite(d->u_max)) { set_err(h, "u_max must be >= 0"); return PLBM_E_ARG; }
    if (d->workspace && (reinterpret_cast<uintptr_t>(d->workspace) & 255u)) {
        set_err(h, "workspace must be 256-byte aligned");
        return PLBM_E_ARG;
    }
    return PLBM_OK;
}

struct Layout {
    int pitch;
    size_t pop_bytes, partial_off, result_off, status_off, total;
    int nblocks;
};

Layout layout_of(const plbm_desc* d) {
    Layout L{};
    L.pitch = (int)align_up((size_t)d->nx, plbm::kPitchAlign);
    const int q = d->dim == 1 ? d->q1 : (d->dim == 2 ? d->q1 * d->q1 : d->q1 * d->q1 * d->q1);
    const size_t rows = (size_t)d->ny * (d->dim == 3 ? d->nz : 1);
    L.pop_bytes = align_up((size_t)q * rows * L.pitch * elem_size(d->prec), 256);
    L.nblocks = (int)(((d->nx + plbm::kBlockX - 1) / plbm::kBlockX) * rows);
    L.partial_off = 2 * L.pop_bytes;
    L.result_off = L.partial_off + align_up((size_t)L.nblocks * plbm::kPartialStride * sizeof(double), 256);
    L.status_off = L.result_off + 256;
    L.total = L.status_off + 256;
    return L;
}

// Positivity gate of Sec. 3.1: every r_i(u, theta0) >= 0 for |u| <= u_max.
bool admissible(int q1, const double* C, double theta0, double u_max, double* worst_u, double* worst_r) {
    const int n = u_max > 0.0 ? 401 : 1;
    double r[plbm::kMaxQ1];
    *worst_r = 1e300;
    for (int k = 0; k < n; ++k) {
        const double u = (n == 1) ? 0.0 : -u_max + 2.0 * u_max * k / (n - 1);
        rule_1d(q1, C, u, theta0, r);
        for (int i = 0; i < q1; ++i) {
            if (r[i] < *worst_r) { *worst_r = r[i]; *worst_u = u; }
        }
    }
    return *worst_r >= -1e-14;
}

#define CK(call)                                                                       \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            set_err(h, "%s failed: %s", #call, cudaGetErrorString(e_));                \
            if (h) h->sticky = PLBM_E_CUDA;                                            \
            return PLBM_E_CUDA;                                                        \
        }                                                                              \
    } while (0)

plbm_status usable(Handle* h, bool need_init = true) {
    if (!h) { set_err(nullptr, "handle is NULL"); return PLBM_E_ARG; }
    if (h->sticky != PLBM_OK) {
        set_err(h, "handle is in error state %d: %s", (int)h->sticky, h->err);
        return h->sticky;
    }
    if (need_init && !h->initialised) { set_err(h, "populations not initialised"); return PLBM_E_STATE; }
    if (cudaSetDevice(h->desc.device) != cudaSuccess) { set_err(h, "cudaSetDevice failed"); return PLBM_E_CUDA; }
    return PLBM_OK;
}

void free_handle(Handle* h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    for (cudaGraphExec_t g : h->sgraph)
        if (g) cudaGraphExecDestroy(g);
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->xfer) {
        cudaStreamSynchronize(h->xfer);
        for (cudaEvent_t e : h->xev)
            if (e) cudaEventDestroy(e);
        cudaStreamDestroy(h->xfer);
    }
    if (h->stage) cudaFree(h->stage);
    if (h->owns_ws && h->ws) cudaFree(h->ws);
    if (h->host_buf) cudaFreeHost(h->host_buf);
    delete h;
}

plbm_status read_status(Handle* h, unsigned* bits) {
    CK(cudaMemcpyAsync(h->host_buf + 8, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    std::memcpy(bits, h->host_buf + 8, sizeof(unsigned));
    return PLBM_OK;
}

// Staging buffer of at least `bytes` and the copy stream with its events (made
// on first use; the previous host-pointer call has synchronised, so the buffer
// is idle).
#define XCK(call)                                                                      \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            set_err(h, "%s failed: %s", #call, cudaGetErrorString(e_));                \
            h->sticky = PLBM_E_CUDA;                                                   \
            return PLBM_E_CUDA;                                                        \
        }                                                                              \
    } while (0)

plbm_status ensure_xfer(Handle* h, size_t bytes) {
    if (!h->xfer) {
        XCK(cudaStreamCreateWithFlags(&h->xfer, cudaStreamNonBlocking));
        for (cudaEvent_t& e : h->xev) XCK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    if (h->stage_bytes < bytes) {
        if (h->stage) XCK(cudaFree(h->stage));
        h->stage = nullptr;
        h->stage_bytes = 0;
        if (cudaMalloc(&h->stage, bytes) != cudaSuccess) {
            cudaGetLastError();
            h->stage = nullptr;
            set_err(h, "staging buffer of %zu bytes: out of device memory", bytes);
            return PLBM_E_NOMEM;
        }
        h->stage_bytes = bytes;
    }
    return PLBM_OK;
}

// Row bands [y0, y1) of a pipelined transfer of an ny-row lattice.
int xfer_bands(const Handle* h) {
    const size_t n = (size_t)h->P.nx * h->P.ny;
    return (n >= kXferMinNodes && h->P.ny >= kXferChunks) ? kXferChunks : 1;
}

// Temporary device buffer for host<->device staging, stream-ordered.
struct Staging {
    void* p = nullptr;
    cudaStream_t s = nullptr;
    ~Staging() { if (p) cudaFreeAsync(p, s); }
};

}  // namespace

namespace plbm {
void set_thread_error(const char* msg) { std::snprintf(g_thread_error, sizeof g_thread_error, "%s", msg); }

bool desc_row_paired(const plbm_desc* d) {
    if (!d || !d->v || d->dim != 2 || d->q1 != 5) return false;
    const int* v = d->v;
    const bool sym5 = v[0] == 0 && v[1] > 0 && v[2] == -v[1] && v[3] > 0 && v[4] == -v[3] && v[1] != v[3];
    return sym5 && d->ny % 2 == 0 && d->prec != PLBM_F64 && !(d->flags & PLBM_FLAG_ISOTHERMAL) &&
           d->bc == PLBM_PERIODIC && !(d->flags & PLBM_FLAG_PLAIN_LAYOUT);
}

bool handle_view(void* hh, HandleView* out) {
    Handle* h = static_cast<Handle*>(hh);
    if (!h || !out || !h->initialised || h->sticky != PLBM_OK) return false;
    out->P = &h->P;
    out->f_cur = h->f[h->cur];
    out->f_next = h->f[h->cur ^ 1];
    out->cur = &h->cur;
    out->prec = h->prec;
    out->stream = h->stream;
    out->steps = &h->steps;
    return true;
}
}  // namespace plbm

extern "C" {

int plbm_abi_version(void) { return PLBM_ABI_VERSION; }

plbm_status plbm_coefficients(int q1, const int* v, double* C_out) {
    if (q1 < 2 || q1 > PLBM_MAX_Q1 || !v || !C_out) { set_err(nullptr, "bad arguments"); return PLBM_E_ARG; }
    if (!lagrange_coefficients(q1, v, C_out)) { set_err(nullptr, "velocities must be distinct"); return PLBM_E_ARG; }
    return PLBM_OK;
}

plbm_status plbm_positivity(const plbm_desc* desc, double u_max, double* min_r) {
    if (!min_r || !(u_max >= 0.0) || !std::isfinite(u_max)) {
        set_err(nullptr, "bad arguments");
        return PLBM_E_ARG;
    }
    plbm_status st = validate(desc, nullptr);
    if (st != PLBM_OK) return st;
    double C[plbm::kMaxQ1 * plbm::kMaxQ1];
    if (!lagrange_coefficients(desc->q1, desc->v, C)) {
        set_err(nullptr, "velocities must be distinct");
        return PLBM_E_ARG;
    }
    double wu = 0.0;
    admissible(desc->q1, C, desc->theta0, u_max, &wu, min_r);
    return PLBM_OK;
}

plbm_status plbm_linear_stability(const plbm_desc* desc, double ux, int nk, double stop_above,
                                  double* max_abs_lambda) {
    if (!max_abs_lambda || nk < 1 || nk > 256 || !std::isfinite(ux)) {
        set_err(nullptr, "bad arguments");
        return PLBM_E_ARG;
    }
    plbm_status st = validate(desc, nullptr);
    if (st != PLBM_OK) return st;
    if (desc->dim == 3) {
        set_err(nullptr, "the linear stability scan covers 1D and 2D lattices");
        return PLBM_E_ARG;
    }
    double C[plbm::kMaxQ1 * plbm::kMaxQ1];
    if (!lagrange_coefficients(desc->q1, desc->v, C)) {
        set_err(nullptr, "velocities must be distinct");
        return PLBM_E_ARG;
    }
    *max_abs_lambda = plbm::spectral_radius(desc->dim, desc->q1, desc->v, C, desc->omega, desc->theta0,
                                            (desc->flags & PLBM_FLAG_ISOTHERMAL) != 0, ux, nk, stop_above);
    return PLBM_OK;
}

size_t plbm_workspace_bytes(const plbm_desc* desc) {
    if (validate(desc, nullptr) != PLBM_OK) return 0;
    return layout_of(desc).total;
}

plbm_status plbm_create(const plbm_desc* desc, plbm_handle* out) {
    if (!out) { set_err(nullptr, "out is NULL"); return PLBM_E_ARG; }
    *out = nullptr;
    plbm_status st = validate(desc, nullptr);
    if (st != PLBM_OK) return st;
    Handle* h = new (std::nothrow) Handle();
    if (!h) { set_err(nullptr, "host allocation failed"); return PLBM_E_NOMEM; }
    h->desc = *desc;
    std::memcpy(h->v, desc->v, sizeof(int) * desc->q1);
    h->desc.v = h->v;
    h->desc.left_state = nullptr;
    h->desc.right_state = nullptr;
    h->stream = static_cast<cudaStream_t>(desc->stream);
    h->prec = (int)desc->prec;
    h->elem = elem_size(desc->prec);

    LatticeParams& P = h->P;
    std::memset(&P, 0, sizeof P);
    const int q1 = desc->q1, dim = desc->dim;
    P.nx = desc->nx;
    P.ny = desc->ny;
    P.dim = dim;
    P.q1 = q1;
    P.q = dim == 1 ? q1 : (dim == 2 ? q1 * q1 : q1 * q1 * q1);
    P.nz = dim == 3 ? desc->nz : 1;
    P.fixed_ends = desc->bc == PLBM_FIXED_ENDS;
    P.isothermal = (desc->flags & PLBM_FLAG_ISOTHERMAL) ? 1 : 0;
    P.omega = desc->omega;
    P.theta0 = desc->theta0;
    P.omegaf = (float)desc->omega;
    P.theta0f = (float)desc->theta0;
    for (int i = 0; i < q1; ++i) {
        P.v[i] = desc->v[i];
        P.vxm[i] = ((-desc->v[i]) % P.nx + P.nx) % P.nx;
        P.vym[i] = ((-desc->v[i]) % P.ny + P.ny) % P.ny;
        P.vzm[i] = ((-desc->v[i]) % P.nz + P.nz) % P.nz;
    }
    if (!lagrange_coefficients(q1, desc->v, P.C)) {
        set_err(nullptr, "velocities must be distinct");
        delete h;
        return PLBM_E_ARG;
    }
    for (int k = 0; k < q1 * q1; ++k) {
        P.Cf[k] = (float)P.C[k];
        P.Cf_lo[k] = (float)(P.C[k] - (double)P.Cf[k]);
    }
    const int* v = desc->v;
    P.sym5 = (q1 == 5 && v[0] == 0 && v[1] > 0 && v[2] == -v[1] && v[3] > 0 && v[4] == -v[3] &&
              v[1] != v[3]) ? 1 : 0;
    if (P.sym5) {
        const double a = v[1], b = v[3];
        P.sa = (float)a;
        P.sb = (float)b;
        P.sa2 = (float)(a * a);
        P.sb2 = (float)(b * b);
        P.kOa = (float)(1.0 / (2.0 * a));
        P.kOb = (float)(1.0 / (2.0 * b * (b * b - a * a)));
        P.kEa = (float)(1.0 / (2.0 * a * a));
        P.kEb = (float)(1.0 / (2.0 * b * b * (b * b - a * a)));
    }
    // Row-paired layout and the two-nodes-per-thread kernel: 2D periodic symmetric
    // five-velocity thermal lattices with an even number of rows, 16/32-bit storage.
    P.paired = (dim == 2 && desc->ny % 2 == 0 && desc->prec != PLBM_F64 && P.sym5 && !P.isothermal &&
                desc->bc == PLBM_PERIODIC && !(desc->flags & PLBM_FLAG_PLAIN_LAYOUT)) ? 1 : 0;
    P.half_ny = P.paired ? desc->ny / 2 : 0;
    // z-paired layout and the two-nodes-per-thread 3D kernel: 16-bit storage, even nz,
    // every |v| <= nz / 2 (one wrap of the pair row per pull).
    int vmax = 0;
    for (int i = 0; i < q1; ++i) vmax = std::max(vmax, std::abs(desc->v[i]));
    // The kernel indexes a population array in 32-bit pair offsets.
    const double pairs = (double)q1 * q1 * q1 * (double)align_up((size_t)desc->nx, plbm::kPitchAlign) *
                         desc->ny * (dim == 3 ? desc->nz : 1) / 2.0;
    P.zpaired = (dim == 3 && desc->nz % 2 == 0 && vmax <= desc->nz / 2 && P.sym5 && !P.isothermal &&
                 (desc->prec == PLBM_F16DEV || desc->prec == PLBM_BF16DEV) && pairs < 4294967296.0) ? 1 : 0;
    P.half_nz = P.zpaired ? desc->nz / 2 : 0;

    if (!(desc->flags & PLBM_FLAG_SKIP_ADMISSIBILITY)) {
        double wu = 0, wr = 0;
        if (!admissible(q1, P.C, desc->theta0, desc->u_max, &wu, &wr)) {
            set_err(nullptr,
                    "inadmissible: r_i(u=%g, theta0=%g) = %g < 0 (positivity range of Sec. 3.1)",
                    wu, desc->theta0, wr);
            delete h;
            return PLBM_E_INADMISSIBLE;
        }
    }

    // Rest equilibrium w0 = f^eq(1, 0, theta0) and the moments it reproduces.
    double mu0[plbm::kMaxQ1];
    mb_moments(0.0, desc->theta0, q1, mu0);
    rule_1d(q1, P.C, 0.0, desc->theta0, P.w1);
    for (int i = 0; i < q1; ++i) {
        P.w1f[i] = (float)P.w1[i];
        P.mu0f[i] = (float)mu0[i];
    }
    if (dim <= 2) {  // 3D kernels form w0 from the 1D weights (q1^3 exceeds the table)
        feq_host(dim, q1, P.C, 1.0, 0.0, 0.0, desc->theta0, P.W0);
        for (int p = 0; p < P.q; ++p) P.W0f[p] = (float)P.W0[p];
    }
    if (P.fixed_ends) {
        const double* L = desc->left_state;
        const double* R = desc->right_state;
        const double thL = P.isothermal ? desc->theta0 : L[2];
        const double thR = P.isothermal ? desc->theta0 : R[2];
        feq_host(dim, q1, P.C, L[0], L[1], 0.0, thL, P.ghostL);
        feq_host(dim, q1, P.C, R[0], R[1], 0.0, thR, P.ghostR);
        for (int p = 0; p < P.q; ++p) {
            P.ghostLg[p] = (float)(P.ghostL[p] - P.W0[p]);
            P.ghostRg[p] = (float)(P.ghostR[p] - P.W0[p]);
        }
    }

    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= desc->device || desc->device < 0) {
        set_err(nullptr, "no usable CUDA device %d (count %d)", desc->device, ndev);
        delete h;
        return PLBM_E_CUDA;
    }
    const Layout L = layout_of(desc);
    P.pitch = L.pitch;
    P.plane = (long long)L.pitch * desc->ny * P.nz;
    h->pop_bytes = L.pop_bytes;
    h->ws_bytes = L.total;
    if (cudaSetDevice(desc->device) != cudaSuccess) {
        set_err(nullptr, "cudaSetDevice(%d) failed", desc->device);
        delete h;
        return PLBM_E_CUDA;
    }
    if (desc->workspace) {
        if (desc->workspace_bytes < L.total) {
            set_err(nullptr, "workspace of %zu bytes is smaller than the %zu bytes needed",
                    desc->workspace_bytes, L.total);
            delete h;
            return PLBM_E_NOMEM;
        }
        h->ws = static_cast<char*>(desc->workspace);
    } else {
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, L.total);
        if (e != cudaSuccess) {
            set_err(nullptr, "cudaMalloc(%zu) failed: %s", L.total, cudaGetErrorString(e));
            delete h;
            return PLBM_E_NOMEM;
        }
        h->ws = static_cast<char*>(p);
        h->owns_ws = true;
    }
    if (cudaMallocHost(reinterpret_cast<void**>(&h->host_buf), 16 * sizeof(double)) != cudaSuccess) {
        set_err(nullptr, "cudaMallocHost failed");
        free_handle(h);
        return PLBM_E_NOMEM;
    }
    h->f[0] = h->ws;
    h->f[1] = h->ws + L.pop_bytes;
    h->partials = reinterpret_cast<double*>(h->ws + L.partial_off);
    h->result = reinterpret_cast<double*>(h->ws + L.result_off);
    h->status = reinterpret_cast<unsigned*>(h->ws + L.status_off);
    P.partials = h->partials;
    P.status = h->status;
    if (cudaMemsetAsync(h->status, 0, 256, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess) {
        set_err(nullptr, "initial status reset failed");
        free_handle(h);
        return PLBM_E_CUDA;
    }
    *out = reinterpret_cast<plbm_handle>(h);
    return PLBM_OK;
}

plbm_status plbm_destroy(plbm_handle hh) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (h && h->in_batch) {
        set_err(h, "instance handles of a batch are released by plbm_batch_destroy");
        return PLBM_E_STATE;
    }
    free_handle(h);
    return PLBM_OK;
}

static plbm::FieldSet field_set(const double* const* d, int nd) {
    plbm::FieldSet F{};
    F.rho = -1;
    F.theta = -1;
    for (int k = 0; k < nd; ++k) {
        if (!d[k]) continue;
        if (k == 0) F.rho = F.count;
        if (k == nd - 1) F.theta = F.count;
        F.field[F.count++] = d[k];
    }
    return F;
}

// After a synchronous (host-pointer) init: PLBM_E_ARG if the field check set a
// status bit; the handle is then left uninitialised.
static plbm_status init_fields_verdict(Handle* h) {
    unsigned bits = 0;
    plbm_status st = read_status(h, &bits);
    if (st != PLBM_OK) return st;
    if (bits) {
        h->initialised = false;
        set_err(h, "initial fields rejected (status 0x%x): non-finite values, rho <= 0 or theta <= 0", bits);
        return PLBM_E_ARG;
    }
    return PLBM_OK;
}

plbm_status plbm_init(plbm_handle hh, const double* rho, const double* ux, const double* uy,
                      const double* theta, int on_device) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    plbm_status st = usable(h, false);
    if (st != PLBM_OK) return st;
    if (h->P.dim == 3) { set_err(h, "3D handle: use plbm_init3"); return PLBM_E_ARG; }
    if (!rho || !ux || (h->P.dim == 2 && !uy) || (!theta && !h->P.isothermal)) {
        set_err(h, "missing field array");
        return PLBM_E_ARG;
    }
    const size_t n = (size_t)h->P.nx * h->P.ny;
    h->cur = 0;
    // the status word is cleared first: the initialisation kernels set its bits for
    // non-finite fields, rho <= 0 or theta <= 0 as they read them
    CK(cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->stream));
    if (on_device) {
        CK(plbm::launch_init(h->prec, h->P, rho, ux, uy, theta, h->f[0], h->stream));
    } else {
        // Band k of the four fields is copied on the copy stream while the kernel
        // initialises band k - 1 on the handle's stream.
        st = ensure_xfer(h, 4 * n * sizeof(double));
        if (st != PLBM_OK) return st;
        double* base = static_cast<double*>(h->stage);
        const double* src[4] = {rho, ux, (uy && h->P.dim == 2) ? uy : nullptr, theta};
        const double* dev[4];
        for (int k = 0; k < 4; ++k) dev[k] = src[k] ? base + k * n : nullptr;
        const int bands = xfer_bands(h);
        const int ny = h->P.ny, nx = h->P.nx;
        for (int b = 0; b < bands; ++b) {
            const int y0 = (int)((long long)ny * b / bands), y1 = (int)((long long)ny * (b + 1) / bands);
            const size_t off = (size_t)y0 * nx, cnt = (size_t)(y1 - y0) * nx;
            for (int k = 0; k < 4; ++k)
                if (src[k])
                    CK(cudaMemcpyAsync(base + k * n + off, src[k] + off, cnt * sizeof(double),
                                       cudaMemcpyHostToDevice, h->xfer));
            CK(cudaEventRecord(h->xev[b], h->xfer));
            CK(cudaStreamWaitEvent(h->stream, h->xev[b], 0));
            CK(plbm::launch_init(h->prec, h->P, dev[0], dev[1], dev[2], dev[3], h->f[0], h->stream, y0, y1));
        }
    }
    h->steps = 0;
    h->initialised = true;
    return on_device ? PLBM_OK : init_fields_verdict(h);
}

plbm_status plbm_check(plbm_handle hh) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    plbm_status st = usable(h);
    if (st != PLBM_OK) return st;
    unsigned bits = 0;
    st = read_status(h, &bits);
    if (st != PLBM_OK) return st;
    if (bits) {
        set_err(h, "diverged (status 0x%x) at or before step %lld", bits, h->steps);
        h->sticky = PLBM_E_DIVERGED;
        return PLBM_E_DIVERGED;
    }
    return PLBM_OK;
}

plbm_status plbm_step(plbm_handle hh, long n) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    plbm_status st = usable(h);
    if (st != PLBM_OK) return st;
    if (n < 0) { set_err(h, "n must be >= 0"); return PLBM_E_ARG; }
    const int ce = h->desc.check_every;
    long s = 0;
    const long long nodes = (long long)h->P.nx * h->P.ny * h->P.nz;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (ce == 0 && nodes <= kGraphMaxNodes && n >= 2 * kGraphSteps &&
        cudaStreamIsCapturing(h->stream, &cap) == cudaSuccess && cap == cudaStreamCaptureStatusNone) {
        // launch-bound lattices: replay a run of kGraphSteps steps, captured on a
        // private stream (any stream, the legacy default one included, can launch it)
        for (; s + kGraphSteps <= n; s += kGraphSteps) {
            cudaGraphExec_t& g = h->sgraph[h->cur];
            if (!g) {
                if (!h->cap) CK(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
                cudaGraph_t graph = nullptr;
                CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
                cudaError_t el = cudaSuccess;
                for (int k = 0, c = h->cur; k < kGraphSteps && el == cudaSuccess; ++k, c ^= 1)
                    el = h->P.dim == 3 ? plbm::launch_step3(h->prec, h->P, h->f[c], h->f[c ^ 1], h->cap)
                                       : plbm::launch_step(h->prec, h->P, h->f[c], h->f[c ^ 1], false, h->cap);
                const cudaError_t ec = cudaStreamEndCapture(h->cap, &graph);
                const cudaError_t ei = (el == cudaSuccess && ec == cudaSuccess)
                                           ? cudaGraphInstantiate(&g, graph, 0) : cudaSuccess;
                if (graph) cudaGraphDestroy(graph);
                CK(el);
                CK(ec);
                CK(ei);
            }
            CK(cudaGraphLaunch(g, h->stream));
            h->steps += kGraphSteps;
        }
    }
    for (; s < n; ++s) {
        if (h->P.dim == 3)
            CK(plbm::launch_step3(h->prec, h->P, h->f[h->cur], h->f[h->cur ^ 1], h->stream));
        else
            CK(plbm::launch_step(h->prec, h->P, h->f[h->cur], h->f[h->cur ^ 1], false, h->stream));
        h->cur ^= 1;
        ++h->steps;
        if (ce > 0 && ((s + 1) % ce == 0) && s + 1 < n) {
            st = plbm_check(hh);
            if (st != PLBM_OK) return st;
        }
    }
    if (ce > 0) return plbm_check(hh);
    return PLBM_OK;
}

plbm_status plbm_moments(plbm_handle hh, double* rho, double* ux, double* uy, double* theta,
                         int on_device) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    plbm_status st = usable(h);
    if (st != PLBM_OK && st != PLBM_E_DIVERGED) return st;
    if (st == PLBM_E_DIVERGED) { set_err(h, "handle diverged"); return st; }
    if (h->P.dim == 3) { set_err(h, "3D handle: use plbm_moments3"); return PLBM_E_ARG; }
    const size_t n = (size_t)h->P.nx * h->P.ny;
    if (on_device) {
        CK(plbm::launch_moments(h->prec, h->P, h->f[h->cur], rho, ux, uy, theta, h->stream));
        return PLBM_OK;
    }
    // The kernel fills band k on the handle's stream while band k - 1 is copied
    // to the host on the copy stream.
    st = ensure_xfer(h, 4 * n * sizeof(double));
    if (st != PLBM_OK) return st;
    double* base = static_cast<double*>(h->stage);
    double* outs[4] = {rho, ux, uy, theta};
    double* dev[4];
    for (int k = 0; k < 4; ++k) dev[k] = outs[k] ? base + k * n : nullptr;
    const int bands = xfer_bands(h);
    const int ny = h->P.ny, nx = h->P.nx;
    for (int b = 0; b < bands; ++b) {
        const int y0 = (int)((long long)ny * b / bands), y1 = (int)((long long)ny * (b + 1) / bands);
        const size_t off = (size_t)y0 * nx, cnt = (size_t)(y1 - y0) * nx;
        CK(plbm::launch_moments(h->prec, h->P, h->f[h->cur], dev[0], dev[1], dev[2], dev[3], h->stream, y0, y1));
        CK(cudaEventRecord(h->xev[b], h->stream));
        CK(cudaStreamWaitEvent(h->xfer, h->xev[b], 0));
        for (int k = 0; k < 4; ++k)
            if (outs[k])
                CK(cudaMemcpyAsync(outs[k] + off, base + k * n + off, cnt * sizeof(double),
                                   cudaMemcpyDeviceToHost, h->xfer));
    }
    CK(cudaStreamSynchronize(h->xfer));
    return PLBM_OK;
}

plbm_status plbm_diagnostics(plbm_handle hh, plbm_diag* out) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !out) { set_err(h, "bad arguments"); return PLBM_E_ARG; }
    if (!h->initialised) { set_err(h, "populations not initialised"); return PLBM_E_STATE; }
    if (h->sticky == PLBM_E_CUDA) { set_err(h, "handle in CUDA error state"); return PLBM_E_CUDA; }
    CK(cudaSetDevice(h->desc.device));
    if (h->P.dim == 3)
        CK(plbm::launch_reduce3(h->prec, h->P, h->f[h->cur], h->result, h->stream));
    else
        CK(plbm::launch_reduce_state(h->prec, h->P, h->f[h->cur], h->result, h->stream));
    CK(cudaMemcpyAsync(h->host_buf, h->result, 7 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(h->host_buf + 8, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    out->mass = h->host_buf[0];
    out->jx = h->host_buf[1];
    out->jy = h->host_buf[2];
    out->energy = h->host_buf[3];
    out->rho_min = h->host_buf[4];
    out->theta_min = h->host_buf[5];
    std::memcpy(&out->status, h->host_buf + 8, sizeof(unsigned));
    out->steps = h->steps;
    return PLBM_OK;
}

plbm_status plbm_step_diagnostics(plbm_handle hh, long n, plbm_diag* out) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    plbm_status st = usable(h);
    if (st != PLBM_OK) return st;
    if (n < 1 || !out) { set_err(h, "n must be >= 1 and out non-NULL"); return PLBM_E_ARG; }
    if (h->P.dim == 3) {
        st = plbm_step(hh, n);
        return st != PLBM_OK ? st : plbm_diagnostics(hh, out);
    }
    if (n > 1) {
        st = plbm_step(hh, n - 1);
        if (st != PLBM_OK) return st;
    }
    CK(plbm::launch_step(h->prec, h->P, h->f[h->cur], h->f[h->cur ^ 1], true, h->stream));
    h->cur ^= 1;
    ++h->steps;
    CK(plbm::launch_finalize(h->P, plbm::step_blocks(h->P), h->result, h->stream));
    CK(cudaMemcpyAsync(h->host_buf, h->result, 7 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(h->host_buf + 8, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    out->mass = h->host_buf[0];
    out->jx = h->host_buf[1];
    out->jy = h->host_buf[2];
    out->energy = h->host_buf[3];
    out->rho_min = h->host_buf[4];
    out->theta_min = h->host_buf[5];
    std::memcpy(&out->status, h->host_buf + 8, sizeof(unsigned));
    out->steps = h->steps;
    return PLBM_OK;
}

plbm_status plbm_conserved(plbm_handle hh, double out[4]) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (h && h->P.dim == 3) { set_err(h, "3D handle: use plbm_conserved3"); return PLBM_E_ARG; }
    plbm_diag d;
    plbm_status st = plbm_diagnostics(hh, &d);
    if (st != PLBM_OK) return st;
    out[0] = d.mass;
    out[1] = d.jx;
    out[2] = d.jy;
    out[3] = d.energy;
    return PLBM_OK;
}

plbm_status plbm_init3(plbm_handle hh, const double* rho, const double* ux, const double* uy, const double* uz,
                       const double* theta, int on_device) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    plbm_status st = usable(h, false);
    if (st != PLBM_OK) return st;
    if (h->P.dim != 3) { set_err(h, "plbm_init3 takes 3D handles"); return PLBM_E_ARG; }
    if (!rho || !ux || !uy || !uz || (!theta && !h->P.isothermal)) {
        set_err(h, "missing field array");
        return PLBM_E_ARG;
    }
    const size_t n = (size_t)h->P.nx * h->P.ny * h->P.nz;
    const double* d[5] = {rho, ux, uy, uz, theta};
    Staging stg;
    stg.s = h->stream;
    if (!on_device) {
        CK(cudaMallocAsync(&stg.p, 5 * n * sizeof(double), h->stream));
        double* base = static_cast<double*>(stg.p);
        for (int k = 0; k < 5; ++k) {
            if (!d[k]) continue;
            CK(cudaMemcpyAsync(base + k * n, d[k], n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
            d[k] = base + k * n;
        }
    }
    h->cur = 0;
    CK(plbm::launch_init3(h->prec, h->P, d[0], d[1], d[2], d[3], d[4], h->f[0], h->stream));
    CK(cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->stream));
    CK(plbm::launch_check_fields(field_set(d, 5), (long long)n, h->status, h->stream));
    h->steps = 0;
    h->initialised = true;
    return on_device ? PLBM_OK : init_fields_verdict(h);
}

plbm_status plbm_moments3(plbm_handle hh, double* rho, double* ux, double* uy, double* uz, double* theta,
                          int on_device) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    plbm_status st = usable(h);
    if (st != PLBM_OK && st != PLBM_E_DIVERGED) return st;
    if (st == PLBM_E_DIVERGED) { set_err(h, "handle diverged"); return st; }
    if (h->P.dim != 3) { set_err(h, "plbm_moments3 takes 3D handles"); return PLBM_E_ARG; }
    const size_t n = (size_t)h->P.nx * h->P.ny * h->P.nz;
    if (on_device) {
        CK(plbm::launch_moments3(h->prec, h->P, h->f[h->cur], rho, ux, uy, uz, theta, h->stream));
        return PLBM_OK;
    }
    Staging stg;
    stg.s = h->stream;
    CK(cudaMallocAsync(&stg.p, 5 * n * sizeof(double), h->stream));
    double* b = static_cast<double*>(stg.p);
    double* outs[5] = {rho, ux, uy, uz, theta};
    CK(plbm::launch_moments3(h->prec, h->P, h->f[h->cur], rho ? b : nullptr, ux ? b + n : nullptr,
                             uy ? b + 2 * n : nullptr, uz ? b + 3 * n : nullptr, theta ? b + 4 * n : nullptr,
                             h->stream));
    for (int k = 0; k < 5; ++k)
        if (outs[k]) CK(cudaMemcpyAsync(outs[k], b + k * n, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return PLBM_OK;
}

plbm_status plbm_conserved3(plbm_handle hh, double out[5]) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !out) { set_err(h, "bad arguments"); return PLBM_E_ARG; }
    if (h->P.dim != 3) { set_err(h, "plbm_conserved3 takes 3D handles"); return PLBM_E_ARG; }
    plbm_diag d;
    plbm_status st = plbm_diagnostics(hh, &d);
    if (st != PLBM_OK) return st;
    out[0] = d.mass;
    out[1] = d.jx;
    out[2] = d.jy;
    out[3] = h->host_buf[6];  // j_z, the seventh entry of the 3D reduction
    out[4] = d.energy;
    return PLBM_OK;
}

plbm_status plbm_get_populations(plbm_handle hh, double* f, int on_device) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !f) { set_err(h, "bad arguments"); return PLBM_E_ARG; }
    if (!h->initialised) { set_err(h, "populations not initialised"); return PLBM_E_STATE; }
    if (h->sticky == PLBM_E_CUDA) { set_err(h, "handle in CUDA error state"); return PLBM_E_CUDA; }
    CK(cudaSetDevice(h->desc.device));
    const size_t n = (size_t)h->P.q * h->P.nx * h->P.ny * h->P.nz;
    auto get = [&](double* dst) {
        return h->P.dim == 3 ? plbm::launch_get_pop3(h->prec, h->P, h->f[h->cur], dst, h->stream)
                             : plbm::launch_get_populations(h->prec, h->P, h->f[h->cur], dst, h->stream);
    };
    if (on_device) {
        CK(get(f));
        return PLBM_OK;
    }
    Staging stg;
    stg.s = h->stream;
    CK(cudaMallocAsync(&stg.p, n * sizeof(double), h->stream));
    CK(get(static_cast<double*>(stg.p)));
    CK(cudaMemcpyAsync(f, stg.p, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return PLBM_OK;
}

plbm_status plbm_set_populations(plbm_handle hh, const double* f, int on_device, int64_t step) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    plbm_status st = usable(h, false);
    if (st != PLBM_OK) return st;
    if (!f) { set_err(h, "populations pointer is NULL"); return PLBM_E_ARG; }
    const size_t n = (size_t)h->P.q * h->P.nx * h->P.ny * h->P.nz;
    const double* src = f;
    Staging stg;
    stg.s = h->stream;
    if (!on_device) {
        CK(cudaMallocAsync(&stg.p, n * sizeof(double), h->stream));
        CK(cudaMemcpyAsync(stg.p, f, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        src = static_cast<const double*>(stg.p);
    }
    h->cur = 0;
    if (h->P.dim == 3)
        CK(plbm::launch_set_pop3(h->prec, h->P, src, h->f[0], h->stream));
    else
        CK(plbm::launch_set_populations(h->prec, h->P, src, h->f[0], h->stream));
    CK(cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->stream));
    if (!on_device) CK(cudaStreamSynchronize(h->stream));
    h->steps = step;
    h->initialised = true;
    return PLBM_OK;
}

// ---------------------------------------------------------------------------
// Checkpoints: a fixed header that describes the lattice, then the stored
// population array byte for byte (its precision and layout), protected by a
// 64-bit FNV-1a checksum over the header (checksum field zero) and the payload.
// ---------------------------------------------------------------------------
namespace {

constexpr char kCkptMagic[8] = {'P', 'L', 'B', 'M', 'C', 'K', 'P', 'T'};
constexpr uint32_t kCkptFormat = 1;

struct CkptHeader {
    char magic[8];
    uint32_t format, header_bytes;
    int32_t abi, dim, q1, nx, ny, nz, prec, bc, isothermal, pitch, paired, zpaired;
    int32_t v[plbm::kMaxQ1];
    double omega, theta0;
    uint64_t ends_digest;   // FNV-1a of the fixed-end ghost populations (0 when periodic)
    int64_t step;
    uint64_t payload_bytes;
    uint64_t checksum;
};

// FNV-1a, 64-bit: for every byte, h = (h xor byte) * 1099511628211.
uint64_t fnv1a(uint64_t h, const void* data, size_t n) {
    const unsigned char* p = static_cast<const unsigned char*>(data);
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}
constexpr uint64_t kFnvOffset = 14695981039346656037ull;

CkptHeader ckpt_header_of(const Handle* h) {
    CkptHeader c;
    std::memset(&c, 0, sizeof c);
    std::memcpy(c.magic, kCkptMagic, sizeof c.magic);
    c.format = kCkptFormat;
    c.header_bytes = sizeof(CkptHeader);
    c.abi = PLBM_ABI_VERSION;
    c.dim = h->P.dim;
    c.q1 = h->P.q1;
    c.nx = h->P.nx;
    c.ny = h->P.ny;
    c.nz = h->P.nz;
    c.prec = h->prec;
    c.bc = h->P.fixed_ends;
    c.isothermal = h->P.isothermal;
    c.pitch = h->P.pitch;
    c.paired = h->P.paired;
    c.zpaired = h->P.zpaired;
    for (int i = 0; i < h->P.q1; ++i) c.v[i] = h->P.v[i];
    c.omega = h->P.omega;
    c.theta0 = h->P.theta0;
    if (h->P.fixed_ends) {
        c.ends_digest = fnv1a(kFnvOffset, h->P.ghostL, sizeof(double) * h->P.q);
        c.ends_digest = fnv1a(c.ends_digest, h->P.ghostR, sizeof(double) * h->P.q);
    }
    c.step = h->steps;
    c.payload_bytes = h->pop_bytes;
    return c;
}

}  // namespace

size_t plbm_checkpoint_bytes(plbm_handle hh) {
    const Handle* h = reinterpret_cast<const Handle*>(hh);
    return h ? sizeof(CkptHeader) + h->pop_bytes : 0;
}

plbm_status plbm_checkpoint_save(plbm_handle hh, void* buf, size_t bytes) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !buf) { set_err(h, "bad arguments"); return PLBM_E_ARG; }
    if (!h->initialised) { set_err(h, "populations not initialised"); return PLBM_E_STATE; }
    if (h->sticky == PLBM_E_CUDA) { set_err(h, "handle in CUDA error state"); return PLBM_E_CUDA; }
    if (bytes < sizeof(CkptHeader) + h->pop_bytes) {
        set_err(h, "checkpoint buffer of %zu bytes, %zu needed", bytes, sizeof(CkptHeader) + h->pop_bytes);
        return PLBM_E_ARG;
    }
    CK(cudaSetDevice(h->desc.device));
    unsigned char* out = static_cast<unsigned char*>(buf);
    CK(cudaMemcpyAsync(out + sizeof(CkptHeader), h->f[h->cur], h->pop_bytes, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    CkptHeader c = ckpt_header_of(h);
    uint64_t sum = fnv1a(kFnvOffset, &c, sizeof c);
    c.checksum = fnv1a(sum, out + sizeof(CkptHeader), h->pop_bytes);
    std::memcpy(out, &c, sizeof c);
    return PLBM_OK;
}

plbm_status plbm_checkpoint_load(plbm_handle hh, const void* buf, size_t bytes) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    plbm_status st = usable(h, false);
    if (st != PLBM_OK) return st;
    if (!buf || bytes < sizeof(CkptHeader)) { set_err(h, "checkpoint too short"); return PLBM_E_CHECKSUM; }
    CkptHeader c;
    std::memcpy(&c, buf, sizeof c);
    if (std::memcmp(c.magic, kCkptMagic, sizeof c.magic) != 0 || c.format != kCkptFormat ||
        c.header_bytes != sizeof(CkptHeader)) {
        set_err(h, "not a checkpoint of this format");
        return PLBM_E_CHECKSUM;
    }
    if (c.payload_bytes != h->pop_bytes || bytes < sizeof(CkptHeader) + c.payload_bytes) {
        set_err(h, "checkpoint payload of %llu bytes, handle holds %zu", (unsigned long long)c.payload_bytes,
                h->pop_bytes);
        return PLBM_E_CHECKSUM;
    }
    const unsigned char* in = static_cast<const unsigned char*>(buf);
    const uint64_t stored = c.checksum;
    c.checksum = 0;
    const uint64_t sum = fnv1a(fnv1a(kFnvOffset, &c, sizeof c), in + sizeof(CkptHeader), c.payload_bytes);
    if (sum != stored) {
        set_err(h, "checkpoint checksum mismatch (stored %016llx, computed %016llx)", (unsigned long long)stored,
                (unsigned long long)sum);
        return PLBM_E_CHECKSUM;
    }
    CkptHeader mine = ckpt_header_of(h);
    mine.step = c.step;
    mine.checksum = 0;
    if (std::memcmp(&mine, &c, sizeof c) != 0) {
        set_err(h, "checkpoint describes another lattice (velocities, omega, theta0, sizes, precision, layout or "
                   "boundary states differ)");
        return PLBM_E_CHECKSUM;
    }
    h->cur = 0;
    CK(cudaMemcpyAsync(h->f[0], in + sizeof(CkptHeader), h->pop_bytes, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->steps = c.step;
    h->initialised = true;
    return PLBM_OK;
}

plbm_status plbm_get_info(plbm_handle hh, int* q, int* pitch, size_t* population_bytes) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) { set_err(nullptr, "handle is NULL"); return PLBM_E_ARG; }
    if (q) *q = h->P.q;
    if (pitch) *pitch = h->P.pitch;
    if (population_bytes) *population_bytes = h->pop_bytes;
    return PLBM_OK;
}

plbm_status plbm_device_populations(plbm_handle hh, void** ptr) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !ptr) { set_err(h, "bad arguments"); return PLBM_E_ARG; }
    *ptr = h->f[h->cur];
    return PLBM_OK;
}

const char* plbm_last_error(plbm_handle hh) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    return h ? h->err : g_thread_error;
}

const char* plbm_status_string(plbm_status s) {
    switch (s) {
        case PLBM_OK: return "PLBM_OK";
        case PLBM_E_ARG: return "PLBM_E_ARG";
        case PLBM_E_CUDA: return "PLBM_E_CUDA";
        case PLBM_E_INADMISSIBLE: return "PLBM_E_INADMISSIBLE";
        case PLBM_E_DIVERGED: return "PLBM_E_DIVERGED";
        case PLBM_E_TIMEOUT: return "PLBM_E_TIMEOUT";
        case PLBM_E_STATE: return "PLBM_E_STATE";
        case PLBM_E_CHECKSUM: return "PLBM_E_CHECKSUM";
        case PLBM_E_NOMEM: return "PLBM_E_NOMEM";
    }
    return "PLBM_E_UNKNOWN";
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched runner.
// ---------------------------------------------------------------------------
namespace {

// The instances fall into groups that one persistent launch per step advances:
// row-paired lattices (2D periodic thermal (0, +-a, +-b), even row count,
// 16/32-bit storage) by k_batch_pair, one group per storage precision; every
// other 2D lattice (odd row counts, FP64, isothermal, other velocity sets with
// q1 <= 5) by k_batch_node, one group per (precision, q1).
struct PairGroup {
    int prec = 0;
    std::vector<int> members;                // indices into Batch::inst
    std::vector<plbm::PairParams> table;
    plbm::PairParams* d_table = nullptr;
    unsigned short* d_tile_inst = nullptr;   // instance (index into table) of every tile
    size_t max_tiles = 0;                    // tiles at the smallest block_x
    int total_tiles = 0;
};

struct NodeGroup {
    int prec = 0, q1 = 0;
    std::vector<int> members;
    plbm::LatticeParams* d_params = nullptr;
    plbm::NodeSpan* d_span = nullptr;
    unsigned short* d_tile_inst = nullptr;
    int total_tiles = 0;
    int ctas = 0;
};

struct Batch {
    std::vector<Handle*> inst;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool owns_stream = false;
    char* ws = nullptr;        // instance workspaces
    char* tables = nullptr;    // group tables
    std::vector<PairGroup> pairs;
    std::vector<NodeGroup> nodes;
    int order = PLBM_BATCH_ORDER_INTERLEAVED;
    int block_x = 128, ctas_per_sm = 0, sms = 0;
    cudaGraphExec_t graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [kind][start parity]
    long long steps = 0;
    char err[512] = "";
};

void batch_err(Batch* b, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    std::snprintf(g_thread_error, sizeof g_thread_error, "%s", buf);
    if (b) std::snprintf(b->err, sizeof b->err, "%s", buf);
}

#define BCK(call)                                                                  \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            batch_err(b, "%s failed: %s", #call, cudaGetErrorString(e_));          \
            return PLBM_E_CUDA;                                                    \
        }                                                                          \
    } while (0)

void drop_graphs(Batch* b) {
    for (auto& row : b->graph)
        for (auto& g : row)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
}

// Occupancy of the row-paired kernel at block_x: the smallest over the paired
// groups' precisions (1 when there are none).
int pair_occupancy(Batch* b, int block_x) {
    int occ = 1 << 20;
    for (const PairGroup& g : b->pairs) {
        int o = 0;
        if (plbm::batch_occupancy(g.prec, block_x, &o) != cudaSuccess || o < 1) o = 1;
        occ = std::min(occ, o);
    }
    return b->pairs.empty() ? 1 : occ;
}

int batch_ctas(Batch* b, int* occ_out = nullptr) {
    const int occ = pair_occupancy(b, b->block_x);
    if (occ_out) *occ_out = occ;
    const int per_sm = b->ctas_per_sm > 0 ? std::min(b->ctas_per_sm, occ) : occ;
    return b->sms * per_sm;
}

int batch_total_tiles(const Batch* b) {
    int t = 0;
    for (const PairGroup& g : b->pairs) t += g.total_tiles;
    for (const NodeGroup& g : b->nodes) t += g.total_tiles;
    return t;
}

// Tile lists of the row-paired groups for the current block_x.
plbm_status batch_table(Batch* b) {
    for (PairGroup& g : b->pairs) {
        int tile = 0;
        for (plbm::PairParams& Q : g.table) {
            Q.tiles_x = (Q.nx + b->block_x - 1) / b->block_x;
            Q.tile_begin = tile;
            tile += Q.tiles_x * plbm::tile_rows(Q);
        }
        g.total_tiles = tile;
        std::vector<unsigned short> ti((size_t)tile);
        for (size_t i = 0; i < g.table.size(); ++i) {
            const plbm::PairParams& Q = g.table[i];
            std::fill(ti.begin() + Q.tile_begin, ti.begin() + Q.tile_begin + Q.tiles_x * plbm::tile_rows(Q),
                      (unsigned short)i);
        }
        BCK(cudaMemcpyAsync(g.d_table, g.table.data(), sizeof(plbm::PairParams) * g.table.size(),
                            cudaMemcpyHostToDevice, b->stream));
        if (tile > 0)
            BCK(cudaMemcpyAsync(g.d_tile_inst, ti.data(), sizeof(unsigned short) * ti.size(),
                                cudaMemcpyHostToDevice, b->stream));
        BCK(cudaStreamSynchronize(b->stream));
    }
    drop_graphs(b);
    return PLBM_OK;
}

void free_batch(Batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graphs(b);
    for (Handle* h : b->inst) {
        if (!h) continue;
        h->in_batch = false;
        free_handle(h);
    }
    if (b->ws) cudaFree(b->ws);
    if (b->tables) cudaFree(b->tables);
    if (b->owns_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

// One step of every instance with the chosen launch scheme (no graph).
plbm_status batch_launch(Batch* b, int scheme, int parity, int ctas) {
    if (scheme == 0) {
        for (const PairGroup& g : b->pairs)
            BCK(plbm::launch_batch(g.prec, g.d_table, (int)g.table.size(), g.total_tiles, b->block_x, ctas, parity,
                                   b->order == PLBM_BATCH_ORDER_INTERLEAVED ? g.d_tile_inst : nullptr, b->stream));
        for (const NodeGroup& g : b->nodes)
            BCK(plbm::launch_batch_node(g.prec, g.q1, g.d_params, g.d_span, g.total_tiles, g.ctas, parity,
                                        g.d_tile_inst, b->stream));
    } else {
        for (Handle* h : b->inst)
            BCK(plbm::launch_step(h->prec, h->P, h->f[parity], h->f[parity ^ 1], false, b->stream));
    }
    return PLBM_OK;
}

// Groups the created instances and builds the groups' device tables.
plbm_status batch_groups(Batch* b) {
    for (size_t i = 0; i < b->inst.size(); ++i) {
        const Handle* h = b->inst[i];
        // the two-nodes-per-thread kernel's groups also take the plain-layout lattices of
        // the same arithmetic (symmetric five-velocity thermal sets, 16/32-bit storage)
        const bool sym5_group = h->P.paired || (h->P.dim == 2 && h->P.sym5 && !h->P.isothermal &&
                                                !h->P.fixed_ends && h->prec != plbm::kF64);
        if (sym5_group) {
            PairGroup* g = nullptr;
            for (PairGroup& c : b->pairs)
                if (c.prec == h->prec) g = &c;
            if (!g) {
                b->pairs.emplace_back();
                g = &b->pairs.back();
                g->prec = h->prec;
            }
            g->members.push_back((int)i);
            g->max_tiles += (size_t)((h->P.nx + 63) / 64) * (size_t)(h->P.paired ? h->P.half_ny : h->P.ny);
        } else {
            if (h->P.dim != 2 || h->P.q1 < 3 || h->P.q1 > 5) {
                batch_err(b, "instance %zu: the batched runner takes 2D lattices with 3 to 5 velocities per axis", i);
                return PLBM_E_ARG;
            }
            NodeGroup* g = nullptr;
            for (NodeGroup& c : b->nodes)
                if (c.prec == h->prec && c.q1 == h->P.q1) g = &c;
            if (!g) {
                b->nodes.emplace_back();
                g = &b->nodes.back();
                g->prec = h->prec;
                g->q1 = h->P.q1;
            }
            g->members.push_back((int)i);
        }
    }
    for (const PairGroup& g : b->pairs)
        if (g.members.size() > 65535) { batch_err(b, "at most 65535 row-paired instances per precision"); return PLBM_E_ARG; }
    for (const NodeGroup& g : b->nodes)
        if (g.members.size() > 65535) { batch_err(b, "at most 65535 instances per group"); return PLBM_E_ARG; }
    // one allocation for every group's tables
    size_t total = 0;
    std::vector<size_t> off;
    for (const PairGroup& g : b->pairs) {
        off.push_back(total);
        total += align_up(sizeof(plbm::PairParams) * g.members.size(), 256);
        off.push_back(total);
        total += align_up(sizeof(unsigned short) * std::max<size_t>(g.max_tiles, 1), 256);
    }
    std::vector<std::vector<unsigned short>> node_tiles(b->nodes.size());
    std::vector<std::vector<plbm::NodeSpan>> spans(b->nodes.size());
    for (size_t k = 0; k < b->nodes.size(); ++k) {
        NodeGroup& g = b->nodes[k];
        int tile = 0;
        for (size_t m = 0; m < g.members.size(); ++m) {
            const Handle* h = b->inst[g.members[m]];
            plbm::NodeSpan sp{};
            sp.f[0] = h->f[0];
            sp.f[1] = h->f[1];
            sp.nx = h->P.nx;
            sp.tiles_x = (h->P.nx + plbm::kBlockX - 1) / plbm::kBlockX;
            sp.tile_begin = tile;
            tile += sp.tiles_x * h->P.ny;
            spans[k].push_back(sp);
            node_tiles[k].insert(node_tiles[k].end(), (size_t)sp.tiles_x * h->P.ny, (unsigned short)m);
        }
        g.total_tiles = tile;
        int occ = 0;
        if (plbm::batch_node_occupancy(g.prec, g.q1, &occ) != cudaSuccess || occ < 1) occ = 1;
        g.ctas = std::max(1, std::min(tile, b->sms * occ));
        off.push_back(total);
        total += align_up(sizeof(plbm::LatticeParams) * g.members.size(), 256);
        off.push_back(total);
        total += align_up(sizeof(plbm::NodeSpan) * g.members.size(), 256);
        off.push_back(total);
        total += align_up(sizeof(unsigned short) * std::max<size_t>(node_tiles[k].size(), 1), 256);
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(total, 256));
    if (e != cudaSuccess) {
        batch_err(b, "cudaMalloc(%zu) failed: %s", total, cudaGetErrorString(e));
        return PLBM_E_NOMEM;
    }
    b->tables = static_cast<char*>(p);
    size_t o = 0;
    for (PairGroup& g : b->pairs) {
        g.d_table = reinterpret_cast<plbm::PairParams*>(b->tables + off[o++]);
        g.d_tile_inst = reinterpret_cast<unsigned short*>(b->tables + off[o++]);
        for (int i : g.members) {
            const Handle* h = b->inst[i];
            plbm::PairParams Q = plbm::pair_params(h->P);
            Q.f[0] = h->f[0];
            Q.f[1] = h->f[1];
            g.table.push_back(Q);
        }
    }
    for (size_t k = 0; k < b->nodes.size(); ++k) {
        NodeGroup& g = b->nodes[k];
        g.d_params = reinterpret_cast<plbm::LatticeParams*>(b->tables + off[o++]);
        g.d_span = reinterpret_cast<plbm::NodeSpan*>(b->tables + off[o++]);
        g.d_tile_inst = reinterpret_cast<unsigned short*>(b->tables + off[o++]);
        std::vector<plbm::LatticeParams> params;
        for (int i : g.members) params.push_back(b->inst[i]->P);
        BCK(cudaMemcpyAsync(g.d_params, params.data(), sizeof(plbm::LatticeParams) * params.size(),
                            cudaMemcpyHostToDevice, b->stream));
        BCK(cudaMemcpyAsync(g.d_span, spans[k].data(), sizeof(plbm::NodeSpan) * spans[k].size(),
                            cudaMemcpyHostToDevice, b->stream));
        if (!node_tiles[k].empty())
            BCK(cudaMemcpyAsync(g.d_tile_inst, node_tiles[k].data(), sizeof(unsigned short) * node_tiles[k].size(),
                                cudaMemcpyHostToDevice, b->stream));
    }
    BCK(cudaStreamSynchronize(b->stream));
    return batch_table(b);
}

}  // namespace

extern "C" {

plbm_status plbm_batch_create(const plbm_desc* descs, int n, void* stream, plbm_batch* out) {
    if (!out || !descs || n < 1) {
        batch_err(nullptr, "bad arguments");
        return PLBM_E_ARG;
    }
    *out = nullptr;
    Batch* b = new (std::nothrow) Batch();
    if (!b) return PLBM_E_NOMEM;
    b->device = descs[0].device;
    std::vector<size_t> off(n);
    size_t total = 0;
    for (int i = 0; i < n; ++i) {
        const plbm_desc& d = descs[i];
        if (d.device != b->device) {
            batch_err(b, "instance %d: all instances need the same device", i);
            delete b;
            return PLBM_E_ARG;
        }
        if (d.dim != 2) {
            batch_err(b, "instance %d: the batched runner takes 2D lattices", i);
            delete b;
            return PLBM_E_ARG;
        }
        const size_t need = plbm_workspace_bytes(&d);
        if (need == 0) {
            batch_err(b, "instance %d: %s", i, g_thread_error);
            delete b;
            return PLBM_E_ARG;
        }
        off[i] = total;
        total += align_up(need, 256);
    }
    if (cudaSetDevice(b->device) != cudaSuccess) {
        batch_err(b, "cudaSetDevice(%d) failed", b->device);
        delete b;
        return PLBM_E_CUDA;
    }
    if (stream) {
        b->stream = static_cast<cudaStream_t>(stream);
    } else {
        // graph capture needs a stream other than the legacy default stream
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            batch_err(b, "cudaStreamCreate failed");
            delete b;
            return PLBM_E_CUDA;
        }
        b->owns_stream = true;
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, total);
    if (e != cudaSuccess) {
        batch_err(b, "cudaMalloc(%zu) failed: %s", total, cudaGetErrorString(e));
        free_batch(b);
        return PLBM_E_NOMEM;
    }
    b->ws = static_cast<char*>(p);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
    b->inst.assign(n, nullptr);
    for (int i = 0; i < n; ++i) {
        plbm_desc d = descs[i];
        d.workspace = b->ws + off[i];
        d.workspace_bytes = align_up(plbm_workspace_bytes(&descs[i]), 256);
        d.stream = b->stream;
        plbm_handle hh = nullptr;
        plbm_status st = plbm_create(&d, &hh);
        if (st != PLBM_OK) {
            batch_err(b, "instance %d: %s", i, g_thread_error);
            free_batch(b);
            return st;
        }
        Handle* h = reinterpret_cast<Handle*>(hh);
        h->in_batch = true;
        b->inst[i] = h;
    }
    plbm_status st = batch_groups(b);
    if (st != PLBM_OK) {
        free_batch(b);
        return st;
    }
    *out = reinterpret_cast<plbm_batch>(b);
    return PLBM_OK;
}

plbm_status plbm_batch_destroy(plbm_batch bb) {
    free_batch(reinterpret_cast<Batch*>(bb));
    return PLBM_OK;
}

plbm_status plbm_batch_instance(plbm_batch bb, int i, plbm_handle* out) {
    Batch* b = reinterpret_cast<Batch*>(bb);
    if (!b || !out || i < 0 || i >= (int)b->inst.size()) {
        batch_err(b, "bad arguments");
        return PLBM_E_ARG;
    }
    *out = reinterpret_cast<plbm_handle>(b->inst[i]);
    return PLBM_OK;
}

plbm_status plbm_batch_step(plbm_batch bb, long n, int mode) {
    Batch* b = reinterpret_cast<Batch*>(bb);
    if (!b || n < 0 || mode < 0 || mode > 3) {
        batch_err(b, "bad arguments");
        return PLBM_E_ARG;
    }
    const int parity0 = b->inst[0]->cur;
    for (size_t i = 0; i < b->inst.size(); ++i) {
        Handle* h = b->inst[i];
        if (h->sticky != PLBM_OK || !h->initialised) {
            batch_err(b, "instance %zu is not initialised or in an error state", i);
            return PLBM_E_STATE;
        }
        if (h->cur != parity0) {
            batch_err(b, "instance %zu was stepped on its own; all instances must be in step", i);
            return PLBM_E_STATE;
        }
    }
    BCK(cudaSetDevice(b->device));
    const int scheme = (mode == PLBM_BATCH_PERSISTENT || mode == PLBM_BATCH_PERSISTENT_GRAPH) ? 0 : 1;
    const bool use_graph = (mode == PLBM_BATCH_PERSISTENT_GRAPH || mode == PLBM_BATCH_PER_INSTANCE_GRAPH);
    int parity = parity0;
    long done = 0;
    const int ctas = batch_ctas(b);  // occupancy query outside any stream capture
    if (use_graph) {
        for (; done + 2 <= n; done += 2) {
            cudaGraphExec_t& g = b->graph[scheme][parity];
            if (!g) {
                cudaGraph_t graph = nullptr;
                BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
                plbm_status st = batch_launch(b, scheme, parity, ctas);
                if (st == PLBM_OK) st = batch_launch(b, scheme, parity ^ 1, ctas);
                cudaError_t ec = cudaStreamEndCapture(b->stream, &graph);
                cudaError_t ei = (st == PLBM_OK && ec == cudaSuccess) ? cudaGraphInstantiate(&g, graph, 0)
                                                                       : cudaSuccess;
                if (graph) cudaGraphDestroy(graph);
                if (st != PLBM_OK) return st;
                BCK(ec);
                BCK(ei);
            }
            BCK(cudaGraphLaunch(g, b->stream));
        }
    }
    for (; done < n; ++done) {
        plbm_status st = batch_launch(b, scheme, parity, ctas);
        if (st != PLBM_OK) return st;
        parity ^= 1;
    }
    if (n % 2) parity = parity0 ^ 1; else parity = parity0;
    for (Handle* h : b->inst) {
        h->cur = parity;
        h->steps += n;
    }
    b->steps += n;
    return PLBM_OK;
}

plbm_status plbm_batch_check(plbm_batch bb, int* first_bad) {
    Batch* b = reinterpret_cast<Batch*>(bb);
    if (!b) return PLBM_E_ARG;
    if (first_bad) *first_bad = -1;
    std::vector<unsigned> bits(b->inst.size(), 0u);
    for (size_t i = 0; i < b->inst.size(); ++i)
        BCK(cudaMemcpyAsync(&bits[i], b->inst[i]->status, sizeof(unsigned), cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    for (size_t i = 0; i < bits.size(); ++i)
        if (bits[i]) {
            if (first_bad) *first_bad = (int)i;
            batch_err(b, "instance %zu diverged (status 0x%x)", i, bits[i]);
            return PLBM_E_DIVERGED;
        }
    return PLBM_OK;
}

plbm_status plbm_batch_set_config(plbm_batch bb, int block_x, int ctas_per_sm) {
    Batch* b = reinterpret_cast<Batch*>(bb);
    if (!b || (block_x != 64 && block_x != 128 && block_x != 256) || ctas_per_sm < 0 || ctas_per_sm > 64) {
        batch_err(b, "block_x must be 64, 128 or 256 and 0 <= ctas_per_sm <= 64");
        return PLBM_E_ARG;
    }
    b->block_x = block_x;
    b->ctas_per_sm = ctas_per_sm;
    return batch_table(b);
}

plbm_status plbm_batch_set_order(plbm_batch bb, int order) {
    Batch* b = reinterpret_cast<Batch*>(bb);
    if (!b || (order != PLBM_BATCH_ORDER_CONTIGUOUS && order != PLBM_BATCH_ORDER_INTERLEAVED)) {
        batch_err(b, "order must be PLBM_BATCH_ORDER_CONTIGUOUS or PLBM_BATCH_ORDER_INTERLEAVED");
        return PLBM_E_ARG;
    }
    b->order = order;
    drop_graphs(b);
    return PLBM_OK;
}

int plbm_batch_get_order(plbm_batch bb) {
    Batch* b = reinterpret_cast<Batch*>(bb);
    return b ? b->order : -1;
}

plbm_status plbm_batch_info(plbm_batch bb, int* ninst, int* total_tiles, int* block_x, int* ctas,
                            int* max_ctas_per_sm) {
    Batch* b = reinterpret_cast<Batch*>(bb);
    if (!b) return PLBM_E_ARG;
    int occ = 0;
    const int c = batch_ctas(b, &occ);
    if (ninst) *ninst = (int)b->inst.size();
    if (total_tiles) *total_tiles = batch_total_tiles(b);
    if (block_x) *block_x = b->block_x;
    if (ctas) *ctas = c;
    if (max_ctas_per_sm) *max_ctas_per_sm = occ;
    return PLBM_OK;
}

plbm_status plbm_batch_groups(plbm_batch bb, int* paired_instances, int* plain_instances, int* launches_per_step) {
    Batch* b = reinterpret_cast<Batch*>(bb);
    if (!b) return PLBM_E_ARG;
    int np = 0, nn = 0;
    for (const PairGroup& g : b->pairs) np += (int)g.members.size();
    for (const NodeGroup& g : b->nodes) nn += (int)g.members.size();
    if (paired_instances) *paired_instances = np;
    if (plain_instances) *plain_instances = nn;
    if (launches_per_step) *launches_per_step = (int)(b->pairs.size() + b->nodes.size());
    return PLBM_OK;
}

plbm_status plbm_batch_tune(plbm_batch bb, int steps_per_trial, int* best_block_x, int* best_ctas_per_sm,
                            double* best_ms_per_step) {
    Batch* b = reinterpret_cast<Batch*>(bb);
    if (!b || steps_per_trial < 1) return PLBM_E_ARG;
    for (Handle* h : b->inst)
        if (!h->initialised) {
            batch_err(b, "initialise every instance before tuning");
            return PLBM_E_STATE;
        }
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0));
    BCK(cudaEventCreate(&e1));
    double best = 1e300;
    int bx_best = 128, cps_best = 0, order_best = PLBM_BATCH_ORDER_INTERLEAVED;
    const int bxs[3] = {64, 128, 256};
    // Without row-paired instances the shape has nothing to choose: one trial.
    const bool any_pairs = !b->pairs.empty();
    for (int order : {PLBM_BATCH_ORDER_CONTIGUOUS, PLBM_BATCH_ORDER_INTERLEAVED}) {
        if (!any_pairs && order != PLBM_BATCH_ORDER_INTERLEAVED) continue;
        for (int bx : bxs) {
            if (!any_pairs && bx != 128) continue;
            const int occ = any_pairs ? pair_occupancy(b, bx) : 1;
            for (int cps = any_pairs ? 1 : 0; cps <= occ; ++cps) {
                if (any_pairs && cps == 0) continue;
                plbm_status st = plbm_batch_set_config(bb, bx, cps);
                if (st == PLBM_OK) st = plbm_batch_set_order(bb, order);
                if (st != PLBM_OK) return st;
                st = plbm_batch_step(bb, 2, PLBM_BATCH_PERSISTENT);
                if (st != PLBM_OK) return st;
                BCK(cudaEventRecord(e0, b->stream));
                st = plbm_batch_step(bb, steps_per_trial, PLBM_BATCH_PERSISTENT);
                if (st != PLBM_OK) return st;
                BCK(cudaEventRecord(e1, b->stream));
                BCK(cudaEventSynchronize(e1));
                float ms = 0.f;
                BCK(cudaEventElapsedTime(&ms, e0, e1));
                const double per = ms / steps_per_trial;
                if (per < best) {
                    best = per;
                    bx_best = bx;
                    cps_best = cps;
                    order_best = order;
                }
                if (!any_pairs) break;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    plbm_status st = plbm_batch_set_config(bb, bx_best, cps_best);
    if (st == PLBM_OK) st = plbm_batch_set_order(bb, order_best);
    if (st != PLBM_OK) return st;
    if (best_block_x) *best_block_x = bx_best;
    if (best_ctas_per_sm) *best_ctas_per_sm = cps_best;
    if (best_ms_per_step) *best_ms_per_step = best;
    return PLBM_OK;
}

const char* plbm_batch_last_error(plbm_batch bb) {
    Batch* b = reinterpret_cast<Batch*>(bb);
    return b ? b->err : g_thread_error;
}

}  // extern "C"
