// Domain decomposition of a periodic 2D lattice into slabs of consecutive rows.
//
// Eq. (eq:srt) read as pull + collide takes a node's populations from at most
// w = max|v| rows away (lattice units, on-lattice velocities, Sec. 2.4), and the
// collision is local.  A slab of rows [y0, y0 + n) therefore advances one step on
// its own once the w rows below and above it hold the current state of its
// neighbours; the rows below are read only by populations moving up (v_y > 0),
// the rows above only by those moving down (v_y < 0).
//
// Each slab here is an ordinary periodic handle of n + 2w rows: rows 0..w-1 are
// the lower halo, w..w+n-1 the slab's own rows, w+n..n+2w-1 the upper halo.  A
// step is the halo exchange (k_halo_copy: the halo populations of every slab
// from the neighbours' own rows, one launch for all slabs) and one ordinary step
// of every slab.  The halo rows' own updates pull across the slab's periodic
// wrap and are discarded: the next exchange overwrites what the slab's rows will
// read, and nothing else of the halo rows is ever read.  Every own row is
// computed from exactly the values the undivided lattice would use, by the same
// per-node code, so the decomposed run equals the undivided one bit for bit.
//
// The slabs of one plbm_slabs live on one device and the exchange is a device
// copy.  plbm_slab_rows and plbm_halo_plan are the host side of the exchange
// (which rows a slab owns; which populations each halo needs) for callers that
// move the halo rows themselves, e.g. between processes.
#include "plbm.h"

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "plbm_internal.h"

namespace {

thread_local char g_slab_error[512] = "";

// Layout facts of one population array (plain or row-paired, see elem_index).
struct ArrayLayout {
    long long plane;
    int pitch, paired, half_ny;
};

// One halo of one slab: w rows from src (rows src_row0..) into dst (rows dst_row0..).
struct HaloCopy {
    const void* src;
    void* dst;
    ArrayLayout ls, ld;
    int src_row0, dst_row0;
    int side;   // 0: lower halo (populations moving up), 1: upper halo (moving down)
};

struct PopList {
    int lo[PLBM_MAX_Q1 * PLBM_MAX_Q1], hi[PLBM_MAX_Q1 * PLBM_MAX_Q1];
    int nlo, nhi;
};

__device__ __forceinline__ long long at(const ArrayLayout& L, int p, int x, int y) {
    if (L.paired) {
        const int hi = y >= L.half_ny;
        const int r = hi ? y - L.half_ny : y;
        return (long long)p * L.plane + (long long)r * 2 * L.pitch + 2LL * x + hi;
    }
    return (long long)p * L.plane + (long long)y * L.pitch + x;
}

// grid.x over nx, grid.y over (copy, halo population, row); one element per thread.
template <typename S>
__global__ void k_halo_copy(const HaloCopy* __restrict__ copies, PopList pops, int w, int nx, int per_copy) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nx) return;
    const int c = blockIdx.y / per_copy;
    const int k = blockIdx.y - c * per_copy;
    const HaloCopy hc = copies[c];
    const int n = hc.side == 0 ? pops.nlo : pops.nhi;
    const int pi = k / w, j = k - pi * w;
    if (pi >= n) return;
    const int p = hc.side == 0 ? pops.lo[pi] : pops.hi[pi];
    static_cast<S*>(hc.dst)[at(hc.ld, p, x, hc.dst_row0 + j)] =
        static_cast<const S*>(hc.src)[at(hc.ls, p, x, hc.src_row0 + j)];
}

struct Slabs {
    int n = 0, w = 0, nx = 0, ny = 0, q1 = 0, q = 0, prec = 0;
    int v[PLBM_MAX_Q1] = {};
    std::vector<int> y0, rows;
    std::vector<plbm_handle> h;
    PopList pops{};
    HaloCopy* d_copies = nullptr;   // [parity][2 n]
    cudaStream_t stream = nullptr;
    bool owns_stream = false;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    long long steps = 0;
    bool initialised = false;
    char err[512] = "";
};

void slab_err(Slabs* s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    std::snprintf(g_slab_error, sizeof g_slab_error, "%s", buf);
    plbm::set_thread_error(buf);
    if (s) std::snprintf(s->err, sizeof s->err, "%s", buf);
}

#define SLCK(call)                                                                 \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            slab_err(s, "%s failed: %s", #call, cudaGetErrorString(e_));           \
            return PLBM_E_CUDA;                                                    \
        }                                                                          \
    } while (0)

ArrayLayout layout_of(const plbm::LatticeParams& P) {
    return ArrayLayout{P.plane, P.pitch, P.paired, P.half_ny};
}

cudaError_t launch_halo(const Slabs* s, int parity) {
    const int per_copy = std::max(s->pops.nlo, s->pops.nhi) * s->w;
    const dim3 grid((s->nx + 127) / 128, 2 * s->n * per_copy);
    const HaloCopy* c = s->d_copies + (size_t)parity * 2 * s->n;
    switch (s->prec) {
        case plbm::kF64: k_halo_copy<double><<<grid, 128, 0, s->stream>>>(c, s->pops, s->w, s->nx, per_copy); break;
        case plbm::kF32: k_halo_copy<float><<<grid, 128, 0, s->stream>>>(c, s->pops, s->w, s->nx, per_copy); break;
        case plbm::kF16Dev: k_halo_copy<__half><<<grid, 128, 0, s->stream>>>(c, s->pops, s->w, s->nx, per_copy); break;
        case plbm::kBF16Dev:
            k_halo_copy<__nv_bfloat16><<<grid, 128, 0, s->stream>>>(c, s->pops, s->w, s->nx, per_copy);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// One decomposed step from array `parity` of every slab: exchange, then step.
plbm_status slab_cycle(Slabs* s, int parity) {
    SLCK(launch_halo(s, parity));
    for (plbm_handle hh : s->h) {
        plbm::HandleView hv{};
        if (!plbm::handle_view(hh, &hv)) {
            slab_err(s, "a slab handle is not usable: %s", plbm_last_error(hh));
            return PLBM_E_STATE;
        }
        void* f[2] = {parity == *hv.cur ? hv.f_cur : hv.f_next, parity == *hv.cur ? hv.f_next : hv.f_cur};
        SLCK(plbm::launch_step(hv.prec, *hv.P, f[0], f[1], false, s->stream));
    }
    return PLBM_OK;
}

void drop_graphs(Slabs* s) {
    for (cudaGraphExec_t& g : s->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

void free_slabs(Slabs* s) {
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    drop_graphs(s);
    for (plbm_handle hh : s->h)
        if (hh) plbm_destroy(hh);
    if (s->d_copies) cudaFree(s->d_copies);
    if (s->stream && s->owns_stream) cudaStreamDestroy(s->stream);
    delete s;
}

}  // namespace

extern "C" {

plbm_status plbm_slab_rows(int ny, int nslabs, int k, int* y0, int* rows) {
    if (ny < 1 || nslabs < 1 || nslabs > ny || k < 0 || k >= nslabs || !y0 || !rows) {
        slab_err(nullptr, "plbm_slab_rows: need 1 <= nslabs <= ny and 0 <= k < nslabs");
        return PLBM_E_ARG;
    }
    const int base = ny / nslabs, extra = ny % nslabs;
    *rows = base + (k < extra ? 1 : 0);
    *y0 = k * base + std::min(k, extra);
    return PLBM_OK;
}

int plbm_halo_width(int q1, const int* v) {
    if (q1 < 1 || q1 > PLBM_MAX_Q1 || !v) return -1;
    int w = 0;
    for (int i = 0; i < q1; ++i) w = std::max(w, v[i] < 0 ? -v[i] : v[i]);
    return w;
}

plbm_status plbm_halo_plan(int q1, const int* v, int side, int* pops, int* count) {
    if (q1 < 1 || q1 > PLBM_MAX_Q1 || !v || (side != -1 && side != 1) || !count) {
        slab_err(nullptr, "plbm_halo_plan: bad arguments");
        return PLBM_E_ARG;
    }
    int n = 0;
    for (int ix = 0; ix < q1; ++ix)
        for (int iy = 0; iy < q1; ++iy) {
            // the rows below are pulled by populations moving up, the rows above by those moving down
            const bool need = side < 0 ? v[iy] > 0 : v[iy] < 0;
            if (!need) continue;
            if (pops) pops[n] = ix * q1 + iy;
            ++n;
        }
    *count = n;
    return PLBM_OK;
}

plbm_status plbm_slabs_create(const plbm_desc* desc, int nslabs, plbm_slabs* out) {
    if (!out || !desc) {
        slab_err(nullptr, "plbm_slabs_create: bad arguments");
        return PLBM_E_ARG;
    }
    *out = nullptr;
    if (desc->dim != 2 || desc->bc != PLBM_PERIODIC || !desc->v || desc->q1 < 1 || desc->q1 > PLBM_MAX_Q1) {
        slab_err(nullptr, "plbm_slabs_create: the decomposition takes periodic 2D lattices");
        return PLBM_E_ARG;
    }
    const int w = plbm_halo_width(desc->q1, desc->v);
    if (nslabs < 1 || w < 1 || (long long)nslabs * w > desc->ny) {
        slab_err(nullptr, "plbm_slabs_create: need 1 <= nslabs and at least max|v| = %d rows per slab", w);
        return PLBM_E_ARG;
    }
    Slabs* s = new (std::nothrow) Slabs();
    if (!s) return PLBM_E_NOMEM;
    s->n = nslabs;
    s->w = w;
    s->nx = desc->nx;
    s->ny = desc->ny;
    s->q1 = desc->q1;
    s->q = desc->q1 * desc->q1;
    s->prec = (int)desc->prec;
    std::memcpy(s->v, desc->v, sizeof(int) * desc->q1);
    if (cudaSetDevice(desc->device) != cudaSuccess) {
        slab_err(s, "plbm_slabs_create: no usable CUDA device %d", desc->device);
        free_slabs(s);
        return PLBM_E_CUDA;
    }
    if (desc->stream) {
        s->stream = static_cast<cudaStream_t>(desc->stream);
    } else {
        // the step graphs are captured on this stream: not the legacy default one
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
            slab_err(s, "plbm_slabs_create: cudaStreamCreate failed");
            free_slabs(s);
            return PLBM_E_CUDA;
        }
        s->owns_stream = true;
    }
    plbm_halo_plan(s->q1, s->v, -1, s->pops.lo, &s->pops.nlo);
    plbm_halo_plan(s->q1, s->v, 1, s->pops.hi, &s->pops.nhi);
    // Both layouts give a node the same bits (the plain-layout kernel runs the
    // single-lane forms of the row-paired arithmetic); slabs of a row-paired lattice
    // take even row counts all the same, so that they keep the faster two-nodes-per-
    // thread kernel (rows + 2w stays even).
    const bool paired = plbm::desc_row_paired(desc);
    s->y0.resize(nslabs);
    s->rows.resize(nslabs);
    s->h.assign(nslabs, nullptr);
    for (int k = 0; k < nslabs; ++k) {
        if (paired) {
            int p0 = 0, np = 0;
            if (plbm_slab_rows(s->ny / 2, nslabs, k, &p0, &np) != PLBM_OK) {
                slab_err(s, "plbm_slabs_create: more slabs than row pairs");
                free_slabs(s);
                return PLBM_E_ARG;
            }
            s->y0[k] = 2 * p0;
            s->rows[k] = 2 * np;
        } else {
            plbm_slab_rows(s->ny, nslabs, k, &s->y0[k], &s->rows[k]);
        }
        if (s->rows[k] < w) {
            slab_err(s, "plbm_slabs_create: slab %d has %d rows, fewer than max|v| = %d", k, s->rows[k], w);
            free_slabs(s);
            return PLBM_E_ARG;
        }
        plbm_desc d = *desc;
        if (!paired) d.flags |= PLBM_FLAG_PLAIN_LAYOUT;
        d.ny = s->rows[k] + 2 * w;
        d.stream = s->stream;
        d.workspace = nullptr;
        d.workspace_bytes = 0;
        d.check_every = 0;
        const plbm_status st = plbm_create(&d, &s->h[k]);
        if (st != PLBM_OK) {
            slab_err(s, "slab %d: %s", k, plbm_last_error(nullptr));
            free_slabs(s);
            return st;
        }
    }
    if (cudaMalloc(&s->d_copies, sizeof(HaloCopy) * 4 * nslabs) != cudaSuccess) {
        slab_err(s, "plbm_slabs_create: cudaMalloc of the copy table failed");
        free_slabs(s);
        return PLBM_E_NOMEM;
    }
    *out = reinterpret_cast<plbm_slabs>(s);
    return PLBM_OK;
}

plbm_status plbm_slabs_destroy(plbm_slabs ss) {
    free_slabs(reinterpret_cast<Slabs*>(ss));
    return PLBM_OK;
}

plbm_status plbm_slabs_slab(plbm_slabs ss, int k, plbm_handle* h, int* y0, int* rows) {
    Slabs* s = reinterpret_cast<Slabs*>(ss);
    if (!s || k < 0 || k >= s->n) {
        slab_err(s, "plbm_slabs_slab: bad arguments");
        return PLBM_E_ARG;
    }
    if (h) *h = s->h[k];
    if (y0) *y0 = s->y0[k];
    if (rows) *rows = s->rows[k];
    return PLBM_OK;
}

plbm_status plbm_slabs_init(plbm_slabs ss, const double* rho, const double* ux, const double* uy,
                            const double* theta) {
    Slabs* s = reinterpret_cast<Slabs*>(ss);
    if (!s || !rho || !ux || !uy || !theta) {
        slab_err(s, "plbm_slabs_init: bad arguments");
        return PLBM_E_ARG;
    }
    const int nx = s->nx, w = s->w;
    std::vector<double> buf;
    for (int k = 0; k < s->n; ++k) {
        const int n = s->rows[k] + 2 * w;
        buf.assign((size_t)4 * n * nx, 0.0);
        const double* src[4] = {rho, ux, uy, theta};
        for (int f = 0; f < 4; ++f)
            for (int j = 0; j < n; ++j) {
                const int y = ((s->y0[k] - w + j) % s->ny + s->ny) % s->ny;
                std::memcpy(&buf[((size_t)f * n + j) * nx], src[f] + (size_t)y * nx, sizeof(double) * nx);
            }
        const size_t plane = (size_t)n * nx;
        const plbm_status st =
            plbm_init(s->h[k], &buf[0], &buf[plane], &buf[2 * plane], &buf[3 * plane], 0);
        if (st != PLBM_OK) {
            slab_err(s, "slab %d: %s", k, plbm_last_error(s->h[k]));
            return st;
        }
    }
    // copy tables for both array parities: lower halo of k from slab k - 1's last
    // w own rows, upper halo from slab k + 1's first w own rows
    std::vector<HaloCopy> tab((size_t)4 * s->n);
    for (int parity = 0; parity < 2; ++parity)
        for (int k = 0; k < s->n; ++k) {
            plbm::HandleView me{}, lo{}, hi{};
            const int kl = (k + s->n - 1) % s->n, kh = (k + 1) % s->n;
            if (!plbm::handle_view(s->h[k], &me) || !plbm::handle_view(s->h[kl], &lo) ||
                !plbm::handle_view(s->h[kh], &hi)) {
                slab_err(s, "plbm_slabs_init: slab handle not usable");
                return PLBM_E_STATE;
            }
            auto arr = [&](const plbm::HandleView& hv) { return parity == *hv.cur ? hv.f_cur : hv.f_next; };
            HaloCopy& a = tab[(size_t)parity * 2 * s->n + 2 * k];
            a.src = arr(lo);
            a.dst = arr(me);
            a.ls = layout_of(*lo.P);
            a.ld = layout_of(*me.P);
            a.src_row0 = s->rows[kl];       // padded rows w + rows - w .. : the last w own rows
            a.dst_row0 = 0;
            a.side = 0;
            HaloCopy& b = tab[(size_t)parity * 2 * s->n + 2 * k + 1];
            b.src = arr(hi);
            b.dst = arr(me);
            b.ls = layout_of(*hi.P);
            b.ld = layout_of(*me.P);
            b.src_row0 = w;                 // the first w own rows
            b.dst_row0 = w + s->rows[k];
            b.side = 1;
        }
    SLCK(cudaMemcpyAsync(s->d_copies, tab.data(), sizeof(HaloCopy) * tab.size(), cudaMemcpyHostToDevice,
                         s->stream));
    SLCK(cudaStreamSynchronize(s->stream));
    drop_graphs(s);
    s->steps = 0;
    s->initialised = true;
    return PLBM_OK;
}

plbm_status plbm_slabs_step(plbm_slabs ss, long n) {
    Slabs* s = reinterpret_cast<Slabs*>(ss);
    if (!s || n < 0) {
        slab_err(s, "plbm_slabs_step: bad arguments");
        return PLBM_E_ARG;
    }
    if (!s->initialised) {
        slab_err(s, "plbm_slabs_step: not initialised");
        return PLBM_E_STATE;
    }
    plbm::HandleView hv{};
    if (!plbm::handle_view(s->h[0], &hv)) {
        slab_err(s, "plbm_slabs_step: slab 0 not usable: %s", plbm_last_error(s->h[0]));
        return PLBM_E_STATE;
    }
    int parity = *hv.cur;
    long done = 0;
    // pairs of decomposed steps replay a CUDA graph captured once per starting parity
    for (; done + 2 <= n; done += 2) {
        cudaGraphExec_t& g = s->graph[parity];
        if (!g) {
            cudaGraph_t graph = nullptr;
            SLCK(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
            plbm_status st = slab_cycle(s, parity);
            if (st == PLBM_OK) st = slab_cycle(s, parity ^ 1);
            const cudaError_t ec = cudaStreamEndCapture(s->stream, &graph);
            const cudaError_t ei =
                (st == PLBM_OK && ec == cudaSuccess) ? cudaGraphInstantiate(&g, graph, 0) : cudaSuccess;
            if (graph) cudaGraphDestroy(graph);
            if (st != PLBM_OK) return st;
            SLCK(ec);
            SLCK(ei);
        }
        SLCK(cudaGraphLaunch(g, s->stream));
    }
    for (; done < n; ++done) {
        const plbm_status st = slab_cycle(s, parity);
        if (st != PLBM_OK) return st;
        parity ^= 1;
    }
    for (plbm_handle hh : s->h) {
        plbm::HandleView v{};
        plbm::handle_view(hh, &v);
        *v.cur = (int)((*v.cur + n) & 1);
        *v.steps += n;
    }
    s->steps += n;
    return PLBM_OK;
}

plbm_status plbm_slabs_moments(plbm_slabs ss, double* rho, double* ux, double* uy, double* theta) {
    Slabs* s = reinterpret_cast<Slabs*>(ss);
    if (!s || !rho || !ux || !uy || !theta) {
        slab_err(s, "plbm_slabs_moments: bad arguments");
        return PLBM_E_ARG;
    }
    const int nx = s->nx, w = s->w;
    std::vector<double> buf;
    for (int k = 0; k < s->n; ++k) {
        const int n = s->rows[k] + 2 * w;
        const size_t plane = (size_t)n * nx;
        buf.assign(4 * plane, 0.0);
        const plbm_status st = plbm_moments(s->h[k], &buf[0], &buf[plane], &buf[2 * plane], &buf[3 * plane], 0);
        if (st != PLBM_OK) {
            slab_err(s, "slab %d: %s", k, plbm_last_error(s->h[k]));
            return st;
        }
        double* dst[4] = {rho, ux, uy, theta};
        for (int f = 0; f < 4; ++f)
            std::memcpy(dst[f] + (size_t)s->y0[k] * nx, &buf[f * plane + (size_t)w * nx],
                        sizeof(double) * (size_t)s->rows[k] * nx);
    }
    return PLBM_OK;
}

plbm_status plbm_slabs_get_populations(plbm_slabs ss, double* f) {
    Slabs* s = reinterpret_cast<Slabs*>(ss);
    if (!s || !f) {
        slab_err(s, "plbm_slabs_get_populations: bad arguments");
        return PLBM_E_ARG;
    }
    const int nx = s->nx, w = s->w;
    std::vector<double> buf;
    for (int k = 0; k < s->n; ++k) {
        const int n = s->rows[k] + 2 * w;
        buf.assign((size_t)s->q * n * nx, 0.0);
        const plbm_status st = plbm_get_populations(s->h[k], buf.data(), 0);
        if (st != PLBM_OK) {
            slab_err(s, "slab %d: %s", k, plbm_last_error(s->h[k]));
            return st;
        }
        for (int p = 0; p < s->q; ++p)
            std::memcpy(f + ((size_t)p * s->ny + s->y0[k]) * nx, &buf[((size_t)p * n + w) * nx],
                        sizeof(double) * (size_t)s->rows[k] * nx);
    }
    return PLBM_OK;
}

const char* plbm_slabs_last_error(plbm_slabs ss) {
    Slabs* s = reinterpret_cast<Slabs*>(ss);
    return s ? s->err : g_slab_error;
}

}  // extern "C"
