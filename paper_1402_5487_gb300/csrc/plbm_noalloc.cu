// plbm_diagnostics_noalloc: global sums and extrema of caller-held FP64
// populations for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: plug-ins whose host application
// owns every allocation (custom allocators, fixed memory budgets), or embedded
// setups that forbid allocation after start-up.  This entry point needs no handle and no
// workspace.  Its only scratch (one partial-sum record per block) lives in the
// file-scope device array below, which every GPU that loads the library holds
// until the process exits.
//
// Set-up: a __device__ array exists once per CUDA context, at a different
// address in each.  The first call made while a given context is current
// looks up the array's address in that context with cudaGetSymbolAddress and
// caches it under the context's unique ID (cuCtxGetId: IDs are never reused,
// so a context destroyed by cudaDeviceReset or cuCtxDestroy and a new one at
// the same handle value never share an entry).  Any context works: the
// device's primary context of the runtime API, or one the caller created and
// made current with the driver API.
//
// Every call shares the one array.  Each block writes its own record before
// the final pass reads it, so nothing has to start at zero and stale contents
// of an earlier call are never read; but two calls that overlap on the GPU (on
// different streams, or from different threads) race on the array and may
// return wrong sums.  Serialise them.
#include "plbm.h"

#include <cstdio>
#include <mutex>

#include <cuda.h>  // CUcontext and the driver's function types; nothing is linked from libcuda
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "plbm_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = PLBM_NOALLOC_MAX_NODES / kThreads;
constexpr int kRecord = 8;     // doubles per block record (6 used)
constexpr int kMaxContexts = 64;  // cached addresses; the oldest entry is replaced first
constexpr int kFinalThreads = 512;

static __device__ __align__(256) double g_noalloc_scratch[kMaxBlocks * kRecord];

struct NodeSet {
    int dim, q1, q, nx, ny;
    int v[PLBM_MAX_Q1];
};

__global__ void __launch_bounds__(kThreads) k_noalloc_partials(const NodeSet L, const double* __restrict__ f,
                                                               double* __restrict__ scratch) {
    const long long n = (long long)blockIdx.x * kThreads + threadIdx.x;
    const long long nodes = (long long)L.nx * L.ny;
    double m = 0.0, jx = 0.0, jy = 0.0, e = 0.0, rmin = 1e300, tmin = 1e300;
    if (n < nodes) {
        for (int p = 0; p < L.q; ++p) {
            const int ix = (L.dim == 1) ? p : p / L.q1;
            const int iy = (L.dim == 1) ? 0 : p % L.q1;
            const double vx = (double)L.v[ix];
            const double vy = (L.dim == 1) ? 0.0 : (double)L.v[iy];
            const double fp = f[(long long)p * nodes + n];
            m += fp;
            jx += vx * fp;
            jy += vy * fp;
            e += (vx * vx + vy * vy) * fp;
        }
        const double ux = jx / m, uy = jy / m;
        rmin = m;
        tmin = (e / m - (ux * ux + uy * uy)) / (double)L.dim;
    }
    __shared__ double sh[6][kThreads];
    sh[0][threadIdx.x] = m;
    sh[1][threadIdx.x] = jx;
    sh[2][threadIdx.x] = jy;
    sh[3][threadIdx.x] = e;
    sh[4][threadIdx.x] = rmin;
    sh[5][threadIdx.x] = tmin;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
            sh[4][threadIdx.x] = fmin(sh[4][threadIdx.x], sh[4][threadIdx.x + s]);
            sh[5][threadIdx.x] = fmin(sh[5][threadIdx.x], sh[5][threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x < 6) scratch[(long long)blockIdx.x * kRecord + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void __launch_bounds__(kFinalThreads) k_noalloc_final(const double* __restrict__ scratch,
                                                                 int nblocks, double* __restrict__ out) {
    __shared__ double sh[6][kFinalThreads];
    double r[6] = {0, 0, 0, 0, 1e300, 1e300};
    for (int b = threadIdx.x; b < nblocks; b += kFinalThreads) {
        const double* q = scratch + (long long)b * kRecord;
        for (int k = 0; k < 4; ++k) r[k] += q[k];
        r[4] = fmin(r[4], q[4]);
        r[5] = fmin(r[5], q[5]);
    }
    for (int k = 0; k < 6; ++k) sh[k][threadIdx.x] = r[k];
    __syncthreads();
    for (int s = kFinalThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
            sh[4][threadIdx.x] = fmin(sh[4][threadIdx.x], sh[4][threadIdx.x + s]);
            sh[5][threadIdx.x] = fmin(sh[5][threadIdx.x], sh[5][threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x < 6) out[threadIdx.x] = sh[threadIdx.x][0];
}

std::mutex g_mutex;

struct ContextSlot {
    unsigned long long id;  // cuCtxGetId of the context; 0 = empty slot
    double* scratch;        // g_noalloc_scratch's device address in that context
};
ContextSlot g_slots[kMaxContexts] = {};
int g_next_slot = 0;
PFN_cuCtxGetCurrent_v4000 g_ctx_get_current = nullptr;
PFN_cuCtxGetId_v12000 g_ctx_get_id = nullptr;

void fail(const char* fmt, const char* a = "", long long n = 0) {
    char buf[256];
    std::snprintf(buf, sizeof buf, fmt, a, n);
    plbm::set_thread_error(buf);
}

// Driver entry points through the runtime (no link-time dependence on libcuda).
bool load_driver_entry_points() {
    if (g_ctx_get_current && g_ctx_get_id) return true;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 4000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
        return false;
    g_ctx_get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(fn);
    fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
        return false;
    g_ctx_get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(fn);
    return true;
}

// Device address of g_noalloc_scratch in the context current on this thread.
// Host code sees g_noalloc_scratch only as a stand-in symbol, so the kernels
// must be given this address.  Called with g_mutex held.
plbm_status scratch_of_current_context(double** out) {
    if (!load_driver_entry_points()) {
        fail("plbm_diagnostics_noalloc: driver entry points cuCtxGetCurrent/cuCtxGetId unavailable%s");
        return PLBM_E_CUDA;
    }
    void* looked_up = nullptr;
    CUcontext ctx = nullptr;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS) {
        fail("plbm_diagnostics_noalloc: cuCtxGetCurrent failed%s");
        return PLBM_E_CUDA;
    }
    if (!ctx) {
        // No context is current on this thread yet: the runtime makes the current
        // device's primary context current on its first call, this lookup.
        const cudaError_t e = cudaGetSymbolAddress(&looked_up, g_noalloc_scratch);
        if (e != cudaSuccess || !looked_up) {
            fail("plbm_diagnostics_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return PLBM_E_CUDA;
        }
        if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) {
            fail("plbm_diagnostics_noalloc: no CUDA context is current%s");
            return PLBM_E_CUDA;
        }
    }
    unsigned long long id = 0;
    if (g_ctx_get_id(ctx, &id) != CUDA_SUCCESS || id == 0) {
        fail("plbm_diagnostics_noalloc: cuCtxGetId failed%s");
        return PLBM_E_CUDA;
    }
    for (const ContextSlot& slot : g_slots) {
        if (slot.id == id) {
            *out = slot.scratch;
            return PLBM_OK;
        }
    }
    if (!looked_up) {
        const cudaError_t e = cudaGetSymbolAddress(&looked_up, g_noalloc_scratch);
        if (e != cudaSuccess || !looked_up) {
            fail("plbm_diagnostics_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return PLBM_E_CUDA;
        }
    }
    g_slots[g_next_slot] = ContextSlot{id, static_cast<double*>(looked_up)};
    g_next_slot = (g_next_slot + 1) % kMaxContexts;
    *out = static_cast<double*>(looked_up);
    return PLBM_OK;
}

}  // namespace

extern "C" plbm_status plbm_diagnostics_noalloc(int dim, int q1, const int* v, int nx, int ny,
                                                const double* f, double* out, void* stream) {
    if ((dim != 1 && dim != 2) || q1 < 1 || q1 > PLBM_MAX_Q1 || !v || !f || !out || nx < 1 || ny < 1 ||
        (dim == 1 && ny != 1)) {
        fail("plbm_diagnostics_noalloc: invalid arguments%s", "");
        return PLBM_E_ARG;
    }
    const long long nodes = (long long)nx * ny;
    if (nodes > PLBM_NOALLOC_MAX_NODES) {
        fail("plbm_diagnostics_noalloc: %s%lld nodes exceed the limit of PLBM_NOALLOC_MAX_NODES "
             "(the size of the static scratch array)", "", nodes);
        return PLBM_E_ARG;
    }
    // An error left pending by earlier, unrelated work is reported as such (and
    // left in place) rather than blamed on this call's launches.
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) {
        fail("plbm_diagnostics_noalloc: a CUDA error from earlier work is pending (not cleared): %s",
             cudaGetErrorString(e));
        return PLBM_E_CUDA;
    }
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        const plbm_status st = scratch_of_current_context(&scratch);
        if (st != PLBM_OK) return st;
    }
    NodeSet L{};
    L.dim = dim;
    L.q1 = q1;
    L.q = dim == 1 ? q1 : q1 * q1;
    L.nx = nx;
    L.ny = ny;
    for (int i = 0; i < q1; ++i) L.v[i] = v[i];
    const int nblocks = (int)((nodes + kThreads - 1) / kThreads);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_noalloc_partials<<<nblocks, kThreads, 0, s>>>(L, f, scratch);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        fail("plbm_diagnostics_noalloc: launch of k_noalloc_partials failed: %s", cudaGetErrorString(e));
        return PLBM_E_CUDA;
    }
    k_noalloc_final<<<1, kFinalThreads, 0, s>>>(scratch, nblocks, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        fail("plbm_diagnostics_noalloc: launch of k_noalloc_final failed: %s", cudaGetErrorString(e));
        return PLBM_E_CUDA;
    }
    return PLBM_OK;
}
