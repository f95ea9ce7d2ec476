// plbm_diagnostics_noalloc: global sums and extrema of caller-held FP64
// populations for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code running inside a CUDA
// graph that is being captured, plug-ins whose host application owns every
// allocation (custom allocators, fixed memory budgets), or embedded setups that
// forbid allocation after start-up.  This entry point needs no handle and no
// workspace.  Its only scratch (one partial-sum record per block) lives in the
// file-scope device array below, which every GPU that loads the library holds
// until the process exits.
//
// Set-up: the first call on a device looks up the device address of that array
// with cudaGetSymbolAddress while the device is current and caches it.  Make the
// first call on each device before any stream capture begins.
//
// Every call shares the one array.  Each block writes its own record before
// the final pass reads it, so nothing has to start at zero and stale contents
// of an earlier call are never read; but two calls that overlap on the GPU (on
// different streams, or from different threads) race on the array and may
// return wrong sums.  Serialise them.
#include "plbm.h"

#include <cstdio>
#include <mutex>

#include <cuda_runtime.h>

#include "plbm_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = PLBM_NOALLOC_MAX_NODES / kThreads;
constexpr int kRecord = 8;     // doubles per block record (6 used)
constexpr int kMaxDevices = 64;
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
double* g_scratch_ptr[kMaxDevices] = {nullptr};

void fail(const char* fmt, const char* a = "", long long n = 0) {
    char buf[256];
    std::snprintf(buf, sizeof buf, fmt, a, n);
    plbm::set_thread_error(buf);
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
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        fail("plbm_diagnostics_noalloc: no usable current CUDA device: %s", cudaGetErrorString(e));
        return PLBM_E_CUDA;
    }
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_scratch_ptr[dev]) {
            // Host code sees g_noalloc_scratch only as a stand-in symbol: the kernel
            // must get the device address, looked up once per device.
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                fail("plbm_diagnostics_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
                return PLBM_E_CUDA;
            }
            g_scratch_ptr[dev] = static_cast<double*>(p);
        }
        scratch = g_scratch_ptr[dev];
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
    k_noalloc_final<<<1, kFinalThreads, 0, s>>>(scratch, nblocks, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        fail("plbm_diagnostics_noalloc: launch failed: %s", cudaGetErrorString(e));
        return PLBM_E_CUDA;
    }
    return PLBM_OK;
}
