// Stream-and-collide launcher for one storage precision (double).  The kernel
// templates live in plbm_device.cuh; this unit only instantiates them so the
// four precisions compile in parallel.
#include "plbm_device.cuh"

namespace plbm {
cudaError_t launch_step_f64(const LatticeParams& P, const void* src, void* dst, bool reduce,
                             cudaStream_t stream) {
    return launch_step_t<double>(P, src, dst, reduce, stream);
}
}  // namespace plbm
