// Stream-and-collide launcher for one storage precision (double).  The kernel
// templates live in plbm_device.cuh; this unit only instantiates them so the
// four precisions compile in parallel.
#include "plbm_device.cuh"

namespace plbm {
cudaError_t launch_step_f64(const LatticeParams& P, const void* src, void* dst, bool reduce,
                             cudaStream_t stream) {
    return launch_step_t<double>(P, src, dst, reduce, stream);
}
cudaError_t launch_batch_node_f64(int q1, const LatticeParams* inst, const NodeSpan* span, int total_tiles, int ctas,
                                 int parity, const unsigned short* tile_inst, cudaStream_t stream) {
    return launch_batch_node_t<double>(q1, inst, span, total_tiles, ctas, parity, tile_inst, stream);
}
cudaError_t batch_node_occupancy_f64(int q1, int* blocks_per_sm) {
    return batch_node_occupancy_t<double>(q1, blocks_per_sm);
}
}  // namespace plbm
