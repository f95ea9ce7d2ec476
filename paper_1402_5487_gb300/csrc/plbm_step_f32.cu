// Stream-and-collide launcher for one storage precision (float).  The kernel
// templates live in plbm_device.cuh; this unit only instantiates them so the
// four precisions compile in parallel.  Row-paired lattices take the
// two-nodes-per-thread kernel of plbm_pair.cuh.
#include "plbm_pair.cuh"

namespace plbm {
cudaError_t launch_step_f32(const LatticeParams& P, const void* src, void* dst, bool reduce,
                             cudaStream_t stream) {
    if (P.paired) return launch_step_pair_t<float>(P, src, dst, reduce, stream);
    if (P.dim == 2 && P.sym5 && !P.isothermal && !P.fixed_ends) return launch_step_sym5_t<float>(P, src, dst, reduce, stream);
    return launch_step_t<float>(P, src, dst, reduce, stream);
}
cudaError_t launch_batch_f32(const PairParams* inst, int ninst, int total_tiles, int block_x, int ctas,
                             int parity, const unsigned short* tile_inst, cudaStream_t stream) {
    return launch_batch_pair_t<float>(inst, ninst, total_tiles, block_x, ctas, parity, tile_inst, stream);
}
cudaError_t batch_occupancy_f32(int block_x, int* blocks_per_sm) {
    return batch_occupancy_t<float>(block_x, blocks_per_sm);
}
cudaError_t launch_batch_node_f32(int q1, const LatticeParams* inst, const NodeSpan* span, int total_tiles, int ctas,
                                 int parity, const unsigned short* tile_inst, cudaStream_t stream) {
    return launch_batch_node_t<float>(q1, inst, span, total_tiles, ctas, parity, tile_inst, stream);
}
cudaError_t batch_node_occupancy_f32(int q1, int* blocks_per_sm) {
    return batch_node_occupancy_t<float>(q1, blocks_per_sm);
}
}  // namespace plbm
