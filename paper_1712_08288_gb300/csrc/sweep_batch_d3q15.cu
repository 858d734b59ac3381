// sweep_batch_d3q15.cu -- D3Q15 instantiations of the batched sweep (many contexts in
// one persistent launch), in 64-node and 32-node tiles, for every storage precision.
#include "sweep.cuh"

namespace lbm {

namespace {
template <class T, class A>
cudaError_t batch_d3q15(int tile_w, bool odd, const void *inst, const TileDesc *tiles, const int *tile_inst,
                      int n_tiles, bool big, bool aligned, bool skew, int blocks_per_sm, cudaStream_t st,
                      bool prepare_only) {
  const A *args = static_cast<const A *>(inst);
  if (tile_w == 32)
    return launch_sweep_batch_t<D3Q15, T, 32>(odd, args, tiles, tile_inst, n_tiles, big, aligned, skew,
                                            blocks_per_sm, st, prepare_only);
  if (tile_w == kTileW)
    return launch_sweep_batch_t<D3Q15, T, kTileW>(odd, args, tiles, tile_inst, n_tiles, big, aligned, skew,
                                                blocks_per_sm, st, prepare_only);
  return cudaErrorInvalidValue;
}
}  // namespace

cudaError_t launch_sweep_batch_d3q15(int precision, int tile_w, bool odd, const void *inst,
                                   const TileDesc *tiles, const int *tile_inst, int n_tiles, bool big,
                                   bool aligned, bool skew, int blocks_per_sm, cudaStream_t st,
                                   bool prepare_only) {
  switch (precision) {
    case 0: return batch_d3q15<double, SweepArgs<double>>(tile_w, odd, inst, tiles, tile_inst, n_tiles, big, aligned, skew, blocks_per_sm, st, prepare_only);
    case 1: return batch_d3q15<float, SweepArgs<float>>(tile_w, odd, inst, tiles, tile_inst, n_tiles, big, aligned, skew, blocks_per_sm, st, prepare_only);
    case 2: return batch_d3q15<__nv_bfloat16, SweepArgs<float>>(tile_w, odd, inst, tiles, tile_inst, n_tiles, big, aligned, skew, blocks_per_sm, st, prepare_only);
    case 3: return batch_d3q15<__half, SweepArgs<float>>(tile_w, odd, inst, tiles, tile_inst, n_tiles, big, aligned, skew, blocks_per_sm, st, prepare_only);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lbm
