// sweep_d2q9.cu -- D2Q9 instantiations of the fused collide / stream / boundary sweep
// of a single context
// (storage: FP64, FP32 deviations, BF16 deviations, FP16 deviations).
#include "sweep.cuh"

namespace lbm {

cudaError_t launch_sweep_d2q9(int precision, bool odd, const SweepArgs<double> &a64,
                           const SweepArgs<float> &a32, const TileDesc *tiles, int n_tiles,
                           const TileDesc *tiles_half, int n_half, cudaStream_t st) {
  switch (precision) {
    case 0: return launch_sweep_t<D2Q9, double>(odd, a64, tiles, n_tiles, tiles_half, n_half, st);
    case 1: return launch_sweep_t<D2Q9, float>(odd, a32, tiles, n_tiles, tiles_half, n_half, st);
    case 2: return launch_sweep_t<D2Q9, __nv_bfloat16>(odd, a32, tiles, n_tiles, tiles_half, n_half, st);
    case 3: return launch_sweep_t<D2Q9, __half>(odd, a32, tiles, n_tiles, tiles_half, n_half, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lbm
