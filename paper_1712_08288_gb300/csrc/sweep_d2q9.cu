// sweep_d2q9.cu -- D2Q9 instantiations of the fused collide / stream / boundary sweep
// of a single context
// (storage: FP64, FP32 deviations, BF16 deviations, FP16 deviations).
#include "sweep.cuh"

namespace lbm {

cudaError_t launch_sweep_d2q9(int precision, bool odd, const SweepArgs<double> &a64,
                           const SweepArgs<float> &a32, const TileDesc *tiles, int n_tiles,
                           int bx, cudaStream_t st) {
  switch (precision) {
    case 0: return launch_sweep_t<D2Q9, double>(odd, a64, tiles, n_tiles, bx, st);
    case 1: return launch_sweep_t<D2Q9, float>(odd, a32, tiles, n_tiles, bx, st);
    case 2: return launch_sweep_t<D2Q9, __nv_bfloat16>(odd, a32, tiles, n_tiles, bx, st);
    case 3: return launch_sweep_t<D2Q9, __half>(odd, a32, tiles, n_tiles, bx, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lbm
