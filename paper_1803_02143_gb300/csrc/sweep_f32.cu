// sweep_f32.cu -- FP32-storage instantiations of the sweep kernels.
#include "sweep_kernels.cuh"

namespace sldg {

cudaError_t launch_sweep_f32(const SweepArgs& a, cudaStream_t st) {
  return launch_sweep_any<PolF32>(a, st);
}

}  // namespace sldg
