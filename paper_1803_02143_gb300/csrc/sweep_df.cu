// sweep_df.cu -- double-float instantiations of the sweep kernels: FP64
// storage, arithmetic on the FP32 pipe (the forward sweeps of FP64 contexts).
#include "sweep_kernels.cuh"

namespace sldg {

cudaError_t launch_sweep_df(const SweepArgs& a, cudaStream_t st) {
  return launch_sweep_any<PolDF>(a, st);
}

}  // namespace sldg
