// sweep_f32.cu -- FP32-storage sweeps: the packed FP32x2 kernels
// (sweep_f32x2.cuh) for forward sweeps of degree 0..2 on aligned layouts,
// the one-lane kernels for everything else (adjoint, degree 3, odd sizes).
#include "sweep_f32x2.cuh"

namespace sldg {

cudaError_t launch_sweep_f32(const SweepArgs& a, cudaStream_t st) {
  const cudaError_t e = launch_sweep_f2(a, st);
  if (e != cudaErrorNotSupported) return e;
  return launch_sweep_any<PolF32>(a, st);
}

}  // namespace sldg
