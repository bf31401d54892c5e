// sweep_f32.cu -- FP32-storage sweeps: the fused X1 X2 pass (sweep_x12.cuh)
// and the packed FP32x2 kernels (sweep_f32x2.cuh) for forward sweeps of
// degree 0..2 on aligned layouts, the one-lane kernels for everything else
// (adjoint, degree 3, odd sizes).
#include "sweep_x12.cuh"

namespace sldg {

cudaError_t launch_sweep_f32(const SweepArgs& a, cudaStream_t st) {
  const cudaError_t e = launch_sweep_f2(a, st);
  if (e != cudaErrorNotSupported || out_of_place(a)) return e;
  return launch_sweep_any<PolF32>(a, st);
}

cudaError_t launch_sweep_x12_f32(void* f, const Grid& g, const void* ab1, const int* s1,
                                 const void* ab2, const int* s2, cudaStream_t st, int* shape,
                                 void* out, const double* fold_w, const double* fold_r) {
  const float* ff = static_cast<const float*>(f);
  float* o = static_cast<float*>(out ? out : f);
  switch (g.n) {
    case 1: return launch_x12_N<1>(ff, o, g, ab1, s1, ab2, s2, st, shape, fold_w, fold_r);
    case 2: return launch_x12_N<2>(ff, o, g, ab1, s1, ab2, s2, st, shape, fold_w, fold_r);
    case 3: return launch_x12_N<3>(ff, o, g, ab1, s1, ab2, s2, st, shape, fold_w, fold_r);
    case 4: return launch_x12_N<4>(ff, o, g, ab1, s1, ab2, s2, st, shape, fold_w, fold_r);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace sldg
