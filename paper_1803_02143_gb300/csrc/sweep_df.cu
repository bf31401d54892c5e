// sweep_df.cu -- double-float instantiations of the sweep kernels: FP64
// storage, arithmetic on the FP32 pipe (the forward sweeps of FP64 contexts).
// The packed FP32x2 kernels (sweep_df2.cuh for x1, sweep_df3.cuh for the
// strided directions) take degrees 0..2 on aligned layouts; everything else
// runs the one-lane double-float kernels.
#include "sweep_df2.cuh"
#include "sweep_df3.cuh"

namespace sldg {

cudaError_t launch_sweep_df(const SweepArgs& a, cudaStream_t st) {
  const cudaError_t e = launch_sweep_df2(a, st);
  if (e != cudaErrorNotSupported) return e;
  if (a.in_df && a.out_df) return launch_sweep_any<PolDFT<true, true>>(a, st);
  if (a.in_df) return launch_sweep_any<PolDFT<true, false>>(a, st);
  if (a.out_df) return launch_sweep_any<PolDFT<false, true>>(a, st);
  return launch_sweep_any<PolDFT<false, false>>(a, st);
}

}  // namespace sldg
