// sweep_df.cu -- double-float instantiations of the sweep kernels: FP64
// storage, arithmetic on the FP32 pipe (the forward sweeps of FP64 contexts).
// The packed FP32x2 kernels (sweep_df2.cuh for x1, sweep_df3.cuh for the
// strided directions) take degrees 0..3 on aligned layouts; everything else
// runs the one-lane double-float kernels.  The fused x pass and the v-sweep
// adjoints with field-gradient partials are instantiated in sweep_df_x12.cu
// and sweep_df_adj.cu (translation units compiled in parallel).
#include "sweep_df2.cuh"
#include "sweep_df3.cuh"

namespace sldg {

// degree 3 (the paper's dG4): the warp-per-pair x1 and the strided kernels
static cudaError_t launch_sweep_df_n4(const SweepArgs& a, cudaStream_t st) {
  if (a.adjoint || (reinterpret_cast<uintptr_t>(a.f) & 15)) return cudaErrorNotSupported;
  auto go = [&](auto in_t, auto out_t) -> cudaError_t {
    constexpr bool I = decltype(in_t)::value, O = decltype(out_t)::value;
    if (a.dim == 0) return out_of_place(a) ? cudaErrorNotSupported : launch_x1_warp_T<4, I, O>(a, st);
    if (a.inner % 2) return cudaErrorNotSupported;
    return launch_strided_df3_T<4, I, O>(a, st);
  };
  using T = std::true_type;
  using F = std::false_type;
  if (a.in_df && a.out_df) return go(T(), T());
  if (a.in_df) return go(T(), F());
  if (a.out_df) return go(F(), T());
  return go(F(), F());
}

cudaError_t launch_sweep_df(const SweepArgs& a, cudaStream_t st) {
  const cudaError_t e = a.n == 4 ? launch_sweep_df_n4(a, st) : launch_sweep_df2(a, st);
  if (e != cudaErrorNotSupported || out_of_place(a)) return e;
  if (a.in_df && a.out_df) return launch_sweep_any<PolDFT<true, true>>(a, st);
  if (a.in_df) return launch_sweep_any<PolDFT<true, false>>(a, st);
  if (a.out_df) return launch_sweep_any<PolDFT<false, true>>(a, st);
  return launch_sweep_any<PolDFT<false, false>>(a, st);
}

}  // namespace sldg
