// sweep_df.cu -- double-float instantiations of the sweep kernels: FP64
// storage, arithmetic on the FP32 pipe (the forward sweeps of FP64 contexts).
// The packed FP32x2 kernels (sweep_df2.cuh for x1, sweep_df3.cuh for the
// strided directions) take degrees 0..3 on aligned layouts; everything else
// runs the one-lane double-float kernels.
#include "sweep_df2.cuh"
#include "sweep_df3.cuh"
#include "sweep_x12_df.cuh"

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

cudaError_t launch_ebar_df(const SweepArgs& a, cudaStream_t st) {
  switch (a.n) {
    case 1: return launch_ebar_df3_T<1>(a, st);
    case 2: return launch_ebar_df3_T<2>(a, st);
    case 3: return launch_ebar_df3_T<3>(a, st);
    case 4: return launch_ebar_df3_T<4>(a, st);
    default: return cudaErrorNotSupported;
  }
}

cudaError_t launch_sweep_x12_df(void* f, const Grid& g, const void* ab1, const int* s1,
                                const void* ab2, const int* s2, int in_df, int out_df,
                                cudaStream_t st, int* shape, void* out) {
  const double* d = static_cast<const double*>(f);
  double* o = static_cast<double*>(out ? out : f);
  auto go = [&](auto nt) -> cudaError_t {
    constexpr int N = decltype(nt)::value;
    if (in_df && out_df) return launch_x12_df_N<N, true, true>(d, o, g, ab1, s1, ab2, s2, st, shape);
    if (in_df) return launch_x12_df_N<N, true, false>(d, o, g, ab1, s1, ab2, s2, st, shape);
    if (out_df) return launch_x12_df_N<N, false, true>(d, o, g, ab1, s1, ab2, s2, st, shape);
    return launch_x12_df_N<N, false, false>(d, o, g, ab1, s1, ab2, s2, st, shape);
  };
  switch (g.n) {
    case 1: return go(std::integral_constant<int, 1>());
    case 2: return go(std::integral_constant<int, 2>());
    case 3: return go(std::integral_constant<int, 3>());
    // Four nodes per cell (degree 3): the X1 phase's lane stride of two cells
    // (64 bytes) makes its shared-memory accesses 8-way bank conflicts, and the
    // fused pass runs slower than the two separate kernels (measured 2.83
    // against 2.43 ms per pass at 32^4 cells): not supported, the caller runs
    // those.
    default: return cudaErrorNotSupported;
  }
}

}  // namespace sldg
