// sweep_df_x12.cu -- the fused X1 X2 pass of FP64 storage in double-float
// arithmetic (sweep_x12_df.cuh), degrees 0..2, every element format.
#include "sweep_x12_df.cuh"

namespace sldg {

cudaError_t launch_sweep_x12_df(void* f, const Grid& g, const void* ab1, const int* s1,
                                const void* ab2, const int* s2, int in_df, int out_df,
                                cudaStream_t st, int* shape, void* out, const double* fold_w,
                                const double* fold_r) {
  const double* d = static_cast<const double*>(f);
  double* o = static_cast<double*>(out ? out : f);
  auto go = [&](auto nt) -> cudaError_t {
    constexpr int N = decltype(nt)::value;
    const double *w = fold_w, *r = fold_r;
    if (in_df && out_df) return launch_x12_df_N<N, true, true>(d, o, g, ab1, s1, ab2, s2, st, shape, w, r);
    if (in_df) return launch_x12_df_N<N, true, false>(d, o, g, ab1, s1, ab2, s2, st, shape, w, r);
    if (out_df) return launch_x12_df_N<N, false, true>(d, o, g, ab1, s1, ab2, s2, st, shape, w, r);
    return launch_x12_df_N<N, false, false>(d, o, g, ab1, s1, ab2, s2, st, shape, w, r);
  };
  switch (g.n) {
    case 1: return go(std::integral_constant<int, 1>());
    case 2: return go(std::integral_constant<int, 2>());
    case 3: return go(std::integral_constant<int, 3>());
    // Four nodes per cell (degree 3): the pass is bound by its double-float
    // arithmetic like the two separate kernels, which it does not beat
    // (2.83 against 2.43 ms per pass at 32^4 cells; 2.39 against 2.33 with
    // an X1 layout free of bank conflicts): not supported, the caller runs
    // those.
    default: return cudaErrorNotSupported;
  }
}

}  // namespace sldg
