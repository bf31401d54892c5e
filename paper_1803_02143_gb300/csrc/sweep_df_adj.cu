// sweep_df_adj.cu -- the double-float v-sweep adjoints with the field-gradient
// partials (k_ebar_df3 of sweep_df3.cuh), degrees 0..3.
#include "sweep_df3.cuh"

namespace sldg {

cudaError_t launch_ebar_df(const SweepArgs& a, cudaStream_t st) {
  switch (a.n) {
    case 1: return launch_ebar_df3_T<1>(a, st);
    case 2: return launch_ebar_df3_T<2>(a, st);
    case 3: return launch_ebar_df3_T<3>(a, st);
    case 4: return launch_ebar_df3_T<4>(a, st);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace sldg
