// sweep_f64.cu -- FP64-FMA instantiations of the sweep kernels (the
// transposed sweeps of FP64 contexts, and forward sweeps on request).
#include "sweep_kernels.cuh"

namespace sldg {

cudaError_t launch_sweep_f64(const SweepArgs& a, cudaStream_t st) {
  if (out_of_place(a)) return cudaErrorNotSupported;  // in place only
  return launch_sweep_any<PolF64>(a, st);
}

size_t sweep_smem_bytes(int prec, int dim, long long D, int lines_per_tile) {
  const size_t es = prec == SLDG_FP64 ? sizeof(double) : sizeof(float);
  return dim == 0 ? x1_smem(es, D, lines_per_tile) : strided_smem(es, D);
}

}  // namespace sldg
