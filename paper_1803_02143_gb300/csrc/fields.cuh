// fields.cuh -- launchers of the non-sweep kernels (fields.cu).
#pragma once

#include "ctx.h"

namespace sldg {

// Spectral tables and work arrays of the Poisson map (see fields.cu).
struct PoissonArgs {
  int D0, D1, K0, K1;
  double k0, k1;  // wavenumbers 2 pi / L_d
  const double2 *F1, *F2, *G1, *G2;
  double2 *T, *R, *U;
};

// abt, abt2, sT (nullable): the transposed sweep in forward form, see MatSet
cudaError_t launch_build_mats(int prec, long long count, const double* src, double dt, double frac,
                              double h, const Basis& b, void* ab, void* dab, void* ab2, int* s,
                              cudaStream_t st, void* abt = nullptr, void* abt2 = nullptr,
                              int* sT = nullptr, void* dab2 = nullptr);
cudaError_t launch_rho(int prec, const void* f, const Grid& g, const float2* wv2, double* part,
                       int chunks, double* rho, cudaStream_t st, int* nlaunch, int df = 0);
cudaError_t launch_sum_rows(const double* part, int rows, long long cols, double scale, double* out,
                            int accumulate, cudaStream_t st);
// *p = v on the stream
cudaError_t launch_set_int(int* p, int v, cudaStream_t st);
// double-float pairs -> IEEE doubles, n elements (in place when dst == src)
cudaError_t launch_df_to_ieee(const void* src, void* dst, long long n, cudaStream_t st);
// the reverse: IEEE doubles to double-float pairs (dst may be src)
cudaError_t launch_ieee_to_df(const void* src, void* dst, long long n, cudaStream_t st);
cudaError_t launch_poisson(const PoissonArgs& a, const double* rho, double* E1, double* E2,
                           cudaStream_t st, int* nlaunch);
cudaError_t launch_poisson_adj(const PoissonArgs& a, const double* Eb1, const double* Eb2,
                               double* rhob, cudaStream_t st, int* nlaunch);
// counter (device, nullable): W goes to out[*counter], which is then advanced
cudaError_t launch_energy(const double* E1, const double* E2, const double* wx, long long Dx,
                          double* out, cudaStream_t st, int* counter = nullptr);
size_t diag_scratch_doubles();
cudaError_t launch_diag(int prec, const void* f, const Grid& g, const double* wx, const double* wv,
                        const double* z2, const double* z3, double* scratch, double* out4,
                        cudaStream_t st, int* nlaunch);
cudaError_t launch_init(int prec, void* f, const Grid& g, int kind, const double* params,
                        const double* zall, double* tab, cudaStream_t st, int* nlaunch);
cudaError_t launch_param_grad(int prec, const void* grad, const Grid& g, int kind,
                              const double* params, const double* zall, double* tab,
                              double* scratch, double* out, cudaStream_t st, int* nlaunch);
cudaError_t launch_rho_adj(int prec, void* lam, const Grid& g, const double* wv,
                           const double* rhob, cudaStream_t st);
cudaError_t launch_energy_adj(double* Eb1, double* Eb2, const double* E1, const double* E2,
                              const double* wx, long long Dx, double c, cudaStream_t st);

}  // namespace sldg
