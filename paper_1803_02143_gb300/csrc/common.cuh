// common.cuh -- shared definitions of the libsldg CUDA translation units.
//
// Grid conventions (Sec. 2-3 of the paper): directions 0..3 = x1, x2, v1, v2;
// D_d = ncell_d * n nodal values per direction (n = degree + 1), nodal index
// i = cell * n + node; f stored f[v2][v1][x2][x1] with x1 fastest.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sldg.h"

namespace sldg {

constexpr int kMaxNodes = 4;  // degree <= 3

// Gauss-Legendre basis on [0,1]: nodes xi, weights w (sum 1) and the
// Lagrange denominators 1 / prod_{m != j} (xi_j - xi_m).
struct Basis {
  int n;
  double xi[kMaxNodes];
  double w[kMaxNodes];
  double inv_den[kMaxNodes];
};

// Lagrange basis polynomial phi_j(t) on the Gauss-Legendre nodes.  NT > 0:
// the node count as a compile-time constant (NT = b.n; the loops unroll and
// the operations are the same); NT = 0: b.n at run time.
template <int NT = 0>
__host__ __device__ inline double lagrange(const Basis& b, int j, double t) {
  const int n = NT > 0 ? NT : b.n;
  double p = b.inv_den[j];
#pragma unroll
  for (int m = 0; m < (NT > 0 ? NT : kMaxNodes); ++m)
    if (m < n && m != j) p *= (t - b.xi[m]);
  return p;
}

// phi_j'(t) = inv_den_j * sum_k prod_{m != j, k} (t - xi_m)
template <int NT = 0>
__host__ __device__ inline double lagrange_d(const Basis& b, int j, double t) {
  const int n = NT > 0 ? NT : b.n;
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < (NT > 0 ? NT : kMaxNodes); ++k) {
    if (k >= n || k == j) continue;
    double p = 1.0;
#pragma unroll
    for (int m = 0; m < (NT > 0 ? NT : kMaxNodes); ++m)
      if (m < n && m != j && m != k) p *= (t - b.xi[m]);
    s += p;
  }
  return s * b.inv_den[j];
}

// Projection matrices of Eq. (AB-sldg) for a sub-cell shift theta in [0,1).
// Target local coordinate t < theta comes from the left source cell i* at
// t + 1 - theta, t >= theta from cell i*+1 at t - theta; the L2 projection
// with the diagonal Gauss-Legendre mass matrix gives
//   A_jl = (1/w_j) int_0^theta phi_j(t) phi_l(t + 1 - theta) dt,
//   B_jl = (1/w_j) int_theta^1 phi_j(t) phi_l(t - theta) dt,
// integrated exactly by n-point Gauss-Legendre on each sub-interval (the
// integrand has degree 2(n-1)).  dA, dB (nullable) are the theta
// derivatives (Leibniz rule).  Row-major j*n + l.  NT as for lagrange.
template <int NT = 0>
__host__ __device__ inline void build_ab(const Basis& b, double theta, double* A, double* B,
                                         double* dA, double* dB) {
  const int n = NT > 0 ? NT : b.n;
  constexpr int U = NT > 0 ? NT : kMaxNodes;  // loop bound the compiler unrolls
  const double om = 1.0 - theta;
#pragma unroll
  for (int j = 0; j < U; ++j) {
    if (j >= n) break;
#pragma unroll
    for (int l = 0; l < U; ++l) {
      if (l >= n) break;
      double a = 0.0, bb = 0.0, da = 0.0, db = 0.0;
#pragma unroll
      for (int q = 0; q < U; ++q) {
        if (q >= n) break;
        const double ta = theta * b.xi[q];
        const double tb = theta + om * b.xi[q];
        const double pa = lagrange<NT>(b, j, ta), pb = lagrange<NT>(b, j, tb);
        a += b.w[q] * pa * lagrange<NT>(b, l, ta + om);
        bb += b.w[q] * pb * lagrange<NT>(b, l, tb - theta);
        if (dA) {
          da += b.w[q] * pa * lagrange_d<NT>(b, l, ta + om);
          db += b.w[q] * pb * lagrange_d<NT>(b, l, tb - theta);
        }
      }
      A[j * n + l] = theta * a / b.w[j];
      B[j * n + l] = om * bb / b.w[j];
      if (dA) {
        const double pj = lagrange<NT>(b, j, theta);
        dA[j * n + l] = (pj * lagrange<NT>(b, l, 1.0) - theta * da) / b.w[j];
        dB[j * n + l] = (-pj * lagrange<NT>(b, l, 0.0) - om * db) / b.w[j];
      }
    }
  }
}

// Split a shift a into s = floor(a/h) and theta = a/h - s in [0,1).
// Division and subtraction are single IEEE operations (no contraction), so
// the integer part agrees with any other correctly rounded evaluation.
__host__ __device__ inline void split_shift(double a, double h, int* s, double* theta) {
#ifdef __CUDA_ARCH__
  const double sigma = __ddiv_rn(a, h);
  const double fl = floor(sigma);
  double th = __dsub_rn(sigma, fl);
#else
  const double sigma = a / h;
  const double fl = floor(sigma);
  double th = sigma - fl;
#endif
  // shifts beyond 2^30 cells are outside any grid this library accepts
  int si = (int)fmin(fmax(fl, -1073741824.0), 1073741824.0);
  if (th >= 1.0) {  // sigma a hair below an integer: theta rounded up to 1
    th = 0.0;
    si += 1;
  }
  *s = si;
  *theta = th;
}

__host__ __device__ inline int wrap_cell(int k, int nc) {
  int r = k % nc;
  return r < 0 ? r + nc : r;
}

// Device-side description of the grid.
struct Grid {
  int n;
  int nc[4];
  long long D[4];
  double lo[4];
  double h[4];
  double dt;
  int vbc;
  long long N;   // all nodal values
  long long Dx;  // x-plane D0 * D1
  long long Dv;  // v-plane D2 * D3
};

}  // namespace sldg
