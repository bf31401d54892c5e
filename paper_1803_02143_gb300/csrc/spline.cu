// spline.cu -- the cubic-spline advection of Sec. 3 (the method the paper
// compares SLDG with) on degree-0 grids: one point per cell, every direction
// periodic.  For each line of n points u_i (spacing h) the periodic cubic
// B-spline interpolant u~(x) = sum_k w_k S(x - x_k) has the coefficients of
//   (w_{i-1} + 4 w_i + w_{i+1}) / 6 = u_i     (indices mod n),
// and the new values are u~(x_i - a): with a/h = s + theta (0 <= theta < 1)
//   6 out_i = theta^3 w_{i-s-2} + (4 - 6 om^2 + 3 om^3) w_{i-s-1}
//           + (4 - 6 theta^2 + 3 theta^3) w_{i-s} + om^3 w_{i-s+1},  om = 1 - theta.
//
// The cyclic system is solved through the factorisation of its symbol
//   (S^-1 + 4 + S) / 6 = (1 + z S)(1 + z S^-1) / (6 z),   z = 2 - sqrt(3),
// S the cyclic shift: a causal recurrence y_i = u_i - z y_{i-1}, an
// anti-causal one v_i = y_i - z v_{i+1}, then w = 6 z v.  Both recurrences
// are periodic; every thread runs its chunk of a line after W warm-up
// points started from zero, which drops terms of weight below
// z^(W+1) / (1 - z) (2^-61 for W = 32, 2^-31 for W = 16): the periodic
// solution to below the rounding of the working precision, with the chunks
// of a line computed in parallel.
//
// A CTA takes 32 lines (a 32-column tile of a strided direction, or 32
// consecutive x1 lines) into shared memory as [n][33] (padded: the lines
// are the columns), four threads per line (chunks of ceil(n/4) points).
#include "ctx.h"

namespace sldg {

namespace {

constexpr int kSplLines = 32;
constexpr int kSplChunks = 4;
constexpr int kSplThreads = kSplLines * kSplChunks;
constexpr int kSplPitch = kSplLines + 1;

template <typename T>
__global__ void k_spline_shifts(long long count, const double* __restrict__ src, double dt,
                                double frac, double h, T* __restrict__ theta,
                                int* __restrict__ svec) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= count) return;
  const double a = __dmul_rn(__dmul_rn(src[e], dt), frac);
  int s;
  double th;
  split_shift(a, h, &s, &th);
  theta[e] = (T)th;
  svec[e] = s;
}

// CONTIG: the lines are contiguous (x1); otherwise element i of line
// (block b, column j) is at b n inner + i inner + j.  KEYCOL: the shift key
// is the column (v-sweeps); otherwise the block (x-sweeps), key =
// (block / key_div) % key_mod.
template <typename T, bool CONTIG, bool KEYCOL>
__global__ void __launch_bounds__(kSplThreads)
    k_spline_sweep(T* __restrict__ f, int n, long long inner, long long outer,
                   long long tiles_per_block, const T* __restrict__ theta,
                   const int* __restrict__ svec, long long key_div, long long key_mod, T z,
                   int W) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* U = reinterpret_cast<T*>(smraw);  // [n][kSplPitch]
  T* Y = U + (size_t)n * kSplPitch;
  const int tid = threadIdx.x;
  long long b0, j0;  // first line: block, column
  int nl;            // lines of this tile
  if (CONTIG) {
    b0 = blockIdx.x * (long long)kSplLines;
    j0 = 0;
    nl = (int)min((long long)kSplLines, outer - b0);
  } else {
    b0 = blockIdx.x / tiles_per_block;
    j0 = (blockIdx.x - b0 * tiles_per_block) * kSplLines;
    nl = (int)min((long long)kSplLines, inner - j0);
  }
  T* base = CONTIG ? f + b0 * n : f + b0 * n * inner + j0;

  // stage: every read coalesced (a warp along a line, or along a row of the
  // column tile); the padded pitch keeps the transposed writes conflict-free
  const int warp = tid / kSplLines, lane = tid % kSplLines;
  constexpr int kWarps = kSplThreads / kSplLines;
  if (CONTIG) {
    for (int l = warp; l < nl; l += kWarps) {
      const T* src = base + (long long)l * n;
      for (int i = lane; i < n; i += kSplLines) U[i * kSplPitch + l] = src[i];
    }
  } else if (lane < nl) {
    for (int i = warp; i < n; i += kWarps) U[i * kSplPitch + lane] = base[(long long)i * inner + lane];
  }
  __syncthreads();

  const int l = tid % kSplLines, c = tid / kSplLines;
  const int C = (n + kSplChunks - 1) / kSplChunks;
  const int ib = min(c * C, n), ie = min(ib + C, n);
  const bool act = l < nl && ib < ie;
  T* Ul = U + l;
  T* Yl = Y + l;
  // causal recurrence y_i = u_i - z y_{i-1}
  if (act) {
    T y = T(0);
    int k = (ib - W) % n;
    if (k < 0) k += n;
    for (int t = 0; t < W; ++t) {
      y = fma(-z, y, Ul[k * kSplPitch]);
      k = k + 1 == n ? 0 : k + 1;
    }
    for (int i = ib; i < ie; ++i) {
      y = fma(-z, y, Ul[i * kSplPitch]);
      Yl[i * kSplPitch] = y;
    }
  }
  __syncthreads();
  // anti-causal recurrence v_i = y_i - z v_{i+1}; w = 6 z v over u
  if (act) {
    T v = T(0);
    int k = (ie - 1 + W) % n;
    for (int t = 0; t < W; ++t) {
      v = fma(-z, v, Yl[k * kSplPitch]);
      k = k == 0 ? n - 1 : k - 1;
    }
    const T sz = T(6) * z;
    for (int i = ie - 1; i >= ib; --i) {
      v = fma(-z, v, Yl[i * kSplPitch]);
      Ul[i * kSplPitch] = sz * v;
    }
  }
  __syncthreads();
  // the interpolant at the shifted points
  if (act) {
    const long long key = KEYCOL ? (j0 + l) % key_mod
                                 : ((CONTIG ? b0 + l : b0) / key_div) % key_mod;
    const T th = theta[key];
    const int s = svec[key];
    const T om = T(1) - th, sixth = T(1) / T(6);
    const T w0 = th * th * th * sixth;
    const T w1 = (T(4) - T(6) * om * om + T(3) * om * om * om) * sixth;
    const T w2 = (T(4) - T(6) * th * th + T(3) * th * th * th) * sixth;
    const T w3 = om * om * om * sixth;
    int k = (ib - s - 2) % n;
    if (k < 0) k += n;
    T c0 = Ul[k * kSplPitch];
    k = k + 1 == n ? 0 : k + 1;
    T c1 = Ul[k * kSplPitch];
    k = k + 1 == n ? 0 : k + 1;
    T c2 = Ul[k * kSplPitch];
    k = k + 1 == n ? 0 : k + 1;
    for (int i = ib; i < ie; ++i) {
      const T c3 = Ul[k * kSplPitch];
      k = k + 1 == n ? 0 : k + 1;
      Yl[i * kSplPitch] = fma(w0, c0, fma(w1, c1, fma(w2, c2, w3 * c3)));
      c0 = c1;
      c1 = c2;
      c2 = c3;
    }
  }
  __syncthreads();
  if (CONTIG) {
    for (int ll = warp; ll < nl; ll += kWarps) {
      T* dst = base + (long long)ll * n;
      for (int i = lane; i < n; i += kSplLines) dst[i] = Y[i * kSplPitch + ll];
    }
  } else if (lane < nl) {
    for (int i = warp; i < n; i += kWarps) base[(long long)i * inner + lane] = Y[i * kSplPitch + lane];
  }
}

template <typename T, bool CONTIG, bool KEYCOL>
cudaError_t launch_spline_T(const SweepArgs& a, cudaStream_t st) {
  const int n = a.nc;
  const size_t smem = 2 * (size_t)n * kSplPitch * sizeof(T);
  if (n < 3 || smem > 227 * 1024) return cudaErrorNotSupported;
  auto kfn = k_spline_sweep<T, CONTIG, KEYCOL>;
  if (smem > 48 * 1024) {
    const cudaError_t e =
        cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const long long tiles_per_block = CONTIG ? 1 : (a.inner + kSplLines - 1) / kSplLines;
  const long long blocks = CONTIG ? (a.outer + kSplLines - 1) / kSplLines : a.outer * tiles_per_block;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  const T z = T(2.0 - 1.7320508075688772);  // 2 - sqrt(3)
  const int W = sizeof(T) == 8 ? 32 : 16;
  kfn<<<(unsigned)blocks, kSplThreads, smem, st>>>(
      static_cast<T*>(a.f), n, a.inner, a.outer, tiles_per_block, static_cast<const T*>(a.ab),
      a.s, a.key_div, a.key_mod, z, W);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_spline_P(const SweepArgs& a, cudaStream_t st) {
  if (a.dim == 0) return launch_spline_T<T, true, false>(a, st);
  if (a.dim == 1) return launch_spline_T<T, false, false>(a, st);
  return launch_spline_T<T, false, true>(a, st);
}

}  // namespace

cudaError_t launch_spline_sweep(const SweepArgs& a, cudaStream_t st) {
  if (out_of_place(a)) return cudaErrorNotSupported;  // in place only
  if (a.n != 1 || !a.periodic || a.adjoint) return cudaErrorNotSupported;
  return a.prec == SLDG_FP32 ? launch_spline_P<float>(a, st) : launch_spline_P<double>(a, st);
}

cudaError_t launch_spline_shifts(int prec, long long count, const double* src, double dt,
                                 double frac, double h, void* theta, int* s, cudaStream_t st) {
  const unsigned blocks = (unsigned)((count + 127) / 128);
  if (prec == SLDG_FP32)
    k_spline_shifts<float><<<blocks, 128, 0, st>>>(count, src, dt, frac, h,
                                                   static_cast<float*>(theta), s);
  else
    k_spline_shifts<double><<<blocks, 128, 0, st>>>(count, src, dt, frac, h,
                                                    static_cast<double*>(theta), s);
  return cudaGetLastError();
}

}  // namespace sldg
